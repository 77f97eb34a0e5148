"""Pins of the oracle's real-valued decomposition (RVD) variant: a complete
list over the 2 nt real levels is exhaustive ML, equal to the complex
model's complete list; N_pe = 1 is the real sorted-QR SIC written as a plain
slicer loop; noise-free recovery; selection against brute force; the PAM
level error model against simulated slicing; the axes join back to the
constellation's points."""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests._ref_helpers import qfunc


def _slot(nr, nt, qam, n_sym, snr_db, seed, noise=True):
    rng = np.random.default_rng(seed)
    pts = oracle.constellation(qam)
    H = (rng.standard_normal((nr, nt)) + 1j * rng.standard_normal((nr, nt))) / math.sqrt(2)
    lab = rng.integers(0, qam, (n_sym, nt))
    s = pts[lab]
    sigma2 = nt / 10 ** (snr_db / 10)
    n = (rng.standard_normal((n_sym, nr)) + 1j * rng.standard_normal((n_sym, nr))) * math.sqrt(sigma2 / 2)
    Y = s @ H.T + (n if noise else 0)
    return H, Y, sigma2, lab


def _front_rvd(H, Y):
    Hr, Yr = oracle.rvd_embed(H, Y)
    Q, R, perm, _ = oracle.sqrd(Hr)
    return R, oracle.qhy(Q, Yr), perm


def test_embedding_reproduces_the_complex_model():
    H, Y, _, lab = _slot(3, 2, 16, 4, 20.0, 1, noise=False)
    Hr, Yr = oracle.rvd_embed(H, Y)
    s = oracle.constellation(16)[lab]
    sr = np.concatenate([s.real, s.imag], axis=-1)
    np.testing.assert_allclose(sr @ Hr.real.T, Yr.real, atol=1e-12)
    assert np.all(Hr.imag == 0) and np.all(Yr.imag == 0)


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_axes_join_back_to_the_constellation(qam):
    pam = oracle.pam_points(qam)
    pts = oracle.constellation(qam)
    L = len(pam)
    nt = 1
    re, im = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    hard_r = np.stack([re.ravel(), im.ravel()], axis=-1).astype(np.uint8)   # [L*L][2]
    llr_r = np.zeros((L * L, 2, oracle.BITS[qam] // 2))
    lab, _ = oracle.join_axes(hard_r, llr_r, qam)
    np.testing.assert_allclose(pts[lab[:, 0]], pam[re.ravel()] + 1j * pam[im.ravel()], atol=1e-15)
    assert len(set(lab[:, 0].tolist())) == qam and nt == 1


@pytest.mark.parametrize("nr,nt,qam,seed", [(2, 2, 4, 1), (3, 2, 16, 2), (3, 3, 4, 3)])
def test_complete_list_is_ml_and_equals_the_complex_model(nr, nt, qam, seed):
    H, Y, sigma2, _ = _slot(nr, nt, qam, 6, 8.0, seed)
    L = 1 << (oracle.BITS[qam] // 2)
    ntr = 2 * nt
    R, Z, perm = _front_rvd(H, Y)
    full = np.array(list(itertools.product(range(1, L + 1), repeat=ntr)), np.uint8)
    o = oracle.detect_rvd(R, Z, perm, full, sigma2, qam)
    # exhaustive ML in the complex model
    pts = oracle.constellation(qam)
    cands = np.array(list(itertools.product(range(qam), repeat=nt)))
    S = pts[cands]                                         # [M^nt][nt]
    for k in range(Y.shape[0]):
        m = np.sum(np.abs(Y[k][None, :] - S @ H.T) ** 2, axis=1)
        best = int(np.argmin(m))
        np.testing.assert_array_equal(o["hard"][k], cands[best])
        # d + ||y||^2 - ||z||^2 is the ML metric (real QR of a tall matrix)
        yr = np.concatenate([Y[k].real, Y[k].imag])
        assert math.isclose(o["ped2"][k][0] + yr @ yr - np.sum(np.abs(Z[k]) ** 2), m[best],
                            rel_tol=1e-9, abs_tol=1e-12)
    # and the complex model's complete list gives the same LLRs
    Q, Rc, pc, _ = oracle.sqrd(H)
    Zc = oracle.qhy(Q, Y)
    fullc = np.array(list(itertools.product(range(1, qam + 1), repeat=nt)), np.uint8)
    oc = oracle.detect(Rc, Zc, pc, fullc, sigma2, qam)
    np.testing.assert_array_equal(o["hard"], oc["hard"])
    np.testing.assert_allclose(o["llr"], oc["llr"], rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("nt,qam", [(2, 16), (4, 64), (8, 4)])
def test_single_path_is_real_sorted_qr_sic(nt, qam):
    H, Y, sigma2, _ = _slot(nt, nt, qam, 5, 15.0, nt + qam)
    R, Z, perm = _front_rvd(H, Y)
    R = np.real(R)
    pam = oracle.pam_points(qam)
    ntr = 2 * nt
    o = oracle.detect_rvd(R, Z, perm, np.ones((1, ntr), np.uint8), sigma2, qam)
    for k in range(Z.shape[0]):
        z = np.real(Z[k])
        s = np.zeros(ntr)
        a = np.zeros(ntr, int)
        for l in range(ntr - 1, -1, -1):
            b = (z[l] - R[l, l + 1:] @ s[l + 1:]) / R[l, l]
            d = (b - pam) ** 2
            a[l] = int(np.lexsort((np.arange(len(pam)), d))[0])   # nearest, ties to the lower label
            s[l] = pam[a[l]]
        hard_r = np.zeros(ntr, np.uint8)
        hard_r[perm] = a
        np.testing.assert_array_equal(o["hard_r"][k], hard_r)


def test_noise_free_slots_are_recovered():
    H, Y, sigma2, lab = _slot(8, 8, 64, 6, 20.0, 9, noise=False)
    out = oracle.detect_slot_rvd(H[None], Y[None], sigma2, 64, 16)
    np.testing.assert_array_equal(out["hard"][0], lab)


def _bruteforce_pam(rdiag, sigma2, qam, n_pe):
    L = 1 << (oracle.BITS[qam] // 2)
    ntr = len(rdiag)
    pe = []
    for r in rdiag:
        x = math.sqrt(3 * r * r / sigma2 / (qam - 1))
        pe.append(max(2 * (1 - 1 / L) * qfunc(x), oracle.PE_FLOOR))
    vecs = np.array(list(itertools.product(range(1, L + 1), repeat=ntr)))[:, ::-1]
    scores = np.zeros(len(vecs))
    for l in range(ntr):
        scores = scores + np.log1p(-pe[l]) + (vecs[:, l] - 1) * math.log(pe[l])
    keys = [vecs[:, l] for l in range(ntr)] + [-scores]
    order = np.lexsort(keys)
    return vecs[order[:n_pe]].astype(np.uint8)


@pytest.mark.parametrize("ntr,qam,n_pe", [(4, 16, 40), (6, 4, 30), (3, 64, 100)])
def test_pam_selection_matches_bruteforce(ntr, qam, n_pe):
    rng = np.random.default_rng(ntr * qam)
    for _ in range(4):
        rdiag = np.sqrt(rng.exponential(1.0, ntr) * 3 + 0.05)
        sigma2 = float(rng.choice([0.05, 0.2, 1.0]))
        paths, score, _ = oracle.select_paths_pam(rdiag, sigma2, qam, n_pe)
        want = _bruteforce_pam(rdiag, sigma2, qam, n_pe)
        sep = np.abs(np.diff(score)) > 1e-9
        ok = np.concatenate([[True], sep]) & np.concatenate([sep, [True]])
        np.testing.assert_array_equal(paths[ok], want[ok])


@pytest.mark.parametrize("qam,snr_db", [(4, 6.0), (16, 14.0), (64, 22.0)])
def test_pam_level_model_matches_simulated_slicing(qam, snr_db):
    # a real level b = s + n / R_ll with noise sigma2/2 per real dimension:
    # simulate the slicer and compare its error rate with the model's Pe
    rng = np.random.default_rng(qam)
    pam = oracle.pam_points(qam)
    sigma2 = 1.0
    gamma = 10 ** (snr_db / 10)
    rll = math.sqrt(gamma * sigma2)
    n = 400_000
    a = rng.integers(0, len(pam), n)
    b = pam[a] + rng.standard_normal(n) * math.sqrt(sigma2 / 2) / rll
    dec = np.argmin(np.abs(b[:, None] - pam[None, :]), axis=1)
    ser = np.mean(dec != a)
    _, _, pe = oracle.select_paths_pam(np.array([rll]), sigma2, qam, 1)
    sd = math.sqrt(pe[0] * (1 - pe[0]) / n)
    assert abs(ser - pe[0]) <= 5 * sd, (ser, pe[0])
