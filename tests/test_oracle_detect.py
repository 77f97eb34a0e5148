"""Pins of the oracle's walks, argmin and max-log LLRs: exhaustive ML on 4x4
QPSK, N_pe = 1 == sorted-QR SIC, full enumeration == ML, noise-free recovery,
the p-th-nearest ranking, and the closed-form MRC bit-error rate."""
import math

import numpy as np
import pytest

import oracle
from paper_2409_14355_gb300 import inputs
from tests._ref_helpers import (all_label_vectors, bit_of, maxlog_llr_bruteforce, ml_metrics,
                                mrc_rayleigh_bpsk_ber)


def _prep(H, Y):
    Q, R, perm, _ = oracle.sqrd(H)
    return R, oracle.qhy(Q, Y), perm


@pytest.mark.parametrize("seed", [0, 1])
def test_full_enumeration_is_exhaustive_ml_4x4_qpsk(seed):
    sl = inputs.make_slot(4, 4, 4, 6, 14, 6.0, "iid", 0.3, 1234 + seed)
    pts = oracle.constellation(4)
    cand = all_label_vectors(4, 4)                   # 256 candidates, user order
    cand_s = pts[cand]
    for c in range(sl.n_sc):
        H = sl.H[c].astype(np.complex128)
        Y = sl.Y[c].astype(np.complex128)
        R, Z, perm = _prep(H, Y)
        paths, _, _ = oracle.select_paths(np.diag(R).real, sl.sigma2, 4, 256)
        out = oracle.detect(R, Z, perm, paths, sl.sigma2, 4, want_all=True)
        for s in range(sl.n_sym):
            met = ml_metrics(H, Y[s], cand_s)
            best = np.argmin(met)
            np.testing.assert_array_equal(out["hard"][s], cand[best])
            # d_best + ||y||^2 - ||z||^2 equals the ML metric
            dml = out["ped2"][s, 0] + np.sum(np.abs(Y[s]) ** 2) - np.sum(np.abs(Z[s]) ** 2)
            assert abs(dml - met[best]) <= 1e-12 * max(met[best], 1.0)
            want = maxlog_llr_bruteforce(met, cand, 2, sl.sigma2, oracle.LLR_MAX)
            np.testing.assert_allclose(out["llr"][s], want, rtol=1e-10, atol=1e-9)


def test_full_enumeration_visits_every_vector_once():
    sl = inputs.make_slot(3, 3, 4, 3, 4, 8.0, "iid", 0.3, 77)
    for c in range(sl.n_sc):
        R, Z, perm = _prep(sl.H[c], sl.Y[c])
        paths, _, _ = oracle.select_paths(np.diag(R).real, sl.sigma2, 4, 64)
        out = oracle.detect(R, Z, perm, paths, sl.sigma2, 4, want_all=True)
        for s in range(sl.n_sym):
            vecs = {tuple(v) for v in out["sym_all"][s]}
            assert len(vecs) == 64


def _sic(R, z, perm, pts):
    """Sorted-QR ZF-SIC: plain slicer loop, bottom level last."""
    nt = R.shape[0]
    s = np.zeros(nt, np.complex128)
    lab = np.zeros(nt, np.int64)
    for l in range(nt - 1, -1, -1):
        b = (z[l] - R[l, l + 1:] @ s[l + 1:]) / R[l, l].real
        lab[l] = int(np.argmin(np.abs(b - pts)))
        s[l] = pts[lab[l]]
    hard = np.zeros(nt, np.int64)
    hard[perm] = lab
    return hard, float(np.sum(np.abs(z - R @ s) ** 2))


@pytest.mark.parametrize("nr,nt,qam", [(4, 4, 4), (8, 8, 16), (16, 16, 64)])
def test_single_path_is_sorted_qr_sic(nr, nt, qam):
    sl = inputs.make_slot(nr, nt, qam, 5, 14, 12.0, "iid", 0.3, 5 + nt)
    pts = oracle.constellation(qam)
    for c in range(sl.n_sc):
        R, Z, perm = _prep(sl.H[c], sl.Y[c])
        paths = np.ones((1, nt), np.uint8)
        out = oracle.detect(R, Z, perm, paths, sl.sigma2, qam)
        for s in range(sl.n_sym):
            hard, d = _sic(R, Z[s], perm, pts)
            np.testing.assert_array_equal(out["hard"][s], hard)
            assert np.isclose(out["ped2"][s, 0], d, rtol=1e-12)
            assert np.isinf(out["ped2"][s, 1])
            B = int(math.log2(qam))
            # one-entry list: every LLR is at the clip value with the decided bit's sign
            for k in range(nt):
                for b in range(B):
                    v = bit_of(hard[k], b, B)
                    assert out["llr"][s, k, b] == (-oracle.LLR_MAX if v else oracle.LLR_MAX)


@pytest.mark.parametrize("nr,nt,qam,n_pe", [(4, 4, 4, 16), (8, 8, 16, 64), (16, 16, 64, 256),
                                             (16, 8, 64, 32)])
def test_noise_free_exact_recovery(nr, nt, qam, n_pe):
    sl = inputs.make_slot(nr, nt, qam, 4, 14, 20.0, "iid", 0.3, 31, noise=False)
    pts = oracle.constellation(qam)
    for c in range(sl.n_sc):
        H = sl.H[c].astype(np.complex128)
        Y = pts[sl.labels[c]] @ H.T
        R, Z, perm = _prep(H, Y)
        paths, _, _ = oracle.select_paths(np.diag(R).real, sl.sigma2, qam, n_pe)
        out = oracle.detect(R, Z, perm, paths, sl.sigma2, qam)
        np.testing.assert_array_equal(out["hard"], sl.labels[c])
        assert np.all(out["ped2"][:, 0] < 1e-20)


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_walk_takes_the_pth_nearest_point(qam):
    # One level: R = [[r]], z = r b  ->  the walk of rank p lands on the p-th
    # point of Q ordered by (|b - q|^2, label).
    pts = oracle.constellation(qam)
    rng = np.random.default_rng(qam)
    r = 1.7
    paths = np.arange(1, qam + 1, dtype=np.uint8)[:, None]
    for _ in range(20):
        b = complex(rng.uniform(-1.3, 1.3), rng.uniform(-1.3, 1.3))
        out = oracle.detect(np.array([[r]]), np.array([[r * b]]), np.array([0]), paths, 1.0, qam,
                            want_all=True)
        dist = np.abs(b - pts) ** 2
        order = np.lexsort((np.arange(qam), dist))
        np.testing.assert_array_equal(out["sym_all"][0, :, 0], order)
        np.testing.assert_allclose(out["ped_all"][0], r * r * dist[order], rtol=1e-12)


def test_llr_sign_agrees_with_hard_decision():
    sl = inputs.make_slot(8, 8, 16, 6, 14, 14.0, "kronecker", 0.3, 8)
    for c in range(sl.n_sc):
        R, Z, perm = _prep(sl.H[c], sl.Y[c])
        paths, _, _ = oracle.select_paths(np.diag(R).real, sl.sigma2, 16, 64)
        out = oracle.detect(R, Z, perm, paths, sl.sigma2, 16)
        for b in range(4):
            bits = bit_of(out["hard"], b, 4)
            llr = out["llr"][:, :, b]
            assert np.all(np.where(bits == 1, llr <= 0, llr >= 0))


def test_slot_driver_equals_per_subcarrier_calls_and_is_thread_invariant():
    sl = inputs.make_slot(8, 8, 16, 7, 14, 15.0, "kronecker", 0.3, 4)
    a = oracle.detect_slot(sl.H, sl.Y, sl.sigma2, 16, 64, n_threads=1, with_mmse=True)
    b = oracle.detect_slot(sl.H, sl.Y, sl.sigma2, 16, 64, n_threads=3, with_mmse=True)
    for k in ("hard", "llr", "ped2", "R", "Z", "paths", "mmse_hard", "mmse_llr"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["threads"] == 1 and b["threads"] == 3
    c = 5
    R, Z, perm = _prep(sl.H[c], sl.Y[c])
    paths, _, _ = oracle.select_paths(np.diag(R).real, sl.sigma2, 16, 64)
    one = oracle.detect(R, Z, perm, paths, sl.sigma2, 16)
    np.testing.assert_array_equal(one["hard"], a["hard"][c])
    np.testing.assert_array_equal(one["llr"], a["llr"][c])
    np.testing.assert_array_equal(paths, a["paths"][c])


def test_mrc_qpsk_ber_matches_closed_form():
    # 1 x 2 QPSK over Rayleigh: N_pe = 1 is maximum-ratio combining + slicing;
    # BER must equal the closed-form L = 2 MRC value at Eb/N0 = 1 / (2 sigma2).
    snr_db = 6.0
    sl = inputs.make_slot(2, 1, 4, 36000, 14, snr_db, "iid", 0.3, 2024)
    out = oracle.detect_slot(sl.H, sl.Y, sl.sigma2, 4, 1)
    nbits = sl.labels.size * 2
    err = 0
    for b in range(2):
        err += np.sum(bit_of(out["hard"], b, 2) != bit_of(sl.labels, b, 2))
    ber = err / nbits
    want = mrc_rayleigh_bpsk_ber(1.0 / (2.0 * sl.sigma2), 2)
    sd = math.sqrt(want * (1 - want) / nbits)
    assert abs(ber - want) < 4 * sd + 1e-4, (ber, want)


@pytest.mark.parametrize("nr,nt,qam", [(2, 3, 4), (3, 4, 4), (2, 2, 16)])
def test_mmse_qr_full_enumeration_is_regularised_ml(nr, nt, qam):
    # More users than antennas: with the MMSE-extended QR and a complete list
    # the decision is argmin ||y - H s||^2 + sigma2 ||s||^2 over all of Q^nt.
    sl = inputs.make_slot(nr, nt, qam, 5, 14, 8.0, "iid", 0.3, 123 + nt)
    pts = oracle.constellation(qam)
    cand = all_label_vectors(qam, nt)
    cand_s = pts[cand]
    n_all = qam ** nt
    out = oracle.detect_slot(sl.H, sl.Y, sl.sigma2, qam, n_all, mmse_qr=True)
    for c in range(sl.n_sc):
        H = sl.H[c].astype(np.complex128)
        Y = sl.Y[c].astype(np.complex128)
        for s in range(sl.n_sym):
            met = ml_metrics(H, Y[s], cand_s) + sl.sigma2 * np.sum(np.abs(cand_s) ** 2, axis=1)
            best = np.argmin(met)
            np.testing.assert_array_equal(out["hard"][c, s], cand[best])
            z = out["Z"][c, s]
            dml = out["ped2"][c, s, 0] + np.sum(np.abs(Y[s]) ** 2) - np.sum(np.abs(z) ** 2)
            assert abs(dml - met[best]) <= 1e-11 * max(met[best], 1.0)


def test_mmse_baseline_handles_more_users_than_antennas():
    sl = inputs.make_slot(4, 6, 16, 3, 14, 20.0, "iid", 0.3, 5)
    for c in range(sl.n_sc):
        H = sl.H[c].astype(np.complex128)
        out = oracle.mmse(H, sl.Y[c], sl.sigma2, 16)
        W = np.linalg.solve(H.conj().T @ H + sl.sigma2 * np.eye(6), H.conj().T)
        mu = np.real(np.diag(W @ H))
        np.testing.assert_allclose(out["xt"] * mu, sl.Y[c].astype(np.complex128) @ W.T,
                                   rtol=1e-10, atol=1e-12)
