"""Property-based pins of the oracle on random tiny systems (hypothesis):
a complete list is exhaustive ML for the complex and the real-valued models
alike, with equal max-log LLRs; the best-first table equals the brute-force
ranking of all M^Nt vectors; noise-free slots are recovered at any N_pe."""
import itertools
import math

import numpy as np
import pytest

import oracle

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


def _system(seed, nr, nt, qam, snr_db, n_sym=3, noise=True):
    rng = np.random.default_rng(seed)
    H = (rng.standard_normal((nr, nt)) + 1j * rng.standard_normal((nr, nt))) / math.sqrt(2)
    lab = rng.integers(0, qam, (n_sym, nt))
    s = oracle.constellation(qam)[lab]
    sigma2 = nt / 10 ** (snr_db / 10)
    n = (rng.standard_normal((n_sym, nr)) + 1j * rng.standard_normal((n_sym, nr))) * math.sqrt(sigma2 / 2)
    return H, s @ H.T + (n if noise else 0), sigma2, lab


systems = st.tuples(st.integers(0, 2 ** 31 - 1), st.sampled_from([(2, 2, 4), (3, 2, 4), (2, 1, 16),
                                                                   (3, 2, 16), (3, 3, 4)]),
                    st.floats(0.0, 20.0))


@settings(max_examples=25, deadline=None)
@given(systems)
def test_complete_lists_are_ml_in_both_models(case):
    seed, (nr, nt, qam), snr_db = case
    H, Y, sigma2, _ = _system(seed, nr, nt, qam, snr_db)
    pts = oracle.constellation(qam)
    cands = np.array(list(itertools.product(range(qam), repeat=nt)))
    metric = np.sum(np.abs(Y[:, None, :] - (pts[cands] @ H.T)[None]) ** 2, axis=2)  # [n_sym][M^nt]
    best = cands[np.argmin(metric, axis=1)]
    # complex model
    Q, R, perm, _ = oracle.sqrd(H)
    Z = oracle.qhy(Q, Y)
    full = np.array(list(itertools.product(range(1, qam + 1), repeat=nt)), np.uint8)
    oc = oracle.detect(R, Z, perm, full, sigma2, qam)
    np.testing.assert_array_equal(oc["hard"], best)
    # real-valued decomposition
    Hr, Yr = oracle.rvd_embed(H, Y)
    Qr, Rr, pr, _ = oracle.sqrd(Hr)
    L = 1 << (oracle.BITS[qam] // 2)
    fr = np.array(list(itertools.product(range(1, L + 1), repeat=2 * nt)), np.uint8)
    orv = oracle.detect_rvd(Rr, oracle.qhy(Qr, Yr), pr, fr, sigma2, qam)
    np.testing.assert_array_equal(orv["hard"], best)
    np.testing.assert_allclose(orv["llr"], oc["llr"], rtol=1e-7, atol=1e-7)


@settings(max_examples=25, deadline=None)
@given(st.integers(0, 2 ** 31 - 1), st.sampled_from([(3, 4), (2, 16), (4, 4)]),
       st.integers(1, 60), st.floats(0.02, 2.0))
def test_table_is_the_brute_force_ranking(seed, shape, n_pe, sigma2):
    nt, qam = shape
    n_pe = min(n_pe, qam ** nt)
    rng = np.random.default_rng(seed)
    rdiag = np.sqrt(rng.exponential(1.0, nt) * 3 + 0.05)
    paths, score, pe = oracle.select_paths(rdiag, sigma2, qam, n_pe)
    vecs = np.array(list(itertools.product(range(1, qam + 1), repeat=nt)))
    scores = np.zeros(len(vecs))
    for l in range(nt):
        scores = scores + np.log1p(-pe[l]) + (vecs[:, l] - 1) * math.log(pe[l])
    order = np.lexsort([vecs[:, l] for l in range(nt)] + [-scores])
    want = vecs[order[:n_pe]]
    # rows whose score is apart from their neighbours sit where brute force puts them
    sep = np.abs(np.diff(score)) > 1e-9 * np.maximum(1.0, np.abs(score[1:]))
    ok = np.concatenate([[True], sep]) & np.concatenate([sep, [True]])
    np.testing.assert_array_equal(paths[ok], want[ok])


@settings(max_examples=20, deadline=None)
@given(st.integers(0, 2 ** 31 - 1), st.sampled_from([(4, 4, 16), (8, 8, 64), (6, 4, 16)]),
       st.integers(1, 40))
def test_noise_free_slots_are_recovered(seed, shape, n_pe):
    nr, nt, qam = shape
    H, Y, sigma2, lab = _system(seed, nr, nt, qam, 20.0, noise=False)
    out = oracle.detect_slot(H[None], Y[None], sigma2, qam, n_pe)
    np.testing.assert_array_equal(out["hard"][0], lab)
