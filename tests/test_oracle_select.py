"""Pins of the oracle's position-vector selection: brute force over all M^Nt
vectors on tiny systems, structural invariants, and a Monte-Carlo check of the
per-level symbol-error model against simulated QAM slicing."""
import math

import numpy as np
import pytest

import oracle
from tests._ref_helpers import qfunc


def _pe_textbook(gamma, M):
    # exact nearest-neighbour SER of square M-QAM at SNR gamma (Proakis eq. 4.3-30)
    # (1 - (1 - p)^2 expanded as p (2 - p) to keep precision at high SNR)
    p = 2.0 * (1.0 - 1.0 / math.sqrt(M)) * qfunc(math.sqrt(3.0 * gamma / (M - 1)))
    return max(p * (2.0 - p), oracle.PE_FLOOR)


def _bruteforce_top(rdiag, sigma2, M, n_pe):
    nt = len(rdiag)
    pe = [_pe_textbook(r * r / sigma2, M) for r in rdiag]
    logp = [[math.log(1.0 - pe[l]) + (k - 1) * math.log(pe[l]) for k in range(M + 1)]
            for l in range(nt)]
    vecs = np.array(np.meshgrid(*[np.arange(1, M + 1)] * nt, indexing="ij")).reshape(nt, -1).T
    scores = np.zeros(len(vecs))
    for l in range(nt):  # same summation order as the definition (level 0 first)
        scores = scores + np.array([logp[l][k] for k in vecs[:, l]])
    # order: score descending, then lexicographically smaller from the top level
    keys = [vecs[:, l] for l in range(nt)] + [-scores]
    order = np.lexsort(keys)
    return vecs[order[:n_pe]].astype(np.uint8), scores[order[:n_pe]]


@pytest.mark.parametrize("nt,M,n_pe,seed", [(4, 4, 16, 1), (4, 4, 256, 2), (2, 16, 40, 3),
                                            (3, 16, 100, 4), (4, 4, 60, 5), (1, 64, 64, 6)])
def test_matches_bruteforce_ranking(nt, M, n_pe, seed):
    rng = np.random.default_rng(seed)
    for _ in range(5):
        rdiag = np.sqrt(rng.exponential(1.0, nt) * 2 + 0.05)
        sigma2 = float(rng.choice([0.1, 0.4, 1.0, 2.5]))
        paths, score, pe = oracle.select_paths(rdiag, sigma2, M, n_pe)
        want, wscore = _bruteforce_top(rdiag, sigma2, M, n_pe)
        np.testing.assert_array_equal(paths, want)
        np.testing.assert_allclose(score, wscore, rtol=1e-12)


def test_equal_levels_break_ties_lexicographically():
    rdiag = np.ones(4)
    paths, score, _ = oracle.select_paths(rdiag, 0.5, 4, 30)
    want, _ = _bruteforce_top(rdiag, 0.5, 4, 30)
    np.testing.assert_array_equal(paths, want)
    # Two equal levels: swapping the two terms of a two-term sum is exact, so
    # (2,1) and (1,2) tie exactly and the lexicographic rule (top level
    # compared first, smaller first) puts (2,1) ahead.
    paths, score, _ = oracle.select_paths(np.ones(2), 0.5, 4, 5)
    assert paths[1].tolist() == [2, 1] and paths[2].tolist() == [1, 2]
    assert score[1] == score[2]


@pytest.mark.parametrize("nt,M,n_pe", [(16, 64, 256), (8, 16, 64), (16, 64, 1024)])
def test_structural_invariants(nt, M, n_pe):
    rng = np.random.default_rng(nt * M)
    rdiag = np.sqrt(rng.exponential(1.0, nt) * 4)
    paths, score, _ = oracle.select_paths(rdiag, 0.05, M, n_pe)
    rows = [tuple(r) for r in paths]
    assert len(set(rows)) == n_pe
    assert rows[0] == (1,) * nt
    assert np.all(np.diff(score) <= 0)
    pos = {r: i for i, r in enumerate(rows)}
    for i, r in enumerate(rows):  # downward closed, parents listed first
        for l in range(nt):
            if r[l] > 1:
                par = list(r)
                par[l] -= 1
                assert pos[tuple(par)] < i
    assert paths.min() >= 1 and paths.max() <= M


@pytest.mark.parametrize("M", [4, 16, 64])
@pytest.mark.parametrize("snr_db", [4.0, 10.0, 16.0])
def test_level_error_model_matches_monte_carlo_slicing(M, snr_db):
    # Pe_l is the SER of nearest-point slicing at SNR gamma = R_ll^2 / sigma2.
    gamma = 10 ** (snr_db / 10)
    if M == 4 and snr_db > 12:
        gamma = 10 ** (8.0 / 10)  # keep the error count measurable
    _, _, pe = oracle.select_paths(np.array([math.sqrt(gamma)]), 1.0, M, 1)
    pts = oracle.constellation(M)
    rng = np.random.default_rng(int(snr_db * 10) + M)
    n = 400_000
    lab = rng.integers(0, M, n)
    x = pts[lab] + (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * math.sqrt(0.5 / gamma)
    dec = np.argmin(np.abs(x[:, None] - pts[None, :]), axis=1)
    ser = np.mean(dec != lab)
    tol = 5 * math.sqrt(pe[0] * (1 - pe[0]) / n) + 1e-5
    assert abs(ser - pe[0]) < tol, (ser, pe[0])


def test_rejects_impossible_sizes():
    with pytest.raises(RuntimeError):
        oracle.select_paths(np.ones(2), 1.0, 4, 17)  # only 16 vectors exist
