"""Pins of the oracle's table-driven rank model: the Monte-Carlo rank
histogram against the closed-form rank probabilities of QPSK and 16QAM,
selection under a cost table against brute force over all M^Nt vectors, and
against the geometric model on a table built from the geometric costs."""
import math

import numpy as np
import pytest

import oracle
from tests._ref_helpers import qfunc


def _binomial_ok(count, n, p, sig=5.0):
    sd = math.sqrt(max(n * p * (1 - p), 1.0))
    return abs(count - n * p) <= sig * sd


@pytest.mark.parametrize("snr_db", [0.0, 5.0, 8.0, 12.0])
def test_qpsk_rank_probabilities_closed_form(snr_db):
    # QPSK (unit energy, points at (+-1, +-1)/sqrt 2): per real axis the noise
    # has variance 1/(2 gamma) and crosses the boundary with probability
    # Q(sqrt gamma).  The sent point ranks first iff neither axis crosses and
    # last (4th) iff both do.
    g = 10 ** (snr_db / 10)
    n = 200_000
    c = oracle.rank_counts_mc(4, [g], n, seed=7)[0]
    assert c.sum() == n
    q = qfunc(math.sqrt(g))
    assert _binomial_ok(c[0], n, (1 - q) ** 2)
    assert _binomial_ok(c[3], n, q * q)
    assert _binomial_ok(c[1] + c[2], n, 2 * q * (1 - q))


@pytest.mark.parametrize("qam,snr_db", [(16, 8.0), (16, 14.0), (16, 20.0), (64, 16.0), (64, 24.0)])
def test_rank_one_is_the_exact_symbol_error_rate(qam, snr_db):
    # square M-QAM: P(correct) = (1 - 2 (1 - 1/sqrt M) Q(sqrt(3 gamma / (M - 1))))^2 (Proakis)
    g = 10 ** (snr_db / 10)
    n = 100_000
    c = oracle.rank_counts_mc(qam, [g], n, seed=11)[0]
    p1 = (1 - 2 * (1 - 1 / math.sqrt(qam)) * qfunc(math.sqrt(3 * g / (qam - 1)))) ** 2
    assert _binomial_ok(c[0], n, p1)


def test_counts_are_reproducible_and_seeded():
    g = [3.0, 30.0]
    a = oracle.rank_counts_mc(64, g, 20_000, seed=5)
    b = oracle.rank_counts_mc(64, g, 20_000, seed=5)
    c = oracle.rank_counts_mc(64, g, 20_000, seed=6)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    assert np.all(a.sum(axis=1) == 20_000)
    # more SNR, more mass on rank 1
    assert a[1, 0] > a[0, 0]


def test_costs_are_zero_at_rank_one_and_nondecreasing():
    counts = oracle.rank_counts_mc(16, [0.5, 5.0, 50.0], 50_000, seed=3)
    cost = oracle.rank_costs(counts, 50_000)
    assert np.all(cost[:, 0] == 0.0)
    assert np.all(np.diff(cost, axis=1) >= 0.0)
    # where the histogram decreases, exp(-c) is the probability ratio
    p = counts[1] / 50_000
    k = 1
    assert counts[1, 0] > counts[1, k] > 0
    assert math.isclose(math.exp(-cost[1, k]), p[k] / p[0], rel_tol=1e-12)
    # ranks never seen: each half as likely as the one before it (ln 2 more)
    assert np.all(np.isfinite(cost))
    c = np.zeros((1, 16), np.int64)
    c[0, :4] = [9000, 700, 250, 50]
    cc = oracle.rank_costs(c, 10_000)[0]
    np.testing.assert_allclose(np.diff(cc[3:]), math.log(2.0), rtol=1e-12)
    assert math.isclose(cc[3], math.log(9000 / 50), rel_tol=1e-12)
    # rank 1 never seen: half a trial
    c0 = np.array([[0, 3, 1, 0]], np.int64)
    assert math.isclose(oracle.rank_costs(c0, 100)[0, 1], max(0.0, math.log(0.5 / 3)), abs_tol=1e-12)


def _bins(rdiag, sigma2, edges):
    r = np.asarray(rdiag, np.float32)
    g = (r * r) / np.float32(sigma2)
    return np.array([int(np.sum(gl >= np.asarray(edges, np.float32))) for gl in g])


def _bruteforce_lut(rdiag, sigma2, M, n_pe, edges, cost):
    nt = len(rdiag)
    b = _bins(rdiag, sigma2, edges)
    vecs = np.array(np.meshgrid(*[np.arange(1, M + 1)] * nt, indexing="ij")).reshape(nt, -1).T
    scores = np.zeros(len(vecs))
    for l in range(nt):
        scores = scores - cost[b[l]][vecs[:, l] - 1].astype(np.float64)
    keys = [vecs[:, l] for l in range(nt)] + [-scores]
    order = np.lexsort(keys)
    return vecs[order[:n_pe]].astype(np.uint8), scores[order[:n_pe]], b


@pytest.mark.parametrize("nt,M,n_pe,seed", [(4, 4, 16, 1), (4, 4, 200, 2), (2, 16, 60, 3),
                                            (3, 16, 120, 4), (1, 64, 40, 5)])
def test_lut_selection_matches_bruteforce(nt, M, n_pe, seed):
    rng = np.random.default_rng(seed)
    n_bins = 6
    edges = np.sort(rng.uniform(0.2, 20.0, n_bins - 1)).astype(np.float32)
    for _ in range(4):
        # random nondecreasing costs with c(1) = 0 (continuous: no exact ties)
        inc = rng.exponential(1.0, (n_bins, M))
        inc[:, 0] = 0.0
        cost = np.cumsum(inc, axis=1).astype(np.float32)
        rdiag = np.sqrt(rng.exponential(1.0, nt) * 3 + 0.05)
        sigma2 = float(rng.choice([0.1, 0.4, 1.0]))
        paths, score, bins = oracle.select_paths_lut(rdiag, sigma2, M, n_pe, edges, cost)
        want, wscore, wb = _bruteforce_lut(rdiag, sigma2, M, n_pe, edges, cost)
        np.testing.assert_array_equal(bins, wb)
        np.testing.assert_array_equal(paths, want)
        np.testing.assert_allclose(score, wscore, rtol=1e-12)


@pytest.mark.parametrize("nt,M,n_pe", [(8, 16, 64), (16, 64, 256)])
def test_geometric_costs_in_a_table_reproduce_the_geometric_model(nt, M, n_pe):
    # one bin per level (edges between the levels' SNRs), costs (k - 1) w_l
    # with w_l = -log Pe_l: the table-driven order is the geometric one
    rng = np.random.default_rng(nt + M)
    rdiag = np.sort(np.sqrt(rng.exponential(1.0, nt) * 4 + 0.1))
    sigma2 = 0.05
    paths_g, score_g, pe = oracle.select_paths(rdiag, sigma2, M, n_pe)
    g = (rdiag.astype(np.float32) ** 2 / np.float32(sigma2)).astype(np.float64)
    order = np.argsort(g)
    gs = g[order]
    assert np.all(np.diff(gs) > 1e-3 * gs[1:])
    edges = np.sqrt(gs[:-1] * gs[1:]).astype(np.float32)
    cost = np.zeros((nt, M), np.float32)
    for b, l in enumerate(order):
        cost[b] = (np.arange(M) * -math.log(pe[l])).astype(np.float32)
    paths_t, score_t, bins = oracle.select_paths_lut(rdiag, sigma2, M, n_pe, edges, cost)
    np.testing.assert_array_equal(np.asarray(bins)[order], np.arange(nt))
    # identical wherever the geometric scores are not within float32 rounding
    # of a neighbour (the table holds float32 costs)
    sep = np.abs(np.diff(score_g)) > 1e-5 * np.abs(score_g[1:]) + 1e-6
    ok = np.concatenate([[True], sep]) & np.concatenate([sep, [True]])
    assert ok.mean() > 0.8
    np.testing.assert_array_equal(paths_t[ok], paths_g[ok])


def test_unseen_rank_tail_recovers_a_halving_law_truncated_by_sampling():
    # A source whose rank probabilities halve from rank to rank (P(k) =
    # 2^-k, renormalised over 16 ranks) sampled with few trials: the deep
    # ranks are never seen.  The true costs are c(k) = (k - 1) ln 2 at every
    # rank; the histogram gives them (up to sampling noise) where it saw
    # ranks, and the tail rule must give them where it did not -- checked
    # against the law itself, not against the rule's own formula.  Counts
    # drawn from the law by the inverse-CDF of a seeded generator.
    rng = np.random.default_rng(17)
    M, trials = 16, 4000
    p = 0.5 ** np.arange(1, M + 1)
    p /= p.sum()
    draws = rng.choice(M, size=trials, p=p)
    counts = np.bincount(draws, minlength=M).astype(np.int64)[None, :]
    seen = int(np.max(np.nonzero(counts[0])[0])) + 1
    assert seen < M - 2                      # the tail really is unseen
    cost = oracle.rank_costs(counts, trials)[0]
    true = np.arange(M) * math.log(2.0)
    # seen ranks: within the sampling error of the true cost (rank counts of a
    # few hundred: a few tenths in log)
    first = [k for k in range(seen) if counts[0, k] >= 30]
    np.testing.assert_allclose(cost[first], true[first], atol=0.35)
    # unseen ranks: the law's step, exactly, from the last seen rank on
    np.testing.assert_allclose(np.diff(cost[seen - 1:]), np.diff(true[seen - 1:]), rtol=1e-12)
    # and the extrapolated costs stay within the sampling error of the truth
    assert np.all(np.abs(cost[seen:] - true[seen:]) <= 1.5)
