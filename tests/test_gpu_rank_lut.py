"""Table-driven rank model on the GPU (mpnl_rank_counts, mpnl_rank_costs,
mpnl_select_paths_lut) against the oracle: the Monte-Carlo histogram from
the same counter-based draws, the cost rule, and the selection under a cost
table -- exact where the oracle's scores are unique at float32."""
import numpy as np
import pytest

import oracle
from paper_2409_14355_gb300 import inputs
from tests import _parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    from paper_2409_14355_gb300 import mpnl

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    mpnl.load_library()
    d = torch.device("cuda", 0)
    torch.cuda.set_device(d)
    return d


def _mpnl():
    from paper_2409_14355_gb300 import mpnl
    return mpnl


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_rank_counts_match_oracle_draw_for_draw(dev, qam):
    mpnl = _mpnl()
    gamma = np.array([0.7, 4.0, 25.0, 300.0])
    n = 60_000
    seed = 0xC0FFEE + qam
    g = mpnl.rank_counts(qam, torch.tensor(gamma, dtype=torch.float64, device=dev), n, seed)
    torch.cuda.synchronize()
    G = g.cpu().numpy()
    O = oracle.rank_counts_mc(qam, gamma, n, seed)
    assert np.all(G.sum(axis=1) == n)
    # the same SplitMix64 draws on both sides; only a rank decided within the
    # last bits of a double (libm vs CUDA log/sincos) could differ
    assert np.max(np.abs(G - O)) <= 2, np.max(np.abs(G - O))


def test_rank_costs_follow_the_rule(dev):
    mpnl = _mpnl()
    rng = np.random.default_rng(4)
    counts = rng.integers(0, 5000, size=(7, 16)).astype(np.int64)
    counts[:, 0] += 20_000
    counts[2, 5:] = 0            # ranks never seen
    counts[3, 1] = counts[3, 0]  # a flat step
    counts[4, 0] = 0             # rank 1 never seen
    n = 100_000
    c = mpnl.rank_costs(torch.from_numpy(counts).to(dev), n)
    torch.cuda.synchronize()
    want = oracle.rank_costs(counts, n)
    np.testing.assert_allclose(c.cpu().numpy(), want.astype(np.float32), rtol=2e-7, atol=1e-7)
    got = c.cpu().numpy()
    assert np.all(got[:, 0] == 0) and np.all(np.diff(got, axis=1) >= 0)


def _scores_lut(paths, bins, cost):
    return -np.sum([cost[bins[l]][paths[:, l] - 1].astype(np.float64)
                    for l in range(paths.shape[1])], axis=0)


@pytest.mark.parametrize("nt,qam,n_pe,snr_db", [
    (4, 4, 16, 10.0), (8, 16, 64, 16.0), (16, 64, 256, 21.0), (16, 64, 64, 30.0),
    (3, 16, 37, 12.0), (16, 64, 1, 15.0),
])
def test_select_paths_lut_matches_oracle(dev, nt, qam, n_pe, snr_db):
    mpnl = _mpnl()
    # a coarse table (few trials: its values only need to be a valid table)
    lut = mpnl.RankLut.build(qam, db_min=-5.0, db_max=45.0, db_step=1.0, n_trials=20_000,
                             seed=99, device=dev)
    edges = lut.edges.cpu().numpy()
    cost = lut.cost.cpu().numpy()
    n_sc = 25
    sl = inputs.make_slot(nt, nt, qam, n_sc, 1, snr_db, "iid", 0.3, 11 + nt * qam + n_pe)
    Rr, _, _, _ = P.oracle_front(sl.H.astype(np.complex128), sl.Y.astype(np.complex128))
    R32 = Rr.astype(np.complex64)
    Rp = torch.from_numpy(np.ascontiguousarray(P.pack_upper(R32))).to(dev)
    paths = mpnl.select_paths_lut(Rp, sl.sigma2, lut,
                                  n_pe, nt)
    torch.cuda.synchronize()
    G = paths.cpu().numpy()
    delta_abs = 1e-4
    n_checked = 0
    for c in range(n_sc):
        rdiag = np.real(np.diag(R32[c])).astype(np.float64)
        n_more = n_pe + 1 if n_pe + 1 <= min(qam ** nt, 1024) else n_pe
        O, so, bins = oracle.select_paths_lut(rdiag, sl.sigma2, qam, n_more, edges, cost)
        g = G[c]
        assert g[0].tolist() == [1] * nt
        assert len({tuple(r) for r in g}) == n_pe
        assert g.min() >= 1 and g.max() <= qam
        sg = _scores_lut(g, bins, cost)
        delta = delta_abs + 1e-5 * np.abs(sg)
        assert np.all(sg >= so[n_pe - 1] - delta), c
        assert np.all(np.diff(sg) <= delta[1:]), c
        if n_more > n_pe and so[n_pe - 1] - so[n_pe] > 2 * (delta_abs + 1e-5 * abs(so[n_pe])):
            assert {tuple(r) for r in g} == {tuple(r) for r in O[:n_pe]}, c
        for i in range(n_pe):
            lo = so[i - 1] - so[i] if i > 0 else np.inf
            hi = so[i] - so[i + 1] if i + 1 < len(so) else np.inf
            if min(lo, hi) > 2 * (delta_abs + 1e-5 * abs(so[i])):
                assert g[i].tolist() == O[i].tolist(), (c, i)
                n_checked += 1
    assert n_checked > 0


def test_select_paths_lut_rejects_bad_tables(dev):
    mpnl = _mpnl()
    lut = mpnl.RankLut.build(16, db_min=0.0, db_max=10.0, db_step=5.0, n_trials=1000, device=dev)
    R = torch.zeros((3, 6), dtype=torch.complex64, device=dev)
    R[:, 0] = 1.0
    R[:, 3] = 1.0
    R[:, 5] = 1.0
    # a table for 64QAM passed with 16QAM dims: refused by the ABI
    import ctypes
    ctx = mpnl.context(dev.index)
    c = mpnl.RankLutC(64, lut.n_bins, lut.edges.data_ptr(), lut.cost.data_ptr())
    d = mpnl.Dims(3, 1, 3, 3, 16, 8)
    out = torch.empty((3, 8, 3), dtype=torch.uint8, device=dev)
    st = mpnl.load_library().mpnl_select_paths_lut(ctx, ctypes.byref(d), R.data_ptr(), 0.1,
                                                   ctypes.byref(c), out.data_ptr(), None, None)
    assert st != 0
    with pytest.raises(ValueError):
        mpnl.RankLut(16, lut.edges[:1], lut.cost)
    with pytest.raises(mpnl.MpnlError):
        mpnl.rank_counts(16, torch.ones(2, dtype=torch.float64, device=dev), 0, 1)
    p = mpnl.select_paths_lut(R, 0.1, lut, 8, 3)
    torch.cuda.synchronize()
    assert p.shape == (3, 8, 3) and p[:, 0].eq(1).all()


def _exact_fixed_point_top(bins, cost, nt, qam, n_pe):
    """The N_pe vectors of smallest fixed-point cost (each level's term the
    float32 table value, capped at 2^20, in units of 2^-32, rounded to the
    nearest unit; integer sums), ties lexicographically smaller from level
    nt-1 down: level by level, all candidates sorted, exact truncation."""
    def q(m, j):
        v = float(min(np.float32(cost[bins[m], j]), np.float32(2.0 ** 20))) * 2.0 ** 32
        return int(np.rint(v))
    cur = [(q(nt - 1, j), (j,)) for j in range(min(qam, n_pe))]
    cur.sort()
    for m in range(nt - 2, -1, -1):
        qs = [q(m, j) for j in range(qam)]
        cur = sorted((v + qs[j], k + (j,)) for v, k in cur for j in range(qam))[:n_pe]
    return np.array([[k[nt - 1 - l] + 1 for l in range(nt)] for _, k in cur], np.uint8)


@pytest.mark.parametrize("nt,qam,n_pe,n_sc,scale", [
    (16, 64, 256, 8, 1.0), (8, 16, 100, 12, 1.0), (4, 4, 64, 12, 1.0), (16, 64, 1024, 3, 1.0),
    (5, 64, 300, 8, 1.0), (3, 16, 200, 8, 3.0e5),
])
def test_select_paths_lut_exact_under_near_ties(dev, nt, qam, n_pe, n_sc, scale):
    """Tables built to make near-ties: rows a few float32 ulps apart, a flat
    step, equal rows.  In float, adding a shift cost can round two list costs
    a ulp apart to one value and swap them under the tie rule; the selection
    ranks by fixed-point terms instead, and must equal the exact top-N_pe of
    that order row for row.  With scale 3e5 the costs run past the 2^20 cap
    (capped terms tie and fall back to the key order)."""
    mpnl = _mpnl()
    rng = np.random.default_rng(1000 + nt * qam + n_pe)
    n_bins = 6
    base = (np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.9, qam - 1))])
            * scale).astype(np.float32)
    cost = np.empty((n_bins, qam), np.float32)
    for b in range(n_bins):
        row = base.copy()
        row[1:] = np.nextafter(row[1:], np.float32(np.inf)) if b % 2 else row[1:]
        if b >= 2:
            row[1:] = row[1:] * np.float32(1.0 + 1e-7 * b)
        if b == 4:
            row[3] = row[2]           # a flat step
        if b == 5:
            row = cost[0].copy()      # a row equal to another
        cost[b] = np.maximum.accumulate(row)
        cost[b, 0] = 0.0
    edges = np.arange(1, n_bins, dtype=np.float32)          # bin b: gamma in [b, b + 1)
    lut = mpnl.RankLut(qam, torch.from_numpy(edges).to(dev), torch.from_numpy(cost).to(dev))
    P_ = nt * (nt + 1) // 2
    bins = rng.integers(0, n_bins, size=(n_sc, nt))
    gamma = bins + 0.5
    R = np.zeros((n_sc, P_), np.complex64)
    for l in range(nt):
        R[:, l * nt - l * (l - 1) // 2] = np.sqrt(gamma[:, l]).astype(np.float32)
    paths = mpnl.select_paths_lut(torch.from_numpy(R).to(dev), 1.0, lut, n_pe, nt)
    torch.cuda.synchronize()
    G = paths.cpu().numpy()
    for c in range(n_sc):
        # the bin the kernel sees: gamma from the float32 diagonal
        rll = R[c, [l * nt - l * (l - 1) // 2 for l in range(nt)]].real.astype(np.float32)
        b_dev = np.array([int(np.sum((rll[l] * rll[l]) / np.float32(1.0) >= edges))
                          for l in range(nt)])
        assert np.array_equal(b_dev, bins[c])
        want = _exact_fixed_point_top(b_dev, cost, nt, qam, n_pe)
        assert np.array_equal(G[c], want), (c, np.nonzero(np.any(G[c] != want, axis=1))[0][:5])
