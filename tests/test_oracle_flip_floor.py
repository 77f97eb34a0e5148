"""Pin of the oracle's near-tie diagnostic `flip_floor`, which decides which
GPU outputs the parity tests hold to bit-exactness.

The claim it carries: a walk whose ranking at some level lies within
tie_eps of a distance tie may, in lower precision, take the neighbouring
point there instead; every walk so perturbed -- at one near-tie or at
several -- still has a PED of at least flip_floor.  If flip_floor were too
high, a detection could be counted as unique at float32 while a perturbed
walk undercuts its best; if it were too low, more detections than needed
would be excluded.  This test enumerates, by brute force on tiny systems,
every walk obtained by swapping near-tied neighbours at any subset of the
near-tie points of a row (lower levels keep their ranks), recomputing each
walk from scratch with numpy, and checks:
  * every perturbed walk's PED is >= flip_floor;
  * flip_floor is attained: some perturbed or unperturbed walk has a partial
    PED through its near-tie level equal to it (so it is not too low);
  * the comparability rule built on it is sound: wherever the tests call a
    decision unique, no perturbed walk reaches the best PED.
"""
import itertools

import numpy as np
import pytest

import oracle
from tests import _parity as P


def _ranked(b, pts):
    """Constellation indices ordered by (distance to b, label)."""
    d = np.abs(b - pts) ** 2
    return sorted(range(len(pts)), key=lambda q: (d[q], q)), d


def _walk(R, z, ranks, pts, swaps):
    """The walk of one row with the choice at the levels in `swaps` replaced
    by the given constellation index; returns (PED, per-level partial PEDs
    before each level, per-level (order, dist, chosen position))."""
    nt = R.shape[0]
    s = np.zeros(nt, complex)
    d = 0.0
    info = {}
    for l in range(nt - 1, -1, -1):
        e = z[l] - np.dot(R[l, l + 1:], s[l + 1:])
        rll = R[l, l].real
        order, dist = _ranked(e / rll, pts)
        k = ranks[l] - 1
        q = swaps.get(l, order[k])
        info[l] = (order, dist, k, d)
        s[l] = pts[q]
        d += rll * rll * dist[q]
    return d, info


@pytest.mark.parametrize("nt,qam,n_pe,tie_eps,seed", [
    (3, 16, 24, 0.15, 1), (3, 4, 8, 0.3, 2), (2, 64, 40, 0.08, 3), (4, 16, 16, 0.1, 4),
    (3, 16, 24, 0.02, 5), (4, 4, 16, 0.05, 6),
])
def test_flip_floor_bounds_every_perturbed_walk(nt, qam, n_pe, tie_eps, seed):
    rng = np.random.default_rng(seed)
    pts = oracle.constellation(qam)
    sigma2 = 0.05
    n_sym = 6
    n_det = 0
    n_comp = 0
    n_pert = 0
    for trial in range(8):
        H = (rng.standard_normal((nt, nt)) + 1j * rng.standard_normal((nt, nt))) / np.sqrt(2)
        Q, R, perm, _ = oracle.sqrd(H)
        labels = rng.integers(0, qam, size=(n_sym, nt))
        Y = pts[labels] @ H.T + np.sqrt(sigma2 / 2) * (
            rng.standard_normal((n_sym, nt)) + 1j * rng.standard_normal((n_sym, nt)))
        Z = oracle.qhy(Q, Y)
        paths, _, _ = oracle.select_paths(np.real(np.diag(R)), sigma2, qam, n_pe)
        o = oracle.detect(R, Z, perm, paths, sigma2, qam, tie_eps=tie_eps)
        for s in range(n_sym):
            floor = o["flip_floor"][s]
            best = o["ped2"][s, 0]
            lowest = np.inf          # smallest PED of any perturbed walk
            attained = np.isinf(floor)
            for row in paths:
                d0, info = _walk(R, Z[s], row, pts, {})
                # near-tie points of the unperturbed walk and their neighbours
                ties = []
                for l, (order, dist, k, dpart) in info.items():
                    g_lo = np.sqrt(dist[order[k]]) - np.sqrt(dist[order[k - 1]]) if k > 0 else np.inf
                    g_hi = (np.sqrt(dist[order[k + 1]]) - np.sqrt(dist[order[k]])
                            if k + 1 < qam else np.inf)
                    alts = []
                    if g_lo < tie_eps:
                        alts.append(order[k - 1])
                    if g_hi < tie_eps:
                        alts.append(order[k + 1])
                    if alts:
                        ties.append((l, alts))
                        # the floor candidate at this point: the partial PED
                        # through the level with the nearer of the two points
                        rll2 = R[l, l].real ** 2
                        near = min(dist[order[k]], dist[order[k - 1]] if k > 0 else np.inf)
                        if np.isclose(dpart + rll2 * near, floor, rtol=1e-12, atol=0):
                            attained = True
                # every subset of near-tie points swapped (at most 3 for size)
                for r in range(1, min(3, len(ties)) + 1):
                    for combo in itertools.combinations(ties, r):
                        for pick in itertools.product(*[alts for _, alts in combo]):
                            sw = {l: q for (l, _), q in zip(combo, pick)}
                            d1, _ = _walk(R, Z[s], row, pts, sw)
                            lowest = min(lowest, d1)
                            n_pert += 1
                            assert d1 >= floor * (1 - 1e-12), (trial, s, d1, floor)
            assert attained, (trial, s, floor)
            n_det += 1
            if np.isfinite(lowest):
                # the rule of the parity tests: a decision counted as unique is
                # one no perturbed walk can take over
                ref = {k: o[k][s:s + 1][None] for k in ("ped2", "flip_floor", "llr")}
                if P.comparable(ref, sigma2)["decision"][0, 0]:
                    n_comp += 1
                    assert lowest > best
    assert n_det == 8 * n_sym and n_pert > 0
    print(f"perturbed walks {n_pert}, unique decisions with perturbations {n_comp}")
