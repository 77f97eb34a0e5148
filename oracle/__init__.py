"""FP64 CPU oracle of the MPNL detection path (ctypes front end).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_2409_14355_gb300``) never imports it and
shares no code with it.

The arithmetic lives in ``mpnl_oracle.c`` (plain C, double precision), which
cites the paper section or the stated reading for every step.  This module
only compiles it with gcc and marshals numpy arrays.

Parity pins (checked by ``tests/test_oracle_*.py`` against things other than
the oracle itself): exhaustive ML on 4x4 QPSK, N_pe = 1 == sorted-QR SIC,
N_pe = M^Nt == ML, QR and path-table invariants, brute-force top-N selection,
noise-free recovery, MMSE vs a direct linear solve, closed-form SISO LLRs,
the closed-form MRC bit-error rate, and for the table-driven rank model the
closed-form rank probabilities of QPSK and 16QAM, brute-force top-N selection
and agreement with the geometric model on a table built from it.  Parity unpinned: how well the selection
heuristic (the per-level error model) matches the paper's own MPNL BER; the
paper prints no numbers for it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpnl_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc_mpnl.so")
_lock = threading.Lock()
_lib = None

LLR_MAX = 20.0
PE_FLOOR = 1e-12
BITS = {4: 2, 16: 4, 64: 6}


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (FMA contraction off)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.orc_constellation.argtypes = [I, P]
            lib.orc_sqrd.argtypes = [I, I, P, P, P, P, P]
            lib.orc_sqrd_mmse.argtypes = [I, I, P, D, P, P, P, P]
            lib.orc_qhy.argtypes = [I, I, I, P, P, P]
            lib.orc_select_paths.argtypes = [I, I, P, D, I, P, P, P]
            lib.orc_detect.argtypes = [I, I, I, P, P, P, I, P, D, P, P, P, P, P, P, D, P]
            lib.orc_mmse.argtypes = [I, I, I, I, P, P, D, P, P, P, P]
            lib.orc_detect_slot.argtypes = [I, I, I, I, I, I, D, P, P, P, P, P, P, P, P, P,
                                            P, P, P, P, P, I, D, P, I]
            LL = ctypes.c_longlong
            lib.orc_rank_counts_mc.argtypes = [I, I, P, LL, ctypes.c_ulonglong, P]
            lib.orc_rank_costs.argtypes = [I, I, P, LL, P]
            lib.orc_select_paths_lut.argtypes = [I, I, P, D, I, P, P, I, P, P, P]
            lib.orc_pam_points.argtypes = [I, P]
            lib.orc_select_paths_pam.argtypes = [I, I, P, D, I, P, P, P]
            lib.orc_detect_pam.argtypes = [I, I, I, P, P, P, I, P, D, P, P, P, P, D, P]
            for f in ("orc_constellation", "orc_sqrd", "orc_sqrd_mmse", "orc_qhy", "orc_select_paths",
                      "orc_detect", "orc_mmse", "orc_detect_slot", "orc_rank_counts_mc",
                      "orc_rank_costs", "orc_select_paths_lut", "orc_pam_points",
                      "orc_select_paths_pam", "orc_detect_pam"):
                getattr(lib, f).restype = I
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _check(st, what):
    if st < 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")
    return st


def constellation(qam: int) -> np.ndarray:
    """Label-indexed unit-energy Gray constellation (TS 38.211 §5.1), complex128[M]."""
    out = np.zeros(qam, np.complex128)
    _check(_load().orc_constellation(qam, _p(out)), "constellation")
    return out


def sqrd(H):
    """Sorted QR of one channel H[nr][nt] -> (Q, R, perm, gap)."""
    H = _c128(H)
    nr, nt = H.shape
    Q = np.zeros((nr, nt), np.complex128)
    R = np.zeros((nt, nt), np.complex128)
    perm = np.zeros(nt, np.int32)
    gap = np.zeros(nt, np.float64)
    _check(_load().orc_sqrd(nr, nt, _p(H), _p(Q), _p(R), _p(perm), _p(gap)), "sqrd")
    return Q, R, perm, gap


def sqrd_mmse(H, sigma2: float):
    """MMSE-extended sorted QR of [H; sigma I] -> (Q_a [(nr+nt)][nt], R, perm, gap).
    z = Q_a^H [y; 0] = qhy(Q_a, [Y | 0])."""
    H = _c128(H)
    nr, nt = H.shape
    Q = np.zeros((nr + nt, nt), np.complex128)
    R = np.zeros((nt, nt), np.complex128)
    perm = np.zeros(nt, np.int32)
    gap = np.zeros(nt, np.float64)
    _check(_load().orc_sqrd_mmse(nr, nt, _p(H), float(sigma2), _p(Q), _p(R), _p(perm), _p(gap)),
           "sqrd_mmse")
    return Q, R, perm, gap


def qhy(Q, Y):
    """z = Q^H y for Y[n_sym][nr] -> Z[n_sym][nt]."""
    Q = _c128(Q)
    Y = _c128(Y)
    nr, nt = Q.shape
    n_sym = Y.shape[0]
    Z = np.zeros((n_sym, nt), np.complex128)
    _check(_load().orc_qhy(nr, nt, n_sym, _p(Q), _p(Y), _p(Z)), "qhy")
    return Z


def select_paths(rdiag, sigma2: float, qam: int, n_pe: int):
    """Best-first position-vector table -> (paths uint8[n_pe][nt], score[n_pe], pe[nt])."""
    rdiag = np.ascontiguousarray(np.asarray(rdiag, np.float64))
    nt = rdiag.shape[0]
    paths = np.zeros((n_pe, nt), np.uint8)
    score = np.zeros(n_pe, np.float64)
    pe = np.zeros(nt, np.float64)
    _check(_load().orc_select_paths(nt, qam, _p(rdiag), float(sigma2), n_pe, _p(paths),
                                    _p(score), _p(pe)), "select_paths")
    return paths, score, pe


def rank_counts_mc(qam: int, gamma, n_trials: int, seed: int) -> np.ndarray:
    """Monte-Carlo rank histogram per SNR (linear) -> int64[n_bins][qam]:
    counts[b][k-1] = trials whose transmitted point ranked k-th."""
    gamma = np.ascontiguousarray(np.asarray(gamma, np.float64))
    counts = np.zeros((gamma.shape[0], qam), np.int64)
    _check(_load().orc_rank_counts_mc(qam, gamma.shape[0], _p(gamma), int(n_trials),
                                      ctypes.c_ulonglong(seed), _p(counts)), "rank_counts_mc")
    return counts


def rank_costs(counts, n_trials: int) -> np.ndarray:
    """Rank costs c(k) = log P(1) - log P(k) (floored, nondecreasing) -> float64[n_bins][qam]."""
    counts = np.ascontiguousarray(np.asarray(counts, np.int64))
    n_bins, qam = counts.shape
    cost = np.zeros((n_bins, qam), np.float64)
    _check(_load().orc_rank_costs(qam, n_bins, _p(counts), int(n_trials), _p(cost)), "rank_costs")
    return cost


def select_paths_lut(rdiag, sigma2: float, qam: int, n_pe: int, edges, cost):
    """Best-first table under the table-driven rank model: per level the bin
    of gamma = R_ll^2 / sigma2 (float32) among the ascending `edges`, costs
    from `cost` (float32 [n_bins][qam]) -> (paths, score, bins)."""
    rdiag = np.ascontiguousarray(np.asarray(rdiag, np.float64))
    edges = np.ascontiguousarray(np.asarray(edges, np.float32))
    cost = np.ascontiguousarray(np.asarray(cost, np.float32))
    nt = rdiag.shape[0]
    n_bins = cost.shape[0]
    assert edges.shape[0] == n_bins - 1 and cost.shape[1] == qam
    paths = np.zeros((n_pe, nt), np.uint8)
    score = np.zeros(n_pe, np.float64)
    bins = np.zeros(nt, np.int32)
    _check(_load().orc_select_paths_lut(nt, qam, _p(rdiag), float(sigma2), n_bins, _p(edges),
                                        _p(cost), n_pe, _p(paths), _p(score), _p(bins)),
           "select_paths_lut")
    return paths, score, bins


def detect(R, Z, perm, paths, sigma2: float, qam: int, want_all: bool = False,
           tie_eps: float = 0.0):
    """Walks + argmin + LLRs for one subcarrier.

    Returns dict(hard, llr, ped2, margin, flip_floor[, ped_all, sym_all]);
    flip_floor is the smallest partial PED at a ranking whose neighbour gap
    is below tie_eps (+inf if none).
    """
    R = _c128(R)
    Z = _c128(Z)
    perm = np.ascontiguousarray(np.asarray(perm, np.int32))
    paths = np.ascontiguousarray(np.asarray(paths, np.uint8))
    nt = R.shape[0]
    n_sym = Z.shape[0]
    n_pe = paths.shape[0]
    B = BITS[qam]
    hard = np.zeros((n_sym, nt), np.uint8)
    llr = np.zeros((n_sym, nt, B), np.float64)
    ped2 = np.zeros((n_sym, 2), np.float64)
    margin = np.zeros(n_sym, np.float64)
    ped_all = np.zeros((n_sym, n_pe), np.float64) if want_all else None
    sym_all = np.zeros((n_sym, n_pe, nt), np.uint8) if want_all else None
    flip = np.zeros(n_sym, np.float64)
    _check(_load().orc_detect(nt, qam, n_sym, _p(R), _p(Z), _p(perm), n_pe, _p(paths),
                              float(sigma2), _p(hard), _p(llr), _p(ped2), _p(margin),
                              _p(ped_all), _p(sym_all), float(tie_eps), _p(flip)), "detect")
    out = dict(hard=hard, llr=llr, ped2=ped2, margin=margin, flip_floor=flip)
    if want_all:
        out["ped_all"] = ped_all
        out["sym_all"] = sym_all
    return out


def mmse(H, Y, sigma2: float, qam: int):
    """Linear MMSE for one subcarrier -> dict(hard, llr, xt, nu)."""
    H = _c128(H)
    Y = _c128(Y)
    nr, nt = H.shape
    n_sym = Y.shape[0]
    B = BITS[qam]
    hard = np.zeros((n_sym, nt), np.uint8)
    llr = np.zeros((n_sym, nt, B), np.float64)
    xt = np.zeros((n_sym, nt), np.complex128)
    nu = np.zeros(nt, np.float64)
    _check(_load().orc_mmse(nr, nt, qam, n_sym, _p(H), _p(Y), float(sigma2), _p(hard),
                            _p(llr), _p(xt), _p(nu)), "mmse")
    return dict(hard=hard, llr=llr, xt=xt, nu=nu)


def detect_slot(H, Y, sigma2: float, qam: int, n_pe: int, paths=None, n_threads: int = 0,
                with_mmse: bool = False, tie_eps: float = 0.0, mmse_qr: bool = False):
    """Steps 1-6 (and 7 with ``with_mmse``) over a whole slot.

    H: [n_sc][nr][nt], Y: [n_sc][n_sym][nr] (any complex dtype; promoted to
    complex128).  Returns a dict of numpy arrays plus ``threads`` (the number
    of host threads the oracle used).
    """
    H = _c128(H)
    Y = _c128(Y)
    n_sc, nr, nt = H.shape
    n_sym = Y.shape[1]
    B = BITS[qam]
    hard = np.zeros((n_sc, n_sym, nt), np.uint8)
    llr = np.zeros((n_sc, n_sym, nt, B), np.float64)
    ped2 = np.zeros((n_sc, n_sym, 2), np.float64)
    R = np.zeros((n_sc, nt, nt), np.complex128)
    perm = np.zeros((n_sc, nt), np.int32)
    Z = np.zeros((n_sc, n_sym, nt), np.complex128)
    paths_out = np.zeros((n_sc, n_pe, nt), np.uint8)
    gap = np.zeros((n_sc, nt), np.float64)
    margin = np.zeros((n_sc, n_sym), np.float64)
    mh = np.zeros((n_sc, n_sym, nt), np.uint8) if with_mmse else None
    ml = np.zeros((n_sc, n_sym, nt, B), np.float64) if with_mmse else None
    pin = None if paths is None else np.ascontiguousarray(np.asarray(paths, np.uint8))
    flip = np.zeros((n_sc, n_sym), np.float64)
    st = _load().orc_detect_slot(n_sc, n_sym, nr, nt, qam, n_pe, float(sigma2), _p(H), _p(Y),
                                 _p(pin), _p(hard), _p(llr), _p(ped2), _p(R), _p(perm), _p(Z),
                                 _p(paths_out), _p(gap), _p(margin), _p(mh), _p(ml),
                                 int(n_threads), float(tie_eps), _p(flip), int(mmse_qr))
    _check(st, "detect_slot")
    out = dict(hard=hard, llr=llr, ped2=ped2, R=R, perm=perm, Z=Z, paths=paths_out,
               sqrd_gap=gap, margin=margin, flip_floor=flip, threads=st)
    if with_mmse:
        out["mmse_hard"] = mh
        out["mmse_llr"] = ml
    return out


# ---------------------------------------------------------------------------
# Real-valued decomposition (RVD) variant: 2 nt real levels, L-PAM each
# ---------------------------------------------------------------------------
def rvd_embed(H, Y):
    """[Re y; Im y] = [[Re H, -Im H]; [Im H, Re H]] [Re s; Im s]: H [..][nr][nt]
    -> [..][2nr][2nt], Y [..][n_sym][nr] -> [..][n_sym][2nr], as complex128
    with zero imaginary parts (so the complex routines run on them)."""
    H = _c128(H)
    Y = _c128(Y)
    top = np.concatenate([H.real, -H.imag], axis=-1)
    bot = np.concatenate([H.imag, H.real], axis=-1)
    Hr = np.concatenate([top, bot], axis=-2).astype(np.complex128)
    Yr = np.concatenate([Y.real, Y.imag], axis=-1).astype(np.complex128)
    return Hr, Yr


def pam_points(qam: int) -> np.ndarray:
    """Axis positions of the L-PAM of a square QAM, indexed by axis label."""
    L = 1 << (BITS[qam] // 2)
    out = np.zeros(L, np.float64)
    _check(_load().orc_pam_points(qam, _p(out)), "pam_points")
    return out


def select_paths_pam(rdiag, sigma2: float, qam: int, n_pe: int):
    """Best-first table over 2 nt real levels (ranks 1..L) -> (paths, score, pe)."""
    rdiag = np.ascontiguousarray(np.asarray(rdiag, np.float64))
    ntr = rdiag.shape[0]
    paths = np.zeros((n_pe, ntr), np.uint8)
    score = np.zeros(n_pe, np.float64)
    pe = np.zeros(ntr, np.float64)
    _check(_load().orc_select_paths_pam(ntr, qam, _p(rdiag), float(sigma2), n_pe, _p(paths),
                                        _p(score), _p(pe)), "select_paths_pam")
    return paths, score, pe


def join_axes(hard_r, llr_r, qam: int):
    """Per-column axis labels / LLRs of the real levels ([..][2nt], [..][2nt][B/2])
    -> user labels [..][nt] and LLRs [..][nt][B]: bits b0 b2 .. of user u from
    column u, b1 b3 .. from column nt + u (TS 38.211 §5.1)."""
    B = BITS[qam]
    H = B // 2
    nt = hard_r.shape[-1] // 2
    re, im = hard_r[..., :nt].astype(np.int64), hard_r[..., nt:].astype(np.int64)
    lab = np.zeros(re.shape, np.int64)
    for t in range(H):
        lab |= ((re >> (H - 1 - t)) & 1) << (B - 1 - 2 * t)
        lab |= ((im >> (H - 1 - t)) & 1) << (B - 2 - 2 * t)
    llr = np.zeros(hard_r.shape[:-1] + (nt, B), np.float64)
    llr[..., 0::2] = llr_r[..., :nt, :]
    llr[..., 1::2] = llr_r[..., nt:, :]
    return lab.astype(np.uint8), llr


def detect_rvd(R, Z, perm, paths, sigma2: float, qam: int, tie_eps: float = 0.0):
    """Walks over the 2 nt real levels of one subcarrier (R real upper
    [2nt][2nt], Z [n_sym][2nt], perm, paths [n_pe][2nt] with ranks 1..L)."""
    R = _c128(R)
    Z = _c128(Z)
    perm = np.ascontiguousarray(np.asarray(perm, np.int32))
    paths = np.ascontiguousarray(np.asarray(paths, np.uint8))
    ntr = R.shape[0]
    n_sym = Z.shape[0]
    Bh = BITS[qam] // 2
    hard_r = np.zeros((n_sym, ntr), np.uint8)
    llr_r = np.zeros((n_sym, ntr, Bh), np.float64)
    ped2 = np.zeros((n_sym, 2), np.float64)
    margin = np.zeros(n_sym, np.float64)
    flip = np.zeros(n_sym, np.float64)
    _check(_load().orc_detect_pam(ntr, qam, n_sym, _p(R), _p(Z), _p(perm), paths.shape[0],
                                  _p(paths), float(sigma2), _p(hard_r), _p(llr_r), _p(ped2),
                                  _p(margin), float(tie_eps), _p(flip)), "detect_pam")
    hard, llr = join_axes(hard_r, llr_r, qam)
    return dict(hard=hard, llr=llr, ped2=ped2, margin=margin, flip_floor=flip, hard_r=hard_r,
                llr_r=llr_r)


def detect_slot_rvd(H, Y, sigma2: float, qam: int, n_pe: int, tie_eps: float = 0.0):
    """The RVD path over a slot, subcarrier by subcarrier: embed, sorted QR of
    the real matrix, z, PAM-level selection, walks, axes joined per user."""
    Hr, Yr = rvd_embed(H, Y)
    n_sc, n_sym = Yr.shape[0], Yr.shape[1]
    ntr = Hr.shape[-1]
    nt = ntr // 2
    B = BITS[qam]
    out = dict(hard=np.zeros((n_sc, n_sym, nt), np.uint8),
               llr=np.zeros((n_sc, n_sym, nt, B)), ped2=np.zeros((n_sc, n_sym, 2)),
               flip_floor=np.zeros((n_sc, n_sym)), R=np.zeros((n_sc, ntr, ntr), np.complex128),
               perm=np.zeros((n_sc, ntr), np.int32), Z=np.zeros((n_sc, n_sym, ntr), np.complex128),
               paths=np.zeros((n_sc, n_pe, ntr), np.uint8))
    for c in range(n_sc):
        Q, R, perm, _ = sqrd(Hr[c])
        Z = qhy(Q, Yr[c])
        paths, _, _ = select_paths_pam(np.real(np.diag(R)), sigma2, qam, n_pe)
        o = detect_rvd(R, Z, perm, paths, sigma2, qam, tie_eps)
        for k in ("hard", "llr", "ped2", "flip_floor"):
            out[k][c] = o[k]
        out["R"][c], out["perm"][c], out["Z"][c], out["paths"][c] = R, perm, Z, paths
    return out
