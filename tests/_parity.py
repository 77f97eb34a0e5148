"""Helpers for the GPU-vs-oracle parity tests (test code only).

Tolerances (the derivations are in the design notes):
* decisions: bit-exact wherever the oracle's best and runner-up PED differ by
  more than 1e-3 relative and no ranking within TIE_EPS of a distance tie can
  reach the best walk (see ``comparable``);
* PEDs: |d_gpu - d_ref| <= 1e-4 d_ref + 1e-6 sum_l R_ll^2;
* LLRs: |L_gpu - L_ref| <= 1e-4 (2 d_best / sigma2 + |L_ref|) + 1e-6 sum_l R_ll^2 / sigma2
  (an LLR is a difference of two PED minima, d_best and d_best + |L| sigma2,
  so its error is bounded relative to those two terms, not to |L|).
"""
from __future__ import annotations

import numpy as np

import oracle

RTOL = 1e-4
GAP_REL = 1e-3        # runner-up vs best PED, relative (decision clarity)
TIE_EPS = 1e-4        # stage-isolated ranking near-tie width, constellation distance units

# End to end, R and z carry the float32 QR's own error, which grows with the
# channel's condition number: tie width and tolerance are 64 u kappa(H)
# per subcarrier (u = 2^-24), floored at the stage-isolated values.
E2E_KAPPA_FACTOR = 64 * 2.0 ** -24


def e2e_reference(H, Y, sigma2, qam, n_pe, with_mmse=True, mmse_qr=False):
    """Oracle run of a whole slot plus per-subcarrier near-tie floors and
    tolerances for comparing the end-to-end GPU path.  With mmse_qr the
    factorised matrix, and so kappa, is the augmented [H; sigma I]."""
    ref = oracle.detect_slot(H, Y, sigma2, qam, n_pe, with_mmse=with_mmse, mmse_qr=mmse_qr)
    H = np.asarray(H, np.complex128)
    if mmse_qr:
        nt = H.shape[-1]
        aug = np.broadcast_to(np.sqrt(sigma2) * np.eye(nt), (H.shape[0], nt, nt))
        H = np.concatenate([H, aug], axis=1)
    kappa = np.linalg.cond(H)
    eps = np.maximum(TIE_EPS * 0.1, E2E_KAPPA_FACTOR * kappa)
    ff = np.zeros(ref["ped2"].shape[:2])
    for c in range(H.shape[0]):
        o = oracle.detect(ref["R"][c], ref["Z"][c], ref["perm"][c], ref["paths"][c], sigma2, qam,
                          tie_eps=eps[c])
        ff[c] = o["flip_floor"]
    ref["flip_floor"] = ff
    ref["rtol"] = np.maximum(RTOL, E2E_KAPPA_FACTOR * kappa)
    ref["kappa"] = kappa
    return ref


def pack_upper(R: np.ndarray) -> np.ndarray:
    """[..., nt, nt] upper-triangular -> [..., nt(nt+1)/2], row by row."""
    nt = R.shape[-1]
    iu = np.triu_indices(nt)
    return R[..., iu[0], iu[1]]


def unpack_upper(Rp: np.ndarray, nt: int) -> np.ndarray:
    out = np.zeros(Rp.shape[:-1] + (nt, nt), Rp.dtype)
    iu = np.triu_indices(nt)
    out[..., iu[0], iu[1]] = Rp
    return out


def oracle_front(H: np.ndarray, Y: np.ndarray):
    """Oracle sorted QR + z per subcarrier: R [n_sc][nt][nt], perm, Z, gap."""
    n_sc, nr, nt = H.shape
    R = np.zeros((n_sc, nt, nt), np.complex128)
    perm = np.zeros((n_sc, nt), np.int32)
    Z = np.zeros((n_sc, Y.shape[1], nt), np.complex128)
    gap = np.zeros((n_sc, nt))
    for c in range(n_sc):
        Q, R[c], perm[c], gap[c] = oracle.sqrd(H[c])
        Z[c] = oracle.qhy(Q, Y[c])
    return R, perm, Z, gap


def oracle_front_mmse(H: np.ndarray, Y: np.ndarray, sigma2: float):
    """Oracle MMSE-extended sorted QR + z = Q_a^H [y; 0] per subcarrier."""
    n_sc, nr, nt = H.shape
    R = np.zeros((n_sc, nt, nt), np.complex128)
    perm = np.zeros((n_sc, nt), np.int32)
    Z = np.zeros((n_sc, Y.shape[1], nt), np.complex128)
    gap = np.zeros((n_sc, nt))
    for c in range(n_sc):
        Q, R[c], perm[c], gap[c] = oracle.sqrd_mmse(H[c], sigma2)
        Ya = np.concatenate([Y[c], np.zeros((Y.shape[1], nt), np.complex128)], axis=1)
        Z[c] = oracle.qhy(Q, Ya)
    return R, perm, Z, gap


def to_fp32_inputs(R: np.ndarray, Z: np.ndarray):
    """Round the oracle's R and Z to the GPU's input precision and derive the
    float32 1 / R_ll the way a caller would."""
    R32 = R.astype(np.complex64)
    Z32 = Z.astype(np.complex64)
    diag32 = np.real(np.diagonal(R32, axis1=-2, axis2=-1)).astype(np.float32)
    inv32 = (1.0 / diag32.astype(np.float64)).astype(np.float32)
    return R32, Z32, inv32


def oracle_detect_all(R, Z, perm, paths, sigma2, qam, tie_eps=TIE_EPS):
    n_sc, n_sym, nt = Z.shape
    B = oracle.BITS[qam]
    out = dict(hard=np.zeros((n_sc, n_sym, nt), np.uint8), llr=np.zeros((n_sc, n_sym, nt, B)),
               ped2=np.zeros((n_sc, n_sym, 2)), margin=np.zeros((n_sc, n_sym)),
               flip_floor=np.zeros((n_sc, n_sym)))
    for c in range(n_sc):
        o = oracle.detect(R[c], Z[c], perm[c], paths[c], sigma2, qam, tie_eps=tie_eps)
        for k in out:
            out[k][c] = o[k]
    return out


def comparable(ref: dict, sigma2: float):
    """Which outputs are unique at float32 precision.

    A ranking within the tie width may resolve the other way on the GPU; the
    walk that takes it still carries at least the partial PED `flip_floor`.
    So an output that is a minimum below flip_floor cannot be disturbed:
      decision    : runner-up > best by GAP_REL, and flip_floor above the best
      best PED    : flip_floor above it
      runner-up   : flip_floor above it
      LLR (k, b)  : flip_floor above the larger of its two minima
                    (d_best + |L| sigma2); clipped LLRs only with no near-tie
    """
    d1, d2 = ref["ped2"][..., 0], ref["ped2"][..., 1]
    ff = ref["flip_floor"]
    pad = 1.0 + 10 * RTOL
    best = ff > d1 * pad
    dec = best & ((d2 - d1) > GAP_REL * np.maximum(d1, 1e-30))
    run = np.isfinite(d2) & (ff > d2 * pad)
    L = ref["llr"]
    clipped = np.abs(L) == oracle.LLR_MAX
    upper = d1[..., None, None] + np.abs(L) * sigma2
    llr = np.where(clipped, np.isinf(ff)[..., None, None], ff[..., None, None] > upper * pad)
    return dict(decision=dec, best=best, runner=run, llr=llr)


def compare_detect(gpu: dict, ref: dict, R: np.ndarray, sigma2: float, rtol=RTOL,
                   what: str = "", sc_mask=None, min_frac: float = 0.5) -> dict:
    """Assert decisions / PEDs / LLRs wherever they are unique (see comparable).
    rtol is a scalar or one value per subcarrier."""
    rtol = np.broadcast_to(np.asarray(rtol, np.float64), (R.shape[0],))[:, None]
    m = comparable(ref, sigma2)
    if sc_mask is not None:
        m = {k: v & (sc_mask[:, None] if v.ndim == 2 else sc_mask[:, None, None, None])
             for k, v in m.items()}
    rdiag2 = np.sum(np.real(np.diagonal(R, axis1=-2, axis2=-1)) ** 2, axis=-1)  # [n_sc]
    scale = rdiag2[:, None] * np.ones(m["best"].shape)
    n = int(m["decision"].sum())
    frac = n / m["decision"].size
    assert frac >= min_frac, f"{what}: only {frac:.2%} of decisions are unique at float32"
    hard_ok = np.all(gpu["hard"] == ref["hard"], axis=-1)
    bad = np.argwhere(m["decision"] & ~hard_ok)
    assert len(bad) == 0, f"{what}: {len(bad)} decision mismatches of {n}, first at {bad[:5].tolist()}"
    d_ref = ref["ped2"][..., 0]
    d_gpu = gpu["ped2"][..., 0].astype(np.float64)
    tol = rtol * d_ref + 1e-6 * scale
    err = np.abs(d_gpu - d_ref)
    mb = m["best"]
    assert np.all(err[mb] <= tol[mb]), f"{what}: best-PED error {np.max((err / tol)[mb]):.3g} x tol"
    mr = m["runner"]
    if mr.any():
        d2r = ref["ped2"][..., 1]
        err2 = np.abs(gpu["ped2"][..., 1].astype(np.float64) - d2r)
        tol2 = rtol * d2r + 1e-6 * scale
        assert np.all(err2[mr] <= tol2[mr]), \
            f"{what}: runner-up PED error {np.max((err2 / tol2)[mr]):.3g} x tol"
    ml = m["llr"]
    if gpu.get("llr") is not None:
        L = ref["llr"]
        Lg = gpu["llr"].astype(np.float64)
        tolL = rtol[..., None, None] * (2 * d_ref[..., None, None] / sigma2 + np.abs(L)) \
            + 1e-6 * scale[..., None, None] / sigma2
        errL = np.abs(Lg - L)
        assert np.all(errL[ml] <= tolL[ml]), \
            f"{what}: LLR error {np.max((errL / tolL)[ml]):.3g} x tol"
        assert ml.mean() >= min_frac * 0.5, f"{what}: only {ml.mean():.2%} of LLRs unique"
    return dict(decisions=n, total=int(m["decision"].size), llrs=int(ml.sum()))
