"""Pins of the oracle's linear MMSE baseline against a direct linear solve and
the closed-form single-user (SISO) max-log LLRs."""
import math

import numpy as np
import pytest

import oracle
from paper_2409_14355_gb300 import inputs


@pytest.mark.parametrize("nr,nt,qam", [(4, 4, 4), (8, 8, 16), (16, 16, 64), (8, 3, 16)])
def test_equaliser_matches_direct_solve(nr, nt, qam):
    sl = inputs.make_slot(nr, nt, qam, 5, 14, 15.0, "kronecker", 0.3, 21)
    for c in range(sl.n_sc):
        H = sl.H[c].astype(np.complex128)
        Y = sl.Y[c].astype(np.complex128)
        out = oracle.mmse(H, Y, sl.sigma2, qam)
        A = H.conj().T @ H + sl.sigma2 * np.eye(nt)
        W = np.linalg.solve(A, H.conj().T)
        xhat = Y @ W.T
        mu = np.real(np.diag(W @ H))
        np.testing.assert_allclose(out["xt"] * mu[None, :], xhat, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(out["nu"], (1 - mu) / mu, rtol=1e-9)
        pts = oracle.constellation(qam)
        want = np.argmin(np.abs(out["xt"][..., None] - pts), axis=-1)
        np.testing.assert_array_equal(out["hard"], want)


def test_single_user_qpsk_llr_closed_form():
    # Nt = 1: x~ = h^H y / ||h||^2, nu = sigma2 / ||h||^2, and the QPSK max-log
    # LLRs are 2 sqrt(2) Re(x~) / nu and 2 sqrt(2) Im(x~) / nu.
    sl = inputs.make_slot(4, 1, 4, 10, 14, 5.0, "iid", 0.3, 8)
    for c in range(sl.n_sc):
        h = sl.H[c].astype(np.complex128)[:, 0]
        Y = sl.Y[c].astype(np.complex128)
        out = oracle.mmse(h[:, None], Y, sl.sigma2, 4)
        nh2 = np.sum(np.abs(h) ** 2)
        xt = (Y @ h.conj()) / nh2
        nu = sl.sigma2 / nh2
        np.testing.assert_allclose(out["xt"][:, 0], xt, rtol=1e-12)
        np.testing.assert_allclose(out["nu"][0], nu, rtol=1e-10)
        np.testing.assert_allclose(out["llr"][:, 0, 0], 2 * math.sqrt(2) * xt.real / nu, rtol=1e-9)
        np.testing.assert_allclose(out["llr"][:, 0, 1], 2 * math.sqrt(2) * xt.imag / nu, rtol=1e-9)


def test_single_user_16qam_llr_piecewise_closed_form():
    # 16QAM, bit b0 (sign of the real part, points at +-1, +-3 over sqrt 10):
    # the max-log LLR is piecewise linear in t = Re(x~) sqrt(10):
    #   |t| <= 2: 4 t / (10 nu);  |t| > 2: 8 (t - sign(t)) / (10 nu).
    sl = inputs.make_slot(2, 1, 16, 20, 14, 3.0, "iid", 0.3, 9)
    for c in range(sl.n_sc):
        out = oracle.mmse(sl.H[c], sl.Y[c], sl.sigma2, 16)
        t = out["xt"][:, 0].real * math.sqrt(10)
        nu = out["nu"][0]
        want = np.where(np.abs(t) <= 2, 4 * t, 8 * (t - np.sign(t))) / (10 * nu)
        np.testing.assert_allclose(out["llr"][:, 0, 0], want, rtol=1e-9, atol=1e-12)
