"""Pins of the oracle's sorted QR (SQRD) and z = Q^H y."""
import numpy as np
import pytest

import oracle
from paper_2409_14355_gb300 import inputs


def _channels(nr, nt, n, seed, channel="iid"):
    return inputs.make_slot(nr, nt, 4, n, 1, 10.0, channel, 0.3, seed).H.astype(np.complex128)


@pytest.mark.parametrize("nr,nt", [(4, 4), (8, 8), (16, 16), (8, 4), (32, 16), (3, 1)])
def test_factorisation_invariants(nr, nt):
    for H in _channels(nr, nt, 12, 11 + nr + nt):
        Q, R, perm, gap = oracle.sqrd(H)
        P = np.eye(nt)[:, perm]
        assert np.linalg.norm(H @ P - Q @ R) / np.linalg.norm(H) < 1e-13
        assert np.linalg.norm(Q.conj().T @ Q - np.eye(nt)) < 1e-13
        assert np.allclose(np.tril(R, -1), 0.0)
        d = np.diag(R)
        assert np.all(d.imag == 0.0) and np.all(d.real > 0)
        assert sorted(perm.tolist()) == list(range(nt))


@pytest.mark.parametrize("nr,nt", [(4, 4), (8, 8), (16, 16), (12, 6)])
def test_sort_order_is_min_residual_norm_bruteforce(nr, nt):
    # At step i the chosen column must have the smallest norm after projecting
    # out the span of the columns already chosen (checked with numpy's QR).
    for H in _channels(nr, nt, 8, 5 + nt, "kronecker"):
        _, R, perm, _ = oracle.sqrd(H)
        for i in range(nt):
            if i:
                Qi, _ = np.linalg.qr(H[:, perm[:i]])
                res = H - Qi @ (Qi.conj().T @ H)
            else:
                res = H
            rest = [c for c in range(nt) if c not in perm[:i]]
            norms = {c: np.linalg.norm(res[:, c]) ** 2 for c in rest}
            cmin = min(rest, key=lambda c: (norms[c], c))
            assert perm[i] == cmin
            assert np.isclose(R[i, i].real ** 2, norms[cmin], rtol=1e-12)


def test_ties_go_to_lower_user_index():
    H = np.eye(4, dtype=np.complex128)  # all columns have the same norm at every step
    _, R, perm, gap = oracle.sqrd(H)
    assert perm.tolist() == [0, 1, 2, 3]
    assert np.allclose(R, np.eye(4))


def test_single_user_reduces_to_mrc():
    rng = np.random.default_rng(3)
    h = (rng.standard_normal((6, 1)) + 1j * rng.standard_normal((6, 1)))
    y = (rng.standard_normal((5, 6)) + 1j * rng.standard_normal((5, 6)))
    Q, R, perm, _ = oracle.sqrd(h)
    z = oracle.qhy(Q, y)
    nh = np.linalg.norm(h)
    assert np.isclose(R[0, 0].real, nh, rtol=1e-14)
    # z / R_11 is the maximum-ratio-combining estimate h^H y / ||h||^2
    np.testing.assert_allclose(z[:, 0] / R[0, 0], (y @ h.conj())[:, 0] / nh ** 2, rtol=1e-12)


@pytest.mark.parametrize("nr,nt,qam", [(4, 4, 4), (8, 8, 16), (16, 16, 64)])
def test_z_noise_free_equals_R_times_permuted_symbols(nr, nt, qam):
    # y = H s  =>  z = Q^H H s = Q^H Q R P^T s = R (P^T s)
    sl = inputs.make_slot(nr, nt, qam, 6, 3, 20.0, "iid", 0.3, 99, noise=False)
    pts = oracle.constellation(qam)
    for c in range(6):
        H = sl.H[c].astype(np.complex128)
        s = pts[sl.labels[c]]                        # [n_sym][nt]
        y = s @ H.T                                  # exact noise-free, float64
        Q, R, perm, _ = oracle.sqrd(H)
        z = oracle.qhy(Q, y)
        np.testing.assert_allclose(z, s[:, perm] @ R.T, atol=1e-12)


def test_z_preserves_energy_in_column_space():
    sl = inputs.make_slot(8, 5, 16, 4, 14, 10.0, "iid", 0.3, 7)
    for c in range(4):
        H = sl.H[c].astype(np.complex128)
        Y = sl.Y[c].astype(np.complex128)
        Q, R, perm, _ = oracle.sqrd(H)
        Z = oracle.qhy(Q, Y)
        # ||y||^2 = ||z||^2 + ||component of y orthogonal to range(H)||^2
        U, _, _ = np.linalg.svd(H, full_matrices=False)
        orth = Y.T - U @ (U.conj().T @ Y.T)
        np.testing.assert_allclose(np.sum(np.abs(Y) ** 2, 1),
                                   np.sum(np.abs(Z) ** 2, 1) + np.sum(np.abs(orth) ** 2, 0),
                                   rtol=1e-12)


@pytest.mark.parametrize("nr,nt", [(7, 12), (2, 3), (8, 8), (4, 16), (16, 16)])
def test_mmse_extended_qr_factorises_the_augmented_channel(nr, nt):
    sl = inputs.make_slot(nr, nt, 4, 6, 3, 15.0, "iid", 0.3, 40 + nr + nt)
    for c in range(sl.n_sc):
        H = sl.H[c].astype(np.complex128)
        Q, R, perm, _ = oracle.sqrd_mmse(H, sl.sigma2)
        Ha = np.vstack([H, np.sqrt(sl.sigma2) * np.eye(nt)])
        P = np.eye(nt)[:, perm]
        assert np.linalg.norm(Ha @ P - Q @ R) / np.linalg.norm(Ha) < 1e-13
        assert np.linalg.norm(Q.conj().T @ Q - np.eye(nt)) < 1e-13
        assert np.allclose(np.tril(R, -1), 0) and np.all(np.real(np.diag(R)) > 0)
        # the pivot order is the minimum residual norm of the augmented columns
        for i in range(nt):
            if i:
                Qi, _ = np.linalg.qr(Ha[:, perm[:i]])
                res = Ha - Qi @ (Qi.conj().T @ Ha)
            else:
                res = Ha
            rest = [k for k in range(nt) if k not in perm[:i]]
            assert perm[i] == min(rest, key=lambda k: (np.linalg.norm(res[:, k]), k))
