"""The seeded slot generator: determinism, shapes, noise level, correlation."""
import numpy as np

from paper_2409_14355_gb300 import inputs


def test_seeded_and_deterministic():
    a = inputs.workload_slot("4x4-qpsk-64sc", 0)
    b = inputs.workload_slot("4x4-qpsk-64sc", 0)
    c = inputs.workload_slot("4x4-qpsk-64sc", 0, extra_seed=1)
    assert np.array_equal(a.H, b.H) and np.array_equal(a.Y, b.Y)
    assert not np.array_equal(a.H, c.H)
    assert a.H.shape == (64, 4, 4) and a.Y.shape == (64, 14, 4) and a.labels.shape == (64, 14, 4)
    assert a.H.dtype == np.complex64 and a.labels.max() < 4


def test_noise_variance_and_channel_power():
    sl = inputs.make_slot(8, 4, 16, 2000, 14, 12.0, "iid", 0.3, 3)
    sl0 = inputs.make_slot(8, 4, 16, 2000, 14, 12.0, "iid", 0.3, 3, noise=False)
    n = (sl.Y - sl0.Y).astype(np.complex128)
    assert abs(np.mean(np.abs(n) ** 2) / sl.sigma2 - 1) < 0.01
    assert abs(sl.sigma2 - 4 / 10 ** 1.2) < 1e-12
    assert abs(np.mean(np.abs(sl.H) ** 2) - 1) < 0.01


def test_kronecker_correlation():
    sl = inputs.make_slot(4, 4, 4, 20000, 1, 10.0, "kronecker", 0.3, 5)
    H = sl.H.astype(np.complex128)
    # E[h_r1,t h_r2,t^*] = rho^|r1 - r2| (transmit side has unit diagonal)
    c01 = np.mean(H[:, 0, 0] * np.conj(H[:, 1, 0]))
    c02 = np.mean(H[:, 0, 0] * np.conj(H[:, 2, 0]))
    assert abs(c01.real - 0.3) < 0.03 and abs(c02.real - 0.09) < 0.03
