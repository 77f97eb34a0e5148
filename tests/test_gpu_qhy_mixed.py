"""z = Q^H y on the tensor cores (mpnl_qhy_mixed, FP16 operands, FP32
accumulation) against its FP64 definition (a matrix product of the same Q
and y): every z_j within the FP16 rounding bound 2^-10 sum_i |Q_ij| |y_i|
(both operands rounded to 11-bit significands), over square, tall, wide
(MMSE-extended antenna rows) and ragged shapes."""
import numpy as np
import pytest

from paper_2409_14355_gb300 import inputs

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


@pytest.mark.parametrize("nr,nt,n_sym,n_sc,mmse", [
    (16, 16, 14, 77, False), (8, 8, 14, 45, False), (4, 4, 14, 33, False),
    (32, 16, 32, 9, False), (5, 3, 7, 21, False), (6, 12, 14, 19, True), (1, 1, 1, 5, False),
])
def test_tensor_core_qhy_within_fp16_rounding(dev, nr, nt, n_sym, n_sc, mmse):
    from paper_2409_14355_gb300 import mpnl
    sl = inputs.make_slot(nr, nt, 16, n_sc, n_sym, 18.0, "iid", 0.3, 3 + nr * nt)
    H = torch.from_numpy(sl.H).to(dev)
    Y = torch.from_numpy(sl.Y).to(dev)
    Q, _, _, _ = mpnl.factor(H, sl.sigma2 if mmse else None)
    Z16 = mpnl.qhy(Q, Y, precision="fp16")
    Z32 = mpnl.qhy(Q, Y)
    torch.cuda.synchronize()
    Qn = Q.cpu().numpy().astype(np.complex128)
    Yn = sl.Y.astype(np.complex128)
    got = Z16.cpu().numpy().astype(np.complex128)
    for c in range(n_sc):
        want = Yn[c] @ Qn[c].conj()                             # [n_sym][nt]: z = Q^H y
        bound = 2.0 ** -10 * (np.abs(Yn[c]) @ np.abs(Qn[c])) + 1e-6   # [n_sym][nt]
        # per real and imaginary part the rounding error is at most 2^-10
        # sum_i |Q_ij| |y_i|, so |dz| at most sqrt(2) times that
        err = np.abs(got[c] - want)
        assert np.all(err <= 1.5 * bound), (c, float(np.max(err / bound)))
    # and it is FP16-close to the FP32 kernel, not equal to it
    d = (Z16 - Z32).abs().max().item()
    assert d > 0 and d < 1e-2 * Z32.abs().max().item()


def test_tensor_core_qhy_does_not_depend_on_the_scale_of_y(dev):
    # y at ADC-like scales (2^12) or tiny ones (2^-12) would overflow or go
    # subnormal in FP16; the kernel normalises each subcarrier's y by a power
    # of two, so z follows the scale exactly
    from paper_2409_14355_gb300 import mpnl
    sl = inputs.make_slot(16, 16, 64, 40, 14, 21.0, "iid", 0.3, 77)
    H = torch.from_numpy(sl.H).to(dev)
    Y = torch.from_numpy(sl.Y).to(dev)
    Q, _, _, _ = mpnl.factor(H)
    z0 = mpnl.qhy(Q, Y, precision="fp16")
    for k in (12, -12, 20):
        zk = mpnl.qhy(Q, Y * (2.0 ** k), precision="fp16")
        torch.cuda.synchronize()
        assert torch.equal(zk, z0 * (2.0 ** k)), k
        assert torch.isfinite(torch.view_as_real(zk)).all(), k
