"""FP64 re-factorisation of ill-conditioned channels: the subcarriers whose
FP32 R has max R_ll / min R_ll above the threshold are redone in FP64 and
then match the oracle to FP32 rounding, with no condition-number factor;
the others are left bit-for-bit as they were."""
import numpy as np
import pytest

from paper_2409_14355_gb300 import inputs
from tests import _parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def dev():
    from paper_2409_14355_gb300 import mpnl

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    mpnl.load_library()
    d = torch.device("cuda", 0)
    torch.cuda.set_device(d)
    return d


def _ill_slot(nr, nt, qam, n_sc, kappa, seed):
    """Channels U diag(s) V^H with singular values from 1 down to 1/kappa."""
    rng = np.random.default_rng(seed)
    H = np.zeros((n_sc, nr, nt), np.complex128)
    for c in range(n_sc):
        U, _ = np.linalg.qr(rng.standard_normal((nr, nr)) + 1j * rng.standard_normal((nr, nr)))
        V, _ = np.linalg.qr(rng.standard_normal((nt, nt)) + 1j * rng.standard_normal((nt, nt)))
        s = np.logspace(0, -np.log10(kappa), nt)
        H[c] = U[:, :nt] @ np.diag(s) @ V.conj().T
    pts = inputs.tx_constellation(qam)
    labels = rng.integers(0, qam, size=(n_sc, 14, nt))
    sigma2 = 1e-6
    Y = np.einsum("crt,cst->csr", H, pts[labels])
    Y = Y + (rng.standard_normal(Y.shape) + 1j * rng.standard_normal(Y.shape)) * np.sqrt(sigma2 / 2)
    return H.astype(np.complex64), Y.astype(np.complex64), sigma2


# sigma I caps the augmented matrix's condition near 1/sigma: a lower threshold there
@pytest.mark.parametrize("nr,nt,mmse_qr,thr", [(8, 8, False, 100.0), (16, 16, False, 100.0),
                                               (12, 6, False, 100.0), (8, 8, True, 10.0)])
def test_refined_subcarriers_match_the_oracle_to_fp32_rounding(dev, nr, nt, mmse_qr, thr):
    from paper_2409_14355_gb300 import mpnl
    H, Y, sigma2 = _ill_slot(nr, nt, 16, 40, 1e4, 11 + nt)
    Hd, Yd = torch.from_numpy(H).to(dev), torch.from_numpy(Y).to(dev)
    s2 = sigma2 if mmse_qr else None
    R, inv_diag, perm, Z = mpnl.preprocess(Hd, Yd, sigma2=s2)
    R32 = R.clone()
    count = torch.zeros(1, dtype=torch.int32, device=dev)
    mpnl.refine_qr(Hd, Yd, R, inv_diag, perm, Z=Z, sigma2=s2, cond_threshold=thr, count=count)
    torch.cuda.synchronize()
    H64, Y64 = H.astype(np.complex128), Y.astype(np.complex128)
    if mmse_qr:
        Rr, pr, Zr, gap = P.oracle_front_mmse(H64, Y64, sigma2)
    else:
        Rr, pr, Zr, gap = P.oracle_front(H64, Y64)
    diag32 = np.real(np.diagonal(P.unpack_upper(R32.cpu().numpy(), nt), axis1=1, axis2=2))
    expect = np.sum(~(diag32.max(1) <= thr * diag32.min(1)))
    assert int(count.item()) == expect > 0
    Rg = P.unpack_upper(R.cpu().numpy().astype(np.complex128), nt)
    Zg = Z.cpu().numpy().astype(np.complex128)
    pg = perm.cpu().numpy()
    R0 = P.unpack_upper(R32.cpu().numpy().astype(np.complex128), nt)
    ok = np.all(gap > 1e-6, axis=1)
    assert ok.mean() > 0.9
    err32, err64 = 0.0, 0.0
    for c in np.flatnonzero(ok):
        np.testing.assert_array_equal(pg[c], pr[c])
        scale = np.max(np.abs(Rr[c]))
        e = np.max(np.abs(Rg[c] - Rr[c]))
        assert e <= 8 * U32 * scale, (c, e / (U32 * scale))
        assert np.max(np.abs(Zg[c] - Zr[c])) <= 8 * U32 * np.max(np.abs(Zr[c])) + 1e-30
        err64 = max(err64, e / scale)
        if np.array_equal(pg[c], pr[c]):
            err32 = max(err32, np.max(np.abs(R0[c] - Rr[c])) / scale)
    assert err32 > 4 * err64  # the FP32 factor was visibly worse


def test_well_conditioned_channels_are_left_alone(dev):
    from paper_2409_14355_gb300 import mpnl
    sl = inputs.make_slot(8, 8, 16, 50, 14, 20.0, "iid", 0.3, 4)
    Hd, Yd = torch.from_numpy(sl.H).to(dev), torch.from_numpy(sl.Y).to(dev)
    R, inv_diag, perm, Z = mpnl.preprocess(Hd, Yd)
    before = [t.clone() for t in (R, inv_diag, perm, Z)]
    count = torch.zeros(1, dtype=torch.int32, device=dev)
    mpnl.refine_qr(Hd, Yd, R, inv_diag, perm, Z=Z, cond_threshold=1e6, count=count)
    torch.cuda.synchronize()
    assert int(count.item()) == 0
    for a, b in zip(before, (R, inv_diag, perm, Z)):
        assert torch.equal(a, b)


def test_refined_stored_q_reproduces_the_factor(dev):
    from paper_2409_14355_gb300 import mpnl
    H, Y, sigma2 = _ill_slot(16, 12, 64, 24, 1e4, 5)
    Hd = torch.from_numpy(H).to(dev)
    Q, R, inv_diag, perm = mpnl.factor(Hd)
    mpnl.refine_qr(Hd, None, R, inv_diag, perm, Q=Q, cond_threshold=10.0)
    torch.cuda.synchronize()
    Qg = Q.cpu().numpy().astype(np.complex128)
    Rg = P.unpack_upper(R.cpu().numpy().astype(np.complex128), 12)
    pg = perm.cpu().numpy()
    for c in range(24):
        Hp = H[c].astype(np.complex128)[:, pg[c]]
        assert np.max(np.abs(Qg[c] @ Rg[c] - Hp)) <= 16 * U32 * np.linalg.norm(H[c])
        assert np.max(np.abs(Qg[c].conj().T @ Qg[c] - np.eye(12))) <= 16 * U32


def test_refine_rejects_a_threshold_below_one(dev):
    from paper_2409_14355_gb300 import mpnl
    sl = inputs.make_slot(4, 4, 4, 3, 14, 20.0, "iid", 0.3, 4)
    Hd, Yd = torch.from_numpy(sl.H).to(dev), torch.from_numpy(sl.Y).to(dev)
    R, inv_diag, perm, Z = mpnl.preprocess(Hd, Yd)
    with pytest.raises(mpnl.MpnlError):
        mpnl.refine_qr(Hd, Yd, R, inv_diag, perm, Z=Z, cond_threshold=0.5)
