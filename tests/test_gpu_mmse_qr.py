"""GPU path with the MMSE-extended sorted QR (more users than antennas, the
regime of §III-IV where MPNL serves e.g. 12 streams on 7 antennas) against
the FP64 oracle: the factorisation of [H; sigma I], then the whole path."""
import math

import numpy as np
import pytest

import oracle
from paper_2409_14355_gb300 import inputs
from tests import _parity as P
from tests._ref_helpers import bit_of

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


def _mpnl():
    from paper_2409_14355_gb300 import mpnl
    return mpnl


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _augmented(H, sigma2):
    nt = H.shape[-1]
    aug = np.broadcast_to(np.sqrt(sigma2) * np.eye(nt), (H.shape[0], nt, nt))
    return np.concatenate([H, aug], axis=1)


@pytest.mark.parametrize("nr,nt,qam,n_sc,n_sym,snr_db", [
    (7, 12, 4, 37, 14, 15.0),     # 12 streams on 7 antennas; ragged n_sc
    (2, 3, 16, 64, 14, 20.0),
    (4, 16, 4, 9, 14, 10.0),      # nr + nt = 20 rows
    (8, 8, 16, 130, 14, 25.0),    # square channel, augmented to 16 rows
    (16, 16, 64, 11, 14, 30.0),   # nr + nt = 32, the row limit
    (16, 8, 64, 5, 32, 20.0),     # 8 + 32 columns: two columns per lane
])
def test_preprocess_mmse_matches_oracle(dev, nr, nt, qam, n_sc, n_sym, snr_db):
    mpnl = _mpnl()
    sl = inputs.make_slot(nr, nt, qam, n_sc, n_sym, snr_db, "iid", 0.3, 300 + nr + nt + n_sc)
    R, inv_diag, perm, Z = mpnl.preprocess(_t(sl.H, dev), _t(sl.Y, dev), sigma2=sl.sigma2)
    torch.cuda.synchronize()
    Rg = P.unpack_upper(R.cpu().numpy().astype(np.complex128), nt)
    pg = perm.cpu().numpy()
    Zg = Z.cpu().numpy().astype(np.complex128)
    ig = inv_diag.cpu().numpy()
    H64 = sl.H.astype(np.complex128)
    Rr, pr, Zr, gap = P.oracle_front_mmse(H64, sl.Y.astype(np.complex128), sl.sigma2)
    Ha = _augmented(H64, sl.sigma2)
    kappa = np.linalg.cond(Ha)
    ok_order = np.all(gap > 1e-4, axis=1)
    assert ok_order.mean() > 0.8
    np.testing.assert_array_equal(pg[ok_order], pr[ok_order])
    for c in np.flatnonzero(ok_order):
        tolR = 100 * U32 * kappa[c] * np.linalg.norm(Ha[c])
        assert np.max(np.abs(Rg[c] - Rr[c])) <= tolR, (c, np.max(np.abs(Rg[c] - Rr[c])), tolR)
        ynorm = np.max(np.linalg.norm(sl.Y[c].astype(np.complex128), axis=-1))
        assert np.max(np.abs(Zg[c] - Zr[c])) <= 100 * U32 * kappa[c] * ynorm
        d = np.real(np.diag(Rr[c]))
        assert np.allclose(ig[c], 1.0 / d, rtol=100 * U32 * kappa[c])
        # the augmented rows bound every diagonal entry from below by sigma
        assert np.all(np.real(np.diag(Rg[c])) >= math.sqrt(sl.sigma2) * (1 - 1e-5))


def _ber(hard, labels, B):
    e = 0
    for b in range(B):
        e += np.sum(bit_of(hard, b, B) != bit_of(labels, b, B))
    return e / (labels.size * B)


@pytest.mark.parametrize("nr,nt,qam,n_sc,snr_db,n_pe", [
    (7, 12, 4, 96, 12.0, 64),
    (7, 12, 4, 96, 18.0, 256),
    (8, 12, 16, 64, 22.0, 128),
    (4, 6, 16, 128, 18.0, 64),
    (16, 16, 64, 48, 25.0, 128),
])
def test_end_to_end_more_users_than_antennas(dev, nr, nt, qam, n_sc, snr_db, n_pe):
    mpnl = _mpnl()
    sl = inputs.make_slot(nr, nt, qam, n_sc, 14, snr_db, "iid", 0.3, 700 + nr * nt + n_pe)
    buf = mpnl.SlotBuffers(n_sc, 14, nr, nt, qam, n_pe, dev, mmse=True)
    mpnl.run_slot(buf, _t(sl.H, dev), _t(sl.Y, dev), sl.sigma2, mmse=True, mmse_qr=True)
    mpnl.check_status()
    g = dict(hard=buf.hard.cpu().numpy(), llr=buf.llr.cpu().numpy(), ped2=buf.ped2.cpu().numpy(),
             paths=buf.paths.cpu().numpy(), perm=buf.perm.cpu().numpy(),
             mmse_hard=buf.mmse_hard.cpu().numpy())
    ref = P.e2e_reference(sl.H, sl.Y, sl.sigma2, qam, n_pe, with_mmse=True, mmse_qr=True)
    B = oracle.BITS[qam]
    ber_g, ber_r = _ber(g["hard"], sl.labels, B), _ber(ref["hard"], sl.labels, B)
    assert abs(ber_g - ber_r) <= 1e-3, (ber_g, ber_r)
    assert abs(_ber(g["mmse_hard"], sl.labels, B) - _ber(ref["mmse_hard"], sl.labels, B)) <= 1e-3
    same_front = np.all(g["perm"] == ref["perm"], axis=1) & np.all(ref["sqrd_gap"] > 1e-4, axis=1)
    same_tab = np.all(g["paths"] == ref["paths"], axis=(1, 2))
    sc_ok = same_front & same_tab
    assert sc_ok.mean() > 0.8, sc_ok.mean()
    P.compare_detect(g, ref, ref["R"], sl.sigma2, rtol=ref["rtol"],
                     what=f"{nr}x{nt} mmse-qr", sc_mask=sc_ok, min_frac=0.4)


def test_mmse_qr_full_list_is_regularised_ml(dev):
    # 2 antennas, 3 QPSK users, all 64 vectors: the GPU decision must be
    # argmin ||y - H s||^2 + sigma2 ||s||^2 over Q^3 wherever that is unique
    mpnl = _mpnl()
    sl = inputs.make_slot(2, 3, 4, 40, 14, 10.0, "iid", 0.3, 4242)
    out = mpnl.detect_slot(_t(sl.H, dev), _t(sl.Y, dev), sl.sigma2, 4, 64, mmse_qr=True)
    ref = P.e2e_reference(sl.H, sl.Y, sl.sigma2, 4, 64, with_mmse=False, mmse_qr=True)
    g = {k: out[k].cpu().numpy() for k in ("hard", "llr", "ped2")}
    P.compare_detect(g, ref, ref["R"], sl.sigma2, rtol=ref["rtol"], what="2x3 full list",
                     min_frac=0.8)


@pytest.mark.parametrize("nr,nt,qam,n_sc,snr_db", [
    (4, 6, 16, 40, 20.0), (7, 12, 4, 30, 15.0), (2, 8, 4, 17, 10.0),
])
def test_mmse_baseline_more_users_than_antennas(dev, nr, nt, qam, n_sc, snr_db):
    mpnl = _mpnl()
    sl = inputs.make_slot(nr, nt, qam, n_sc, 14, snr_db, "iid", 0.3, 901 + nr + nt)
    hard, llr = mpnl.linear_mmse(_t(sl.H, dev), _t(sl.Y, dev), sl.sigma2, qam)
    torch.cuda.synchronize()
    hg, lg = hard.cpu().numpy(), llr.cpu().numpy().astype(np.float64)
    L = int(round(math.sqrt(qam)))
    scale = math.sqrt(2.0 * (qam - 1) / 3.0)
    n_cmp = 0
    for c in range(n_sc):
        H = sl.H[c].astype(np.complex128)
        o = oracle.mmse(H, sl.Y[c], sl.sigma2, qam)
        A = H.conj().T @ H + sl.sigma2 * np.eye(nt)
        eps = 64 * U32 * np.linalg.cond(A)
        xt, nu = o["xt"], o["nu"]

        def bdist(v):
            t = v * scale
            mids = np.arange(-(L - 2), L - 1, 2)
            return np.min(np.abs(t[..., None] - mids), axis=-1) / scale
        safe = np.minimum(bdist(xt.real), bdist(xt.imag)) > eps * (1 + np.abs(xt))
        assert np.all(hg[c][safe] == o["hard"][safe])
        n_cmp += safe.sum()
        tol = eps * (np.abs(o["llr"]) + 4 * (1 + np.abs(xt[..., None])) ** 2 / nu[None, :, None])
        assert np.all(np.abs(lg[c] - o["llr"]) <= tol), c
    assert n_cmp > 0.8 * hg.size


def test_preprocess_mmse_argument_errors(dev):
    mpnl = _mpnl()
    sl = inputs.make_slot(7, 12, 4, 4, 14, 15.0, "iid", 0.3, 3)
    H, Y = _t(sl.H, dev), _t(sl.Y, dev)
    with pytest.raises(mpnl.MpnlError):
        mpnl.preprocess(H, Y)                       # plain QR needs nt <= nr
    with pytest.raises(mpnl.MpnlError):
        mpnl.preprocess(H, Y, sigma2=0.0)           # sigma2 must be > 0
    H20 = torch.zeros((2, 20, 16), dtype=torch.complex64, device=dev)
    Y20 = torch.zeros((2, 14, 20), dtype=torch.complex64, device=dev)
    with pytest.raises(mpnl.MpnlError):
        mpnl.preprocess(H20, Y20, sigma2=0.5)       # 20 + 16 rows > 32
    R, inv_diag, perm, Z = mpnl.preprocess(H, Y, sigma2=sl.sigma2)
    torch.cuda.synchronize()
    assert perm.shape == (4, 12)
