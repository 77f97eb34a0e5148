"""GPU path (through the C ABI) vs the FP64 oracle, element by element.

Stage-isolated tests feed every kernel the oracle's own intermediates rounded
to the kernel's input precision (complex64 / float32) and run the oracle on
exactly those rounded values; end-to-end tests run the whole GPU path on the
generator's slot and the oracle on the same slot.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2409_14355_gb300 import inputs
from tests import _parity as P
from tests._ref_helpers import all_label_vectors, bit_of, ml_metrics

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


# --------------------------------------------------------------------------
# a1 + a2: sorted QR and z = Q^H y
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nr,nt,qam,n_sc,n_sym,channel", [
    (4, 4, 4, 64, 14, "iid"),
    (8, 8, 16, 937, 14, "kronecker"),     # ragged: not a multiple of the 4 warps per CTA
    (16, 16, 64, 130, 14, "iid"),
    (6, 3, 16, 5, 14, "kronecker"),
    (32, 16, 64, 9, 32, "iid"),           # 16 + 32 columns: two columns per lane, 32 rows
    (16, 16, 64, 3, 1, "iid"),
    (2, 1, 4, 7, 14, "iid"),
])
def test_preprocess_matches_oracle(dev, nr, nt, qam, n_sc, n_sym, channel):
    mpnl = _mpnl()
    sl = inputs.make_slot(nr, nt, qam, n_sc, n_sym, 18.0, channel, 0.3, 100 + nr + nt + n_sc)
    R, inv_diag, perm, Z = mpnl.preprocess(_t(sl.H, dev), _t(sl.Y, dev))
    torch.cuda.synchronize()
    Rg = P.unpack_upper(R.cpu().numpy().astype(np.complex128), nt)
    pg = perm.cpu().numpy()
    Zg = Z.cpu().numpy().astype(np.complex128)
    ig = inv_diag.cpu().numpy()
    Rr, pr, Zr, gap = P.oracle_front(sl.H.astype(np.complex128), sl.Y.astype(np.complex128))
    H64 = sl.H.astype(np.complex128)
    kappa = np.linalg.cond(H64)
    # subcarriers whose pivot choice is a near-tie at some step (relative norm
    # gap below 1e-4) may legitimately order differently in float32
    ok_order = np.all(gap > 1e-4, axis=1)
    assert ok_order.mean() > 0.8
    np.testing.assert_array_equal(pg[ok_order], pr[ok_order])
    for c in np.flatnonzero(ok_order):
        tolR = 100 * U32 * kappa[c] * np.linalg.norm(H64[c])
        assert np.max(np.abs(Rg[c] - Rr[c])) <= tolR, (c, np.max(np.abs(Rg[c] - Rr[c])), tolR)
        ynorm = np.max(np.linalg.norm(sl.Y[c].astype(np.complex128), axis=-1))
        assert np.max(np.abs(Zg[c] - Zr[c])) <= 100 * U32 * kappa[c] * ynorm
        d = np.real(np.diag(Rr[c]))
        assert np.allclose(ig[c], 1.0 / d, rtol=100 * U32 * kappa[c])
        assert np.all(np.imag(np.diag(Rg[c])) == 0) and np.all(np.real(np.diag(Rg[c])) > 0)


# --------------------------------------------------------------------------
# a3: position-vector selection
# --------------------------------------------------------------------------
def _scores(paths, pe):
    """FP64 log-probability of each row under the oracle's per-level model."""
    lp1 = np.log1p(-pe)
    lpe = np.log(pe)
    return np.sum(lp1[None, :] + (paths.astype(np.float64) - 1) * lpe[None, :], axis=1)


@pytest.mark.parametrize("nt,qam,n_pe,snr_db", [
    (4, 4, 16, 10.0), (4, 4, 256, 10.0), (8, 16, 64, 10.0), (8, 16, 64, 25.0),
    (16, 64, 64, 15.0), (16, 64, 256, 30.0), (16, 64, 1024, 21.0), (3, 16, 37, 12.0),
    (1, 64, 64, 20.0), (16, 64, 1, 15.0),
])
def test_select_paths_matches_oracle(dev, nt, qam, n_pe, snr_db):
    mpnl = _mpnl()
    n_sc = 25  # not a multiple of the subcarriers one CTA takes
    sl = inputs.make_slot(nt, nt, qam, n_sc, 1, snr_db, "iid", 0.3, 7 + nt * qam + n_pe)
    Rr, _, _, _ = P.oracle_front(sl.H.astype(np.complex128), sl.Y.astype(np.complex128))
    R32 = Rr.astype(np.complex64)
    paths = mpnl.select_paths(_t(P.pack_upper(R32), dev), sl.sigma2, qam, n_pe, nt)
    torch.cuda.synchronize()
    G = paths.cpu().numpy()
    delta_abs = 1e-4
    for c in range(n_sc):
        rdiag = np.real(np.diag(R32[c])).astype(np.float64)
        n_more = n_pe + 1 if n_pe + 1 <= min(qam ** nt, 1024) else n_pe
        O, so, pe = oracle.select_paths(rdiag, sl.sigma2, qam, n_more)
        g = G[c]
        assert g[0].tolist() == [1] * nt
        assert len({tuple(r) for r in g}) == n_pe
        assert g.min() >= 1 and g.max() <= qam
        sg = _scores(g, pe)
        delta = delta_abs + 1e-5 * np.abs(sg)
        # every GPU row is within the tolerance of the oracle's N_pe-th best score
        assert np.all(sg >= so[n_pe - 1] - delta), c
        # GPU rows come in non-increasing score order up to near-ties
        assert np.all(np.diff(sg) <= delta[1:]), c
        # where the N_pe-th and (N_pe+1)-th scores are clearly apart the set is unique
        if n_more > n_pe and so[n_pe - 1] - so[n_pe] > 2 * (delta_abs + 1e-5 * abs(so[n_pe])):
            assert {tuple(r) for r in g} == {tuple(r) for r in O[:n_pe]}, c
        # rows whose score is clearly separated from all others sit at the oracle's position
        for i in range(n_pe):
            lo = so[i - 1] - so[i] if i > 0 else np.inf
            hi = so[i] - so[i + 1] if i + 1 < len(so) else np.inf
            if min(lo, hi) > 2 * (delta_abs + 1e-5 * abs(so[i])):
                assert g[i].tolist() == O[i].tolist(), (c, i)


# --------------------------------------------------------------------------
# a4-a6: walks, argmin, LLRs -- stage isolated
# --------------------------------------------------------------------------
def _stage_isolated(dev, nr, nt, qam, n_sc, snr_db, n_pe, channel="iid", seed=0, noise=True):
    mpnl = _mpnl()
    sl = inputs.make_slot(nr, nt, qam, n_sc, 14, snr_db, channel, 0.3, seed, noise)
    Rr, pr, Zr, _ = P.oracle_front(sl.H.astype(np.complex128), sl.Y.astype(np.complex128))
    R32, Z32, inv32 = P.to_fp32_inputs(Rr, Zr)
    paths = np.zeros((n_sc, n_pe, nt), np.uint8)
    for c in range(n_sc):
        paths[c] = oracle.select_paths(np.real(np.diag(R32[c])).astype(np.float64), sl.sigma2,
                                       qam, n_pe)[0]
    hard, llr, ped2 = mpnl.detect(_t(P.pack_upper(R32), dev), _t(inv32, dev),
                                  _t(pr.astype(np.uint8), dev), _t(paths, dev), _t(Z32, dev),
                                  sl.sigma2, qam)
    mpnl.check_status()
    gpu = dict(hard=hard.cpu().numpy(), llr=llr.cpu().numpy(), ped2=ped2.cpu().numpy())
    ref = P.oracle_detect_all(R32.astype(np.complex128), Z32.astype(np.complex128), pr, paths,
                              sl.sigma2, qam)
    return sl, gpu, ref, R32.astype(np.complex128)


@pytest.mark.parametrize("nr,nt,qam,n_sc,snr_db,n_pe,channel", [
    (4, 4, 4, 64, 10.0, 16, "iid"),
    (4, 4, 4, 64, 10.0, 256, "iid"),
    (8, 8, 16, 96, 10.0, 64, "kronecker"),
    (8, 8, 16, 96, 25.0, 64, "kronecker"),
    (16, 16, 64, 20, 15.0, 64, "iid"),
    (16, 16, 64, 20, 30.0, 256, "iid"),
    (16, 16, 64, 6, 21.0, 1024, "iid"),
    (5, 3, 16, 33, 12.0, 37, "kronecker"),
    (4, 1, 64, 17, 20.0, 64, "iid"),
    (16, 16, 64, 9, 24.0, 1, "iid"),
    (16, 12, 16, 11, 16.0, 300, "iid"),
])
def test_detect_stage_isolated(dev, nr, nt, qam, n_sc, snr_db, n_pe, channel):
    sl, gpu, ref, R = _stage_isolated(dev, nr, nt, qam, n_sc, snr_db, n_pe, channel,
                                      seed=nr * 31 + n_pe)
    # the larger the list, the more rankings per detection come near a tie
    P.compare_detect(gpu, ref, R, sl.sigma2, what=f"{nr}x{nt} q{qam} npe{n_pe}",
                     min_frac=0.5 if n_pe < 1024 else 0.2)


def test_detect_full_list_is_exhaustive_ml(dev):
    # N_pe = |Q|^Nt on 4x4 QPSK: the GPU's decisions are the brute-force ML ones
    sl, gpu, ref, R = _stage_isolated(dev, 4, 4, 4, 32, 4.0, 256, seed=5)
    pts = oracle.constellation(4)
    cand = all_label_vectors(4, 4)
    H = sl.H.astype(np.complex128)
    Y = sl.Y.astype(np.complex128)
    mask = P.comparable(ref, sl.sigma2)["decision"]
    n = 0
    for c in range(sl.n_sc):
        for s in range(sl.n_sym):
            if mask[c, s]:
                met = ml_metrics(H[c], Y[c, s], pts[cand])
                assert gpu["hard"][c, s].tolist() == cand[np.argmin(met)].tolist()
                n += 1
    assert n > 0.8 * mask.size


def test_detect_noise_free_recovery(dev):
    sl, gpu, ref, R = _stage_isolated(dev, 16, 16, 64, 8, 20.0, 64, seed=3, noise=False)
    np.testing.assert_array_equal(gpu["hard"], sl.labels)


def test_detect_llr_signs_match_decisions(dev):
    sl, gpu, ref, R = _stage_isolated(dev, 8, 8, 16, 40, 14.0, 64, "kronecker", seed=9)
    for b in range(4):
        bits = bit_of(gpu["hard"], b, 4)
        llr = gpu["llr"][..., b]
        assert np.all(np.where(bits == 1, llr <= 0, llr >= 0))


# --------------------------------------------------------------------------
# whole path, end to end
# --------------------------------------------------------------------------
def _end_to_end(dev, sl, n_pe, with_mmse=True):
    mpnl = _mpnl()
    buf = mpnl.SlotBuffers(sl.n_sc, sl.n_sym, sl.nr, sl.nt, sl.qam, n_pe, dev, mmse=with_mmse)
    mpnl.run_slot(buf, _t(sl.H, dev), _t(sl.Y, dev), sl.sigma2, mmse=with_mmse)
    mpnl.check_status()
    g = dict(hard=buf.hard.cpu().numpy(), llr=buf.llr.cpu().numpy(), ped2=buf.ped2.cpu().numpy(),
             paths=buf.paths.cpu().numpy(), perm=buf.perm.cpu().numpy())
    if with_mmse:
        g["mmse_hard"] = buf.mmse_hard.cpu().numpy()
        g["mmse_llr"] = buf.mmse_llr.cpu().numpy()
    ref = P.e2e_reference(sl.H, sl.Y, sl.sigma2, sl.qam, n_pe, with_mmse=with_mmse)
    return g, ref


def _ber(hard, labels, B):
    e = 0
    for b in range(B):
        e += np.sum(bit_of(hard, b, B) != bit_of(labels, b, B))
    return e / (labels.size * B)


@pytest.mark.parametrize("name,snr_index,n_pe,n_sc", [
    ("4x4-qpsk-64sc", 0, 16, None),
    ("4x4-qpsk-64sc", 0, 256, None),
    ("8x8-16qam-936sc", 0, 64, None),
    ("8x8-16qam-936sc", 5, 64, None),
    ("16x16-64qam-3276sc", 0, 64, 96),
    ("16x16-64qam-3276sc", 5, 128, 96),
])
def test_end_to_end_slot(dev, name, snr_index, n_pe, n_sc):
    sl = inputs.workload_slot(name, snr_index, n_sc=n_sc)
    g, ref = _end_to_end(dev, sl, n_pe)
    B = oracle.BITS[sl.qam]
    # BER within 1e-3 of the oracle's at this SNR point
    assert abs(_ber(g["hard"], sl.labels, B) - _ber(ref["hard"], sl.labels, B)) <= 1e-3
    assert abs(_ber(g["mmse_hard"], sl.labels, B) - _ber(ref["mmse_hard"], sl.labels, B)) <= 1e-3
    # decisions on clear detections of subcarriers where both sides built the
    # same ordering and the same table
    same_front = np.all(g["perm"] == ref["perm"], axis=1) & np.all(ref["sqrd_gap"] > 1e-4, axis=1)
    same_tab = np.all(g["paths"] == ref["paths"], axis=(1, 2))
    sc_ok = same_front & same_tab
    assert sc_ok.mean() > 0.8, sc_ok.mean()
    P.compare_detect(g, ref, ref["R"], sl.sigma2, rtol=ref["rtol"], what=name, sc_mask=sc_ok,
                     min_frac=0.4)


def test_full_size_slot_sampled(dev):
    # the bench configuration (3276 subcarriers, N_pe = 256), checked on a
    # sample of subcarriers the oracle can afford
    mpnl = _mpnl()
    sl = inputs.workload_slot("16x16-64qam-3276sc", 2)
    n_pe = 256
    buf = mpnl.SlotBuffers(sl.n_sc, sl.n_sym, sl.nr, sl.nt, sl.qam, n_pe, dev, mmse=True)
    mpnl.run_slot(buf, _t(sl.H, dev), _t(sl.Y, dev), sl.sigma2, mmse=True)
    mpnl.check_status()
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(sl.n_sc, 12, replace=False))
    idx[-1] = sl.n_sc - 1  # include the last (ragged-tail) subcarrier
    ref = P.e2e_reference(sl.H[idx], sl.Y[idx], sl.sigma2, sl.qam, n_pe)
    g = dict(hard=buf.hard.cpu().numpy()[idx], llr=buf.llr.cpu().numpy()[idx],
             ped2=buf.ped2.cpu().numpy()[idx])
    paths = buf.paths.cpu().numpy()[idx]
    perm = buf.perm.cpu().numpy()[idx]
    sc_ok = np.all(perm == ref["perm"], axis=1) & np.all(paths == ref["paths"], axis=(1, 2)) \
        & np.all(ref["sqrd_gap"] > 1e-4, axis=1)
    assert sc_ok.sum() >= 6
    P.compare_detect(g, ref, ref["R"], sl.sigma2, rtol=ref["rtol"], what="full slot",
                     sc_mask=sc_ok, min_frac=0.3)
    assert np.mean(buf.mmse_hard.cpu().numpy()[idx] == ref["mmse_hard"]) > 0.999


# --------------------------------------------------------------------------
# a7: linear MMSE
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nr,nt,qam,n_sc,snr_db,channel", [
    (4, 4, 4, 64, 10.0, "iid"), (8, 8, 16, 200, 25.0, "kronecker"),
    (16, 16, 64, 40, 30.0, "iid"), (6, 2, 64, 13, 20.0, "iid"), (32, 16, 16, 5, 15.0, "iid"),
])
def test_mmse_matches_oracle(dev, nr, nt, qam, n_sc, snr_db, channel):
    mpnl = _mpnl()
    sl = inputs.make_slot(nr, nt, qam, n_sc, 14, snr_db, channel, 0.3, 55 + nr + n_sc)
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
        eps = 64 * U32 * np.linalg.cond(A)  # Cholesky solve: O(n u kappa) relative error
        xt, nu = o["xt"], o["nu"]
        # distance of each equalised coordinate to the nearest decision boundary
        def bdist(v):
            t = v * scale
            mids = np.arange(-(L - 2), L - 1, 2)
            return np.min(np.abs(t[..., None] - mids), axis=-1) / scale
        safe = (np.minimum(bdist(xt.real), bdist(xt.imag)) > eps * (1 + np.abs(xt)))
        assert np.all(hg[c][safe] == o["hard"][safe])
        n_cmp += safe.sum()
        tol = eps * (np.abs(o["llr"]) + 4 * (1 + np.abs(xt[..., None])) ** 2 / nu[None, :, None])
        assert np.all(np.abs(lg[c] - o["llr"]) <= tol), c
    assert n_cmp > 0.8 * hg.size


# --------------------------------------------------------------------------
# edge cases and argument errors
# --------------------------------------------------------------------------
def test_empty_slot_is_a_noop(dev):
    mpnl = _mpnl()
    H = torch.empty((0, 4, 4), dtype=torch.complex64, device=dev)
    Y = torch.empty((0, 14, 4), dtype=torch.complex64, device=dev)
    R, inv_diag, perm, Z = mpnl.preprocess(H, Y)
    paths = mpnl.select_paths(R, 0.4, 4, 16, 4)
    hard, llr, ped2 = mpnl.detect(R, inv_diag, perm, paths, Z, 0.4, 4)
    mh, ml = mpnl.linear_mmse(H, Y, 0.4, 4)
    mpnl.check_status()
    assert hard.shape == (0, 14, 4) and mh.shape == (0, 14, 4)


def test_invalid_arguments_raise(dev):
    mpnl = _mpnl()
    sl = inputs.make_slot(4, 4, 4, 8, 14, 10.0, "iid", 0.3, 1)
    H, Y = _t(sl.H, dev), _t(sl.Y, dev)
    R, inv_diag, perm, Z = mpnl.preprocess(H, Y)
    with pytest.raises(mpnl.MpnlError) as e:
        mpnl.select_paths(R, 0.4, 8, 16, 4)       # qam 8 unsupported
    assert e.value.code == mpnl.ERR_INVALID_ARG
    with pytest.raises(mpnl.MpnlError):
        mpnl.select_paths(R, 0.4, 4, 257, 4)      # more rows than 4^4 vectors
    with pytest.raises(mpnl.MpnlError):
        mpnl.select_paths(R, -1.0, 4, 16, 4)      # sigma2 <= 0
    with pytest.raises(mpnl.MpnlError):
        mpnl.select_paths(R, float("inf"), 4, 16, 4)
    paths = mpnl.select_paths(R, 0.4, 4, 16, 4)
    with pytest.raises(mpnl.MpnlError):
        mpnl.detect(R, inv_diag, perm, paths, Z, 0.0, 4)
    Hw = torch.zeros((2, 3, 4), dtype=torch.complex64, device=dev)  # nt > nr
    with pytest.raises(mpnl.MpnlError):
        mpnl.preprocess(Hw, torch.zeros((2, 14, 3), dtype=torch.complex64, device=dev))
    # the C ABI itself refuses pageable host memory (a kernel would fault on it)
    lib = mpnl.load_library()
    ctx = mpnl.context(0)
    host = np.zeros(4096, np.complex64)
    d = mpnl.Dims(8, 14, 4, 4, 4, 16)
    st = lib.mpnl_preprocess(ctx, ctypes.byref(d), ctypes.c_void_p(host.ctypes.data),
                             ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                             ctypes.c_void_p(inv_diag.data_ptr()),
                             ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(Z.data_ptr()),
                             None, None)
    assert st == mpnl.ERR_INVALID_ARG
    assert b"H" in lib.mpnl_last_error(ctx)
    d17 = mpnl.Dims(8, 14, 17, 17, 4, 16)
    assert lib.mpnl_workspace_bytes(ctypes.byref(d17)) == 0
    st = lib.mpnl_select_paths(ctx, ctypes.byref(d17), ctypes.c_void_p(R.data_ptr()),
                               ctypes.c_float(0.4), ctypes.c_void_p(paths.data_ptr()), None, None)
    assert st == mpnl.ERR_INVALID_ARG


def test_bad_path_entries_are_clamped_and_reported(dev):
    mpnl = _mpnl()
    sl = inputs.make_slot(4, 4, 4, 8, 14, 10.0, "iid", 0.3, 2)
    R, inv_diag, perm, Z = mpnl.preprocess(_t(sl.H, dev), _t(sl.Y, dev))
    paths = mpnl.select_paths(R, sl.sigma2, 4, 16, 4)
    mpnl.check_status()
    bad = paths.clone()
    bad[0, 3, 1] = 0
    bad[5, 7, 2] = 99
    hard, llr, ped2 = mpnl.detect(R, inv_diag, perm, bad, Z, sl.sigma2, 4)
    with pytest.raises(mpnl.MpnlError) as e:
        mpnl.check_status()
    assert e.value.code == mpnl.ERR_INVALID_ARG
    mpnl.check_status()  # the flag was cleared
    assert torch.all(hard < 4)


def test_host_entry_point_matches_device_path(dev):
    mpnl = _mpnl()
    sl = inputs.workload_slot("8x8-16qam-936sc", 2, n_sc=200)
    Hh = torch.from_numpy(sl.H).pin_memory()
    Yh = torch.from_numpy(sl.Y).pin_memory()
    out_h = mpnl.detect_slot(Hh, Yh, sl.sigma2, sl.qam, 64, mmse=True)
    out_d = mpnl.detect_slot(_t(sl.H, dev), _t(sl.Y, dev), sl.sigma2, sl.qam, 64, mmse=True)
    assert out_h["hard"].device.type == "cpu"
    for k in ("hard", "llr", "ped2", "mmse_hard", "mmse_llr"):
        assert torch.equal(out_h[k], out_d[k].cpu()), k


def test_mmse_llr_array_on_a_4_byte_boundary(dev):
    """The ABI promises 4-byte alignment for float arrays: an LLR array that
    starts 4 bytes past an 8-byte boundary gets the same values (the kernel
    writes pairs only when the array is 8-byte aligned)."""
    import ctypes
    mpnl = _mpnl()
    sl = inputs.make_slot(8, 8, 16, 40, 14, 15.0, "iid", 0.3, 9)
    H, Y = _t(sl.H, dev), _t(sl.Y, dev)
    hard, llr = mpnl.linear_mmse(H, Y, sl.sigma2, sl.qam)
    buf = torch.zeros(llr.numel() + 1, dtype=torch.float32, device=dev)
    hard2 = torch.empty_like(hard)
    d = mpnl.Dims(sl.n_sc, 14, sl.nr, sl.nt, sl.qam, 1)
    st = mpnl.load_library().mpnl_linear_mmse(
        mpnl.context(dev.index), ctypes.byref(d), H.data_ptr(), Y.data_ptr(),
        ctypes.c_float(sl.sigma2), hard2.data_ptr(), buf.data_ptr() + 4, None, None)
    torch.cuda.synchronize()
    assert st == mpnl.OK
    assert torch.equal(hard2, hard)
    assert torch.equal(buf[1:].view_as(llr), llr)
