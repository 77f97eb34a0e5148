"""The streaming host API (mpnl.SlotPipeline): slots submitted from pinned
host memory with several in flight give, slot by slot, the same results as
the per-call path run on the device copy of that slot alone."""
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


@pytest.mark.parametrize("name,n_pe,n_sc,depth,precision", [
    ("8x8-16qam-936sc", 64, 97, 2, "fp32"),
    ("16x16-64qam-3276sc", 256, 45, 3, "fp32"),
    ("4x4-qpsk-64sc", 16, 64, 1, "fp16"),
])
def test_pipeline_equals_each_slot_alone(dev, name, n_pe, n_sc, depth, precision):
    from paper_2409_14355_gb300 import mpnl
    slots = [inputs.workload_slot(name, 0, n_sc=n_sc, extra_seed=k) for k in range(5)]
    s0 = slots[0]
    pipe = mpnl.SlotPipeline(n_sc, 14, s0.nr, s0.nt, s0.qam, n_pe, dev, depth=depth,
                             mmse=True, precision=precision)
    host = [(torch.from_numpy(sl.H).pin_memory(), torch.from_numpy(sl.Y).pin_memory())
            for sl in slots]
    got, pending = [], []
    for k, (H, Y) in enumerate(host):
        pending.append((k, pipe.submit(H, Y, slots[k].sigma2)))
        if len(pending) == depth:
            k0, t = pending.pop(0)
            got.append((k0, {n: v.clone() for n, v in pipe.result(t).items()}))
    for k0, t in pending:
        got.append((k0, {n: v.clone() for n, v in pipe.result(t).items()}))
    pipe.check_status()
    for k, res in got:
        sl = slots[k]
        ref = mpnl.SlotBuffers(n_sc, 14, sl.nr, sl.nt, sl.qam, n_pe, dev, mmse=True)
        H = torch.from_numpy(sl.H).to(dev)
        Y = torch.from_numpy(sl.Y).to(dev)
        mpnl.run_slot(ref, H, Y, sl.sigma2, mmse=True, precision=precision)
        torch.cuda.synchronize()
        for n, v in res.items():
            assert torch.equal(v, getattr(ref, n).cpu()), (k, n)
    assert pipe.h2d_bytes == (host[0][0].numel() + host[0][1].numel()) * 8
    # a ticket whose buffers were reused is refused
    if depth == 1:
        t1 = pipe.submit(*host[0], slots[0].sigma2)
        pipe.submit(*host[1], slots[1].sigma2)
        with pytest.raises(ValueError):
            pipe.result(t1)
        torch.cuda.synchronize()


@pytest.mark.parametrize("mmse_qr,precision,pinned", [(False, "fp32", False), (True, "fp16", True)])
def test_c_abi_slot_call_with_host_buffers(dev, mmse_qr, precision, pinned):
    # mpnl_detect_slot straight through ctypes: host H and Y (pageable or
    # pinned), host outputs, a caller workspace; bit-identical to the
    # per-call steps on device copies
    import ctypes

    import numpy as np
    from paper_2409_14355_gb300 import mpnl
    lib = mpnl.load_library()
    sl = inputs.make_slot(6, 8 if mmse_qr else 6, 16, 53, 14, 17.0, "iid", 0.3, 9)
    n_pe = 48
    flags = mpnl.SLOT_MMSE | (mpnl.SLOT_FP16 if precision == "fp16" else 0) \
        | (mpnl.SLOT_MMSE_QR if mmse_qr else 0)
    H, Y = torch.from_numpy(sl.H), torch.from_numpy(sl.Y)
    if pinned:
        H, Y = H.pin_memory(), Y.pin_memory()
    out = mpnl.SlotOutputs(sl.n_sc, 14, sl.nt, sl.qam, mmse=True, pin=pinned)
    d = mpnl.Dims(sl.n_sc, 14, sl.nr, sl.nt, sl.qam, n_pe)
    nbytes = lib.mpnl_slot_workspace_bytes(ctypes.byref(d), flags)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    ctx = mpnl.context(dev.index)
    st = torch.cuda.current_stream(dev)
    P = ctypes.c_void_p
    args = [P(H.data_ptr()), P(Y.data_ptr()), P(out.hard.data_ptr()), P(out.llr.data_ptr()),
            P(out.ped2.data_ptr()), P(out.mmse_hard.data_ptr()), P(out.mmse_llr.data_ptr()),
            flags]
    assert lib.mpnl_detect_slot(ctx, ctypes.byref(d), ctypes.c_float(sl.sigma2), *args,
                                P(ws.data_ptr()), nbytes, P(st.cuda_stream)) == mpnl.OK
    st.synchronize()
    mpnl.check_status()
    ref = mpnl.SlotBuffers(sl.n_sc, 14, sl.nr, sl.nt, sl.qam, n_pe, dev, mmse=True)
    mpnl.run_slot(ref, H.to(dev), Y.to(dev), sl.sigma2, mmse=True, precision=precision,
                  mmse_qr=mmse_qr)
    torch.cuda.synchronize()
    for name, v in out.as_dict().items():
        assert torch.equal(v, getattr(ref, name).cpu()), name
    # a workspace too small, or not 256-byte aligned, is refused before anything runs
    assert lib.mpnl_detect_slot(ctx, ctypes.byref(d), ctypes.c_float(sl.sigma2), *args,
                                P(ws.data_ptr()), nbytes - 1, P(st.cuda_stream)) \
        == mpnl.ERR_INVALID_ARG
    assert lib.mpnl_detect_slot(ctx, ctypes.byref(d), ctypes.c_float(sl.sigma2), *args,
                                P(ws.data_ptr() + 16), nbytes, P(st.cuda_stream)) \
        == mpnl.ERR_INVALID_ARG
    assert np.all(out.hard.numpy() < sl.qam)


@pytest.mark.parametrize("precision,mmse", [("fp32", True), ("fp16", False)])
def test_slot_graph_replays_the_path(dev, precision, mmse):
    """SlotGraph: a replay gives the per-call path's results on whatever the
    fixed H and Y hold, slot after slot."""
    from paper_2409_14355_gb300 import mpnl
    slots = [inputs.make_slot(8, 8, 16, 61, 14, 15.0, "iid", 0.3, 700 + k) for k in range(3)]
    sl = slots[0]
    H = torch.from_numpy(sl.H).to(dev)
    Y = torch.from_numpy(sl.Y).to(dev)
    buf = mpnl.SlotBuffers(sl.n_sc, 14, sl.nr, sl.nt, sl.qam, 64, dev, mmse=mmse)
    g = mpnl.SlotGraph(buf, H, Y, sl.sigma2, mmse=mmse, precision=precision)
    ref = mpnl.SlotBuffers(sl.n_sc, 14, sl.nr, sl.nt, sl.qam, 64, dev, mmse=mmse)
    for s in slots:
        H.copy_(torch.from_numpy(s.H))
        Y.copy_(torch.from_numpy(s.Y))
        g.replay()
        mpnl.run_slot(ref, H, Y, sl.sigma2, mmse=mmse, precision=precision)
        torch.cuda.synchronize()
        for name in ("paths", "hard", "llr", "ped2") + (("mmse_hard", "mmse_llr") if mmse else ()):
            assert torch.equal(getattr(buf, name), getattr(ref, name)), name
    mpnl.check_status()
