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
