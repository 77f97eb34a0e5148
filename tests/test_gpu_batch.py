"""Mixed-size batches in persistent launches (mpnl_batch_*): every unit's
results in the mix equal the per-call path on that unit alone, with and
without a captured CUDA graph; launch-shape knobs leave results unchanged."""
import pytest

from paper_2409_14355_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUTS = ("R", "inv_diag", "perm", "Z", "paths", "hard", "llr", "ped2")


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


def _specs():
    # a scaled-down mixed batch plus a unit with more users than antennas
    specs = inputs.mixed_units(14, seed=20240914, sc_scale=0.05)
    specs.append(inputs.UnitSpec(4, 6, 16, 37, 64, 18.0, "iid", 99))
    return specs


def _fill(dev, specs):
    mpnl = _mpnl()
    units, slots = [], []
    for k, u in enumerate(specs):
        sl = inputs.unit_slot(u)
        buf = mpnl.SlotBuffers(u.n_sc, 14, u.nr, u.nt, u.qam, u.n_pe, dev, mmse=True)
        buf.H.copy_(torch.from_numpy(sl.H))
        buf.Y.copy_(torch.from_numpy(sl.Y))
        mmse_qr = u.nt > u.nr or k % 5 == 3
        precision = "fp16" if k % 4 == 2 else "fp32"
        units.append((buf, sl.sigma2, mmse_qr, k % 3 != 1, precision))
        slots.append(sl)
    return units, slots


def _alone(dev, unit):
    mpnl = _mpnl()
    buf, sigma2, mmse_qr, mmse, precision = unit
    n_sc, n_sym, nr, nt, qam, n_pe = buf.dims
    ref = mpnl.SlotBuffers(n_sc, n_sym, nr, nt, qam, n_pe, dev, mmse=mmse)
    mpnl.run_slot(ref, buf.H, buf.Y, sigma2, mmse=mmse, mmse_qr=mmse_qr, precision=precision)
    return ref


def _assert_same(unit, ref, k):
    buf, _, _, mmse, _ = unit
    names = OUTS + (("mmse_hard", "mmse_llr") if mmse else ())
    for name in names:
        a, b = getattr(buf, name), getattr(ref, name)
        assert torch.equal(a, b), (k, name, buf.dims)


def test_batch_results_equal_each_unit_alone(dev):
    mpnl = _mpnl()
    units, _ = _fill(dev, _specs())
    batch = mpnl.Batch(units, dev)
    batch.run()
    mpnl.check_status()
    torch.cuda.synchronize()
    for k, unit in enumerate(units):
        _assert_same(unit, _alone(dev, unit), k)
    batch.close()


def test_sharing_sms_leaves_results_unchanged(dev):
    mpnl = _mpnl()
    units, _ = _fill(dev, _specs()[:6])
    batch = mpnl.Batch(units, dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    # leaving room on the SMs, or one CTA per work item (short CTAs) instead
    # of persistent ones, changes how the work is spread, never the results
    for graph in (False, True):
        for share, short in ((True, False), (False, True), (True, True)):
            with torch.cuda.stream(side):
                batch.run(graph=graph, stream=side, share_sms=share, short_ctas=short)
            side.synchronize()
            mpnl.check_status()
            for k, unit in enumerate(units):
                _assert_same(unit, _alone(dev, unit), k)
    batch.close()


def test_batch_graph_replay_follows_new_inputs(dev):
    mpnl = _mpnl()
    specs = _specs()
    units, _ = _fill(dev, specs)
    batch = mpnl.Batch(units, dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        batch.run(graph=True, stream=side)
    side.synchronize()
    for k, unit in enumerate(units):
        _assert_same(unit, _alone(dev, unit), k)
    # new received symbols in the same buffers: the replayed graph reads them
    for k, (buf, _, _, _, _) in enumerate(units):
        sl = inputs.unit_slot(inputs.UnitSpec(**{**specs[k].__dict__, "seed": specs[k].seed + 1}))
        buf.Y.copy_(torch.from_numpy(sl.Y))
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        batch.run(graph=True, stream=side)
    side.synchronize()
    mpnl.check_status()
    for k, unit in enumerate(units):
        _assert_same(unit, _alone(dev, unit), k)
    batch.close()


def test_batch_rejects_bad_items(dev):
    mpnl = _mpnl()
    units, _ = _fill(dev, _specs()[:3])
    bad = list(units)
    buf, s2, mq, mm, prec = bad[1]
    bad[1] = (buf, -1.0, mq, mm, prec)
    with pytest.raises(mpnl.MpnlError) as e:
        mpnl.Batch(bad, dev)
    assert "item 1" in str(e.value)
    b = mpnl.Batch(units, dev)
    with pytest.raises(mpnl.MpnlError):
        b.run(graph=True, stream=torch.cuda.default_stream(dev))  # legacy stream cannot be captured
    b.close()


@pytest.mark.parametrize("name,n_pe,n_sc", [("16x16-64qam-3276sc", 256, 40),
                                            ("8x8-16qam-936sc", 64, 61),
                                            ("4x4-qpsk-64sc", 16, 64)])
def test_launch_knobs_do_not_change_results(dev, name, n_pe, n_sc):
    mpnl = _mpnl()
    sl = inputs.workload_slot(name, 0, n_sc=n_sc)
    H = torch.from_numpy(sl.H).to(dev)
    Y = torch.from_numpy(sl.Y).to(dev)
    out = []
    for sym in (2, 1):
        for warps in (1, 2, 4):
            t = mpnl.Tuning()
            a, b, c = mpnl.problem_class(sl.nt, sl.qam, n_pe)
            t.detect_sym[a][b][c] = sym
            t.select_warps[a][b][c] = warps
            mpnl.set_tuning(t)
            try:
                buf = mpnl.SlotBuffers(n_sc, 14, sl.nr, sl.nt, sl.qam, n_pe, dev, mmse=False)
                mpnl.run_slot(buf, H, Y, sl.sigma2, mmse=False)
                torch.cuda.synchronize()
                out.append(buf)
            finally:
                mpnl.set_tuning(None)
    for buf in out[1:]:
        for name_ in ("paths", "hard", "llr", "ped2"):
            assert torch.equal(getattr(buf, name_), getattr(out[0], name_)), name_
    with pytest.raises(mpnl.MpnlError):
        t = mpnl.Tuning()
        t.select_warps[0][0][0] = 3
        mpnl.set_tuning(t)


def test_autotuner_picks_valid_knobs(dev):
    from paper_2409_14355_gb300 import autotune
    mpnl = _mpnl()
    units = inputs.mixed_units(4, seed=7, sc_scale=0.03)
    t, report = autotune.tune(units, dev.index, reps=2)
    d = autotune.to_dict(t)
    assert d["persistent_ctas_per_sm"] in (2, 3)
    for u in units:
        a, b, c = mpnl.problem_class(u.nt, u.qam, u.n_pe)
        assert d["detect_sym"][a][b][c] in (1, 2)
        assert d["select_warps"][a][b][c] in (1, 2, 4)
    assert d["persistent_select_warps"] in (1, 2, 4)
    assert report["classes"] and report["batch_ms"]
    # the tuner leaves the built-in knobs installed
    assert autotune.to_dict(mpnl.get_tuning()) == autotune.to_dict(mpnl.Tuning())


def test_refine_stage_equals_the_per_call_refinement(dev):
    # units flagged MPNL_ITEM_REFINE_QR get the FP64 re-factorisation right
    # after their sorted QR in the batch: the results equal the per-call path
    # with mpnl_refine_qr at the same threshold; ill-conditioned channels
    # make sure the stage changes something
    from tests.test_gpu_refine import _ill_slot

    mpnl = _mpnl()
    units, plain = [], []
    for k, (nr, nt, qam, n_pe, mmse_qr, prec) in enumerate(
            [(8, 8, 16, 64, False, "fp16"), (16, 16, 64, 128, False, "fp32"),
             (12, 6, 16, 32, False, "fp16"), (8, 8, 4, 64, True, "fp16")]):
        H, Y, sigma2 = _ill_slot(nr, nt, qam, 21 + k, 1e5, 40 + k)
        sigma2 = max(sigma2, 1e-3)
        for lst, refine in ((units, True), (plain, False)):
            buf = mpnl.SlotBuffers(H.shape[0], 14, nr, nt, qam, n_pe, dev, mmse=False)
            buf.H.copy_(torch.from_numpy(H))
            buf.Y.copy_(torch.from_numpy(Y))
            lst.append((buf, sigma2, mmse_qr, False, prec, refine))
    for lst in (units, plain):
        batch = mpnl.Batch(lst, dev)
        batch.run()
        torch.cuda.synchronize()
        batch.close()
    mpnl.check_status()
    changed = 0
    for k, unit in enumerate(units):
        buf, sigma2, mmse_qr, _, prec, _ = unit
        n_sc, n_sym, nr, nt, qam, n_pe = buf.dims
        ref = mpnl.SlotBuffers(n_sc, n_sym, nr, nt, qam, n_pe, dev, mmse=False)
        mpnl.run_slot(ref, buf.H, buf.Y, sigma2, mmse=False, mmse_qr=mmse_qr, precision=prec,
                      refine_threshold=1e3)
        torch.cuda.synchronize()
        for name in OUTS:
            assert torch.equal(getattr(buf, name), getattr(ref, name)), (k, name)
        changed += int(not torch.equal(buf.R, plain[k][0].R))
    assert changed >= 3
