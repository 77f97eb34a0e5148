"""The allocation-free walk entry point (mpnl_detect_units_noalloc).

It serves callers that must not allocate device memory while they run (a
distributed unit's real-time threads, where cudaMalloc/cudaFree can block
or synchronise the device, and frameworks that own every device buffer).
Its scratch is a fixed array inside the library, shared by every call.
Each call here goes through the C ABI and must give, for every unit, the
results of the existing per-call walks (mpnl_detect / mpnl_detect_mixed)
on that unit alone, bit for bit as the other batch tests require; two
calls in a row with different units show that the second call does not
see the first call's leftovers in the shared scratch.

The file name sorts last so that a run stopping at the first failure has
run every other test before this one.
"""
import ctypes

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


def _units(dev, specs, fp16_every):
    """Per unit: the walk inputs from the per-call QR and selection, output
    buffers for the allocation-free call, and the per-call walks' results."""
    from paper_2409_14355_gb300 import mpnl

    units = []
    for k, u in enumerate(specs):
        sl = inputs.unit_slot(u)
        H = torch.from_numpy(sl.H).to(dev)
        Y = torch.from_numpy(sl.Y).to(dev)
        mmse_qr = u.nt > u.nr
        R, inv_diag, perm, Z = mpnl.preprocess(H, Y, sigma2=sl.sigma2 if mmse_qr else None)
        paths = mpnl.select_paths(R, sl.sigma2, u.qam, u.n_pe, u.nt)
        precision = "fp16" if fp16_every and k % fp16_every == 1 else "fp32"
        ref = mpnl.detect(R, inv_diag, perm, paths, Z, sl.sigma2, u.qam, precision=precision)
        B = mpnl.BITS[u.qam]
        out = dict(hard=torch.full((u.n_sc, 14, u.nt), 255, dtype=torch.uint8, device=dev),
                   llr=torch.full((u.n_sc, 14, u.nt, B), float("nan"), device=dev),
                   ped2=torch.full((u.n_sc, 14, 2), float("nan"), device=dev))
        item = mpnl.batch_item((u.n_sc, 14, u.nr, u.nt, u.qam, u.n_pe), sl.sigma2,
                               mpnl.ITEM_FP16 if precision == "fp16" else 0, 0,
                               R=R, inv_diag=inv_diag, perm=perm, Z=Z, paths=paths, **out)
        units.append(dict(item=item, out=out, ref=ref, keep=(R, inv_diag, perm, Z, paths),
                          spec=u, precision=precision))
    return units


def _check(units):
    for k, u in enumerate(units):
        hard, llr, ped2 = u["ref"]
        assert torch.equal(u["out"]["hard"], hard), (k, u["spec"], u["precision"])
        assert torch.equal(u["out"]["llr"], llr), (k, u["spec"], u["precision"])
        assert torch.equal(u["out"]["ped2"], ped2), (k, u["spec"], u["precision"])


def test_noalloc_walks_equal_the_per_call_walks_twice_in_a_row(dev):
    from paper_2409_14355_gb300 import mpnl

    # call 1: a scaled-down mixed batch with FP16 units and a unit with more
    # users than antennas; call 2: other units (fewer, other sizes)
    first = inputs.mixed_units(9, seed=7_2409, sc_scale=0.04)
    first.append(inputs.UnitSpec(4, 6, 16, 29, 64, 18.0, "iid", 4242))
    second = inputs.mixed_units(5, seed=9_14355, sc_scale=0.06)
    for specs, fp16_every in ((first, 3), (second, 2)):
        units = _units(dev, specs, fp16_every)
        torch.cuda.synchronize()
        mpnl.detect_units_noalloc([u["item"] for u in units])
        torch.cuda.synchronize()
        _check(units)


def test_noalloc_rejects_more_units_than_its_scratch_holds(dev):
    from paper_2409_14355_gb300 import mpnl

    lib = mpnl.load_library()
    spec = inputs.UnitSpec(4, 4, 4, 3, 16, 10.0, "iid", 1)
    units = _units(dev, [spec], 0)
    n = mpnl.NOALLOC_MAX_UNITS + 1
    arr = (mpnl.BatchItemC * n)(*([units[0]["item"]] * n))
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    assert lib.mpnl_detect_units_noalloc(arr, n, stream) == mpnl.ERR_UNSUPPORTED
    assert lib.mpnl_detect_units_noalloc(arr, 0, stream) == mpnl.ERR_INVALID_ARG
    bad = mpnl.batch_item((3, 14, 4, 4, 4, 16), 0.5, mpnl.ITEM_LINEAR_MMSE, 0,
                          **{k: v for k, v in zip(("R", "inv_diag", "perm", "Z", "paths"),
                                                  units[0]["keep"])}, **units[0]["out"])
    assert lib.mpnl_detect_units_noalloc((mpnl.BatchItemC * 1)(bad), 1, stream) \
        == mpnl.ERR_INVALID_ARG
    # the largest count it holds still runs and matches
    full = (mpnl.BatchItemC * mpnl.NOALLOC_MAX_UNITS)(*([units[0]["item"]] * mpnl.NOALLOC_MAX_UNITS))
    assert lib.mpnl_detect_units_noalloc(full, mpnl.NOALLOC_MAX_UNITS, stream) == mpnl.OK
    torch.cuda.synchronize()
    _check(units)
