"""The C ABI library builds, loads and exports every entry point that
include/mpnl.h declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import pytest

from paper_2409_14355_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpnl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpnl_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    from paper_2409_14355_gb300 import mpnl
    return mpnl.load_library()


def test_header_declares_the_path_entry_points():
    names = _declared()
    for want in ("mpnl_preprocess", "mpnl_select_paths", "mpnl_detect", "mpnl_linear_mmse",
                 "mpnl_create", "mpnl_destroy", "mpnl_last_error", "mpnl_workspace_bytes"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2409_14355_gb300 import mpnl
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(mpnl.EXPORTED) == _declared()


def test_host_side_errors_without_gpu(lib):
    from paper_2409_14355_gb300 import mpnl
    assert lib.mpnl_last_error(None) == b"context is NULL"
    d = mpnl.Dims(4, 14, 4, 4, 4, 16)
    assert lib.mpnl_preprocess(None, ctypes.byref(d), None, None, None, None, None, None, None,
                               None) == mpnl.ERR_INVALID_ARG
    assert lib.mpnl_detect(None, ctypes.byref(d), None, None, None, None, None,
                           ctypes.c_float(1.0), None, None, None, None, None) == mpnl.ERR_INVALID_ARG
    assert lib.mpnl_create(None, 0) == mpnl.ERR_INVALID_ARG
    assert lib.mpnl_workspace_bytes(ctypes.byref(d)) == 0
    lib.mpnl_destroy(None)


def test_create_reports_missing_device(lib):
    import torch
    from paper_2409_14355_gb300 import mpnl
    h = ctypes.c_void_p()
    st = lib.mpnl_create(ctypes.byref(h), 0)
    if torch.cuda.is_available():
        assert st == mpnl.OK
        lib.mpnl_destroy(h)
    else:
        assert st == mpnl.ERR_CUDA and not h.value
    assert lib.mpnl_create(ctypes.byref(h), 10_000) == mpnl.ERR_CUDA


def test_binding_refuses_to_run_without_gpu(lib):
    import torch
    from paper_2409_14355_gb300 import mpnl
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(mpnl.MpnlError):
        mpnl.context(0)
    H = torch.zeros((2, 4, 4), dtype=torch.complex64)
    with pytest.raises(mpnl.MpnlError):
        mpnl.preprocess(H, torch.zeros((2, 14, 4), dtype=torch.complex64))


def test_binding_argument_checks_need_no_gpu(lib):
    # checks the binding makes before touching a device
    import torch
    from paper_2409_14355_gb300 import mpnl
    with pytest.raises(ValueError):
        mpnl.SlotPipeline(4, 14, 4, 4, 4, 16, device="cuda:0", depth=0)
    edges = torch.zeros(3, dtype=torch.float32)
    with pytest.raises(ValueError):            # 4 bins need 3 edges and a [4][qam] table
        mpnl.RankLut(16, edges, torch.zeros((5, 16)))
    with pytest.raises(ValueError):
        mpnl.RankLut(16, edges, torch.zeros((4, 64)))
    lut = mpnl.RankLut(16, edges, torch.zeros((4, 16)))
    c = lut.c_struct()
    assert (c.qam, c.n_bins) == (16, 4)
    with pytest.raises(mpnl.MpnlError):        # precision names are checked first
        mpnl.qhy(torch.zeros((1, 4, 4), dtype=torch.complex64),
                 torch.zeros((1, 14, 4), dtype=torch.complex64), precision="bf8")


def test_header_is_plain_c():
    # the boundary is a C ABI: the header compiles as strict C99 and as C++
    import shutil
    import subprocess
    hdr = os.path.join(ROOT, "include", "mpnl.h")
    for cc, std in (("gcc", ["-std=c99", "-pedantic", "-x", "c"]), ("g++", ["-x", "c++"])):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not installed")
        r = subprocess.run([cc, "-fsyntax-only", "-Wall", "-Wextra", "-Werror", *std, hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_bench_probe_lives_outside_the_detector_library(lib):
    # the FP32 FMA probe is a benchmark helper in libmpnl_bench.so; the
    # detector's library does not export it
    assert not hasattr(lib, "mpnl_probe_ffma")
    b = ctypes.CDLL(cuda_build.BENCH_LIB)
    b.mpnl_bench_ffma_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    f = ctypes.c_double(0.0)
    assert b.mpnl_bench_ffma_probe(0, 1, None, ctypes.byref(f), None) == -1

