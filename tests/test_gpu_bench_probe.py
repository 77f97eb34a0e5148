"""The benchmark's FP32 FMA probe (libmpnl_bench.so): it runs, reports the
floating-point operations it performs, and refuses bad arguments."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_ffma_probe_runs_and_counts_its_flops():
    from paper_2409_14355_gb300 import build as cuda_build

    assert torch.cuda.is_available()
    cuda_build.build()
    lib = ctypes.CDLL(cuda_build.BENCH_LIB)
    lib.mpnl_bench_ffma_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    dev = torch.device("cuda", 0)
    out = torch.empty(3 * 256, dtype=torch.float32, device=dev)
    f = ctypes.c_double(0.0)
    st = torch.cuda.current_stream(dev)
    assert lib.mpnl_bench_ffma_probe(3, 100, ctypes.c_void_p(out.data_ptr()), ctypes.byref(f),
                                     ctypes.c_void_p(st.cuda_stream)) == 0
    torch.cuda.synchronize()
    assert f.value == 2 * 8 * 256 * 3 * 100
    v = out.cpu().numpy()
    assert np.all(np.isfinite(v)) and np.all(v > 0)
    # more than 1e13 flop, or host memory, is refused
    assert lib.mpnl_bench_ffma_probe(3, 10 ** 9, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.byref(f), None) == -1
    host = torch.empty(256, dtype=torch.float32)
    assert lib.mpnl_bench_ffma_probe(1, 1, ctypes.c_void_p(host.data_ptr()), ctypes.byref(f),
                                     None) == -1
