// FP32 FMA throughput probe for the benchmark (libmpnl_bench.so, not the
// detector's library): the measured counterpart of the derived ALU peak (SMs
// x 128 FP32 lanes x 2 flop x clock) that the walk kernel is compared
// against.  Every thread runs kChains independent fmaf chains for `iters`
// rounds, so each SM sub-partition always has independent FMAs to issue; the
// sum is stored so the chains are not removed.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) ffma_probe_kernel(float *__restrict__ out, int iters,
                                                         float x, float y)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], x, y);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// Enqueue the probe: n_blocks CTAs of 256 threads on `stream`; *flops gets
// the floating-point operations it performs (2 per fmaf).  `out` is device
// memory of n_blocks * 256 floats.  Returns 0, -1 for bad arguments (n_blocks
// < 1, iters < 1, NULL pointers, more than 1e13 flop: the probe never runs
// long), -3 for a failed launch.
extern "C" int mpnl_bench_ffma_probe(int n_blocks, int iters, float *out, double *flops,
                                     void *stream)
{
    if (n_blocks < 1 || iters < 1 || !out || !flops) return -1;
    const double f = 2.0 * kChains * 256.0 * (double)n_blocks * (double)iters;
    if (f > 1e13) return -1;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, out) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return -1;
    }
    // x < 1 and y > 0: every chain converges to y / (1 - x), no overflow
    ffma_probe_kernel<<<n_blocks, 256, 0, (cudaStream_t)stream>>>(out, iters, 0.999f, 1e-3f);
    if (cudaGetLastError() != cudaSuccess) return -3;
    *flops = f;
    return 0;
}
