// FP32 FMA throughput probe: the measured counterpart of the derived ALU peak
// (SMs x 128 FP32 lanes x 2 flop x clock) that the walk kernel is compared
// against.  Every thread runs kChains independent fmaf chains for `iters`
// rounds, so each SM sub-partition always has independent FMAs to issue; the
// sum is stored so the chains are not removed.  Not part of the detector.
#include "mpnl.h"
#include "mpnl_internal.h"

namespace mpnl {
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

cudaError_t launch_ffma_probe(int n_blocks, int iters, float *out, cudaStream_t stream)
{
    // x < 1 and y > 0: every chain converges to y / (1 - x), no overflow
    ffma_probe_kernel<<<n_blocks, 256, 0, stream>>>(out, iters, 0.999f, 1e-3f);
    return cudaGetLastError();
}

double ffma_probe_flops(int n_blocks, int iters)
{
    return 2.0 * kChains * 256.0 * (double)n_blocks * (double)iters;
}

}  // namespace mpnl
