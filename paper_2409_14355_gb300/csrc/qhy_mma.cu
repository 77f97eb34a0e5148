// z = Q^H y on the tensor cores with FP16 operands and FP32 accumulation
// (mpnl_qhy_mixed): the per-call kernel, a warp per subcarrier; the warp's
// work is in qhy_mma.cuh (shared with the persistent batch kernel).
#include "mpnl_internal.h"
#include "qhy_mma.cuh"

namespace mpnl {
namespace {

constexpr int kQmWarps = 4;

__global__ void __launch_bounds__(kQmWarps * 32)
qhy_mma_kernel(int n_sc, int n_sym, int nr, int nt, const float2 *__restrict__ Q,
               const float2 *__restrict__ Y, float2 *__restrict__ Z)
{
    const int warp = threadIdx.x >> 5;
    const int sc = blockIdx.x * kQmWarps + warp;
    if (sc >= n_sc) return;  // only __syncwarp inside
    qhy_mma_warp(sc, n_sym, nr, nt, Q, Y, Z, warp * qm_layout(n_sym, nr, nt).bytes);
}

}  // namespace

size_t qhy_mma_warp_bytes(int n_sym, int nr, int nt) { return qm_layout(n_sym, nr, nt).bytes; }

cudaError_t launch_qhy_mma(int n_sc, int n_sym, int nr, int nt, const float2 *Q, const float2 *Y,
                           float2 *Z, cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    const size_t smem = (size_t)qm_layout(n_sym, nr, nt).bytes * kQmWarps;
    cudaError_t e = allow_dynamic_smem(qhy_mma_kernel, smem);
    if (e != cudaSuccess) return e;
    qhy_mma_kernel<<<(n_sc + kQmWarps - 1) / kQmWarps, kQmWarps * 32, smem, stream>>>(
        n_sc, n_sym, nr, nt, Q, Y, Z);
    return cudaGetLastError();
}

}  // namespace mpnl
