// Evaluation of the N_pe position vectors (walks, argmin, max-log LLRs):
// host-side dispatch.  The kernels are in detect_impl.cuh and are instantiated
// in detect_f32.cu and detect_f16.cu.
#include "detect_impl.cuh"

namespace mpnl {

size_t detect_smem_bytes(int nt, int qam, int n_pe, int n_sym)
{
    const int NT = nt <= 4 ? 4 : (nt <= 8 ? 8 : 16);
    const int B = qam == 4 ? 2 : (qam == 16 ? 4 : 6);
    // the larger of the two precisions' layouts (a batch mixes them)
    const int W = (NT * B + 31) / 32;
    const int a = det_layout(NT, B, n_pe, n_sym, W, false).bytes;
    const int b = det_layout(NT, B, n_pe, n_sym, W, true).bytes;
    return (size_t)(a > b ? a : b);
}

cudaError_t launch_detect(int n_sc, int n_sym, int nt, int qam, int n_pe, float sigma2,
                          const float2 *R, const float *inv_diag, const uint8_t *perm,
                          const uint8_t *paths, const float2 *Z, uint8_t *hard, float *llr,
                          float *ped2, unsigned *status, bool f16, int sym, cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    const DetArgs a{n_sym, nt, n_pe, sigma2, R, inv_diag, perm, paths, Z, hard, llr, ped2, status};
    return f16 ? launch_detect_f16(n_sc, a, qam, sym, stream)
               : launch_detect_f32(n_sc, a, qam, sym, stream);
}

}  // namespace mpnl
