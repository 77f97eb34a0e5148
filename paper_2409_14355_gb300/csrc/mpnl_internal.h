// Internal launcher interface between the C ABI (mpnl_api.cu) and the kernel
// translation units.  Each launcher validates nothing (the ABI layer did),
// enqueues its kernel(s) on `stream` and returns cudaGetLastError().
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpnl {

// sigma > 0: MMSE-extended factorisation of [H; sigma I] (mpnl_preprocess_mmse).
cudaError_t launch_preprocess(int n_sc, int n_sym, int nr, int nt, float sigma, const float2 *H,
                              const float2 *Y, float2 *R, float *inv_diag, uint8_t *perm,
                              float2 *Z, cudaStream_t stream);

cudaError_t launch_select_paths(int n_sc, int nt, int qam, int n_pe, float sigma2,
                                const float2 *R, uint8_t *paths, cudaStream_t stream);

// f16: residuals in half2 with FP32 ranking / PED and an FP32 re-check of
// the best and runner-up paths (mpnl_detect_mixed); false: all FP32.
cudaError_t launch_detect(int n_sc, int n_sym, int nt, int qam, int n_pe, float sigma2,
                          const float2 *R, const float *inv_diag, const uint8_t *perm,
                          const uint8_t *paths, const float2 *Z, uint8_t *hard, float *llr,
                          float *ped2, unsigned *status, bool f16, cudaStream_t stream);

cudaError_t launch_mmse(int n_sc, int n_sym, int nr, int nt, int qam, float sigma2,
                        const float2 *H, const float2 *Y, uint8_t *hard, float *llr,
                        cudaStream_t stream);

// FP32 FMA throughput probe (mpnl_probe_ffma): 256-thread CTAs.
cudaError_t launch_ffma_probe(int n_blocks, int iters, float *out, cudaStream_t stream);
double ffma_probe_flops(int n_blocks, int iters);

// Device status bits (mpnl_check_status).
constexpr unsigned kStatusBadPathEntry = 1u;

}  // namespace mpnl
