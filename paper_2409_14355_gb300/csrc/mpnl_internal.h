// Internal launcher interface between the C ABI (mpnl_api.cu) and the kernel
// translation units.  Each launcher validates nothing (the ABI layer did),
// enqueues its kernel(s) on `stream` and returns cudaGetLastError().
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct mpnl_ctx;

namespace mpnl {

// Context plumbing for the calls defined outside mpnl_api.cu: begin (checks
// the context, makes its device current, clears the message), its device,
// and an error return with the message "what: detail" (detail may be empty).
int api_begin(mpnl_ctx *ctx);
int api_device(const mpnl_ctx *ctx);
int api_fail(mpnl_ctx *ctx, int code, const char *what, const char *detail);

// Arguments of one detection problem (one radio unit's slot): sizes and the
// caller's device arrays, indexed by subcarrier inside the walk kernel.
struct DetArgs {
    int n_sym, nt, n_pe;
    float sigma2;
    const float2 *Rp;
    const float *inv_diag;
    const uint8_t *perm;
    const uint8_t *paths;
    const float2 *Z;
    uint8_t *hard;
    float *llr;
    float *ped2;
    unsigned *status;
};

// sigma > 0: MMSE-extended factorisation of [H; sigma I] (mpnl_preprocess_mmse).
// n_sym may be 0 (factor only; Y and Z unused); Q (nullable) receives the
// antenna rows of Q, [n_sc][nr][nt].
cudaError_t launch_preprocess(int n_sc, int n_sym, int nr, int nt, float sigma, const float2 *H,
                              const float2 *Y, float2 *R, float *inv_diag, uint8_t *perm,
                              float2 *Z, float2 *Q, cudaStream_t stream);

// FP64 re-factorisation where max R_ll / min R_ll > threshold (mpnl_refine_qr);
// Y/Z and Q nullable (n_sym 0 / no Q); n_refined (nullable) counts the
// subcarriers redone.
cudaError_t launch_refine(int n_sc, int n_sym, int nr, int nt, float sigma, float threshold,
                          const float2 *H, const float2 *Y, float2 *R, float *inv_diag,
                          uint8_t *perm, float2 *Z, float2 *Q, int *n_refined,
                          cudaStream_t stream);

// z = Q^H y from a stored Q (mpnl_qhy).
cudaError_t launch_qhy(int n_sc, int n_sym, int nr, int nt, const float2 *Q, const float2 *Y,
                       float2 *Z, cudaStream_t stream);
// The same on the tensor cores, FP16 operands, FP32 accumulation (mpnl_qhy_mixed).
cudaError_t launch_qhy_mma(int n_sc, int n_sym, int nr, int nt, const float2 *Q, const float2 *Y,
                           float2 *Z, cudaStream_t stream);
size_t qhy_mma_warp_bytes(int n_sym, int nr, int nt);

// warps: threads of one subcarrier's merges, 32 x (1, 2 or 4).
cudaError_t launch_select_paths(int n_sc, int nt, int qam, int n_pe, float sigma2,
                                const float2 *R, uint8_t *paths, int warps, cudaStream_t stream);

// Table-driven rank model (mpnl_select_paths_lut): edges [n_bins - 1],
// cost [n_bins][qam], device pointers.
cudaError_t launch_select_paths_lut(int n_sc, int nt, int qam, int n_pe, float sigma2,
                                    const float2 *R, const float *edges, const float *cost,
                                    int n_bins, uint8_t *paths, int warps, cudaStream_t stream);

// Monte-Carlo rank histogram (mpnl_rank_counts): counts [n_bins][qam] are
// zeroed and filled; gamma [n_bins] device doubles.
cudaError_t launch_rank_counts(int qam, int n_bins, const double *gamma, long long n_trials,
                               unsigned long long seed, unsigned long long *counts,
                               cudaStream_t stream);
// Rank costs from the histogram (mpnl_rank_costs): cost [n_bins][qam].
cudaError_t launch_rank_costs(int qam, int n_bins, const unsigned long long *counts,
                              long long n_trials, float *cost, cudaStream_t stream);

// Real-valued decomposition (mpnl_rvd_embed, mpnl_select_paths_pam,
// mpnl_detect_rvd): the embedding, the PAM-level selection over ntr = 2 nt
// real levels, and the real walks (nt = users; R, perm, Z over 2 nt levels).
cudaError_t launch_rvd_embed(int n_sc, int n_sym, int nr, int nt, const float2 *H, const float2 *Y,
                             float2 *Hr, float2 *Yr, cudaStream_t stream);
cudaError_t launch_select_paths_pam(int n_sc, int ntr, int qam, int n_pe, float sigma2,
                                    const float2 *R, uint8_t *paths, int warps,
                                    cudaStream_t stream);
cudaError_t launch_detect_rvd(int n_sc, int n_sym, int nt, int qam, int n_pe, float sigma2,
                              const float2 *R, const float *inv_diag, const uint8_t *perm,
                              const uint8_t *paths, const float2 *Z, uint8_t *hard, float *llr,
                              float *ped2, unsigned *status, cudaStream_t stream);
size_t rvd_smem_bytes(int nt, int qam, int n_pe, int n_sym);

// f16: residuals in half2 with FP32 ranking / PED and an FP32 re-check of
// the best and runner-up paths (mpnl_detect_mixed); false: all FP32.
// sym: symbols per lane (1 or 2; a tuning knob, results do not depend on it).
cudaError_t launch_detect(int n_sc, int n_sym, int nt, int qam, int n_pe, float sigma2,
                          const float2 *R, const float *inv_diag, const uint8_t *perm,
                          const uint8_t *paths, const float2 *Z, uint8_t *hard, float *llr,
                          float *ped2, unsigned *status, bool f16, int sym, cudaStream_t stream);
size_t detect_smem_bytes(int nt, int qam, int n_pe, int n_sym);
// The two precisions' launchers live in their own translation units.
cudaError_t launch_detect_f32(int n_sc, const DetArgs &a, int qam, int sym, cudaStream_t stream);
cudaError_t launch_detect_f16(int n_sc, const DetArgs &a, int qam, int sym, cudaStream_t stream);

cudaError_t launch_mmse(int n_sc, int n_sym, int nr, int nt, int qam, float sigma2,
                        const float2 *H, const float2 *Y, uint8_t *hard, float *llr,
                        cudaStream_t stream);

// One radio unit's slot in a batch (mpnl_batch_*), as the persistent kernels
// read it from device memory.  The work items of a stage are the
// subcarriers of the units taking part in it; the stage's start[] holds
// their prefix sums (n_items + 1 entries, zero-length for units outside).
struct BatchItem {
    int n_sc, n_sym, nr, nt, qam, n_pe;
    float sigma2, sigma;  // sigma > 0: MMSE-extended QR (sigma = sqrt(sigma2))
    int sym;              // symbols per lane of the walk kernel
    int mmse;             // also run the linear MMSE baseline
    int f16;              // walks with FP16 residuals (mpnl_detect_mixed's arithmetic)
    int factor_sym;       // symbols the sorted-QR stage carries along (n_sym or 0)
    float refine_threshold;  // FP64 re-factorisation stage: max R_ll / min R_ll threshold
    float2 *Q;            // antenna rows of Q (nullable; required by the Q^H y stage)
    const float2 *H, *Y;
    float2 *R;
    float *inv_diag;
    uint8_t *perm;
    float2 *Z;
    uint8_t *paths;
    uint8_t *hard;
    float *llr;
    float *ped2;
    uint8_t *mmse_hard;
    float *mmse_llr;
};

// Unit of work item w: the largest i with start[i] <= w.
__device__ __forceinline__ int find_item(const int *start, int n_items, int w)
{
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Persistent batch launchers: `counter` is a device int reset to 0 before
// the launch; shared memory per worker is the maximum over the batch.
size_t preprocess_warp_bytes(int n_sym, int nr, int nt);
size_t qhy_warp_bytes(int n_sym, int nr, int nt);
cudaError_t launch_qhy_batch(const BatchItem *items, const int *start, int n_items,
                             int *counter, int warp_bytes, int grid, cudaStream_t stream);
cudaError_t launch_preprocess_batch(const BatchItem *items, const int *start, int n_items,
                                    int *counter, int warp_bytes, int grid, cudaStream_t stream);
size_t select_group_bytes(int n_pe);
cudaError_t launch_select_batch(const BatchItem *items, const int *start, int n_items,
                                int *counter, int group_bytes, int warps, int grid,
                                cudaStream_t stream);
cudaError_t launch_detect_batch(const BatchItem *items, const int *start, int n_items,
                                int *counter, unsigned *status, size_t smem, int grid,
                                cudaStream_t stream);
size_t refine_warp_bytes(int rows, int nt, int n_sym);
cudaError_t launch_refine_batch(const BatchItem *items, const int *start, int n_items,
                                int *counter, int warp_bytes, int grid, cudaStream_t stream);
size_t mmse_warp_bytes(int n_sym, int nr, int nt);
cudaError_t launch_mmse_batch(const BatchItem *items, const int *start, int n_items,
                              int *counter, int warp_bytes, int grid, cudaStream_t stream);

// Device status bits (mpnl_check_status).
constexpr unsigned kStatusBadPathEntry = 1u;

}  // namespace mpnl
