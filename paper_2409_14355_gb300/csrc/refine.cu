// FP64 re-factorisation of ill-conditioned channels.
//
// The FP32 sorted QR loses accuracy in proportion to the channel's condition
// number.  After it, one warp per subcarrier estimates the condition from
// the FP32 R as max R_ll / min R_ll (a lower bound on kappa(R) = kappa(H),
// cheap and usually within a small factor of it); where the estimate exceeds
// the caller's threshold, the warp recomputes the whole sorted QR -- and z,
// and Q if it is kept -- in FP64 and overwrites the outputs (rounded to
// FP32 once, at the end).  Everything else is left as it was.
//
// The FP64 factorisation is the modified Gram-Schmidt of the FP32 kernel,
// with the columns [H | y_0 .. y_{n_sym-1}] (and sigma I below H for the
// MMSE-extended variant) in shared memory, row-major so that lane c reading
// column c touches consecutive words: lane c owns column c (two columns per
// lane when nt + n_sym > 32).
#include <float.h>

#include "mpnl_common.cuh"
#include "mpnl_internal.h"

namespace mpnl {
namespace {

constexpr int kRefWarps = 2;

__host__ __device__ inline int ref_cols(int nt, int n_sym) { return nt + n_sym; }

__host__ __device__ inline size_t ref_warp_bytes(int rows, int nt, int n_sym)
{
    // matrix (rows x cols double2), q (rows double2), R rows (nt x nt double2),
    // z (n_sym x nt double2), diag (nt double), perm (nt int)
    const size_t c = (size_t)ref_cols(nt, n_sym);
    size_t b = (size_t)rows * c * 16 + (size_t)rows * 16 + (size_t)nt * nt * 16 +
               (size_t)n_sym * nt * 16 + (size_t)nt * 8 + (size_t)nt * 4;
    return (b + 15) & ~(size_t)15;
}

// One subcarrier by one warp, in its shared-memory region `base` (at least
// ref_warp_bytes(rows, nt, n_sym)); Y and Z NULL (n_sym 0) when z is not
// formed here, Qout and n_refined nullable.
__device__ __forceinline__ void refine_warp(int sc, int n_sym, int nr, int nt, double sigma,
                                            float threshold, const float2 *__restrict__ H,
                                            const float2 *__restrict__ Y, float2 *__restrict__ Rp,
                                            float *__restrict__ inv_diag,
                                            uint8_t *__restrict__ perm_out,
                                            float2 *__restrict__ Z, float2 *__restrict__ Qout,
                                            int *__restrict__ n_refined, unsigned char *base)
{
    const int lane = threadIdx.x & 31;
    const int P = nt * (nt + 1) / 2;
    float2 *gR = Rp + (size_t)sc * P;

    // condition estimate from the FP32 diagonal
    float dmax = 0.f, dmin = FLT_MAX;
    for (int l = lane; l < nt; l += 32) {
        const float d = gR[l * nt - l * (l - 1) / 2].x;
        dmax = fmaxf(dmax, d);
        dmin = fminf(dmin, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
    }
    // NaN or zero diagonals also take the FP64 path
    const bool redo = !(dmax <= threshold * dmin) || !(dmin > 0.f);
    if (!redo) return;
    if (lane == 0 && n_refined != nullptr) atomicAdd(n_refined, 1);

    const int rows = sigma > 0.0 ? nr + nt : nr;
    const int cols = ref_cols(nt, n_sym);
    double2 *sM = reinterpret_cast<double2 *>(base);  // [rows][cols]
    double2 *sQ = sM + (size_t)rows * cols;
    double2 *sRt = sQ + rows;                          // [i][user column]
    double2 *sZ = sRt + nt * nt;                       // [s][i]
    double *sRd = reinterpret_cast<double *>(sZ + n_sym * nt);
    int *sPerm = reinterpret_cast<int *>(sRd + nt);

    const float2 *gH = H + (size_t)sc * nr * nt;
    const float2 *gY = Y + (size_t)sc * n_sym * nr;
    for (int k = lane; k < rows * cols; k += 32) {
        const int r = k / cols, c = k - r * cols;
        double2 v = make_double2(0.0, 0.0);
        if (r < nr) {
            if (c < nt) {
                const float2 h = gH[r * nt + c];
                v = make_double2(h.x, h.y);
            } else {
                const float2 y = gY[(c - nt) * nr + r];
                v = make_double2(y.x, y.y);
            }
        } else if (c == r - nr) {
            v = make_double2(sigma, 0.0);
        }
        sM[k] = v;
    }
    __syncwarp();

    // lane c owns columns c and c + 32
    bool placed0 = !(lane < nt);
    for (int i = 0; i < nt; ++i) {
        double nrm = INFINITY;
        if (!placed0) {
            double s = 0.0;
            for (int r = 0; r < rows; ++r) {
                const double2 v = sM[r * cols + lane];
                s = fma(v.x, v.x, fma(v.y, v.y, s));
            }
            nrm = (s <= DBL_MAX) ? s : DBL_MAX;
        }
        double bn = nrm;
        int bl = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double on = __shfl_xor_sync(0xffffffffu, bn, o);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (on < bn || (on == bn && ol < bl)) {
                bn = on;
                bl = ol;
            }
        }
        const int piv = bl;
        const double rii = sqrt(bn);
        const double inv = 1.0 / rii;
        for (int r = lane; r < rows; r += 32) {
            const double2 v = sM[r * cols + piv];
            sQ[r] = make_double2(v.x * inv, v.y * inv);
        }
        if (lane == 0) {
            sRd[i] = rii;
            sPerm[i] = piv;
        }
        if (lane == piv) placed0 = true;
        __syncwarp();
        if (Qout != nullptr)
            for (int r = lane; r < nr; r += 32)
                Qout[((size_t)sc * nr + r) * nt + i] = make_float2((float)sQ[r].x, (float)sQ[r].y);
        for (int c = lane; c < cols; c += 32) {
            // channel columns (c < nt <= 16, so c == lane) only while unplaced;
            // the pivot was marked placed above; symbol columns always
            if (c < nt && placed0) continue;
            double ax = 0.0, ay = 0.0;  // q^H col
            for (int r = 0; r < rows; ++r) {
                const double2 q = sQ[r], v = sM[r * cols + c];
                ax = fma(q.x, v.x, fma(q.y, v.y, ax));
                ay = fma(q.x, v.y, fma(-q.y, v.x, ay));
            }
            for (int r = 0; r < rows; ++r) {
                const double2 q = sQ[r];
                double2 v = sM[r * cols + c];
                v.x -= fma(ax, q.x, -ay * q.y);
                v.y -= fma(ax, q.y, ay * q.x);
                sM[r * cols + c] = v;
            }
            if (c < nt) sRt[i * nt + c] = make_double2(ax, ay);
            else sZ[(c - nt) * nt + i] = make_double2(ax, ay);
        }
        __syncwarp();
    }

    for (int k = lane; k < P; k += 32) {
        int i = 0, rem = k;
        while (rem >= nt - i) {
            rem -= nt - i;
            ++i;
        }
        const int j = i + rem;
        const double2 v = (j == i) ? make_double2(sRd[i], 0.0) : sRt[i * nt + sPerm[j]];
        gR[k] = make_float2((float)v.x, (float)v.y);
    }
    if (lane < nt) {
        inv_diag[(size_t)sc * nt + lane] = (float)(1.0 / sRd[lane]);
        perm_out[(size_t)sc * nt + lane] = (uint8_t)sPerm[lane];
    }
    if (Z != nullptr) {
        float2 *gZ = Z + (size_t)sc * n_sym * nt;
        for (int k = lane; k < n_sym * nt; k += 32)
            gZ[k] = make_float2((float)sZ[k].x, (float)sZ[k].y);
    }
}

__global__ void __launch_bounds__(kRefWarps * 32)
refine_kernel(int n_sc, int n_sym, int nr, int nt, double sigma, float threshold,
              const float2 *__restrict__ H, const float2 *__restrict__ Y, float2 *__restrict__ Rp,
              float *__restrict__ inv_diag, uint8_t *__restrict__ perm_out,
              float2 *__restrict__ Z, float2 *__restrict__ Qout, int *__restrict__ n_refined,
              int warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int sc = blockIdx.x * kRefWarps + warp;
    if (sc >= n_sc) return;  // warp-local work only
    refine_warp(sc, n_sym, nr, nt, sigma, threshold, H, Y, Rp, inv_diag, perm_out, Z, Qout,
                n_refined, smem_raw + (size_t)warp * warp_bytes);
}

// The refinement stage of a batch (units with MPNL_ITEM_REFINE_QR, right
// after their sorted QR): warps take (unit, subcarrier) items from a global
// counter; z is redone only where the QR stage formed it.
__global__ void __launch_bounds__(kRefWarps * 32)
refine_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ start,
                    int n_items, int *__restrict__ counter, int warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *base = smem_raw + (size_t)warp * warp_bytes;
    const int total = start[n_items];
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(counter, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= total) break;
        const int i = find_item(start, n_items, w);
        const BatchItem &it = items[i];
        const bool z = it.factor_sym > 0;
        refine_warp(w - start[i], z ? it.factor_sym : 0, it.nr, it.nt, (double)it.sigma,
                    it.refine_threshold, it.H, z ? it.Y : nullptr, it.R, it.inv_diag, it.perm,
                    z ? it.Z : nullptr, it.Q, nullptr, base);
        __syncwarp();  // the region is reused for the warp's next item
    }
}

}  // namespace

size_t refine_warp_bytes(int rows, int nt, int n_sym) { return ref_warp_bytes(rows, nt, n_sym); }

cudaError_t launch_refine_batch(const BatchItem *items, const int *start, int n_items,
                                int *counter, int warp_bytes, int grid, cudaStream_t stream)
{
    const size_t smem = (size_t)warp_bytes * kRefWarps;
    cudaError_t e = allow_dynamic_smem(refine_batch_kernel, smem);
    if (e != cudaSuccess) return e;
    refine_batch_kernel<<<grid, kRefWarps * 32, smem, stream>>>(items, start, n_items, counter,
                                                                 warp_bytes);
    return cudaGetLastError();
}

cudaError_t launch_refine(int n_sc, int n_sym, int nr, int nt, float sigma, float threshold,
                          const float2 *H, const float2 *Y, float2 *R, float *inv_diag,
                          uint8_t *perm, float2 *Z, float2 *Q, int *n_refined,
                          cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    const int rows = sigma > 0.f ? nr + nt : nr;
    const int wb = (int)ref_warp_bytes(rows, nt, n_sym);
    const size_t smem = (size_t)wb * kRefWarps;
    cudaError_t e = allow_dynamic_smem(refine_kernel, smem);
    if (e != cudaSuccess) return e;
    const int grid = (n_sc + kRefWarps - 1) / kRefWarps;
    refine_kernel<<<grid, kRefWarps * 32, smem, stream>>>(n_sc, n_sym, nr, nt, (double)sigma,
                                                           threshold, H, Y, R, inv_diag, perm, Z, Q,
                                                           n_refined, wb);
    return cudaGetLastError();
}

}  // namespace mpnl
