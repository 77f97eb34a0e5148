// Channel pre-processing: sorted QR (SQRD) of H and z = Q^H y, one warp per
// subcarrier.
//
// The warp factorises the augmented matrix [H | y_0 ... y_{n_sym-1}] by
// modified Gram-Schmidt: lane c owns column c (columns nt.. are the received
// symbol vectors).  At step i the not-yet-placed channel column with the
// smallest residual norm is picked (tie: lower user index), normalised into
// q_i, and every remaining column -- channel or symbol -- is projected:
// r = q_i^H col, col -= r q_i.  For a channel column r is R_i,col; for a
// symbol column r is z_i = q_i^H y (exact arithmetic gives the same value as
// Q^H y, and Q never has to be stored).  The 14 symbols sharing one channel
// ride along as 14 extra lanes, so Q^H Y costs no extra pass.
//
// H and Y tiles are staged through shared memory with coalesced 8-byte loads;
// the pivot column is broadcast through shared memory.
#include <float.h>

#include "mpnl_common.cuh"
#include "mpnl_internal.h"
#include "qhy_mma.cuh"

namespace mpnl {
namespace {

constexpr int kWarpsPerCta = 4;

struct WarpSmem {
    int off_h, off_y, off_q, off_rt, off_z, off_rd, off_perm, bytes;
};

__host__ __device__ inline WarpSmem warp_smem_layout(int nr, int nt, int n_sym)
{
    WarpSmem s;
    int o = 0;
    s.off_h = o;
    o += nr * nt * 8;
    s.off_y = o;
    o += n_sym * nr * 8;
    s.off_q = o;
    o += (nr + nt) * 8;
    s.off_rt = o;
    o += nt * nt * 8;
    s.off_z = o;
    o += n_sym * nt * 8;
    s.off_rd = o;
    o += nt * 4;
    s.off_perm = o;
    o += nt * 4;
    s.bytes = (o + 15) & ~15;
    return s;
}

// sigma > 0 selects the MMSE-extended variant: the channel columns are
// augmented with sigma * I below the nr antenna rows and the symbol columns
// with zeros (H_a = [H; sigma I], y_a = [y; 0]), so the factorisation has
// nr + nt rows; nr may then be smaller than nt.
// One subcarrier by one warp, in the warp's shared-memory region at byte
// offset base_off of the dynamic shared memory (at least
// warp_smem_layout(nr, nt, n_sym).bytes).  Inlined into the per-call and the batch
// kernels alike (identical arithmetic: no contraction, see the build flags).
template <int NR, int CS>
__device__ __forceinline__ void sqrd_qhy_warp(int sc, int n_sym, int nr, int nt, float sigma,
                                           const float2 *__restrict__ H,
                                           const float2 *__restrict__ Y,
                                           float2 *__restrict__ Rp,
                                           float *__restrict__ inv_diag,
                                           uint8_t *__restrict__ perm_out,
                                           float2 *__restrict__ Z, float2 *__restrict__ Qout,
                                           int base_off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + base_off;
    const int lane = threadIdx.x & 31;
    const WarpSmem L = warp_smem_layout(nr, nt, n_sym);
    float2 *sH = reinterpret_cast<float2 *>(base + L.off_h);
    float2 *sY = reinterpret_cast<float2 *>(base + L.off_y);
    float2 *sQ = reinterpret_cast<float2 *>(base + L.off_q);
    float2 *sRt = reinterpret_cast<float2 *>(base + L.off_rt);
    float2 *sZ = reinterpret_cast<float2 *>(base + L.off_z);
    float *sRd = reinterpret_cast<float *>(base + L.off_rd);
    int *sPerm = reinterpret_cast<int *>(base + L.off_perm);

    // coalesced staging of this subcarrier's H and Y tiles
    const float2 *gH = H + (size_t)sc * nr * nt;
    const float2 *gY = Y + (size_t)sc * n_sym * nr;
    for (int k = lane; k < nr * nt; k += 32) sH[k] = gH[k];
    for (int k = lane; k < n_sym * nr; k += 32) sY[k] = gY[k];
    __syncwarp();

    const int ncols = nt + n_sym;
    const int nra = sigma > 0.f ? nr + nt : nr;  // rows of the (augmented) matrix
    float2 col[CS][NR];
#pragma unroll
    for (int cs = 0; cs < CS; ++cs) {
        const int c = lane + 32 * cs;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            float2 v = make_float2(0.f, 0.f);
            if (r < nr) {
                if (c < nt) v = sH[r * nt + c];
                else if (c < ncols) v = sY[(c - nt) * nr + r];
            } else if (r < nra && c < nt && r - nr == c) {
                v = make_float2(sigma, 0.f);
            }
            col[cs][r] = v;
        }
    }
    // channel columns are always slot 0, lanes 0..nt-1 (nt <= 16)
    bool placed = !(lane < nt);

    for (int i = 0; i < nt; ++i) {
        // placed (or absent) columns carry +inf, live ones a finite key (a NaN
        // norm maps to FLT_MAX), so every lane agrees on the pivot
        float nrm = INFINITY;
        if (!placed) {
            float s = 0.f;
#pragma unroll
            for (int r = 0; r < NR; ++r) s = fmaf(col[0][r].x, col[0][r].x, fmaf(col[0][r].y, col[0][r].y, s));
            nrm = (s <= FLT_MAX) ? s : FLT_MAX;
        }
        // warp argmin of (norm, user index)
        float bn = nrm;
        int bl = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float on = __shfl_xor_sync(0xffffffffu, bn, o);
            int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (on < bn || (on == bn && ol < bl)) {
                bn = on;
                bl = ol;
            }
        }
        const int piv = bl;
        const float rii = sqrtf(bn);
        if (lane == piv) {
            const float inv = 1.0f / rii;
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (r < nra) sQ[r] = make_float2(col[0][r].x * inv, col[0][r].y * inv);
            sRd[i] = rii;
            sPerm[i] = piv;
            placed = true;
        }
        __syncwarp();
        if (Qout != nullptr)  // column i of Q (antenna rows only), for z = Q^H y later
            for (int r = lane; r < nr; r += 32) Qout[((size_t)sc * nr + r) * nt + i] = sQ[r];
#pragma unroll
        for (int cs = 0; cs < CS; ++cs) {
            const int c = lane + 32 * cs;
            // channel columns not yet placed (the pivot was placed just above),
            // and every symbol column
            const bool use = (c < nt) ? !placed : (c < ncols);
            if (use) {
                float ax = 0.f, ay = 0.f;  // q^H col
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (r < nra) {
                        const float2 q = sQ[r];
                        ax = fmaf(q.x, col[cs][r].x, fmaf(q.y, col[cs][r].y, ax));
                        ay = fmaf(q.x, col[cs][r].y, fmaf(-q.y, col[cs][r].x, ay));
                    }
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (r < nra) {
                        const float2 q = sQ[r];
                        col[cs][r].x -= ax * q.x - ay * q.y;
                        col[cs][r].y -= ax * q.y + ay * q.x;
                    }
                }
                if (c < nt) sRt[i * nt + c] = make_float2(ax, ay);
                else sZ[(c - nt) * nt + i] = make_float2(ax, ay);
            }
        }
        __syncwarp();
    }

    // packed R (row-major upper triangle), 1/R_ll, perm, Z
    const int P = nt * (nt + 1) / 2;
    float2 *gR = Rp + (size_t)sc * P;
    for (int k = lane; k < P; k += 32) {
        int i = 0, rem = k;
        while (rem >= nt - i) {
            rem -= nt - i;
            ++i;
        }
        const int j = i + rem;
        gR[k] = (j == i) ? make_float2(sRd[i], 0.f) : sRt[i * nt + sPerm[j]];
    }
    if (lane < nt) {
        inv_diag[(size_t)sc * nt + lane] = 1.0f / sRd[lane];
        perm_out[(size_t)sc * nt + lane] = (uint8_t)sPerm[lane];
    }
    float2 *gZ = Z + (size_t)sc * n_sym * nt;
    for (int k = lane; k < n_sym * nt; k += 32) gZ[k] = sZ[k];
    __syncwarp();  // the region may be reused for the warp's next subcarrier
}

// Six CTAs per SM (at most 85 registers a thread) where that costs next
// to no spills (8 bytes for nr = 16): a 3276-subcarrier slot (819 CTAs)
// then runs in one wave on 152 SMs instead of one full wave and a 7% tail.
template <int NR, int CS>
__global__ void __launch_bounds__(kWarpsPerCta * 32, (NR <= 16 && CS == 1) ? 6 : 1)
sqrd_qhy_kernel(int n_sc, int n_sym, int nr, int nt, float sigma, const float2 *__restrict__ H,
                const float2 *__restrict__ Y, float2 *__restrict__ Rp,
                float *__restrict__ inv_diag, uint8_t *__restrict__ perm_out,
                float2 *__restrict__ Z, float2 *__restrict__ Qout)
{
    const int warp = threadIdx.x >> 5;
    const int sc = blockIdx.x * kWarpsPerCta + warp;
    if (sc >= n_sc) return;  // only __syncwarp inside: per-warp early exit is safe
    const WarpSmem L = warp_smem_layout(nr, nt, n_sym);
    sqrd_qhy_warp<NR, CS>(sc, n_sym, nr, nt, sigma, H, Y, Rp, inv_diag, perm_out, Z, Qout,
                          warp * L.bytes);
}

// Persistent variant over a batch of radio units of mixed sizes: every warp
// takes (unit, subcarrier) work items from a global counter until the batch
// is exhausted and runs the instance that fits the unit's sizes.  `start`
// holds this stage's prefix sums (units outside the stage have none).
__global__ void __launch_bounds__(kWarpsPerCta * 32)
sqrd_qhy_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ start,
                      int n_items, int *__restrict__ counter, int warp_bytes)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int base = warp * warp_bytes;
    const int total = start[n_items];
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(counter, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= total) break;
        const int i = find_item(start, n_items, w);
        const BatchItem &it = items[i];
        const int sc = w - start[i];
        const int ns = it.factor_sym;  // 0: factor only (no symbols ride along)
        const int rows = it.sigma > 0.f ? it.nr + it.nt : it.nr;
        const bool two = it.nt + ns > 32;
#define MPNL_PRE_W(NRV)                                                                          \
    do {                                                                                         \
        if (two)                                                                                 \
            sqrd_qhy_warp<NRV, 2>(sc, ns, it.nr, it.nt, it.sigma, it.H, it.Y, it.R, it.inv_diag, \
                                  it.perm, it.Z, it.Q, base);                                    \
        else                                                                                     \
            sqrd_qhy_warp<NRV, 1>(sc, ns, it.nr, it.nt, it.sigma, it.H, it.Y, it.R, it.inv_diag, \
                                  it.perm, it.Z, it.Q, base);                                    \
    } while (0)
        if (rows <= 4) MPNL_PRE_W(4);
        else if (rows <= 8) MPNL_PRE_W(8);
        else if (rows <= 16) MPNL_PRE_W(16);
        else MPNL_PRE_W(32);
#undef MPNL_PRE_W
    }
}

// z = Q^H y for every symbol of one subcarrier, by one warp: Q (nr x nt)
// and the symbols' y staged in shared memory with coalesced loads, then
// lane k computes outputs (symbol, level) k, k + 32, ... as nr-term complex
// dot products (FP32, explicit FMAs).
__device__ __forceinline__ void qhy_warp(int sc, int n_sym, int nr, int nt,
                                         const float2 *__restrict__ Q,
                                         const float2 *__restrict__ Y, float2 *__restrict__ Z,
                                         int base_off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sQ = reinterpret_cast<float2 *>(smem_raw + base_off);
    float2 *sY = sQ + nr * nt;
    const int lane = threadIdx.x & 31;
    const float2 *gQ = Q + (size_t)sc * nr * nt;
    const float2 *gY = Y + (size_t)sc * n_sym * nr;
    for (int k = lane; k < nr * nt; k += 32) sQ[k] = gQ[k];
    for (int k = lane; k < n_sym * nr; k += 32) sY[k] = gY[k];
    __syncwarp();
    float2 *gZ = Z + (size_t)sc * n_sym * nt;
    for (int k = lane; k < n_sym * nt; k += 32) {
        const int s = k / nt, i = k - s * nt;
        float zx = 0.f, zy = 0.f;  // conj(q) . y
        for (int r = 0; r < nr; ++r) {
            const float2 q = sQ[r * nt + i], y = sY[s * nr + r];
            zx = fmaf(q.x, y.x, fmaf(q.y, y.y, zx));
            zy = fmaf(q.x, y.y, fmaf(-q.y, y.x, zy));
        }
        gZ[k] = make_float2(zx, zy);
    }
    __syncwarp();  // the region may be reused for the warp's next subcarrier
}

__global__ void __launch_bounds__(kWarpsPerCta * 32)
qhy_kernel(int n_sc, int n_sym, int nr, int nt, const float2 *__restrict__ Q,
           const float2 *__restrict__ Y, float2 *__restrict__ Z, int warp_bytes)
{
    const int warp = threadIdx.x >> 5;
    const int sc = blockIdx.x * kWarpsPerCta + warp;
    if (sc >= n_sc) return;
    qhy_warp(sc, n_sym, nr, nt, Q, Y, Z, warp * warp_bytes);
}

__global__ void __launch_bounds__(kWarpsPerCta * 32)
qhy_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ start,
                 int n_items, int *__restrict__ counter, int warp_bytes)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = start[n_items];
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(counter, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= total) break;
        const int i = find_item(start, n_items, w);
        const BatchItem &it = items[i];
        // FP16-residual units take the tensor-core Q^H y of the mixed path
        if (it.f16) qhy_mma_warp(w - start[i], it.n_sym, it.nr, it.nt, it.Q, it.Y, it.Z,
                                 warp * warp_bytes);
        else qhy_warp(w - start[i], it.n_sym, it.nr, it.nt, it.Q, it.Y, it.Z, warp * warp_bytes);
    }
}

template <int NR, int CS>
cudaError_t launch_tpl(int n_sc, int n_sym, int nr, int nt, float sigma, const float2 *H,
                       const float2 *Y, float2 *R, float *inv_diag, uint8_t *perm, float2 *Z,
                       float2 *Q, cudaStream_t stream)
{
    const WarpSmem L = warp_smem_layout(nr, nt, n_sym);
    const size_t smem = (size_t)L.bytes * kWarpsPerCta;
    {
        cudaError_t e = allow_dynamic_smem(sqrd_qhy_kernel<NR, CS>, smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = (n_sc + kWarpsPerCta - 1) / kWarpsPerCta;
    sqrd_qhy_kernel<NR, CS><<<grid, kWarpsPerCta * 32, smem, stream>>>(n_sc, n_sym, nr, nt, sigma,
                                                                       H, Y, R, inv_diag, perm, Z,
                                                                       Q);
    return cudaGetLastError();
}

}  // namespace

size_t preprocess_warp_bytes(int n_sym, int nr, int nt) { return warp_smem_layout(nr, nt, n_sym).bytes; }

size_t qhy_warp_bytes(int n_sym, int nr, int nt)
{
    return (((size_t)nr * nt + (size_t)n_sym * nr) * 8 + 15) & ~(size_t)15;
}

cudaError_t launch_qhy(int n_sc, int n_sym, int nr, int nt, const float2 *Q, const float2 *Y,
                       float2 *Z, cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    const int wb = (int)qhy_warp_bytes(n_sym, nr, nt);
    const size_t smem = (size_t)wb * kWarpsPerCta;
    cudaError_t e = allow_dynamic_smem(qhy_kernel, smem);
    if (e != cudaSuccess) return e;
    const int grid = (n_sc + kWarpsPerCta - 1) / kWarpsPerCta;
    qhy_kernel<<<grid, kWarpsPerCta * 32, smem, stream>>>(n_sc, n_sym, nr, nt, Q, Y, Z, wb);
    return cudaGetLastError();
}

cudaError_t launch_qhy_batch(const BatchItem *items, const int *start, int n_items,
                             int *counter, int warp_bytes, int grid, cudaStream_t stream)
{
    const size_t smem = (size_t)warp_bytes * kWarpsPerCta;
    cudaError_t e = allow_dynamic_smem(qhy_batch_kernel, smem);
    if (e != cudaSuccess) return e;
    qhy_batch_kernel<<<grid, kWarpsPerCta * 32, smem, stream>>>(items, start, n_items, counter,
                                                                warp_bytes);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_batch(const BatchItem *items, const int *start, int n_items,
                                    int *counter, int warp_bytes, int grid, cudaStream_t stream)
{
    const size_t smem = (size_t)warp_bytes * kWarpsPerCta;
    cudaError_t e = allow_dynamic_smem(sqrd_qhy_batch_kernel, smem);
    if (e != cudaSuccess) return e;
    sqrd_qhy_batch_kernel<<<grid, kWarpsPerCta * 32, smem, stream>>>(items, start, n_items, counter,
                                                                     warp_bytes);
    return cudaGetLastError();
}

cudaError_t launch_preprocess(int n_sc, int n_sym, int nr, int nt, float sigma, const float2 *H,
                              const float2 *Y, float2 *R, float *inv_diag, uint8_t *perm,
                              float2 *Z, float2 *Q, cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    const bool two = nt + n_sym > 32;
    const int rows = sigma > 0.f ? nr + nt : nr;
#define MPNL_PRE(NRV)                                                                          \
    return two ? launch_tpl<NRV, 2>(n_sc, n_sym, nr, nt, sigma, H, Y, R, inv_diag, perm, Z, Q, stream) \
               : launch_tpl<NRV, 1>(n_sc, n_sym, nr, nt, sigma, H, Y, R, inv_diag, perm, Z, Q, stream)
    if (rows <= 4) MPNL_PRE(4);
    if (rows <= 8) MPNL_PRE(8);
    if (rows <= 16) MPNL_PRE(16);
    MPNL_PRE(32);
#undef MPNL_PRE
}

}  // namespace mpnl
