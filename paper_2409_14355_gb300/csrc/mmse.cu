// Linear MMSE baseline, one warp per subcarrier (4 subcarriers per CTA).
//
//   A = H^H H + sigma2 I = L L^H        (right-looking Cholesky in shared memory)
//   W = A^{-1} H^H                      (lane r solves for receive column r)
//   (A^{-1})_kk = || L^{-1} e_k ||^2    (lane k)
//   mu_k = (W H)_kk = 1 - sigma2 (A^{-1})_kk  (since W H = I - sigma2 A^{-1})
//   nu_k = (1 - mu_k) / mu_k = sigma2 a_kk / (1 - sigma2 a_kk)
//   x~_k = (W y)_k / mu_k,  one lane per (symbol, user) pair
// The identity for mu avoids the cancellation in 1 - mu at high SNR.  For a
// square Gray QAM the max-log LLR of a bit separates: the other axis
// contributes the same minimum to both hypotheses and cancels, so each LLR is
// a 1-D minimum over the grid points of its own axis.
#include "mpnl_common.cuh"
#include "mpnl_internal.h"

namespace mpnl {
namespace {

constexpr int kWarps = 4;

struct MmseSmem {
    int off_h, off_y, off_l, off_w, off_nu, off_imu, bytes;
};

__host__ __device__ inline MmseSmem mmse_smem_layout(int nr, int nt, int n_sym)
{
    MmseSmem s;
    int o = 0;
    s.off_h = o;
    o += nr * (nt + 1) * 8;  // rows padded by one element: column reads spread over banks
    s.off_y = o;
    o += n_sym * nr * 8;
    s.off_l = o;
    o += nt * (nt + 1) * 8;
    s.off_w = o;
    o += nt * (nr + 1) * 8;
    s.off_nu = o;
    o += nt * 4;
    s.off_imu = o;
    o += nt * 4;
    s.bytes = (o + 15) & ~15;
    return s;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)  // a * conj(b)
{
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// One subcarrier by one warp, in the warp's shared-memory region at byte
// offset base_off (at least mmse_smem_layout(nr, nt, n_sym).bytes).  Inlined
// into the per-call and the batch kernels alike (no contraction).
template <int NT, int QAM>
__device__ __forceinline__ void mmse_warp(int sc, int n_sym, int nr, int nt, float sigma2,
                                       const float2 *__restrict__ H,
                                       const float2 *__restrict__ Y,
                                       uint8_t *__restrict__ hard, float *__restrict__ llr,
                                       int base_off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + base_off;
    constexpr int B = Qam<QAM>::B;
    constexpr int HB = B / 2;
    constexpr int LQ = Qam<QAM>::L;
    const int lane = threadIdx.x & 31;
    const MmseSmem S = mmse_smem_layout(nr, nt, n_sym);
    float2 *sH = reinterpret_cast<float2 *>(base + S.off_h);
    float2 *sY = reinterpret_cast<float2 *>(base + S.off_y);
    float2 *sL = reinterpret_cast<float2 *>(base + S.off_l);  // A, then its Cholesky factor
    float2 *sW = reinterpret_cast<float2 *>(base + S.off_w);
    // row strides, one element longer than the rows: lanes that walk a
    // column (16 lanes reading W rows, H columns, L columns) hit different
    // banks instead of one
    const int ldh = nt + 1, ldl = nt + 1, ldw = nr + 1;
    float *sNu = reinterpret_cast<float *>(base + S.off_nu);
    float *sImu = reinterpret_cast<float *>(base + S.off_imu);

    const float2 *gH = H + (size_t)sc * nr * nt;
    const float2 *gY = Y + (size_t)sc * n_sym * nr;
    for (int k = lane; k < nr * nt; k += 32) {
        const int r = k / nt;
        sH[r * ldh + (k - r * nt)] = gH[k];
    }
    for (int k = lane; k < n_sym * nr; k += 32) sY[k] = gY[k];
    __syncwarp();

    // lower triangle of A = H^H H + sigma2 I
    for (int k = lane; k < nt * nt; k += 32) {
        const int i = k / nt, j = k - i * nt;
        if (j > i) continue;
        float2 a = make_float2(0.f, 0.f);
        for (int r = 0; r < nr; ++r) {
            const float2 hi = sH[r * ldh + i], hj = sH[r * ldh + j];
            a.x = fmaf(hi.x, hj.x, fmaf(hi.y, hj.y, a.x));
            a.y = fmaf(hi.x, hj.y, fmaf(-hi.y, hj.x, a.y));
        }
        if (i == j) a = make_float2(a.x + sigma2, 0.f);
        sL[i * ldl + j] = a;
    }
    __syncwarp();
    // Cholesky, right-looking: at step j column j is finished (L_jj = the
    // square root of the updated diagonal, L_ij = the updated entry / L_jj)
    // and every trailing entry (i, m), i >= m > j, loses L_ij conj(L_mj).  An
    // entry receives its terms in the order 0, 1, ..., as the left-looking
    // recurrence subtracts them, in the same arithmetic (the diagonal's real
    // part loses |L_mj|^2); the trailing updates spread over the lanes.
    for (int j = 0; j < nt; ++j) {
        const float ljj = sqrtf(sL[j * ldl + j].x);
        for (int i = j + 1 + lane; i < nt; i += 32) {
            const float2 t = sL[i * ldl + j];
            sL[i * ldl + j] = make_float2(t.x / ljj, t.y / ljj);
        }
        __syncwarp();
        if (lane == 0) sL[j * ldl + j] = make_float2(ljj, 0.f);
        const int w = nt - 1 - j;  // trailing order
        for (int p = lane; p < w * (w + 1) / 2; p += 32) {
            // p-th trailing entry, row by row: row ii holds ii + 1 entries
            int ii = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
            if ((ii + 1) * (ii + 2) / 2 <= p) ++ii;
            if (ii * (ii + 1) / 2 > p) --ii;
            const int i = j + 1 + ii, m = j + 1 + (p - ii * (ii + 1) / 2);
            const float2 q = cmulc(sL[i * ldl + j], sL[m * ldl + j]);
            float2 v = sL[i * ldl + m];
            v.x -= q.x;
            v.y -= q.y;
            sL[i * ldl + m] = v;
        }
        __syncwarp();
    }
    // W = A^{-1} H^H, lane r handles receive antenna r (column r of H^H)
    for (int r = lane; r < nr; r += 32) {
        float2 u[NT];
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            if (i < nt) {
                const float2 h = sH[r * ldh + i];
                float2 t = make_float2(h.x, -h.y);
#pragma unroll
                for (int k = 0; k < i; ++k) {
                    const float2 p = cmul(sL[i * ldl + k], u[k]);
                    t.x -= p.x;
                    t.y -= p.y;
                }
                const float il = 1.0f / sL[i * ldl + i].x;
                u[i] = make_float2(t.x * il, t.y * il);
            }
        }
#pragma unroll
        for (int i = NT - 1; i >= 0; --i) {
            if (i < nt) {
                float2 t = u[i];
#pragma unroll
                for (int k = i + 1; k < NT; ++k) {
                    if (k < nt) {
                        const float2 p = cmulc(u[k], sL[k * ldl + i]);  // conj(L_ki) v_k
                        t.x -= p.x;
                        t.y -= p.y;
                    }
                }
                const float il = 1.0f / sL[i * ldl + i].x;
                u[i] = make_float2(t.x * il, t.y * il);
                sW[i * ldw + r] = u[i];
            }
        }
    }
    // (A^{-1})_kk from L^{-1} e_k, then nu_k and 1 / mu_k
    if (lane < nt) {
        const int k = lane;
        float2 u[NT];
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            if (i < nt && i >= k) {
                float2 t = make_float2(i == k ? 1.f : 0.f, 0.f);
#pragma unroll
                for (int m = 0; m < i; ++m) {
                    if (m >= k) {
                        const float2 p = cmul(sL[i * ldl + m], u[m]);
                        t.x -= p.x;
                        t.y -= p.y;
                    }
                }
                const float il = 1.0f / sL[i * ldl + i].x;
                u[i] = make_float2(t.x * il, t.y * il);
                acc = fmaf(u[i].x, u[i].x, fmaf(u[i].y, u[i].y, acc));
            } else {
                u[i] = make_float2(0.f, 0.f);
            }
        }
        const float e = sigma2 * acc;  // 1 - mu_k
        sNu[k] = e / (1.0f - e);
        sImu[k] = 1.0f / (1.0f - e);
    }
    __syncwarp();

    // equalise, slice, LLRs: lane per (symbol, user)
    for (int t = lane; t < n_sym * nt; t += 32) {
        const int s = t / nt, k = t - s * nt;
        float2 x = make_float2(0.f, 0.f);
        for (int r = 0; r < nr; ++r) {
            const float2 p = cmul(sW[k * ldw + r], sY[s * nr + r]);
            x.x += p.x;
            x.y += p.y;
        }
        const float imu = sImu[k];
        x.x *= imu;
        x.y *= imu;
        const size_t det = (size_t)sc * n_sym + s;
        float dd;
        const int ire = axis_nearest<QAM>(x.x, dd);
        const int iim = axis_nearest<QAM>(x.y, dd);
        hard[det * nt + k] =
            (uint8_t)join_label<QAM>(Qam<QAM>::axis_label(ire), Qam<QAM>::axis_label(iim));
        if (llr != nullptr) {
            const float inu = 1.0f / sNu[k];
            // squared distances to the axis points, once per axis
            float dx[LQ], dy[LQ];
#pragma unroll
            for (int i = 0; i < LQ; ++i) {
                const float a = x.x - axis_pos<QAM>(i), c = x.y - axis_pos<QAM>(i);
                dx[i] = a * a;
                dy[i] = c * c;
            }
            float lv[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int tb = b >> 1;  // bit position within the axis label, MSB first
                float m0 = INFINITY, m1 = INFINITY;
#pragma unroll
                for (int i = 0; i < LQ; ++i) {
                    const float dv = (b & 1) ? dy[i] : dx[i];
                    if ((Qam<QAM>::axis_label(i) >> (HB - 1 - tb)) & 1) m1 = fminf(m1, dv);
                    else m0 = fminf(m0, dv);
                }
                lv[b] = (m1 - m0) * inu;
            }
            // B is even, so every row is as aligned as the array: pairs when
            // that is 8 bytes (the ABI promises only 4)
            float *row = llr + (det * nt + k) * B;
            if ((reinterpret_cast<uintptr_t>(llr) & 7u) == 0) {
#pragma unroll
                for (int b = 0; b < B; b += 2)
                    reinterpret_cast<float2 *>(row)[b >> 1] = make_float2(lv[b], lv[b + 1]);
            } else {
#pragma unroll
                for (int b = 0; b < B; ++b) row[b] = lv[b];
            }
        }
    }
    __syncwarp();  // the region may be reused for the warp's next subcarrier
}

template <int NT, int QAM>
__global__ void __launch_bounds__(kWarps * 32, 4)
mmse_kernel(int n_sc, int n_sym, int nr, int nt, float sigma2, const float2 *__restrict__ H,
            const float2 *__restrict__ Y, uint8_t *__restrict__ hard, float *__restrict__ llr)
{
    const int warp = threadIdx.x >> 5;
    const int sc = blockIdx.x * kWarps + warp;
    if (sc >= n_sc) return;  // warp-local work only
    const MmseSmem S = mmse_smem_layout(nr, nt, n_sym);
    mmse_warp<NT, QAM>(sc, n_sym, nr, nt, sigma2, H, Y, hard, llr, warp * S.bytes);
}

template <int NT>
__device__ __forceinline__ void mmse_warp_qam(const BatchItem &it, int sc, int base)
{
    switch (it.qam) {
    case 4: mmse_warp<NT, 4>(sc, it.n_sym, it.nr, it.nt, it.sigma2, it.H, it.Y, it.mmse_hard, it.mmse_llr, base); break;
    case 16: mmse_warp<NT, 16>(sc, it.n_sym, it.nr, it.nt, it.sigma2, it.H, it.Y, it.mmse_hard, it.mmse_llr, base); break;
    default: mmse_warp<NT, 64>(sc, it.n_sym, it.nr, it.nt, it.sigma2, it.H, it.Y, it.mmse_hard, it.mmse_llr, base); break;
    }
}

// Persistent variant over a batch of radio units of mixed sizes (units
// without the baseline are skipped).
__global__ void __launch_bounds__(kWarps * 32, 4)
mmse_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ start, int n_items,
                  int *__restrict__ counter, int warp_bytes)
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
        if (!it.mmse) continue;
        const int sc = w - start[i];
        if (it.nt <= 4) mmse_warp_qam<4>(it, sc, base);
        else if (it.nt <= 8) mmse_warp_qam<8>(it, sc, base);
        else mmse_warp_qam<16>(it, sc, base);
    }
}

template <int NT, int QAM>
cudaError_t launch_tpl(int n_sc, int n_sym, int nr, int nt, float sigma2, const float2 *H,
                       const float2 *Y, uint8_t *hard, float *llr, cudaStream_t stream)
{
    const MmseSmem S = mmse_smem_layout(nr, nt, n_sym);
    const size_t smem = (size_t)S.bytes * kWarps;
    {
        cudaError_t e = allow_dynamic_smem(mmse_kernel<NT, QAM>, smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = (n_sc + kWarps - 1) / kWarps;
    mmse_kernel<NT, QAM><<<grid, kWarps * 32, smem, stream>>>(n_sc, n_sym, nr, nt, sigma2, H, Y,
                                                              hard, llr);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_nt(int qam, int n_sc, int n_sym, int nr, int nt, float sigma2,
                      const float2 *H, const float2 *Y, uint8_t *hard, float *llr,
                      cudaStream_t stream)
{
    switch (qam) {
    case 4: return launch_tpl<NT, 4>(n_sc, n_sym, nr, nt, sigma2, H, Y, hard, llr, stream);
    case 16: return launch_tpl<NT, 16>(n_sc, n_sym, nr, nt, sigma2, H, Y, hard, llr, stream);
    default: return launch_tpl<NT, 64>(n_sc, n_sym, nr, nt, sigma2, H, Y, hard, llr, stream);
    }
}

}  // namespace

size_t mmse_warp_bytes(int n_sym, int nr, int nt) { return mmse_smem_layout(nr, nt, n_sym).bytes; }

cudaError_t launch_mmse_batch(const BatchItem *items, const int *start, int n_items,
                              int *counter, int warp_bytes, int grid, cudaStream_t stream)
{
    const size_t smem = (size_t)warp_bytes * kWarps;
    cudaError_t e = allow_dynamic_smem(mmse_batch_kernel, smem);
    if (e != cudaSuccess) return e;
    mmse_batch_kernel<<<grid, kWarps * 32, smem, stream>>>(items, start, n_items, counter,
                                                           warp_bytes);
    return cudaGetLastError();
}

cudaError_t launch_mmse(int n_sc, int n_sym, int nr, int nt, int qam, float sigma2,
                        const float2 *H, const float2 *Y, uint8_t *hard, float *llr,
                        cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    if (nt <= 4) return launch_nt<4>(qam, n_sc, n_sym, nr, nt, sigma2, H, Y, hard, llr, stream);
    if (nt <= 8) return launch_nt<8>(qam, n_sc, n_sym, nr, nt, sigma2, H, Y, hard, llr, stream);
    return launch_nt<16>(qam, n_sc, n_sym, nr, nt, sigma2, H, Y, hard, llr, stream);
}

}  // namespace mpnl
