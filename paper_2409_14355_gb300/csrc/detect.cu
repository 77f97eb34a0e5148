// Evaluation of the N_pe position vectors: one CTA per subcarrier, one thread
// per (row of the table) walk, looping over the subcarrier's OFDM symbols so
// that R, 1/R_ll, perm and the table are staged once and reused 14 times.
//
// Walk of row p for symbol z (all in registers):
//   e := z
//   for l = nt-1 .. 0:
//     b   = e_l / R_ll
//     s_l = the p_l-th closest constellation point to b (distance, then label)
//     d  += R_ll^2 |b - s_l|^2
//     e_i -= R_il s_l   for every i < l   (interference of the new decision)
// R is read column by column from shared memory; every lane of a warp reads
// the same element at the same time (broadcast), so the loads cost one
// shared-memory wavefront each.
//
// Reductions per symbol, all in shared memory:
//   argmin of (d, row)     : one 64-bit atomicMin per walk
//   runner-up d            : warp redux + one atomicMin per warp
//   max-log LLR minima     : per (level, bit, bit value) a warp redux
//                            (__reduce_min_sync on the float bits, valid for
//                            d >= 0) and one shared atomicMin per warp.
#include "mpnl_common.cuh"
#include "mpnl_internal.h"

namespace mpnl {
namespace {

// p-th closest point (p >= 1) of the square constellation to b = (bx, by),
// ordered by (squared distance, label).  Returns the squared distance and the
// point's label and coordinates.
//
// p == 1 is plain per-axis slicing.  For p > 1 each axis is first ordered by
// distance (ties: smaller axis label) by walking outwards from the nearest
// grid point; the 2-D order is then enumerated over the "staircase" of
// (row i, column j) pairs: popping (i, j) exposes (i, j + 1), and popping
// (i, 0) also exposes (i + 1, 0).  Each pair's parent sorts no later than the
// pair itself, so p pops give the p-th point exactly.
template <int QAM>
__device__ __forceinline__ float kth_point(float bx, float by, int p, int &label, float &sx,
                                           float &sy)
{
    constexpr int L = Qam<QAM>::L;
    float dre0, dim0;
    const int ire = axis_nearest<QAM>(bx, dre0);
    const int iim = axis_nearest<QAM>(by, dim0);
    if (p == 1) {
        label = join_label<QAM>(Qam<QAM>::axis_label(ire), Qam<QAM>::axis_label(iim));
        sx = axis_pos<QAM>(ire);
        sy = axis_pos<QAM>(iim);
        return dre0 + dim0;
    }
    int ore[L], oim[L];
    float dre[L], dim[L];
    ore[0] = ire;
    dre[0] = dre0;
    oim[0] = iim;
    dim[0] = dim0;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        const float x = ax == 0 ? bx : by;
        int *ord = ax == 0 ? ore : oim;
        float *dd = ax == 0 ? dre : dim;
        int lo = ord[0] - 1, hi = ord[0] + 1;
        for (int n = 1; n < L; ++n) {
            float dl = INFINITY, dh = INFINITY;
            if (lo >= 0) {
                dl = x - axis_pos<QAM>(lo);
                dl *= dl;
            }
            if (hi < L) {
                dh = x - axis_pos<QAM>(hi);
                dh *= dh;
            }
            bool take_lo;
            if (lo < 0) take_lo = false;
            else if (hi >= L) take_lo = true;
            else take_lo = dl < dh || (dl == dh && Qam<QAM>::axis_label(lo) < Qam<QAM>::axis_label(hi));
            if (take_lo) {
                ord[n] = lo;
                dd[n] = dl;
                --lo;
            } else {
                ord[n] = hi;
                dd[n] = dh;
                ++hi;
            }
        }
    }
    int col[L];
    col[0] = 0;
    int na = 1;
    int ba = 0;
    float bd = 0.f;
    int blab = 0;
    for (int pop = 1; pop <= p; ++pop) {
        ba = -1;
        bd = INFINITY;
        blab = 0x7fffffff;
        for (int a = 0; a < na; ++a) {
            if (col[a] >= L) continue;
            const float dv = dre[a] + dim[col[a]];
            const int lv = join_label<QAM>(Qam<QAM>::axis_label(ore[a]),
                                           Qam<QAM>::axis_label(oim[col[a]]));
            if (ba < 0 || dv < bd || (dv == bd && lv < blab)) {  // ba < 0: NaN-safe
                bd = dv;
                blab = lv;
                ba = a;
            }
        }
        if (pop == p) break;
        if (col[ba] == 0 && ba == na - 1 && na < L) {
            col[na] = 0;
            ++na;
        }
        ++col[ba];
    }
    label = blab;
    sx = axis_pos<QAM>(ore[ba]);
    sy = axis_pos<QAM>(oim[col[ba]]);
    return bd;
}

struct DetSmem {
    int off_rc, off_r2, off_invd, off_z, off_perm, off_tab, off_d, off_lab, off_slot, bytes;
};

__host__ __device__ inline int align16(int o) { return (o + 15) & ~15; }

__host__ __device__ inline DetSmem det_smem_layout(int NT, int B, int n_pe)
{
    DetSmem s;
    int o = 0;
    s.off_rc = o;
    o = align16(o + NT * NT * 8);
    s.off_z = o;
    o = align16(o + NT * 8);
    s.off_r2 = o;
    o = align16(o + NT * 4);
    s.off_invd = o;
    o = align16(o + NT * 4);
    s.off_perm = o;
    o = align16(o + NT * 4);
    s.off_slot = o;
    o = align16(o + NT * B * 2 * 4);
    s.off_d = o;
    o = align16(o + n_pe * 4);
    s.off_tab = o;  // rows of NT bytes, 16-byte aligned base
    o = align16(o + n_pe * NT);
    s.off_lab = o;
    o = align16(o + n_pe * NT);
    s.bytes = o;
    return s;
}

// The NT rank bytes of one table row, read from shared memory with one
// vector load (NT is 4, 8 or 16, and rows are NT-byte aligned).
template <int NT>
struct RowRanks {
    uint32_t w[NT / 4];
    __device__ __forceinline__ void load(const uint8_t *row)
    {
        if constexpr (NT == 16) {
            const uint4 v = *reinterpret_cast<const uint4 *>(row);
            w[0] = v.x;
            w[1] = v.y;
            w[2] = v.z;
            w[3] = v.w;
        } else if constexpr (NT == 8) {
            const uint2 v = *reinterpret_cast<const uint2 *>(row);
            w[0] = v.x;
            w[1] = v.y;
        } else {
            w[0] = *reinterpret_cast<const uint32_t *>(row);
        }
    }
    __device__ __forceinline__ int get(int l) const { return (w[l >> 2] >> (8 * (l & 3))) & 0xff; }
};

template <int NT, int QAM>
__global__ void __launch_bounds__(256, 2)
detect_walk_kernel(int n_sym, int nt, int n_pe, float sigma2, const float2 *__restrict__ Rp,
                   const float *__restrict__ inv_diag, const uint8_t *__restrict__ perm,
                   const uint8_t *__restrict__ paths, const float2 *__restrict__ Z,
                   uint8_t *__restrict__ hard, float *__restrict__ llr, float *__restrict__ ped2,
                   unsigned *__restrict__ status)
{
    constexpr int B = Qam<QAM>::B;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long s_best;
    __shared__ unsigned s_second;

    const DetSmem S = det_smem_layout(NT, B, n_pe);
    float2 *sRc = reinterpret_cast<float2 *>(smem_raw + S.off_rc);  // sRc[l*NT+i] = R[i][l], i < l
    float2 *sZ = reinterpret_cast<float2 *>(smem_raw + S.off_z);
    float *sR2 = reinterpret_cast<float *>(smem_raw + S.off_r2);
    float *sInvd = reinterpret_cast<float *>(smem_raw + S.off_invd);
    int *sPerm = reinterpret_cast<int *>(smem_raw + S.off_perm);
    unsigned *sSlot = reinterpret_cast<unsigned *>(smem_raw + S.off_slot);
    float *sD = reinterpret_cast<float *>(smem_raw + S.off_d);
    uint8_t *sTab = smem_raw + S.off_tab;
    uint8_t *sLab = smem_raw + S.off_lab;

    const int sc = blockIdx.x;
    const int tid = threadIdx.x;
    const int T = blockDim.x;
    const int lane = tid & 31;

    // ---- stage the subcarrier's R, 1/R_ll, perm and position-vector table
    const int P = nt * (nt + 1) / 2;
    for (int k = tid; k < P; k += T) {
        int i = 0, rem = k;
        while (rem >= nt - i) {
            rem -= nt - i;
            ++i;
        }
        const int j = i + rem;
        const float2 v = Rp[(size_t)sc * P + k];
        if (i == j) sR2[i] = v.x * v.x;
        else sRc[j * NT + i] = v;
    }
    if (tid < nt) {
        sInvd[tid] = inv_diag[(size_t)sc * nt + tid];
        sPerm[tid] = perm[(size_t)sc * nt + tid];
    }
    for (int k = tid; k < n_pe * NT; k += T) sTab[k] = 1;  // padding levels >= nt
    __syncthreads();
    for (int k = tid; k < n_pe * nt; k += T) {
        const int r = k / nt, l = k - r * nt;
        int v = paths[(size_t)sc * n_pe * nt + k];
        if (v < 1 || v > QAM) {
            atomicOr(status, kStatusBadPathEntry);
            v = v < 1 ? 1 : QAM;
        }
        sTab[r * NT + l] = (uint8_t)v;
    }
    __syncthreads();

    for (int sym = 0; sym < n_sym; ++sym) {
        const size_t det = (size_t)sc * n_sym + sym;
        if (tid < nt) sZ[tid] = Z[det * nt + tid];
        for (int k = tid; k < NT * B * 2; k += T) sSlot[k] = kInfBits;
        if (tid == 0) {
            s_best = ~0ull;
            s_second = kInfBits;
        }
        __syncthreads();

        for (int base = 0; base < n_pe; base += T) {
            const int row = base + tid;
            const bool active = row < n_pe;
            float d = INFINITY;
            int lab[NT];
#pragma unroll
            for (int l = 0; l < NT; ++l) lab[l] = 0;
            if (active) {
                RowRanks<NT> pr;
                pr.load(sTab + row * NT);
                float2 e[NT];
#pragma unroll
                for (int l = 0; l < NT; ++l) e[l] = l < nt ? sZ[l] : make_float2(0.f, 0.f);
                d = 0.f;
#pragma unroll
                for (int l = NT - 1; l >= 0; --l) {
                    if (l < nt) {
                        const float iv = sInvd[l];
                        const float bx = e[l].x * iv, by = e[l].y * iv;
                        float sx, sy;
                        int lb;
                        const float dist = kth_point<QAM>(bx, by, pr.get(l), lb, sx, sy);
                        d = fmaf(sR2[l], dist, d);
                        lab[l] = lb;
#pragma unroll
                        for (int i = 0; i < l; ++i) {
                            const float2 r = sRc[l * NT + i];
                            e[i].x -= r.x * sx - r.y * sy;
                            e[i].y -= r.x * sy + r.y * sx;
                        }
                    }
                }
                sD[row] = d;
#pragma unroll
                for (int l = 0; l < NT; ++l)
                    if (l < nt) sLab[row * NT + l] = (uint8_t)lab[l];
                atomicMin(&s_best, ((unsigned long long)fbits(d) << 32) | (unsigned)row);
            }
            if (llr != nullptr) {
                const unsigned db = active ? fbits(d) : kInfBits;
#pragma unroll
                for (int l = 0; l < NT; ++l) {
                    if (l < nt) {
#pragma unroll
                        for (int b = 0; b < B; ++b) {
                            const bool one = (lab[l] >> (B - 1 - b)) & 1;
                            const unsigned m0 = __reduce_min_sync(0xffffffffu, one ? kInfBits : db);
                            const unsigned m1 = __reduce_min_sync(0xffffffffu, one ? db : kInfBits);
                            if (lane == 0) {
                                atomicMin(&sSlot[(l * B + b) * 2], m0);
                                atomicMin(&sSlot[(l * B + b) * 2 + 1], m1);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();

        const int best_row = (int)(s_best & 0xffffffffull);
        if (ped2 != nullptr) {
            for (int base = 0; base < n_pe; base += T) {
                const int row = base + tid;
                const unsigned v = (row < n_pe && row != best_row) ? fbits(sD[row]) : kInfBits;
                const unsigned m = __reduce_min_sync(0xffffffffu, v);
                if (lane == 0) atomicMin(&s_second, m);
            }
            __syncthreads();
            if (tid == 0) {
                ped2[det * 2] = sD[best_row];
                ped2[det * 2 + 1] = __uint_as_float(s_second);
            }
        }
        if (tid < nt) hard[det * nt + sPerm[tid]] = sLab[best_row * NT + tid];
        if (llr != nullptr) {
            for (int k = tid; k < nt * B; k += T) {
                const int l = k / B, b = k - l * B;
                const unsigned m0 = sSlot[(l * B + b) * 2], m1 = sSlot[(l * B + b) * 2 + 1];
                float v;
                if (m1 == kInfBits) v = kLlrMax;
                else if (m0 == kInfBits) v = -kLlrMax;
                else v = (__uint_as_float(m1) - __uint_as_float(m0)) / sigma2;
                llr[(det * nt + sPerm[l]) * B + b] = v;
            }
        }
        __syncthreads();
    }
}

template <int NT, int QAM>
cudaError_t launch_tpl(int n_sc, int n_sym, int nt, int n_pe, float sigma2, const float2 *R,
                       const float *inv_diag, const uint8_t *perm, const uint8_t *paths,
                       const float2 *Z, uint8_t *hard, float *llr, float *ped2, unsigned *status,
                       cudaStream_t stream)
{
    const DetSmem S = det_smem_layout(NT, Qam<QAM>::B, n_pe);
    const size_t smem = S.bytes;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(detect_walk_kernel<NT, QAM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int threads = ((n_pe + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    detect_walk_kernel<NT, QAM><<<n_sc, threads, smem, stream>>>(
        n_sym, nt, n_pe, sigma2, R, inv_diag, perm, paths, Z, hard, llr, ped2, status);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_nt(int qam, int n_sc, int n_sym, int nt, int n_pe, float sigma2,
                      const float2 *R, const float *inv_diag, const uint8_t *perm,
                      const uint8_t *paths, const float2 *Z, uint8_t *hard, float *llr,
                      float *ped2, unsigned *status, cudaStream_t stream)
{
    switch (qam) {
    case 4:
        return launch_tpl<NT, 4>(n_sc, n_sym, nt, n_pe, sigma2, R, inv_diag, perm, paths, Z, hard,
                                 llr, ped2, status, stream);
    case 16:
        return launch_tpl<NT, 16>(n_sc, n_sym, nt, n_pe, sigma2, R, inv_diag, perm, paths, Z, hard,
                                  llr, ped2, status, stream);
    default:
        return launch_tpl<NT, 64>(n_sc, n_sym, nt, n_pe, sigma2, R, inv_diag, perm, paths, Z, hard,
                                  llr, ped2, status, stream);
    }
}

}  // namespace

cudaError_t launch_detect(int n_sc, int n_sym, int nt, int qam, int n_pe, float sigma2,
                          const float2 *R, const float *inv_diag, const uint8_t *perm,
                          const uint8_t *paths, const float2 *Z, uint8_t *hard, float *llr,
                          float *ped2, unsigned *status, cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    if (nt <= 4)
        return launch_nt<4>(qam, n_sc, n_sym, nt, n_pe, sigma2, R, inv_diag, perm, paths, Z, hard,
                            llr, ped2, status, stream);
    if (nt <= 8)
        return launch_nt<8>(qam, n_sc, n_sym, nt, n_pe, sigma2, R, inv_diag, perm, paths, Z, hard,
                            llr, ped2, status, stream);
    return launch_nt<16>(qam, n_sc, n_sym, nt, n_pe, sigma2, R, inv_diag, perm, paths, Z, hard,
                         llr, ped2, status, stream);
}

}  // namespace mpnl
