// Evaluation of the N_pe position vectors of every (subcarrier, symbol):
// SIC / partial-Euclidean-distance walks, argmin, max-log LLRs.
//
// One CTA per subcarrier; R, 1/R_ll, perm, the table and the subcarrier's 14
// z vectors are staged in shared memory once.  A warp takes 32 rows of the
// table for one symbol; each lane runs one walk with its whole state in
// registers:
//
//   e := z
//   for l = nt-1 .. 0:
//     b   = e_l / R_ll
//     s_l = the p_l-th closest constellation point to b (distance, then label)
//     d  += R_ll^2 |b - s_l|^2
//     e_i -= R_il s_l   for every i < l          (4 FFMA per complex term)
//
// Column l of R is read with 16-byte shared loads that every lane of the warp
// issues for the same address (one broadcast wavefront per two complex
// entries).  Rank 1 (the SIC choice, most entries of the table) is plain
// per-axis slicing; higher ranks enumerate the nearest points in order.
//
// Reductions, without contended atomics:
//   warp:  argmin key (d, row) by shuffles; runner-up d and, for every
//          (level, bit), the minimum d over the warp's rows whose bit differs
//          from the warp-best row's bit, by redux.sync;
//   CTA:   per (symbol, level, bit, value) a u32 atomicMin on shared memory
//          (one per warp, distinct addresses across lanes); per symbol a
//          64-bit atomicMin on the argmin key (one per warp);
//   final: one thread per (symbol, level, bit) forms the LLR.
#include "mpnl_common.cuh"
#include "mpnl_internal.h"

namespace mpnl {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// --------------------------------------------------------------------------
// ranking: p-th closest constellation point
// --------------------------------------------------------------------------

// Grid indices of one axis in order of distance to x: the nearest index i0,
// then alternately one step towards x and one step away, until one side runs
// out, then the rest of the longer side.  (For x within half a spacing of
// grid point i0 the distances grow as f, 2 - f, 2 + f, 4 - f, ... in
// half-spacing units, f <= 1, so the zig-zag is the sorted order.)
template <int QAM>
struct AxisOrder {
    int i0, s, m, lon;
    __device__ __forceinline__ AxisOrder(float x, int nearest)
    {
        constexpr int L = Qam<QAM>::L;
        i0 = nearest;
        s = (x >= axis_pos<QAM>(i0)) ? 1 : -1;
        const int a = s > 0 ? L - 1 - i0 : i0;  // room on the near side
        const int c = L - 1 - a;                  // room on the far side
        m = a < c ? a : c;
        lon = a > c ? s : -s;                     // direction of the longer side
    }
    __device__ __forceinline__ int idx(int n) const
    {
        if (n <= 2 * m) {
            const int k = (n + 1) >> 1;
            return (n & 1) ? i0 + s * k : i0 - s * k;
        }
        return i0 + lon * (n - m);
    }
};

template <int QAM>
__device__ __forceinline__ int grid_label(int ire, int iim)
{
    return join_label<QAM>(Qam<QAM>::axis_label(ire), Qam<QAM>::axis_label(iim));
}

// p-th closest point (p >= 1) to b = (bx, by) by (squared distance, label);
// returns the squared distance, writes the label and the coordinates.
// p == 1 is per-axis slicing.  Otherwise the 2-D order is enumerated over the
// "staircase" of (row a, column c) pairs of the two axis orders: popping
// (a, c) exposes (a, c + 1), popping (a, 0) also exposes (a + 1, 0); every
// pair's predecessor sorts no later, so p pops reach the p-th point.  The
// per-row column pointers are packed 4 bits each in one register.
template <int QAM>
__device__ __forceinline__ float kth_point(float bx, float by, int p, int &label, float &sx,
                                           float &sy)
{
    constexpr int L = Qam<QAM>::L;
    float dre, dim;
    const int ire = axis_nearest<QAM>(bx, dre);
    const int iim = axis_nearest<QAM>(by, dim);
    if (p <= 1) {
        label = grid_label<QAM>(ire, iim);
        sx = axis_pos<QAM>(ire);
        sy = axis_pos<QAM>(iim);
        return dre + dim;
    }
    const AxisOrder<QAM> ore(bx, ire), oim(by, iim);
    unsigned cols = 0;
    int na = 1;
    int ba = 0, bi = ire, bj = iim;
    float bd = 0.f;
    for (int pop = 1; pop <= QAM; ++pop) {
        ba = -1;
        bd = INFINITY;
        int blab = 0;
        for (int a = 0; a < na; ++a) {
            const int c = (cols >> (4 * a)) & 0xF;
            if (c >= L) continue;
            const int ia = ore.idx(a), ic = oim.idx(c);
            const float dx = bx - axis_pos<QAM>(ia), dy = by - axis_pos<QAM>(ic);
            const float v = dx * dx + dy * dy;
            bool take = ba < 0 || v < bd;  // ba < 0 takes the first candidate (NaN-safe)
            if (!take && v == bd) {        // exact tie: lower label first
                if (blab < 0) blab = grid_label<QAM>(bi, bj);
                take = grid_label<QAM>(ia, ic) < blab;
            }
            if (take) {
                ba = a;
                bi = ia;
                bj = ic;
                bd = v;
                blab = -1;
            }
        }
        if (pop >= p) break;
        const int bc = (cols >> (4 * ba)) & 0xF;
        if (bc == 0 && ba == na - 1 && na < L) ++na;
        cols += 1u << (4 * ba);
    }
    label = grid_label<QAM>(bi, bj);
    sx = axis_pos<QAM>(bi);
    sy = axis_pos<QAM>(bj);
    return bd;
}

// --------------------------------------------------------------------------
// per-walk state helpers
// --------------------------------------------------------------------------

// The NT rank bytes of one table row (rows are NT-byte aligned in shared memory).
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

// Labels of the NT levels of one walk, B bits each, packed into 32-bit words.
template <int NT, int B>
struct Labels {
    static constexpr int PER = 32 / B;                  // levels per word
    static constexpr int WORDS = (NT + PER - 1) / PER;
    uint32_t w[WORDS];
    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int k = 0; k < WORDS; ++k) w[k] = 0;
    }
    __device__ __forceinline__ void set(int l, int lab) { w[l / PER] |= (uint32_t)lab << (B * (l % PER)); }
    __device__ __forceinline__ int get(int l) const { return (w[l / PER] >> (B * (l % PER))) & ((1 << B) - 1); }
};

__host__ __device__ inline int a16(int o) { return (o + 15) & ~15; }

struct DetSmem {
    int off_rc, off_r2, off_invd, off_perm, off_z, off_tab, off_m, off_best, off_wmin,
        off_second, off_blab, bytes;
};

__host__ __device__ inline DetSmem det_layout(int NT, int B, int n_pe, int n_sym, int WORDS)
{
    const int chunks = (n_pe + 31) / 32;
    DetSmem s;
    int o = 0;
    s.off_rc = o;
    o = a16(o + NT * NT * 8);
    s.off_r2 = o;
    o = a16(o + NT * 4);
    s.off_invd = o;
    o = a16(o + NT * 4);
    s.off_perm = o;
    o = a16(o + NT * 4);
    s.off_z = o;
    o = a16(o + n_sym * NT * 8);
    s.off_tab = o;
    o = a16(o + chunks * 32 * NT);
    s.off_m = o;
    o = a16(o + n_sym * NT * B * 2 * 4);
    s.off_best = o;
    o = a16(o + n_sym * 8);
    s.off_wmin = o;
    o = a16(o + n_sym * chunks * 4);
    s.off_second = o;
    o = a16(o + n_sym * chunks * 4);
    s.off_blab = o;
    o = a16(o + n_sym * chunks * WORDS * 4);
    s.bytes = o;
    return s;
}

template <int NT, int QAM>
__global__ void __launch_bounds__(kThreads, 2)
detect_walk_kernel(int n_sym, int nt, int n_pe, float sigma2, const float2 *__restrict__ Rp,
                   const float *__restrict__ inv_diag, const uint8_t *__restrict__ perm,
                   const uint8_t *__restrict__ paths, const float2 *__restrict__ Z,
                   uint8_t *__restrict__ hard, float *__restrict__ llr, float *__restrict__ ped2,
                   unsigned *__restrict__ status)
{
    constexpr int B = Qam<QAM>::B;
    using Lab = Labels<NT, B>;
    constexpr int WORDS = Lab::WORDS;
    extern __shared__ __align__(16) unsigned char smem[];
    const int chunks = (n_pe + 31) / 32;
    const DetSmem S = det_layout(NT, B, n_pe, n_sym, WORDS);
    float2 *sRc = reinterpret_cast<float2 *>(smem + S.off_rc);  // sRc[l*NT + i] = R_il, i < l
    float *sR2 = reinterpret_cast<float *>(smem + S.off_r2);
    float *sInvd = reinterpret_cast<float *>(smem + S.off_invd);
    int *sPerm = reinterpret_cast<int *>(smem + S.off_perm);
    float2 *sZ = reinterpret_cast<float2 *>(smem + S.off_z);
    uint8_t *sTab = smem + S.off_tab;
    unsigned *sM = reinterpret_cast<unsigned *>(smem + S.off_m);
    unsigned long long *sBest = reinterpret_cast<unsigned long long *>(smem + S.off_best);
    unsigned *sWmin = reinterpret_cast<unsigned *>(smem + S.off_wmin);
    unsigned *sSecond = reinterpret_cast<unsigned *>(smem + S.off_second);
    uint32_t *sBlab = reinterpret_cast<uint32_t *>(smem + S.off_blab);

    const int sc = blockIdx.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;

    // ---- stage the subcarrier
    const int P = nt * (nt + 1) / 2;
    for (int k = tid; k < P; k += kThreads) {
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
    for (int k = tid; k < NT; k += kThreads) {
        if (k < nt) {
            sInvd[k] = inv_diag[(size_t)sc * nt + k];
            sPerm[k] = perm[(size_t)sc * nt + k];
        }
    }
    for (int k = tid; k < n_sym * nt; k += kThreads)
        sZ[(k / nt) * NT + (k % nt)] = Z[(size_t)sc * n_sym * nt + k];
    for (int k = tid; k < chunks * 32 * NT; k += kThreads) {
        const int r = k / NT, l = k - r * NT;
        int v = 1;  // padding rows and levels: rank 1
        if (r < n_pe && l < nt) {
            v = paths[((size_t)sc * n_pe + r) * nt + l];
            if (v < 1 || v > QAM) {
                atomicOr(status, kStatusBadPathEntry);
                v = v < 1 ? 1 : QAM;
            }
        }
        sTab[k] = (uint8_t)v;
    }
    for (int k = tid; k < n_sym * NT * B * 2; k += kThreads) sM[k] = kInfBits;
    for (int k = tid; k < n_sym; k += kThreads) sBest[k] = ~0ull;
    __syncthreads();

    // ---- walks: warp item = (chunk of 32 rows, symbol)
    for (int item = warp; item < chunks * n_sym; item += kWarps) {
        const int chunk = item / n_sym, s = item - chunk * n_sym;
        const int row = chunk * 32 + lane;
        const bool active = row < n_pe;
        RowRanks<NT> pr;
        pr.load(sTab + row * NT);
        float ex[NT], ey[NT];
#pragma unroll
        for (int l = 0; l < NT; ++l) {
            const float2 z = sZ[s * NT + l];
            ex[l] = z.x;
            ey[l] = z.y;
        }
        Lab lab;
        lab.clear();
        float d = 0.f;
#pragma unroll
        for (int l = NT - 1; l >= 0; --l) {
            if (l < nt) {
                const float iv = sInvd[l];
                int lb;
                float sx, sy;
                const float dist = kth_point<QAM>(ex[l] * iv, ey[l] * iv, pr.get(l), lb, sx, sy);
                d = fmaf(sR2[l], dist, d);
                lab.set(l, lb);
                const float4 *col = reinterpret_cast<const float4 *>(sRc + l * NT);
#pragma unroll
                for (int i2 = 0; i2 < NT / 2; ++i2) {
                    if (2 * i2 < l) {
                        const float4 r = col[i2];  // R_{2i2,l}, R_{2i2+1,l}
                        ex[2 * i2] = fmaf(-r.x, sx, fmaf(r.y, sy, ex[2 * i2]));
                        ey[2 * i2] = fmaf(-r.x, sy, fmaf(-r.y, sx, ey[2 * i2]));
                        if (2 * i2 + 1 < l) {
                            ex[2 * i2 + 1] = fmaf(-r.z, sx, fmaf(r.w, sy, ex[2 * i2 + 1]));
                            ey[2 * i2 + 1] = fmaf(-r.z, sy, fmaf(-r.w, sx, ey[2 * i2 + 1]));
                        }
                    }
                }
            }
        }

        // warp argmin of (d, row)
        const unsigned db = active ? fbits(d) : kInfBits;
        unsigned long long key = active ? (((unsigned long long)db << 32) | (unsigned)row) : ~0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
            key = k2 < key ? k2 : key;
        }
        const int blane = (int)(key & 0xffffffffull) - chunk * 32;
        const unsigned wmin = (unsigned)(key >> 32);
        const unsigned second = __reduce_min_sync(0xffffffffu, lane == blane ? kInfBits : db);
        Lab bl;
#pragma unroll
        for (int k = 0; k < WORDS; ++k) bl.w[k] = __shfl_sync(0xffffffffu, lab.w[k], blane & 31);
        if (lane == 0) {
            atomicMin(&sBest[s], key);
            sWmin[s * chunks + chunk] = wmin;
            sSecond[s * chunks + chunk] = second;
#pragma unroll
            for (int k = 0; k < WORDS; ++k) sBlab[(s * chunks + chunk) * WORDS + k] = bl.w[k];
        }
        if (llr != nullptr) {
            // per (level, bit): the warp-best row's bit value bb has minimum
            // wmin; the other value's minimum comes from one redux
            unsigned mine_other[3] = {kInfBits, kInfBits, kInfBits};
            int mine_bb[3] = {0, 0, 0};
#pragma unroll
            for (int l = 0; l < NT; ++l) {
                if (l < nt) {
                    const int x = lab.get(l) ^ bl.get(l);  // bits that differ from the best row
                    const int bbl = bl.get(l);
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        const int sh = B - 1 - b;
                        const unsigned v = ((x >> sh) & 1) ? db : kInfBits;
                        const unsigned mo = __reduce_min_sync(0xffffffffu, v);
                        const int slot = l * B + b;
                        if (lane == (slot & 31)) {
                            mine_other[slot >> 5] = mo;
                            mine_bb[slot >> 5] = (bbl >> sh) & 1;
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int slot = lane + 32 * q;
                if (slot < nt * B) {
                    unsigned *mm = sM + (s * NT * B + slot) * 2;
                    atomicMin(mm + mine_bb[q], wmin);
                    atomicMin(mm + (1 - mine_bb[q]), mine_other[q]);
                }
            }
        }
    }
    __syncthreads();

    // ---- per-symbol results
    for (int s = warp; s < n_sym; s += kWarps) {
        const size_t det = (size_t)sc * n_sym + s;
        const unsigned long long key = sBest[s];
        const int brow = (int)(key & 0xffffffffull);
        const int bchunk = brow >> 5;
        if (lane < nt) {
            const uint32_t w = sBlab[(s * chunks + bchunk) * WORDS + lane / Lab::PER];
            hard[det * nt + sPerm[lane]] = (uint8_t)((w >> (B * (lane % Lab::PER))) & ((1 << B) - 1));
        }
        if (ped2 != nullptr) {
            unsigned sec = kInfBits;
            for (int c = lane; c < chunks; c += 32)
                sec = min(sec, c == bchunk ? sSecond[s * chunks + c] : sWmin[s * chunks + c]);
            sec = __reduce_min_sync(0xffffffffu, sec);
            if (lane == 0) {
                ped2[det * 2] = __uint_as_float((unsigned)(key >> 32));
                ped2[det * 2 + 1] = __uint_as_float(sec);
            }
        }
        if (llr != nullptr) {
            for (int slot = lane; slot < nt * B; slot += 32) {
                const int l = slot / B, b = slot - l * B;
                const unsigned *mm = sM + (s * NT * B + slot) * 2;
                float v;
                if (mm[1] == kInfBits) v = kLlrMax;
                else if (mm[0] == kInfBits) v = -kLlrMax;
                else v = (__uint_as_float(mm[1]) - __uint_as_float(mm[0])) / sigma2;
                llr[(det * nt + sPerm[l]) * B + b] = v;
            }
        }
    }
}

template <int NT, int QAM>
cudaError_t launch_tpl(int n_sc, int n_sym, int nt, int n_pe, float sigma2, const float2 *R,
                       const float *inv_diag, const uint8_t *perm, const uint8_t *paths,
                       const float2 *Z, uint8_t *hard, float *llr, float *ped2, unsigned *status,
                       cudaStream_t stream)
{
    const DetSmem S = det_layout(NT, Qam<QAM>::B, n_pe, n_sym, Labels<NT, Qam<QAM>::B>::WORDS);
    const size_t smem = S.bytes;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(detect_walk_kernel<NT, QAM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    detect_walk_kernel<NT, QAM><<<n_sc, kThreads, smem, stream>>>(
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
