// Evaluation of the N_pe position vectors of every (subcarrier, symbol):
// SIC / partial-Euclidean-distance walks, argmin, max-log LLRs.
//
// One CTA per subcarrier; R, 1/R_ll, perm, the table and the subcarrier's z
// vectors are staged in shared memory once.  A warp takes 32 rows of the
// table for two OFDM symbols; each lane runs the walks of one row for both
// symbols with the whole state in registers:
//
//   e := z
//   for l = nt-1 .. 0:
//     b   = e_l / R_ll
//     s_l = the p_l-th closest constellation point to b (distance, then label)
//     d  += R_ll^2 |b - s_l|^2
//     e_i -= R_il s_l   for every i < l          (4 FFMA per complex term)
//
// Column l of R is read with 16-byte shared loads that all lanes issue for the
// same address (broadcast) and that serve both symbols.
//
// Ranking.  Rank 1 (the SIC choice; ~90% of the entries below the first
// level) is per-axis rounding to the grid; rank 2 compares the two next
// neighbours; higher ranks enumerate the nearest points in order (out of
// line).  The first detected level sees the same b for every row, so its
// ordered neighbour list is built once per symbol and looked up.  Rows are
// sorted in the CTA by how far they deviate from rank 1 below the first
// level, so that lanes needing the slower paths share warps.
//
// Reductions, without contended atomics:
//   warp:  argmin key (d, row) by shuffles; runner-up d and, for every
//          (level, bit), the minimum d over the warp's rows whose bit differs
//          from the warp-best row's bit, by redux.sync;
//   CTA:   per (symbol, level, bit, value) a u32 atomicMin on shared memory
//          (one per warp, distinct addresses across lanes); per symbol a
//          64-bit atomicMin on the argmin key (one per warp);
//   final: one lane per (symbol, level, bit) forms the LLR.
#pragma once

#include <cuda_fp16.h>

#include "mpnl_common.cuh"
#include "mpnl_internal.h"

namespace mpnl {
namespace {

constexpr int kThreads = 256;
// Three CTAs per SM (about 80 registers a thread): measured faster than two
// with more registers, and than four (64 registers: the FP32 walks spill,
// 1.52 against 1.33 ms on the bench slot); the FP16-residual walks keep
// their shift register in half the registers and run four (1.64 against
// 1.69 ms).  The shared memory of the bench shape (52 KB) fits either way.
constexpr int kCtasPerSm = 3;
constexpr int ctas_per_sm(bool f16) { return f16 ? 4 : kCtasPerSm; }
constexpr int kWarps = kThreads / 32;
constexpr int kTopList = 64;  // entries of the first-level neighbour list
constexpr int kList2 = 128;   // per symbol: entries of all second-level lists together

// A neighbour-list entry in 8 bytes: the squared distance, and the label
// with the point's two grid indices (the point itself is axis_pos of them).
__device__ __forceinline__ uint2 list_entry(float d, int lab, int ix, int iy)
{
    return make_uint2(__float_as_uint(d), (unsigned)lab | ((unsigned)ix << 8) | ((unsigned)iy << 16));
}

template <int QAM>
__device__ __forceinline__ void list_point(uint2 e, float &x, float &y, float &d, int &lab)
{
    d = __uint_as_float(e.x);
    lab = (int)(e.y & 0xffu);
    x = axis_pos<QAM>((int)((e.y >> 8) & 0xffu));
    y = axis_pos<QAM>((int)((e.y >> 16) & 0xffu));
}

// --------------------------------------------------------------------------
// ranking
// --------------------------------------------------------------------------

// Nearest grid index along one axis by rounding (an exact midpoint goes to
// the smaller axis label); returns the index, writes the squared distance and
// the grid coordinate.  Round-half-even is corrected only on the rare exact
// midpoint (|u - rint(u)| == 0.5, where u - 0.5 is the floor exactly).
template <int QAM>
__device__ __forceinline__ int axis_round(float x, float &d, float &pos)
{
    constexpr int L = Qam<QAM>::L;
    const float u = fmaf(x, 0.5f * Qam<QAM>::kScale, 0.5f * (float)(L - 1));
    float fr = rintf(u);
    if (fabsf(u - fr) == 0.5f) {
        const float fl = u - 0.5f;
        if (fl >= 0.f && fl < (float)(L - 1)) {
            const int a = (int)fl;
            fr = Qam<QAM>::axis_label(a) < Qam<QAM>::axis_label(a + 1) ? fl : fl + 1.f;
        }
    }
    fr = fminf(fmaxf(fr, 0.f), (float)(L - 1));
    pos = fmaf(fr, 2.f * Qam<QAM>::kInvScale, -(float)(L - 1) * Qam<QAM>::kInvScale);
    const float df = x - pos;
    d = df * df;
    return (int)fr;
}

template <int QAM>
__device__ __forceinline__ int axis_round(float x, float &d)
{
    float pos;
    return axis_round<QAM>(x, d, pos);
}

// The next grid index after i0 in distance order along an axis (one step
// towards x, or away when the constellation ends there).
template <int QAM>
__device__ __forceinline__ int axis_next(float x, int i0)
{
    constexpr int L = Qam<QAM>::L;
    const int s = x >= axis_pos<QAM>(i0) ? 1 : -1;
    const int n = i0 + s;
    return (n >= 0 && n < L) ? n : i0 - s;
}

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

// Coordinates of a label (inverse of grid_label).
template <int QAM>
__device__ __forceinline__ float2 label_point(int lab)
{
    constexpr int H = Qam<QAM>::B / 2;
    constexpr int L = Qam<QAM>::L;
    int lre = 0, lim = 0;
#pragma unroll
    for (int t = 0; t < H; ++t) {
        lre = (lre << 1) | ((lab >> (2 * (H - 1 - t) + 1)) & 1);
        lim = (lim << 1) | ((lab >> (2 * (H - 1 - t))) & 1);
    }
    int ire = 0, iim = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        if (Qam<QAM>::axis_label(i) == lre) ire = i;
        if (Qam<QAM>::axis_label(i) == lim) iim = i;
    }
    return make_float2(axis_pos<QAM>(ire), axis_pos<QAM>(iim));
}

// The third closest point (p = 3), the same answer as the enumeration below
// by the same arithmetic, in closed form: after the nearest point (row 0, column 0
// of the staircase) the second pop is the better of (0, 1) and (1, 0); if it
// was (1, 0) the third is the best of (0, 1), (1, 1) and (2, 0), else the
// better of (0, 2) and (1, 0) -- candidates taken in row order, the first
// valid one first, a later one replacing it on a smaller distance or an
// equal distance with a smaller label.  p = 3 is most of the ranks >= 3 a
// table holds, and this skips the enumeration loop.
template <int QAM>
__device__ __forceinline__ float third_point(float bx, float by, int ire, int iim, int &oi,
                                             int &oj)
{
    constexpr int L = Qam<QAM>::L;
    const AxisOrder<QAM> ore(bx, ire), oim(by, iim);
    auto dist = [&](int ia, int ic) {
        const float dx = bx - axis_pos<QAM>(ia), dy = by - axis_pos<QAM>(ic);
        return dx * dx + dy * dy;
    };
    int bi, bj;
    float bd;
    bool have = false;
    auto offer = [&](int ia, int ic) {
        const float v = dist(ia, ic);
        bool take = !have || v < bd;
        if (!take && v == bd) take = grid_label<QAM>(ia, ic) < grid_label<QAM>(bi, bj);
        if (take) {
            bi = ia;
            bj = ic;
            bd = v;
        }
        have = true;
    };
    const int x1 = ore.idx(1), y1 = oim.idx(1);
    offer(ire, y1);  // row 0, column 1
    offer(x1, iim);  // row 1, column 0
    const bool row1 = bi == x1 && bj == iim && !(x1 == ire && iim == y1);
    have = false;
    if (row1) {
        offer(ire, y1);                       // row 0, column 1
        offer(x1, y1);                        // row 1, column 1
        if (L > 2) offer(ore.idx(2), iim);    // row 2, column 0
    } else {
        if (L > 2) offer(ire, oim.idx(2));    // row 0, column 2
        offer(x1, iim);                       // row 1, column 0
    }
    oi = bi;
    oj = bj;
    return bd;
}

// p-th closest point (p >= 3) by (squared distance, label), out of line (p = 3
// in closed form, above).  The 2-D order is
// enumerated over the "staircase" of (row a, column c) pairs of the two axis
// orders: popping (a, c) exposes (a, c + 1), popping (a, 0) also exposes
// (a + 1, 0); every pair's predecessor sorts no later, so p pops reach the
// p-th point.  The per-row column pointers are packed 4 bits each.
// Writes the grid indices, returns the squared distance.
template <int QAM>
__device__ __noinline__ float kth_point_slow(float bx, float by, int p, int ire, int iim,
                                             int &oi, int &oj)
{
    if (p == 3) return third_point<QAM>(bx, by, ire, iim, oi, oj);
    constexpr int L = Qam<QAM>::L;
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
    oi = bi;
    oj = bj;
    return bd;
}

// The first detected level sees the same b = z_{nt-1} / R for every row, so
// its ordered neighbour list is built once per symbol by one warp: lane j
// holds points j and j + 32, and a bitonic sort of their (distance, label)
// keys over the warp orders them.  Entry r: distance, label, grid indices.
template <int QAM>
__device__ __forceinline__ void top_list(float bx, float by, int kmax, uint2 *list)
{
    // keys (distance bits, label, grid index): as unsigned 64-bit integers
    // they order by (distance, label); a bitonic sort over the warp puts the
    // e-th closest point at element e = lane + 32 k
    constexpr int M = QAM;
    constexpr int PER = (M + 31) / 32;
    constexpr int E = 32 * PER;
    const int lane = threadIdx.x & 31;
    unsigned long long key[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = lane + 32 * k;  // q = grid index: iy * L + ix
        const int ix = q % Qam<QAM>::L, iy = q / Qam<QAM>::L;
        const float dx = bx - axis_pos<QAM>(ix), dy = by - axis_pos<QAM>(iy);
        const float dq = dx * dx + dy * dy;
        key[k] = q < M ? (((unsigned long long)__float_as_uint(dq) << 32) |
                          ((unsigned)grid_label<QAM>(ix, iy) << 8) | (unsigned)q)
                       : ~0ull;
    }
#pragma unroll
    for (int size = 2; size <= E; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int e = lane + 32 * k;
                const bool up = (e & size) == 0;
                if (stride >= 32) {  // partner in the same lane (PER == 2, stride 32)
                    if (k == 0) {
                        const unsigned long long a = key[0], c = key[1];
                        const bool swap = (a > c) == up;
                        key[0] = swap ? c : a;
                        key[1] = swap ? a : c;
                    }
                } else {
                    const unsigned long long o = __shfl_xor_sync(0xffffffffu, key[k], stride);
                    const bool lower = (e & stride) == 0;
                    const bool keep_min = lower == up;
                    key[k] = keep_min ? (o < key[k] ? o : key[k]) : (o > key[k] ? o : key[k]);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = lane + 32 * k;
        if (e < kmax && e < M) {
            const int q = (int)(key[k] & 0xffu);
            const float dq = __uint_as_float((unsigned)(key[k] >> 32));
            list[e] = list_entry(dq, (int)((key[k] >> 8) & 0xffu), q % Qam<QAM>::L,
                                 q / Qam<QAM>::L);
        }
    }
}

// The len nearest points to b in order, by one thread: the staircase
// enumeration of kth_point_slow, emitting every pop.  Entry r: distance,
// label, grid indices.
template <int QAM>
__device__ __forceinline__ void nearest_list(float bx, float by, int len, uint2 *out)
{
    constexpr int L = Qam<QAM>::L;
    float d0;
    const int ire = axis_round<QAM>(bx, d0);
    const int iim = axis_round<QAM>(by, d0);
    const AxisOrder<QAM> ore(bx, ire), oim(by, iim);
    unsigned cols = 0;
    int na = 1;
    for (int pop = 0; pop < len; ++pop) {
        int ba = -1, bi = 0, bj = 0, blab = 0;
        float bd = INFINITY;
        for (int a = 0; a < na; ++a) {
            const int c = (cols >> (4 * a)) & 0xF;
            if (c >= L) continue;
            const int ia = ore.idx(a), ic = oim.idx(c);
            const float dx = bx - axis_pos<QAM>(ia), dy = by - axis_pos<QAM>(ic);
            const float v = dx * dx + dy * dy;
            const int lv = grid_label<QAM>(ia, ic);
            if (ba < 0 || v < bd || (v == bd && lv < blab)) {
                ba = a;
                bi = ia;
                bj = ic;
                bd = v;
                blab = lv;
            }
        }
        out[pop] = list_entry(bd, blab, bi, bj);
        const int bc = (cols >> (4 * ba)) & 0xF;
        if (bc == 0 && ba == na - 1 && na < L) ++na;
        cols += 1u << (4 * ba);
    }
}

// --------------------------------------------------------------------------
// per-walk state helpers
// --------------------------------------------------------------------------

// Labels of the NT levels of one walk, B bits each, packed contiguously:
// level l occupies bits [B l, B l + B) of the WORDS-word integer.  The walk
// visits levels nt-1 .. 0 and pushes each label in at the bottom, so no
// register is ever indexed by the (run-time) level.
template <int NT, int B>
struct Labels {
    static constexpr int WORDS = (NT * B + 31) / 32;
    uint32_t w[WORDS];
    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int k = 0; k < WORDS; ++k) w[k] = 0;
    }
    __device__ __forceinline__ void push(int lab)
    {
#pragma unroll
        for (int k = WORDS - 1; k > 0; --k) w[k] = __funnelshift_l(w[k - 1], w[k], B);
        w[0] = (w[0] << B) | (uint32_t)lab;
    }
    // level l for a run-time l, without indexing the register array
    __device__ __forceinline__ int get_rt(int l) const
    {
        const int bit = B * l, k = bit >> 5, off = bit & 31;
        const uint32_t w0 = w[0];
        const uint32_t w1 = WORDS > 1 ? w[WORDS > 1 ? 1 : 0] : 0u;
        const uint32_t w2 = WORDS > 2 ? w[WORDS > 2 ? 2 : 0] : 0u;
        const uint32_t lo = k == 0 ? w0 : (k == 1 ? w1 : w2);
        const uint32_t hi = k == 0 ? w1 : (k == 1 ? w2 : 0u);
        return (int)(__funnelshift_r(lo, hi, off) & ((1u << B) - 1));
    }
    // level l (a compile-time constant after unrolling)
    __device__ __forceinline__ int get(int l) const
    {
        const int bit = B * l, k = bit >> 5, off = bit & 31;
        uint32_t v = w[k] >> off;
        if (off + B > 32 && k + 1 < WORDS) v |= w[k + 1] << (32 - off);
        return (int)(v & ((1u << B) - 1));
    }
};

// Level l's label from packed words in memory (run-time l).
template <int B>
__device__ __forceinline__ int label_at(const uint32_t *w, int l)
{
    const int bit = B * l, k = bit >> 5, off = bit & 31;
    uint32_t v = w[k] >> off;
    if (off + B > 32) v |= w[k + 1] << (32 - off);
    return (int)(v & ((1u << B) - 1));
}

__host__ __device__ inline int a16(int o) { return (o + 15) & ~15; }
__host__ __device__ inline int pow2_at_least(int n)
{
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

struct DetSmem {
    int off_rc, off_r2, off_invd, off_perm, off_z, off_tab, off_order, off_m, off_best, off_wmin,
        off_second, off_blab, off_top, off_l2, off_lut, off_rh, off_rd, off_pt, off_rp, off_scr,
        bytes;
};

// Small per-CTA counters of one subcarrier, kept in the dynamic shared
// memory rather than as function-scope __shared__ arrays: every instance of
// the walk body would otherwise add its own static copy to a kernel that
// calls several instances (the persistent batch kernel), cutting its
// residency.  Ints: k1[65], off1[65], use2, kmax, hist[256], wsum[warps],
// and the largest magnitude of R and z (FP16 instances).
constexpr int kScrK1 = 0, kScrOff1 = 65, kScrUse2 = 130, kScrKmax = 131, kScrHist = 132,
              kScrWsum = 388, kScrMax = 388 + kWarps, kScrInts = 389 + kWarps;
static_assert(kThreads == 256, "the row sort gives each thread one of the 256 buckets");

// f16: the layout of the mixed-precision instances (half2 columns of R and
// the runner-up rows for the FP32 re-check) instead of the FP32 instances'
// packed-FMA columns of R.
__host__ __device__ inline DetSmem det_layout(int NT, int B, int n_pe, int n_sym, int WORDS,
                                              bool f16)
{
    const int chunks = (n_pe + 31) / 32;
    const int np2 = pow2_at_least(chunks * 32);
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
    o = a16(o + (n_sym + 1) * NT * 8);
    s.off_tab = o;
    o = a16(o + chunks * 32 * NT);
    s.off_order = o;  // row buckets, then the rows in walk order
    o = a16(o + (np2 + chunks * 32) * 4);
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
    s.off_top = o;
    o = a16(o + (n_sym + 1) * kTopList * 8);
    s.off_l2 = o;
    o = a16(o + (n_sym + 1) * kList2 * 8);
    s.off_lut = o;  // 2-D label of grid point (ire, iim) at ire * 8 + iim
    o = a16(o + 64);
    s.off_rh = s.off_rd = s.off_pt = s.off_rp = o;
    if (f16) {
        // mixed precision: R columns as half2 pairs (scaled), the diagonal of
        // R and the constellation points by label for the FP32 replays
        s.off_rh = o;
        o = a16(o + NT * NT * 8);
        s.off_rd = o;
        o = a16(o + NT * 4);
        s.off_pt = o;
        o = a16(o + 64 * 8);
    } else {
        // FP32: each term of the columns of R as {-Re, -Re, Im, Im} for the
        // packed FMAs of the cancellation
        s.off_rp = o;
        o = a16(o + NT * NT * 16);
    }
    s.off_scr = o;
    o = a16(o + kScrInts * 4);
    s.bytes = o;
    return s;
}

// In-warp transpose of a 32 x 32 bit matrix: lane p holds row p on entry
// and column p on return (bit q of the result = bit p of lane q's row).
// Five butterfly stages exchange ever smaller blocks with the partner lane.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x)
{
    const int lane = threadIdx.x & 31;
    const uint32_t masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int j = 16 >> t;
        const uint32_t m = masks[t];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? (((y >> j) & m) | (x & ~m)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

// Warp-level results of one symbol for the 32 walks a warp just finished.
//
// The 32 keys (PED bits, table row, sorted position) are sorted across the
// warp (bitonic, over shuffles).  Position 0 is the warp's best walk,
// position 1 its runner-up.  For the LLRs, X = label bits XOR the best
// walk's label bits marks, per (level, bit), the walks on the other side of
// the best walk's bit.  With X laid out by sorted position, a bit transpose
// gives lane t, for packed bit j = 32 k + t, the set of positions that have
// bit j; the first of them has the smallest PED, which is the other side's
// warp minimum.  So every (level, bit) costs one shared atomicMin per side,
// on addresses distinct across lanes.
template <int NT, int B>
__device__ __forceinline__ void warp_reduce_symbol(bool valid, bool active, int row, int chunk,
                                                   int chunks, int nt, float d,
                                                   const Labels<NT, B> &lab, int s,
                                                   unsigned long long *sBest, unsigned *sWmin,
                                                   unsigned *sSecond, uint32_t *sBlab,
                                                   unsigned *sM, bool want_llr)
{
    using Lab = Labels<NT, B>;
    constexpr int WORDS = Lab::WORDS;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned db = active ? fbits(d) : kInfBits;
    // key: PED bits, table row (the tie-break), then the sorted position
    unsigned long long key =
        active ? (((unsigned long long)db << 32) | ((unsigned)row << 16) | (unsigned)(chunk * 32 + lane))
               : ~0ull;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(FULL, key, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            key = keep_min ? (o < key ? o : key) : (o > key ? o : key);
        }
    }
    const unsigned long long best = __shfl_sync(FULL, key, 0);
    const unsigned long long runner = __shfl_sync(FULL, key, 1);
    const int blane = (int)(best & 31u);  // lane of the warp's best row
    const unsigned wmin = (unsigned)(best >> 32);
    const unsigned second = (unsigned)(runner >> 32);
    Lab bl;
#pragma unroll
    for (int k = 0; k < WORDS; ++k) bl.w[k] = __shfl_sync(FULL, lab.w[k], blane);
    if (!valid) return;  // (warp-uniform) second symbol slot beyond n_sym
    if (lane == 0) {
        atomicMin(&sBest[s], best);
        sWmin[s * chunks + chunk] = wmin;
        sSecond[s * chunks + chunk] = second;
#pragma unroll
        for (int k = 0; k < WORDS; ++k) sBlab[(s * chunks + chunk) * WORDS + k] = bl.w[k];
    }
    if (!want_llr) return;
    const int src = (int)(key & 31u);  // original lane of this sorted position
    const bool real = key != ~0ull;
    const unsigned dp = (unsigned)(key >> 32);
#pragma unroll
    for (int k = 0; k < WORDS; ++k) {
        const uint32_t xm = lab.w[k] ^ bl.w[k];
        const uint32_t xs = __shfl_sync(FULL, xm, src);
        const uint32_t col = warp_transpose32(real ? xs : 0u);  // positions having bit 32 k + lane
        const int owner = col ? __ffs(col) - 1 : 0;
        const unsigned dmin = __shfl_sync(FULL, dp, owner);
        const int j = 32 * k + lane;  // packed bit: level j / B, bit (j % B) from the LSB
        if (j < nt * B) {
            const int l = j / B, bpos = j - l * B;
            const int bb = (bl.w[k] >> lane) & 1;  // the best row's bit
            unsigned *mm = sM + (s * NT * B + l * B + (B - 1 - bpos)) * 2;
            atomicMin(mm + bb, wmin);
            if (col) atomicMin(mm + (1 - bb), dmin);
        }
    }
}

// half2 variant: e + (-Re,-Re)*(sx,sy) + (Im,-Im)*(sy,sx) per complex term.
template <int W, int NT, int SYM>
__device__ __forceinline__ void cancel_shift_h(__half2 (&eh)[SYM][NT], const uint2 *colh,
                                               const __half2 (&sh)[SYM], const __half2 (&sw)[SYM])
{
    static_assert(W < NT, "the shift reads entry W");
    const uint4 *c4 = reinterpret_cast<const uint4 *>(colh);
#pragma unroll
    for (int i2 = 0; i2 < (W + 1) / 2; ++i2) {
        const uint4 r = c4[i2];
        const __half2 a0 = *reinterpret_cast<const __half2 *>(&r.x);
        const __half2 b0 = *reinterpret_cast<const __half2 *>(&r.y);
        const __half2 a1 = *reinterpret_cast<const __half2 *>(&r.z);
        const __half2 b1 = *reinterpret_cast<const __half2 *>(&r.w);
        const int i = 2 * i2;
#pragma unroll
        for (int k = 0; k < SYM; ++k) {
            eh[k][i] = __hfma2(b0, sw[k], __hfma2(a0, sh[k], eh[k][i + 1]));
            if (i + 1 < W) eh[k][i + 1] = __hfma2(b1, sw[k], __hfma2(a1, sh[k], eh[k][i + 2]));
        }
    }
}

// Width dispatch: levels are grouped four at a time so that a level pays for
// at most three unused terms (widths 15, 11, 7, 3 for NT = 16); level 0
// needs no cancellation.  l is warp-uniform, so the branches do not diverge.
template <int NT, int SYM>
__device__ __forceinline__ void cancel_level_h(int l, __half2 (&eh)[SYM][NT], const uint2 *colh,
                                               const __half2 (&sh)[SYM], const __half2 (&sw)[SYM])
{
    if constexpr (NT == 16) {
        if (l > 11) cancel_shift_h<15>(eh, colh, sh, sw);
        else if (l > 7) cancel_shift_h<11>(eh, colh, sh, sw);
        else if (l > 3) cancel_shift_h<7>(eh, colh, sh, sw);
        else if (l > 0) cancel_shift_h<3>(eh, colh, sh, sw);
    } else if constexpr (NT == 8) {
        if (l > 3) cancel_shift_h<7>(eh, colh, sh, sw);
        else if (l > 0) cancel_shift_h<3>(eh, colh, sh, sw);
    } else {
        if (l > 0) cancel_shift_h<3>(eh, colh, sh, sw);
    }
}

// FP32 cancellation with packed FMAs (two FP32 FMAs per instruction):
// e'[i] = e[i+1] - R_{l-1-i, l} s as
//   e'[i] = (-Re R, -Re R) * (sx, sy) + ((Im R, Im R) * (sy, -sx) + e[i+1]),
// component by component the same two roundings as the scalar form
// fmaf(-Re R, sx, fmaf(Im R, sy, ex)), fmaf(-Re R, sy, fmaf(-Im R, sx, ey)).
// col = the staged column l as {-Re, -Re, Im, Im} per term (a broadcast
// 16-byte load serving SYM walks); q = (sy, -sx).
template <int W, int NT, int SYM>
__device__ __forceinline__ void cancel_shift2(float2 (&e)[SYM][NT], const float4 *col,
                                              const float2 (&sv)[SYM], const float2 (&q)[SYM])
{
    static_assert(W < NT, "the shift reads entry W");
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const float4 r = col[i];
        const float2 a = make_float2(r.x, r.y), b = make_float2(r.z, r.w);
#pragma unroll
        for (int k = 0; k < SYM; ++k) e[k][i] = __ffma2_rn(a, sv[k], __ffma2_rn(b, q[k], e[k][i + 1]));
    }
}

template <int NT, int SYM>
__device__ __forceinline__ void cancel_level2(int l, float2 (&e)[SYM][NT], const float4 *col,
                                              const float2 (&sv)[SYM], const float2 (&q)[SYM])
{
    if constexpr (NT == 16) {
        if (l > 11) cancel_shift2<15>(e, col, sv, q);
        else if (l > 7) cancel_shift2<11>(e, col, sv, q);
        else if (l > 3) cancel_shift2<7>(e, col, sv, q);
        else if (l > 0) cancel_shift2<3>(e, col, sv, q);
    } else if constexpr (NT == 8) {
        if (l > 3) cancel_shift2<7>(e, col, sv, q);
        else if (l > 0) cancel_shift2<3>(e, col, sv, q);
    } else {
        if (l > 0) cancel_shift2<3>(e, col, sv, q);
    }
}

template <int V>
struct IntTag {
    static constexpr int value = V;
};

// FP32 replay of a walk's vector x (its labels): the metric
// ||z - R x||^2, accumulated level by level in the walk's order as
// |e_l - R_ll x_l|^2 with e_l = z_l - sum_{j>l} R_lj x_j formed in FP32 by
// the shift-register cancellation.  The mixed-precision walks choose their
// vectors with FP16 residuals; every metric they report comes from here.
// z: the symbol's staged z; col: columns of R bottom-up as in sRr; rd: R_ll;
// pt: constellation points by label.
template <int NT, int B>
__device__ __forceinline__ float replay_metric(const float2 *z, const float2 *col, const float *rd,
                                               const float2 *pt, int nt, const Labels<NT, B> &lab)
{
    float ex[NT], ey[NT];
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        const int lz = nt - 1 - i;
        const float2 v = lz >= 0 ? z[lz] : make_float2(0.f, 0.f);
        ex[i] = v.x;
        ey[i] = v.y;
    }
    float m = 0.f;
#pragma unroll 1
    for (int l = nt - 1; l >= 0; --l) {
        const float2 x = pt[lab.get_rt(l)];
        const float r = rd[l];
        const float dx = fmaf(-r, x.x, ex[0]), dy = fmaf(-r, x.y, ey[0]);
        m = fmaf(dx, dx, fmaf(dy, dy, m));
        // e'[i] = e[i+1] - R_{l-1-i, l} x, width grouped by four levels
        const float4 *c4 = reinterpret_cast<const float4 *>(col + l * NT);
        auto shift = [&](auto wtag) {
            constexpr int W = decltype(wtag)::value;
#pragma unroll
            for (int i2 = 0; i2 < (W + 1) / 2; ++i2) {
                const float4 rr = c4[i2];
                const int i = 2 * i2;
                ex[i] = fmaf(-rr.x, x.x, fmaf(rr.y, x.y, ex[i + 1]));
                ey[i] = fmaf(-rr.x, x.y, fmaf(-rr.y, x.x, ey[i + 1]));
                if (i + 1 < W) {
                    ex[i + 1] = fmaf(-rr.z, x.x, fmaf(rr.w, x.y, ex[i + 2]));
                    ey[i + 1] = fmaf(-rr.z, x.y, fmaf(-rr.w, x.x, ey[i + 2]));
                }
            }
        };
        if constexpr (NT == 16) {
            if (l > 11) shift(IntTag<15>{});
            else if (l > 7) shift(IntTag<11>{});
            else if (l > 3) shift(IntTag<7>{});
            else if (l > 0) shift(IntTag<3>{});
        } else if constexpr (NT == 8) {
            if (l > 3) shift(IntTag<7>{});
            else if (l > 0) shift(IntTag<3>{});
        } else {
            if (l > 0) shift(IntTag<3>{});
        }
    }
    return m;
}

// One subcarrier of a slot, by one CTA of kThreads threads.
// F16: the interference-cancelled residuals e are kept as half2 (re, im) and
// updated with two HFMA2 per complex term; b, the ranking and the PED stay in
// FP32, and the final best and runner-up paths are re-checked in FP32.
// SYM: symbols per lane -- a warp item is 32 table rows x SYM symbols, and
// the staged column of R serves SYM walks per load.
template <int NT, int QAM, bool F16, int SYM>
__device__ __forceinline__ void detect_body(const DetArgs &args, int sc, unsigned char *smem)
{
    const int n_sym = args.n_sym, nt = args.nt, n_pe = args.n_pe;
    const float sigma2 = args.sigma2;
    const float2 *__restrict__ Rp = args.Rp;
    const float *__restrict__ inv_diag = args.inv_diag;
    const uint8_t *__restrict__ perm = args.perm;
    const uint8_t *__restrict__ paths = args.paths;
    const float2 *__restrict__ Z = args.Z;
    uint8_t *__restrict__ hard = args.hard;
    float *__restrict__ llr = args.llr;
    float *__restrict__ ped2 = args.ped2;
    unsigned *__restrict__ status = args.status;
    constexpr int B = Qam<QAM>::B;
    constexpr int L = Qam<QAM>::L;
    using Lab = Labels<NT, B>;
    constexpr int WORDS = Lab::WORDS;
    const int chunks = (n_pe + 31) / 32;
    const int nrows = chunks * 32;
    const int np2 = pow2_at_least(nrows);
    const DetSmem S = det_layout(NT, B, n_pe, n_sym, WORDS, F16);
    // sRr[l*NT + i] = R_{l-1-i, l} for i < l (column l of R above the
    // diagonal, bottom-up: the order the shift-register walk consumes it)
    float2 *sRr = reinterpret_cast<float2 *>(smem + S.off_rc);
    float *sR2 = reinterpret_cast<float *>(smem + S.off_r2);
    float *sInvd = reinterpret_cast<float *>(smem + S.off_invd);
    int *sPerm = reinterpret_cast<int *>(smem + S.off_perm);
    float2 *sZ = reinterpret_cast<float2 *>(smem + S.off_z);
    uint8_t *sTab = smem + S.off_tab;
    unsigned *sOrder = reinterpret_cast<unsigned *>(smem + S.off_order);
    unsigned *sM = reinterpret_cast<unsigned *>(smem + S.off_m);
    unsigned long long *sBest = reinterpret_cast<unsigned long long *>(smem + S.off_best);
    unsigned *sWmin = reinterpret_cast<unsigned *>(smem + S.off_wmin);
    unsigned *sSecond = reinterpret_cast<unsigned *>(smem + S.off_second);
    uint32_t *sBlab = reinterpret_cast<uint32_t *>(smem + S.off_blab);
    uint2 *sTop = reinterpret_cast<uint2 *>(smem + S.off_top);
    uint2 *sL2 = reinterpret_cast<uint2 *>(smem + S.off_l2);
    int *sScr = reinterpret_cast<int *>(smem + S.off_scr);
    int *s_k1 = sScr + kScrK1, *s_off1 = sScr + kScrOff1;  // QAM + 1 entries each
    int &s_use2 = sScr[kScrUse2];
    uint8_t *sLut = smem + S.off_lut;
    uint2 *sRh = reinterpret_cast<uint2 *>(smem + S.off_rh);  // sRr as {(-Re,-Re), (Im,-Im)} half2
    float4 *sRp = reinterpret_cast<float4 *>(smem + S.off_rp);  // sRr as {-Re, -Re, Im, Im}
    float *sRd = reinterpret_cast<float *>(smem + S.off_rd);    // R_ll (FP16 replays)
    float2 *sPt = reinterpret_cast<float2 *>(smem + S.off_pt);  // point of each label
    int &s_kmax = sScr[kScrKmax];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;

    // ---- stage the subcarrier
    const int P = nt * (nt + 1) / 2;
    const float2 *gR = Rp + (size_t)sc * P;
    // FP16 residuals: the subcarrier's R and z are scaled by the power of two
    // 2^-x that brings their largest component into [0.5, 1) -- exact, and
    // within FP16's range (+-65504, subnormal below 2^-14) for any caller
    // scale; b = e / R_ll multiplies the scale back (1/R_ll times 2^x).
    [[maybe_unused]] float hscale = 1.f, hunscale = 1.f;
    if constexpr (F16) {
        unsigned mx = 0u;
        for (int k = tid; k < P; k += kThreads) {
            const float2 v = gR[k];
            mx = max(mx, max(__float_as_uint(fabsf(v.x)), __float_as_uint(fabsf(v.y))));
        }
        for (int k = tid; k < n_sym * nt; k += kThreads) {
            const float2 v = Z[(size_t)sc * n_sym * nt + k];
            mx = max(mx, max(__float_as_uint(fabsf(v.x)), __float_as_uint(fabsf(v.y))));
        }
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (tid == 0) sScr[kScrMax] = 0;
        __syncthreads();
        if (lane == 0) atomicMax(reinterpret_cast<unsigned *>(sScr + kScrMax), mx);
        __syncthreads();
        const float m = __uint_as_float((unsigned)sScr[kScrMax]);
        if (m > 0.f && m < INFINITY) {  // finite and nonzero (NaN bits compare above inf)
            int x;
            frexpf(m, &x);
            x = min(max(x, -100), 100);
            hscale = ldexpf(1.f, -x);
            hunscale = ldexpf(1.f, x);
        }
    }
    for (int k = tid; k < NT * NT; k += kThreads) {
        const int l = k / NT, i = k - l * NT;
        float2 v = make_float2(0.f, 0.f);  // entries i >= l feed only stale registers
        if (l < nt && i < l) {
            const int r = l - 1 - i;  // R_{r,l}: packed row r starts at r nt - r(r-1)/2
            v = gR[r * nt - (r * (r - 1)) / 2 + (l - r)];
        }
        sRr[k] = v;
        if constexpr (!F16) sRp[k] = make_float4(-v.x, -v.x, v.y, v.y);
        if constexpr (F16) {
            const float rx = v.x * hscale, ry = v.y * hscale;
            const __half2 a = __floats2half2_rn(-rx, -rx), b = __floats2half2_rn(ry, -ry);
            sRh[k] = make_uint2(*reinterpret_cast<const unsigned *>(&a),
                                *reinterpret_cast<const unsigned *>(&b));
        }
    }
    for (int l = tid; l < nt; l += kThreads) {
        const float2 v = gR[l * nt - (l * (l - 1)) / 2];
        sR2[l] = v.x * v.x;
        if constexpr (F16) sRd[l] = v.x;
    }
    if constexpr (F16) {
        for (int k = tid; k < QAM; k += kThreads) sPt[k] = label_point<QAM>(k);
    }
    for (int k = tid; k < NT; k += kThreads) {
        if (k < nt) {
            const float iv = inv_diag[(size_t)sc * nt + k];
            sInvd[k] = iv;
            sPerm[k] = perm[(size_t)sc * nt + k];
        }
    }
    for (int k = tid; k < (n_sym + 1) * NT; k += kThreads) {
        const int s = k / NT, l = k - s * NT;
        sZ[k] = (s < n_sym && l < nt) ? Z[((size_t)sc * n_sym + s) * nt + l] : make_float2(0.f, 0.f);
    }
    if (tid < L * 8) {
        const int ire = tid >> 3, iim = tid & 7;
        sLut[tid] = (uint8_t)(iim < L ? grid_label<QAM>(ire, iim) : 0);
    }
    if (tid == 0) s_kmax = 1;
    for (int k = tid; k <= QAM; k += kThreads) s_k1[k] = 0;
    __syncthreads();
    // table, clamped; the order of the rows (a counting sort into 256
    // buckets, padding rows last): a warp pays for a ranking path at a level
    // if any of its lanes takes it there, so rows are grouped by the levels
    // at which they leave rank 1 below the two list-served levels -- rows
    // with a rank >= 4 first, by that rank, largest first (their enumeration
    // loop runs rank-many steps); then those whose largest rank is 3, by
    // the highest level holding it; then rows with a single rank 2, by its
    // level; with two, by (lower, upper) level; with more, by the lowest;
    // rows that stay at rank 1 last.
    // Also: the largest first-level rank, and per first-level rank the
    // largest second-level rank (the lengths of the second-level lists).
    int *s_hist = sScr + kScrHist, *s_wsum = sScr + kScrWsum;  // 256 buckets, kWarps sums
    s_hist[tid] = 0;
    __syncthreads();
    int kmax = 1;
    for (int r = tid; r < np2; r += kThreads) {
        if (r < nrows) {
            int mx = 1, ndev = 0, d1 = 0, d2 = 0, hi3 = 0, top = 1, second = 1;
            // a 16-level row is one 16-byte load (rows are 16-byte aligned then)
            const bool vec = NT == 16 && nt == 16 && r < n_pe;
            uint4 row4 = make_uint4(0u, 0u, 0u, 0u);
            if (vec) row4 = *reinterpret_cast<const uint4 *>(paths + ((size_t)sc * n_pe + r) * 16);
            const unsigned rw[4] = {row4.x, row4.y, row4.z, row4.w};
#pragma unroll
            for (int l = 0; l < NT; ++l) {
                int v = 1;  // padding rows and levels: rank 1
                if (r < n_pe && l < nt) {
                    v = vec ? (int)((rw[l >> 2] >> (8 * (l & 3))) & 0xffu)
                            : paths[((size_t)sc * n_pe + r) * nt + l];
                    if (v < 1 || v > QAM) {
                        atomicOr(status, kStatusBadPathEntry);
                        v = v < 1 ? 1 : QAM;
                    }
                    if (l == nt - 1) {
                        kmax = max(kmax, v);
                        top = v;
                    } else if (l == nt - 2) {
                        second = v;
                    } else if (v > 1) {  // levels visited bottom-up
                        if (ndev == 0) d1 = l;
                        else if (ndev == 1) d2 = l;
                        ++ndev;
                        if (v > 2) hi3 = l;
                        mx = max(mx, v);
                    }
                }
                sTab[r * NT + l] = (uint8_t)v;
            }
            if (r < n_pe) {
                if (nt >= 2) atomicMax(&s_k1[top], second);
                d1 = min(d1, 13);  // levels below nt - 2 <= 14
                d2 = min(d2, 13);
                const int h3 = min(hi3, 13);
                int bucket;
                if (mx >= 4) bucket = 7 - min(mx - 4, 7);               // 0 .. 7
                else if (mx == 3) bucket = 8 + h3;                      // 8 .. 21
                else if (ndev == 0) bucket = 240;
                else if (ndev == 1) bucket = 22 + d1;                   // 22 .. 35
                else if (ndev == 2) bucket = 36 + d1 * 14 + d2;         // 36 .. 217
                else bucket = 218 + d1;                                 // 218 .. 230
                sOrder[r] = (unsigned)bucket;
                atomicAdd(&s_hist[sOrder[r]], 1);
            }
        }
    }
    atomicMax(&s_kmax, kmax);
    for (int k = tid; k < n_sym * NT * B * 2; k += kThreads) sM[k] = kInfBits;
    for (int k = tid; k < n_sym; k += kThreads) sBest[k] = ~0ull;
    __syncthreads();
    {  // exclusive scan of the 256 bucket counts, one per thread
        const int v = s_hist[tid];
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) s_wsum[warp] = inc;
        __syncthreads();
        int base = 0;
        for (int w = 0; w < warp; ++w) base += s_wsum[w];
        s_hist[tid] = base + inc - v;  // now the bucket's next free position
    }
    __syncthreads();
    // scatter: real rows by bucket (order inside a bucket does not matter:
    // every result is a minimum or a per-row value), padding rows after them
    for (int r = tid; r < nrows; r += kThreads) {
        const int pos = r < n_pe ? atomicAdd(&s_hist[sOrder[r]], 1) : r;
        sOrder[np2 + pos] = (unsigned)r;
    }
    __syncthreads();
    // symbol slots the walks visit (SYM per warp item; with SYM = 2 and an
    // odd n_sym the last slot walks the zero vector of row n_sym)
    const int nsl = SYM * ((n_sym + SYM - 1) / SYM);
    // ordered neighbours of b = z_{nt-1} / R_{nt-1,nt-1}, one warp per symbol
    {
        const int kmx = s_kmax;
        const float iv = sInvd[nt - 1];
        for (int s = warp; s < nsl; s += kWarps) {
            const float2 z = sZ[s * NT + nt - 1];
            top_list<QAM>(z.x * iv, z.y * iv, kmx, sTop + s * kTopList);
        }
        if (tid == 0) {  // offsets of the second-level lists (one per first-level rank)
            int o = 0;
            for (int a = 1; a <= kmx; ++a) {
                s_off1[a] = o;
                o += s_k1[a];
            }
            s_use2 = nt >= 2 && o <= kList2;
        }
    }
    __syncthreads();
    // Second level: rows that took the same first-level rank a see the same
    // b = (z_{nt-2} - R_{nt-2,nt-1} s(a)) / R_{nt-2,nt-2}, so one ordered list
    // per (symbol, a) serves them all -- as long as the lists fit.
    if (s_use2) {
        const int kmx = s_kmax;
        const int l = nt - 2;
        const float iv = sInvd[l];
        const float2 r = sRr[(nt - 1) * NT];  // R_{nt-2, nt-1}
        for (int it = tid; it < nsl * kmx; it += kThreads) {  // one thread per list
            const int s = it / kmx, a = 1 + it - s * kmx;
            const int len = s_k1[a];
            if (len == 0) continue;
            float qx, qy, qd;
            int qlab;
            list_point<QAM>(sTop[s * kTopList + a - 1], qx, qy, qd, qlab);
            const float2 z = sZ[s * NT + l];
            const float ex = z.x - (r.x * qx - r.y * qy);
            const float ey = z.y - (r.x * qy + r.y * qx);
            nearest_list<QAM>(ex * iv, ey * iv, len, sL2 + s * kList2 + s_off1[a]);
        }
        __syncthreads();
    }
    const bool use2 = s_use2 != 0;

    // ---- walks: warp item = (chunk of 32 rows, group of SYM symbols)
    const int groups = (n_sym + SYM - 1) / SYM;
    const int l_list = use2 ? nt - 2 : nt - 1;  // levels >= l_list are list-served
    for (int item = warp; item < chunks * groups; item += kWarps) {
        const int chunk = item / groups, s0 = SYM * (item - chunk * groups);
        const int row = (int)sOrder[np2 + chunk * 32 + lane];
        const bool active = row < n_pe;
        const uint8_t *trow = sTab + row * NT;
        Lab lab[SYM];
        float d[SYM];
        {
            // shift register: when level l is decided, e[k][i] = e_{l-i} of
            // symbol s0 + k; entries i > l are stale and never read
            [[maybe_unused]] float2 e2[SYM][NT];
            [[maybe_unused]] __half2 eh[SYM][NT];
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                const int lz = nt - 1 - i;
#pragma unroll
                for (int k = 0; k < SYM; ++k) {
                    const float2 z = lz >= 0 ? sZ[(s0 + k) * NT + lz] : make_float2(0.f, 0.f);
                    if constexpr (F16) eh[k][i] = __floats2half2_rn(z.x * hscale, z.y * hscale);
                    else e2[k][i] = z;
                }
            }
#pragma unroll
            for (int k = 0; k < SYM; ++k) lab[k].clear();
#pragma unroll
            for (int k = 0; k < SYM; ++k) d[k] = 0.f;
            int p_top = 1;
#pragma unroll 1
            for (int l = nt - 1; l >= 0; --l) {
                const int p = trow[l];
                float sx[SYM], sy[SYM], dist[SYM];
                int lb[SYM];
                if (l >= l_list) {  // list-served levels (warp-uniform branch)
                    const uint2 *lst;
                    int stride;
                    if (l == nt - 1) {
                        p_top = p;
                        lst = sTop + s0 * kTopList + p - 1;
                        stride = kTopList;
                    } else {
                        lst = sL2 + s0 * kList2 + s_off1[p_top] + p - 1;
                        stride = kList2;
                    }
#pragma unroll
                    for (int k = 0; k < SYM; ++k)
                        list_point<QAM>(lst[k * stride], sx[k], sy[k], dist[k], lb[k]);
                } else {
                    const float iv = sInvd[l];
                    int ire[SYM], iim[SYM];
                    float dre[SYM], dim[SYM];
#pragma unroll
                    for (int k = 0; k < SYM; ++k) {
                        float bx, by;
                        if constexpr (F16) {
                            const float2 f = __half22float2(eh[k][0]);
                            bx = f.x * (iv * hunscale);
                            by = f.y * (iv * hunscale);
                            ire[k] = axis_round<QAM>(bx, dre[k], sx[k]);
                            iim[k] = axis_round<QAM>(by, dim[k], sy[k]);
                        } else {
                            bx = e2[k][0].x * iv;
                            by = e2[k][0].y * iv;
                            ire[k] = axis_round<QAM>(bx, dre[k], sx[k]);
                            iim[k] = axis_round<QAM>(by, dim[k], sy[k]);
                        }
                        if (p == 2) {
                            // second nearest: the next point along one axis
                            const int nre = axis_next<QAM>(bx, ire[k]);
                            const int nim = axis_next<QAM>(by, iim[k]);
                            float a = bx - axis_pos<QAM>(nre), c = by - axis_pos<QAM>(nim);
                            const float d_re = a * a + dim[k];  // (nre, iim)
                            const float d_im = dre[k] + c * c;  // (ire, nim)
                            bool take_re = d_re < d_im;
                            if (d_re == d_im) take_re = sLut[nre * 8 + iim[k]] < sLut[ire[k] * 8 + nim];
                            if (take_re) {
                                ire[k] = nre;
                                dre[k] = d_re;
                                sx[k] = axis_pos<QAM>(nre);
                            } else {
                                iim[k] = nim;
                                dre[k] = d_im;
                                sy[k] = axis_pos<QAM>(nim);
                            }
                            dim[k] = 0.f;
                        } else if (p > 2) {
                            int oi, oj;
                            dre[k] = kth_point_slow<QAM>(bx, by, p, ire[k], iim[k], oi, oj);
                            dim[k] = 0.f;
                            ire[k] = oi;
                            iim[k] = oj;
                            sx[k] = axis_pos<QAM>(oi);
                            sy[k] = axis_pos<QAM>(oj);
                        }
                        dist[k] = dre[k] + dim[k];
                        lb[k] = sLut[ire[k] * 8 + iim[k]];
                    }
                }
                const float r2 = sR2[l];
#pragma unroll
                for (int k = 0; k < SYM; ++k) {
                    d[k] = fmaf(r2, dist[k], d[k]);
                    lab[k].push(lb[k]);
                }
                if constexpr (F16) {
                    __half2 sh[SYM], sw[SYM];
#pragma unroll
                    for (int k = 0; k < SYM; ++k) {
                        sh[k] = __floats2half2_rn(sx[k], sy[k]);
                        sw[k] = __floats2half2_rn(sy[k], sx[k]);
                    }
                    cancel_level_h<NT>(l, eh, sRh + l * NT, sh, sw);
                } else {
                    float2 sv[SYM], q[SYM];
#pragma unroll
                    for (int k = 0; k < SYM; ++k) {
                        sv[k] = make_float2(sx[k], sy[k]);
                        q[k] = make_float2(sy[k], -sx[k]);
                    }
                    cancel_level2<NT>(l, e2, sRp + l * NT, sv, q);
                }
            }
            if constexpr (F16) {
                // every reported metric is the FP32 metric of the walk's vector
#pragma unroll
                for (int k = 0; k < SYM; ++k)
                    d[k] = replay_metric<NT, B>(sZ + (s0 + k) * NT, sRr, sRd, sPt, nt, lab[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < SYM; ++k)
            warp_reduce_symbol<NT, B>(s0 + k < n_sym, active, row, chunk, chunks, nt, d[k], lab[k],
                                      s0 + k, sBest, sWmin, sSecond, sBlab, sM, llr != nullptr);
    }
    __syncthreads();

    // ---- per-symbol results
    for (int s = warp; s < n_sym; s += kWarps) {
        const size_t det = (size_t)sc * n_sym + s;
        const unsigned long long key = sBest[s];
        const unsigned bd = (unsigned)(key >> 32);
        int bc = (int)((key & 0xffffu) >> 5);  // chunk of the best row's sorted position
        if (bc >= chunks) bc = 0;
        if (lane < nt)
            hard[det * nt + sPerm[lane]] = (uint8_t)label_at<B>(sBlab + (s * chunks + bc) * WORDS, lane);
        if (ped2 != nullptr) {
            unsigned sec = kInfBits;
            for (int c = lane; c < chunks; c += 32)
                sec = min(sec, c == bc ? sSecond[s * chunks + c] : sWmin[s * chunks + c]);
            sec = __reduce_min_sync(0xffffffffu, sec);
            if (lane == 0) {
                ped2[det * 2] = __uint_as_float(bd);
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

// A subcarrier's detection as a separate (not inlined) function, for the
// persistent batch kernel: each instance gets its own register allocation
// instead of the union over all instances.  It addresses the kernel's
// dynamic shared memory directly (shared-window loads).  Its arithmetic is
// that of the inlined per-call kernel (no contraction, see the build flags).
template <int NT, int QAM, bool F16, int SYM>
__device__ __noinline__ void detect_sc(const DetArgs args, int sc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    detect_body<NT, QAM, F16, SYM>(args, sc, smem);
}

template <int NT, int QAM, bool F16, int SYM>
__global__ void __launch_bounds__(kThreads, ctas_per_sm(F16)) detect_walk_kernel(DetArgs args)
{
    extern __shared__ __align__(16) unsigned char smem[];
    detect_body<NT, QAM, F16, SYM>(args, blockIdx.x, smem);
}

template <int NT, int QAM, bool F16, int SYM>
cudaError_t launch_sym(int n_sc, const DetArgs &a, cudaStream_t stream)
{
    const size_t smem =
        det_layout(NT, Qam<QAM>::B, a.n_pe, a.n_sym, Labels<NT, Qam<QAM>::B>::WORDS, F16).bytes;
    {
        cudaError_t e = allow_dynamic_smem(detect_walk_kernel<NT, QAM, F16, SYM>, smem);
        if (e != cudaSuccess) return e;
    }
    detect_walk_kernel<NT, QAM, F16, SYM><<<n_sc, kThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int NT, bool F16>
cudaError_t launch_nt(int qam, int n_sc, const DetArgs &a, int sym, cudaStream_t stream)
{
    switch (qam) {
    case 4:
        return sym == 1 ? launch_sym<NT, 4, F16, 1>(n_sc, a, stream)
                        : launch_sym<NT, 4, F16, 2>(n_sc, a, stream);
    case 16:
        return sym == 1 ? launch_sym<NT, 16, F16, 1>(n_sc, a, stream)
                        : launch_sym<NT, 16, F16, 2>(n_sc, a, stream);
    default:
        return sym == 1 ? launch_sym<NT, 64, F16, 1>(n_sc, a, stream)
                        : launch_sym<NT, 64, F16, 2>(n_sc, a, stream);
    }
}

template <bool F16>
cudaError_t launch_prec(int n_sc, const DetArgs &a, int qam, int sym, cudaStream_t stream)
{
    if (a.nt <= 4) return launch_nt<4, F16>(qam, n_sc, a, sym, stream);
    if (a.nt <= 8) return launch_nt<8, F16>(qam, n_sc, a, sym, stream);
    return launch_nt<16, F16>(qam, n_sc, a, sym, stream);
}

}  // namespace
}  // namespace mpnl
