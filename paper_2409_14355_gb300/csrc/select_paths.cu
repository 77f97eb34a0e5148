// Position-vector pre-selection, one group of G warps per subcarrier.
//
// Each level l gets a cost weight w_l = -log Pe_l from its SNR
// gamma_l = R_ll^2 / sigma2 (square-QAM symbol-error rate, floored); with the
// geometric rank model P_l(k) = (1 - Pe_l) Pe_l^(k-1) the log-probability of
// a vector p is a constant minus cost(p) = sum_l (p_l - 1) w_l.  The N_pe
// vectors of smallest cost (ties: lexicographically smaller from level nt-1
// down) are the N_pe most probable ones, in the order a best-first search
// would pop them.
//
// Instead of a sequential priority queue the CTA builds the answer level by
// level with sorted merges, all in shared memory:
//   L := [ all-ones ]                                  (cost 0)
//   for each level m (top first):
//     B := L
//     for j = 1, 2, ...:  B := first N_pe of merge(B, L shifted by j at level m)
//       (the shifted list adds j w_m to every cost and sets p_m = 1 + j; it
//        stays sorted, and once its first entry sorts after B's last entry no
//        later shift can contribute, so the loop stops there)
//     L := B
// Truncating to N_pe after every level is exact: a vector in the final top
// N_pe has its restriction to the levels seen so far (ones elsewhere) ahead of
// it in the order, so that restriction is in the partial top N_pe.
// Each merge is a merge path: every thread finds where its slice of the
// output (N_pe / (32 G) entries) starts by one co-rank binary search and
// merges from there.  G = 1 (a warp, no barrier) for short lists; G = 2 for
// N_pe >= 256, where halving the serial slice outweighs a two-warp named
// barrier per merge.  A CTA holds several independent groups.  Shifts whose
// cost exceeds an upper bound on the final N_pe-th cost are skipped; for
// N_pe >= 64 the bound comes from the vectors that deviate at one or two
// levels (about 1.1 times the true N_pe-th cost on 16 levels, against about
// 6 times from single deviations alone), so most shifts never start.  (Not
// for a cost table: counting its pairs takes a binary search per row lookup
// and cost more than it saved.)
//
// Costs are 64-bit fixed point (units of 2^-32): each float shift cost j w_m
// converts exactly (or to within 2^-33 below 2^-9), and list costs are exact
// integer sums of them.  So a shifted list is as sorted as the list it came
// from -- in float, two costs a ulp apart can round to one value after the
// shift and swap places under the tie rule, and a merge path over an
// unsorted input can drop or repeat an entry.  A shift cost is taken as at
// most 2^20 (16 levels of it stay below 2^57).
//
// A vector is keyed by 16 bytes (two u64, level nt-1 in the most significant
// byte): comparing keys as unsigned integers is the lexicographic order from
// the top level down, and the key bytes are the ranks written out.  For
// N_pe >= 128 a narrower form runs first (select_group_narrow): one u64 key
// with a field per level only as wide as the bound allows, and two lists
// merged into in place, so that a group needs under half the shared memory.
//
// The bound is tightened from the single-deviation bound where there is
// one; where all single deviations together are fewer than N_pe (none), the
// bisection starts from the largest cost of a two-deviation vector instead,
// provided that N_pe of those exist (16 levels of 64-QAM at N_pe 1024:
// 5.3 -> 1.8 ms for 3276 subcarriers).
#include "mpnl_common.cuh"
#include "mpnl_internal.h"

namespace mpnl {
namespace {

__device__ __forceinline__ bool before(unsigned long long ca, unsigned long long ha,
                                       unsigned long long la, unsigned long long cb,
                                       unsigned long long hb, unsigned long long lb)
{
    return ca < cb || (ca == cb && (ha < hb || (ha == hb && la < lb)));
}

// byte position of level l in the (hi, lo) key: top level first
__device__ __forceinline__ void level_shift(int nt, int l, bool &in_hi, int &shift)
{
    const int t = nt - 1 - l;
    in_hi = t < 8;
    shift = in_hi ? 56 - 8 * t : 56 - 8 * (t - 8);
}

constexpr int kSelMaxWarps = 4;
constexpr int kBoundIters = 10;    // bisection steps of the pair-count bound
constexpr int kBoundMinPe = 64;    // shorter lists keep the single-deviation bound
constexpr float kCostScale = 4294967296.f;  // fixed-point units per unit of cost (2^32)
constexpr float kCostMax = 1048576.f;       // largest shift cost represented (2^20)
constexpr unsigned long long kNoBound = ~0ull;

__host__ __device__ inline size_t sel_group_bytes(int n_pe)
{
    // 3 lists x (8 + 8 + 8) bytes (keys, fixed-point costs), then the bound
    // and w[]; 16-byte multiple so that the next group's keys stay aligned
    return ((size_t)n_pe * 72 + 8 + kMaxNt * 4 + 15) & ~(size_t)15;
}

template <int G>
__device__ __forceinline__ void group_sync(int group)
{
    static_assert(G == 1 || kSelMaxWarps / G <= 2, "named barriers 1 and 2 only");
    if constexpr (G == 1) {
        __syncwarp();
    } else if (group == 0) {
        asm volatile("bar.sync 1, %0;" ::"n"(32 * G) : "memory");
    } else {
        asm volatile("bar.sync 2, %0;" ::"n"(32 * G) : "memory");
    }
}

// Table-driven rank model (mpnl_select_paths_lut): the cost of rank 1 + j
// at level l is a row of a caller's table instead of j w_l.  The row is the
// level's SNR bin: the number of the ascending edges e with
// gamma_l = R_ll^2 / sigma2 >= e (all in float).  Rows start at 0 and are
// nondecreasing, which is all the merges below need.
struct RankLut {
    const float *edges;  // [n_bins - 1]
    const float *cost;   // [n_bins][qam]
    int n_bins;
};

// Cost models: the geometric rank model of square M-QAM levels, a caller's
// rank-cost table, or the geometric model of the L-PAM levels of the
// real-valued decomposition (ranks 1..L, Pe = 2 (1 - 1/L) Q(.) per level).
enum SelMode { kSelGeo = 0, kSelLut = 1, kSelPam = 2 };

// Cost of rank 1 + j at level m under the cost model (w: the levels'
// weights, or for a table the levels' bins), and the same in fixed point
// (rounded to nearest, clamped to kCostMax).
template <int QAM, int MODE>
__device__ __forceinline__ float sel_shift_cost(const float *w, const RankLut &lut, int m, int j)
{
    if constexpr (MODE == kSelLut) return __ldg(lut.cost + (size_t)__float_as_int(w[m]) * QAM + j);
    else return (float)j * w[m];
}

template <int QAM, int MODE>
__device__ __forceinline__ unsigned long long sel_shift_q(const float *w, const RankLut &lut, int m,
                                                          int j)
{
    return __float2ull_rn(fminf(sel_shift_cost<QAM, MODE>(w, lut, m, j), kCostMax) * kCostScale);
}

// The weights w[] of one subcarrier's levels and an upper bound *s_bound on
// its final N_pe-th cost (fixed point; kNoBound: none), in the group's
// shared memory, by the group of G warps; ends with a group barrier.
template <int QAM, int G, int MODE>
__device__ __forceinline__ void sel_setup(int sc, int nt, int n_pe, float sigma2,
                                          const float2 *__restrict__ Rp, float *w,
                                          unsigned long long *s_bound, int group, int tid,
                                          const RankLut &lut)
{
    constexpr bool LUT = MODE == kSelLut;
    constexpr bool PAM = MODE == kSelPam;
    constexpr int RK = PAM ? Qam<QAM>::L : QAM;  // ranks per level
    constexpr unsigned FULL = 0xffffffffu;
    const int P = nt * (nt + 1) / 2;
    if (LUT && tid < nt) {  // w[l] holds the level's table row (its bin)
        const int l = tid;
        const float rll = Rp[(size_t)sc * P + l * nt - l * (l - 1) / 2].x;
        const float sq = rll * rll;
        const float gamma = sq / sigma2;
        int b = 0;
        for (int e = 0; e < lut.n_bins - 1; ++e)
            if (gamma >= __ldg(lut.edges + e)) b = e + 1;
        w[l] = __int_as_float(b);
    } else if (!LUT && tid < nt) {
        const int l = tid;
        const float rll = Rp[(size_t)sc * P + l * nt - l * (l - 1) / 2].x;
        const float gamma = rll * rll / sigma2;
        const float x = sqrtf(3.0f * gamma / (float)(QAM - 1));
        const float qf = 0.5f * erfcf(x * 0.70710678118654752f);
        constexpr float c = 2.0f * (1.0f - 1.0f / (float)Qam<QAM>::L);  // 2 (1 - 1/sqrt(M))
        const float cq = c * qf;
        // square QAM: 1 - (1 - cq)^2 = cq (2 - cq) without cancellation; an
        // L-PAM level: cq
        float pe = PAM ? cq : cq * (2.0f - cq);
        pe = fmaxf(pe, kPeFloor);
        w[l] = -logf(pe);
    }
    group_sync<G>(group);
    auto shift_cost = [&](int m, int j) -> float {
        return sel_shift_cost<QAM, MODE>(w, lut, m, j);
    };
    // Number of deviations j >= 1 at level m whose shift cost j w_m is at
    // most r (linear costs; conservative: r w_m^-1 in float, and callers pass
    // an r already shaded below the value they test).
    auto count_upto = [&](int m, float r) -> int {
        if (!(r >= 0.f)) return 0;
        const int c = (int)floorf(r * __frcp_rn(w[m]));
        return c < 0 ? 0 : (c > RK - 1 ? RK - 1 : c);
    };
    // Tightening of the single-deviation bound v1 (bits of a float, +inf for
    // none; the first warp, all lanes): the vectors that deviate at one or
    // two levels are valid vectors too, so the smallest v at which N_pe of
    // those cost at most v is also an upper bound on the final N_pe-th cost
    // -- about 1.1 times it on 16 levels, where v1 is about 6 times it.  A
    // bisection over (0, v1] with the count split over the lanes: lane
    // (a, h) takes level a's single deviations (h = 0) and its pairs (a, a +
    // k mod nt) for k = 1 + h, 3 + h, ... <= nt / 2 (the pair at k = nt / 2
    // only from a < nt / 2), each pair as a loop over the deviations of the
    // level with the larger first shift cost and a count at the other.  The
    // count is conservative: it is taken at v (1 - 1e-5), far below the
    // rounding of any two-term cost, so every vector counted costs less than
    // v in float; the result is padded upward and returned in fixed point
    // (kNoBound: none).
    auto tighten_bound = [&](unsigned v1bits) -> unsigned long long {
        const bool pairs = !LUT && nt >= 2 && n_pe >= kBoundMinPe;  // linear costs only
        const int lane = tid & 31, a = lane & 15, h = lane >> 4;
        // vectors with one or two deviations costing at most v (1 - 1e-5),
        // all-ones included (all lanes of the first warp)
        auto count_pairs = [&](float v) -> int {
            const float vp = v * (1.0f - 1e-5f);
            int cnt = 0;
            if (a < nt) {
                if (h == 0) cnt += count_upto(a, vp);
                for (int k = 1 + h; 2 * k <= nt; k += 2) {
                    if (2 * k == nt && a >= k) continue;
                    const int b = a + k < nt ? a + k : a + k - nt;
                    const bool ao = shift_cost(a, 1) >= shift_cost(b, 1);
                    const int o = ao ? a : b, q = ao ? b : a;
                    for (int j = 1; j < RK; ++j) {
                        const float r = vp - shift_cost(o, j);
                        if (!(r >= 0.f)) break;
                        cnt += count_upto(q, r);
                    }
                }
            }
            return (int)__reduce_add_sync(FULL, (unsigned)cnt) + 1;
        };
        float hi_v;
        if (v1bits != 0x7f800000u) {
            hi_v = __uint_as_float(v1bits);
        } else {
            // fewer single-deviation vectors than N_pe: start from the most
            // a two-deviation vector can cost, if enough of those exist
            if (!pairs) return kNoBound;
            float mx = 0.f;
            for (int m = 0; m < nt; ++m) mx = fmaxf(mx, shift_cost(m, RK - 1));
            hi_v = 2.0f * mx;
            if (count_pairs(hi_v) < n_pe) return kNoBound;
        }
        if (pairs) {
            float lo_v = 0.f;
            for (int it = 0; it < kBoundIters; ++it) {
                const float mid = 0.5f * (lo_v + hi_v);
                if (count_pairs(mid) >= n_pe) hi_v = mid;
                else lo_v = mid;
            }
        }
        // in fixed point: a vector counted costs less than hi_v, and its
        // fixed-point cost is the exact sum of its float shift costs (each
        // to within half a unit), far inside the padding
        const float b = fminf(hi_v * (1.0f + 1e-4f) + 1e-6f, kCostMax * (float)kMaxNt);
        return __float2ull_ru(b * kCostScale) + 16ull;
    };
    // Upper bound on the final N_pe-th cost: the vectors that deviate from
    // all-ones at a single level (cost j w_l) plus all-ones itself are valid
    // vectors, so if N_pe of them cost <= v, the answer's N_pe-th cost is
    // <= v.  Shifts whose first entry j w_m exceeds the bound cannot
    // contribute and are skipped (the bound is padded against rounding).
    // The count of single-deviation vectors with cost <= j w_l is monotone in
    // j, so thread l of the first warp binary-searches the smallest j that
    // reaches N_pe.  The count never exceeds the exact one: v (1 - 1e-6) /
    // w_m is formed with a rounded reciprocal (relative error below 2^-22 <<
    // 1e-6), so the quotient stays below the exact v / w_m and its floor
    // cannot overshoot.
    if (LUT && tid < 32) {
        // the same bound with the table's rows: count(v) = 1 + the number of
        // (m, j >= 1) with cost(m, j) <= v, a binary search per row (rows are
        // nondecreasing); exact comparisons, no rounding to guard against
        unsigned bbits = 0x7f800000u;
        if (tid < nt) {
            const int l = tid;
            auto count = [&](float v) {
                int cnt = 1;
                for (int m = 0; m < nt; ++m) {
                    int lo_j = 0, hi_j = RK - 1;  // cost(m, 0) = 0 <= v
                    while (lo_j < hi_j) {
                        const int mid = (lo_j + hi_j + 1) >> 1;
                        if (shift_cost(m, mid) <= v) lo_j = mid;
                        else hi_j = mid - 1;
                    }
                    cnt += lo_j;
                }
                return cnt;
            };
            if (count(shift_cost(l, RK - 1)) >= n_pe) {
                int lo_j = 1, hi_j = RK - 1;
                while (lo_j < hi_j) {
                    const int mid = (lo_j + hi_j) >> 1;
                    if (count(shift_cost(l, mid)) >= n_pe) hi_j = mid;
                    else lo_j = mid + 1;
                }
                bbits = __float_as_uint(shift_cost(l, lo_j));
            }
        }
        bbits = __reduce_min_sync(FULL, bbits);
        const unsigned long long bq = tighten_bound(bbits);
        if (tid == 0) *s_bound = bq;
    } else if (!LUT && tid < 32) {
        unsigned bbits = 0x7f800000u;  // +inf
        if (tid < nt) {
            const float wl = w[tid];
            float inv[kMaxNt];
#pragma unroll
            for (int m = 0; m < kMaxNt; ++m) inv[m] = m < nt ? 1.0f / w[m] : 0.f;
            auto count = [&](int j) {
                const float v = (float)j * wl * (1.0f - 1e-6f);
                int cnt = 1;
#pragma unroll
                for (int m = 0; m < kMaxNt; ++m) {
                    const int c = (int)floorf(v * inv[m]);
                    cnt += m < nt ? (c < 0 ? 0 : (c > RK - 1 ? RK - 1 : c)) : 0;
                }
                return cnt;
            };
            if (count(RK - 1) >= n_pe) {
                int lo_j = 1, hi_j = RK - 1;  // count(hi_j) >= n_pe
                while (lo_j < hi_j) {
                    const int mid = (lo_j + hi_j) >> 1;
                    if (count(mid) >= n_pe) hi_j = mid;
                    else lo_j = mid + 1;
                }
                bbits = __float_as_uint((float)lo_j * wl);
            }
        }
        bbits = __reduce_min_sync(FULL, bbits);
        const unsigned long long bq = tighten_bound(bbits);
        if (tid == 0) *s_bound = bq;
    }
    group_sync<G>(group);
}

// One subcarrier by one group of G warps (thread tid of the group, which is
// group number `group` of its CTA), in the group's shared-memory region at
// byte offset base_off (at least sel_group_bytes(n_pe)).  Inlined into
// the per-call and the batch kernels alike (no contraction).  LUT: costs
// from the table `lut` (else the geometric model, w_l = -log Pe_l).
template <int QAM, int G, int MODE = kSelGeo>
__device__ __forceinline__ void select_group_body(int sc, int nt, int n_pe, float sigma2,
                                               const float2 *__restrict__ Rp,
                                               uint8_t *__restrict__ paths, int base_off,
                                               int group, int tid, RankLut lut = RankLut{})
{
    constexpr int RK = MODE == kSelPam ? Qam<QAM>::L : QAM;  // ranks per level
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + base_off;
    constexpr int T = 32 * G;  // threads per subcarrier
    // three lists (struct of arrays) addressed as base + list * n_pe, so that
    // the list index stays arithmetic (no pointer arrays in local memory)
    unsigned long long *HI = reinterpret_cast<unsigned long long *>(base);
    unsigned long long *LO = HI + 3 * n_pe;
    unsigned long long *CO = LO + 3 * n_pe;
    unsigned long long *s_bound = CO + 3 * n_pe;
    float *w = reinterpret_cast<float *>(s_bound + 1);
#define hi(b) (HI + (size_t)(b) * n_pe)
#define lo(b) (LO + (size_t)(b) * n_pe)
#define cost(b) (CO + (size_t)(b) * n_pe)

    sel_setup<QAM, G, MODE>(sc, nt, n_pe, sigma2, Rp, w, s_bound, group, tid, lut);
    auto shift_q = [&](int m, int j) -> unsigned long long {
        return sel_shift_q<QAM, MODE>(w, lut, m, j);
    };
    const unsigned long long bound = *s_bound;  // fixed point; kNoBound: none
    // The first level processed (nt-1) in closed form: starting from the
    // all-ones vector, its list is the arithmetic sequence j * w (rank j + 1
    // at that level), already sorted, cut at N_pe, at M and at the bound --
    // exactly what the shift-and-merge steps would produce one by one.
    int li = 0, nL = 1;
    {
        const int mt = nt - 1;
        while (nL < RK && nL < n_pe && shift_q(mt, nL) <= bound) ++nL;
        unsigned long long h = 0, o = 0;
        for (int l = 0; l < nt; ++l) {
            bool in_hi;
            int sh;
            level_shift(nt, l, in_hi, sh);
            if (in_hi) h |= 1ull << sh;
            else o |= 1ull << sh;
        }
        bool in_hi;
        int sh;
        level_shift(nt, mt, in_hi, sh);
        for (int j = tid; j < nL; j += T) {
            const unsigned long long add = (unsigned long long)j << sh;
            hi(0)[j] = h + (in_hi ? add : 0ull);
            lo(0)[j] = o + (in_hi ? 0ull : add);
            cost(0)[j] = shift_q(mt, j);
        }
    }
    group_sync<G>(group);
    for (int m = nt - 2; m >= 0; --m) {
        bool in_hi;
        int sh;
        level_shift(nt, m, in_hi, sh);
        int bi = li, nB = nL;          // B starts as L itself (read only)
        int oi = (li + 1) % 3;         // first output buffer
        for (int j = 1; j < RK; ++j) {
            const unsigned long long add = (unsigned long long)j << sh;
            const unsigned long long cj = shift_q(m, j);
            if (cj > bound) break;
            // first entry of the shifted list vs the last entry of B
            {
                const unsigned long long c0 = cost(li)[0] + cj;
                const unsigned long long h0 = hi(li)[0] + (in_hi ? add : 0ull);
                const unsigned long long l0 = lo(li)[0] + (in_hi ? 0ull : add);
                if (nB == n_pe &&
                    !before(c0, h0, l0, cost(bi)[nB - 1], hi(bi)[nB - 1], lo(bi)[nB - 1]))
                    break;
            }
            const int nOut = min(n_pe, nB + nL);
            // Merge path: thread t writes outputs [k0, k1).  A co-rank binary
            // search finds how many of the first k0 outputs come from B (the
            // rest from the shifted list C), then the thread merges onward.
            const int per = (nOut + T - 1) / T;
            const int k0 = min(nOut, tid * per), k1 = min(nOut, k0 + per);
            if (k0 < k1) {
                int lo_i = max(0, k0 - nL), hi_i = min(k0, nB);
                while (lo_i < hi_i) {
                    const int i = (lo_i + hi_i) >> 1, jj = k0 - i;  // jj >= 1, i < nB
                    const unsigned long long cc = cost(li)[jj - 1] + cj;
                    const unsigned long long hc = hi(li)[jj - 1] + (in_hi ? add : 0ull);
                    const unsigned long long lc = lo(li)[jj - 1] + (in_hi ? 0ull : add);
                    if (before(cost(bi)[i], hi(bi)[i], lo(bi)[i], cc, hc, lc)) lo_i = i + 1;
                    else hi_i = i;
                }
                int i = lo_i, jj = k0 - lo_i;
                for (int k = k0; k < k1; ++k) {
                    unsigned long long ca = 0ull, cc = 0ull;
                    unsigned long long ha = 0, la = 0, hc = 0, lc = 0;
                    if (i < nB) {
                        ca = cost(bi)[i];
                        ha = hi(bi)[i];
                        la = lo(bi)[i];
                    }
                    if (jj < nL) {
                        cc = cost(li)[jj] + cj;
                        hc = hi(li)[jj] + (in_hi ? add : 0ull);
                        lc = lo(li)[jj] + (in_hi ? 0ull : add);
                    }
                    const bool take_b = jj >= nL || (i < nB && before(ca, ha, la, cc, hc, lc));
                    cost(oi)[k] = take_b ? ca : cc;
                    hi(oi)[k] = take_b ? ha : hc;
                    lo(oi)[k] = take_b ? la : lc;
                    if (take_b) ++i;
                    else ++jj;
                }
            }
            group_sync<G>(group);
            nB = nOut;
            // next output goes to the buffer that is neither L nor the new B
            bi = oi;
            oi = 3 - li - bi;
        }
        li = bi;
        nL = nB;
    }

    // write the table: row r, level l -> byte of the key
    uint8_t *out = paths + (size_t)sc * n_pe * nt;
    for (int k = tid; k < n_pe * nt; k += T) {
        const int r = k / nt, l = k - r * nt;
        bool in_hi;
        int sh;
        level_shift(nt, l, in_hi, sh);
        const unsigned long long v = in_hi ? hi(li)[r] : lo(li)[r];
        out[k] = (uint8_t)((v >> sh) & 0xffull);
    }
#undef hi
#undef lo
#undef cost
    group_sync<G>(group);  // the region may be reused for the group's next subcarrier
}

// Narrow keys (the per-call geometric selection, N_pe >= kNarrowMinPe).  A
// level m's rank offset p_m - 1 never exceeds j_m, the largest j whose shift
// cost is within the bound (the merges stop there), so the key needs only
// ceil(log2(j_m + 1)) bits for level m: fields packed with level nt-1 most
// significant, so that comparing keys as integers is still the lexicographic
// order from the top level down.  With the tightened bound that is under 40
// bits on 16 levels of 64-QAM (N_pe 256 and 1024, 15-30 dB), so a key is one
// u64 and an entry 16 bytes; and with two lists -- the previous level's list
// L and the list B being built, merged into in place -- a group's state is
// 32 N_pe + 108 bytes, under half of the general body's, so that the groups
// of a 3276-subcarrier slot fit on the GPU at once.  The merges, their order
// and their stopping rules are the general body's, so the tables are the
// same.  A subcarrier whose fields need more than 64 bits marks its table (a
// 0 in its first entry, which is otherwise rank 1) and is left to
// select_paths_rest_kernel.
__host__ __device__ inline size_t narrow_group_bytes(int n_pe)
{
    // 2 lists x (8 + 8) bytes, the bound, w[], field offsets and widths, a flag
    return ((size_t)n_pe * 32 + 8 + kMaxNt * 4 + kMaxNt * 2 + 4 + 15) & ~(size_t)15;
}

constexpr int kNarrowPer = 4;  // outputs a thread holds per pass of an in-place merge
// Shorter lists fit on the GPU at once with the general body already, which
// is then faster: no in-place barriers, no second launch (measured on 16x16
// 64-QAM, N_pe 64: 0.072 against 0.076 ms; N_pe 128: 0.108 against 0.103).
constexpr int kNarrowMinPe = 128;

__device__ __forceinline__ bool before_n(unsigned long long ca, unsigned long long ka,
                                         unsigned long long cb, unsigned long long kb)
{
    return ca < cb || (ca == cb && ka < kb);
}

template <int QAM, int G>
__device__ __forceinline__ void select_group_narrow(int sc, int nt, int n_pe, float sigma2,
                                                    const float2 *__restrict__ Rp,
                                                    uint8_t *__restrict__ paths, int base_off,
                                                    int group, int tid)
{
    constexpr int RK = QAM;
    constexpr int T = 32 * G;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + base_off;
    unsigned long long *CO = reinterpret_cast<unsigned long long *>(base);  // [2][n_pe] costs
    unsigned long long *KY = CO + 2 * n_pe;                                  // [2][n_pe] keys
    unsigned long long *s_bound = KY + 2 * n_pe;
    float *w = reinterpret_cast<float *>(s_bound + 1);
    uint8_t *s_off = reinterpret_cast<uint8_t *>(w + kMaxNt);  // field offset per level
    uint8_t *s_bits = s_off + kMaxNt;                            // field width per level
    int *s_ok = reinterpret_cast<int *>(s_bits + kMaxNt);
#define nco(b) (CO + (size_t)(b) * n_pe)
#define nky(b) (KY + (size_t)(b) * n_pe)

    const RankLut lut{};
    sel_setup<QAM, G, kSelGeo>(sc, nt, n_pe, sigma2, Rp, w, s_bound, group, tid, lut);
    auto shift_q = [&](int m, int j) -> unsigned long long {
        return sel_shift_q<QAM, kSelGeo>(w, lut, m, j);
    };
    const unsigned long long bound = *s_bound;
    // field widths: the largest rank offset each level can take under the
    // bound, found with the merges' own fixed-point comparison
    if (tid < 32) {
        int bits = 0;
        if (tid < nt) {
            int jm = 0;
            while (jm + 1 < RK && shift_q(tid, jm + 1) <= bound) ++jm;
            bits = jm ? 32 - __clz(jm) : 0;
        }
        int incl = bits;  // inclusive sum over levels 0..tid
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (tid >= o) incl += v;
        }
        if (tid < nt) {
            s_off[tid] = (uint8_t)(incl - bits);
            s_bits[tid] = (uint8_t)bits;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        if (tid == 0) *s_ok = total <= 64;
    }
    group_sync<G>(group);
    uint8_t *out = paths + (size_t)sc * n_pe * nt;
    if (!*s_ok) {
        if (tid == 0) out[0] = 0;  // left to the general body
        group_sync<G>(group);
        return;
    }
    // the first level (nt-1) in closed form, as in the general body
    int li = 0, nL = 1;
    {
        const int mt = nt - 1;
        while (nL < RK && nL < n_pe && shift_q(mt, nL) <= bound) ++nL;
        const int sh = s_off[mt];  // below 64 whenever nL > 1
        for (int j = tid; j < nL; j += T) {
            nco(0)[j] = shift_q(mt, j);
            nky(0)[j] = j ? (unsigned long long)j << sh : 0ull;
        }
    }
    group_sync<G>(group);
    for (int m = nt - 2; m >= 0; --m) {
        const int sh = s_off[m];
        int bi = li, nB = nL;  // B starts as L itself (read only)
        const int oi = 1 - li;
        for (int j = 1; j < RK; ++j) {
            const unsigned long long cj = shift_q(m, j);
            if (cj > bound) break;
            const unsigned long long add = (unsigned long long)j << sh;  // level m has a field
            if (nB == n_pe &&
                !before_n(nco(li)[0] + cj, nky(li)[0] + add, nco(bi)[nB - 1], nky(bi)[nB - 1]))
                break;
            const int nOut = min(n_pe, nB + nL);
            // co-rank of output k0: how many of the first k0 outputs come from B
            auto co_rank = [&](int k0) {
                int lo_i = max(0, k0 - nL), hi_i = min(k0, nB);
                while (lo_i < hi_i) {
                    const int i = (lo_i + hi_i) >> 1, jj = k0 - i;  // jj >= 1, i < nB
                    if (before_n(nco(bi)[i], nky(bi)[i], nco(li)[jj - 1] + cj, nky(li)[jj - 1] + add))
                        lo_i = i + 1;
                    else
                        hi_i = i;
                }
                return lo_i;
            };
            if (bi == li) {
                // the level's first merge: B is L, the result goes to the other list
                const int per = (nOut + T - 1) / T;
                const int k0 = min(nOut, tid * per), k1 = min(nOut, k0 + per);
                if (k0 < k1) {
                    int i = co_rank(k0), jj = k0 - i;
                    for (int k = k0; k < k1; ++k) {
                        unsigned long long ca = 0ull, ka = 0ull, cc = 0ull, kc = 0ull;
                        if (i < nB) {
                            ca = nco(bi)[i];
                            ka = nky(bi)[i];
                        }
                        if (jj < nL) {
                            cc = nco(li)[jj] + cj;
                            kc = nky(li)[jj] + add;
                        }
                        const bool take_b = jj >= nL || (i < nB && before_n(ca, ka, cc, kc));
                        nco(oi)[k] = take_b ? ca : cc;
                        nky(oi)[k] = take_b ? ka : kc;
                        if (take_b) ++i;
                        else ++jj;
                    }
                }
                group_sync<G>(group);
                bi = oi;
            } else {
                // in place in B: passes over the outputs from the back.  A
                // pass reads only entries of B below its end, which no pass
                // has written yet, into registers; the group meets; then it
                // writes.  Outputs that stay where they are are not written.
                for (int end = nOut; end > 0; end -= T * kNarrowPer) {
                    const int start = max(0, end - T * kNarrowPer);
                    const int per = (end - start + T - 1) / T;
                    const int k0 = min(end, start + tid * per), k1 = min(end, k0 + per);
                    unsigned long long rc[kNarrowPer], rk[kNarrowPer];
                    bool moved = false;
                    if (k0 < k1) {
                        int i = co_rank(k0), jj = k0 - i;
                        moved = jj != 0;
#pragma unroll
                        for (int q = 0; q < kNarrowPer; ++q) {
                            rc[q] = rk[q] = 0ull;
                            if (k0 + q < k1) {
                                unsigned long long ca = 0ull, ka = 0ull, cc = 0ull, kc = 0ull;
                                if (i < nB) {
                                    ca = nco(bi)[i];
                                    ka = nky(bi)[i];
                                }
                                if (jj < nL) {
                                    cc = nco(li)[jj] + cj;
                                    kc = nky(li)[jj] + add;
                                }
                                const bool take_b = jj >= nL || (i < nB && before_n(ca, ka, cc, kc));
                                rc[q] = take_b ? ca : cc;
                                rk[q] = take_b ? ka : kc;
                                if (take_b) {
                                    ++i;
                                } else {
                                    ++jj;
                                    moved = true;
                                }
                            }
                        }
                    }
                    group_sync<G>(group);
                    if (moved) {
#pragma unroll
                        for (int q = 0; q < kNarrowPer; ++q)
                            if (k0 + q < k1) {
                                nco(bi)[k0 + q] = rc[q];
                                nky(bi)[k0 + q] = rk[q];
                            }
                    }
                }
                group_sync<G>(group);
            }
            nB = nOut;
        }
        li = bi;
        nL = nB;
    }

    // the table: row r, level l -> 1 + the key's field for l
    for (int k = tid; k < n_pe * nt; k += T) {
        const int r = k / nt, l = k - r * nt;
        const int b = s_bits[l];
        const unsigned long long v = nky(li)[r];
        out[k] = (uint8_t)(1 + (b ? (int)((v >> s_off[l]) & ((1ull << b) - 1ull)) : 0));
    }
#undef nco
#undef nky
    group_sync<G>(group);
}

template <int QAM, int G>
__global__ void __launch_bounds__(kSelMaxWarps * 32)
select_paths_kernel(int n_sc, int nt, int n_pe, float sigma2, const float2 *__restrict__ Rp,
                    uint8_t *__restrict__ paths)
{
    constexpr int T = 32 * G;
    const int group = threadIdx.x / T, tid = threadIdx.x % T;
    const int sc = blockIdx.x * (blockDim.x / T) + group;
    if (sc >= n_sc) return;  // whole groups leave; each group syncs only itself
    select_group_body<QAM, G>(sc, nt, n_pe, sigma2, Rp, paths,
                              group * (int)sel_group_bytes(n_pe), group, tid);
}

// Two warps a subcarrier: at most 40 registers, so that twelve CTAs (24
// subcarriers) fit on an SM; one warp: the shared memory allows 24 anyway.
template <int QAM, int G>
__global__ void __launch_bounds__(kSelMaxWarps * 32, G == 2 ? 12 : 1)
select_paths_narrow_kernel(int n_sc, int nt, int n_pe, float sigma2,
                           const float2 *__restrict__ Rp, uint8_t *__restrict__ paths)
{
    constexpr int T = 32 * G;
    const int group = threadIdx.x / T, tid = threadIdx.x % T;
    const int sc = blockIdx.x * (blockDim.x / T) + group;
    if (sc >= n_sc) return;
    select_group_narrow<QAM, G>(sc, nt, n_pe, sigma2, Rp, paths,
                                group * (int)narrow_group_bytes(n_pe), group, tid);
}

// The subcarriers select_paths_narrow_kernel left (a 0 in the first entry of
// their table), by the general body; groups stride over the subcarriers and
// skip the others after one byte.
template <int QAM, int G>
__global__ void __launch_bounds__(kSelMaxWarps * 32)
select_paths_rest_kernel(int n_sc, int nt, int n_pe, float sigma2, const float2 *__restrict__ Rp,
                         uint8_t *__restrict__ paths)
{
    constexpr int T = 32 * G;
    const int group = threadIdx.x / T, tid = threadIdx.x % T;
    const int groups = blockDim.x / T;
    for (int sc = blockIdx.x * groups + group; sc < n_sc; sc += gridDim.x * groups) {
        if (paths[(size_t)sc * n_pe * nt] != 0) continue;  // the same for the whole group
        select_group_body<QAM, G>(sc, nt, n_pe, sigma2, Rp, paths,
                                  group * (int)sel_group_bytes(n_pe), group, tid);
    }
}

template <int QAM, int G>
__global__ void __launch_bounds__(kSelMaxWarps * 32)
select_paths_lut_kernel(int n_sc, int nt, int n_pe, float sigma2, const float2 *__restrict__ Rp,
                        uint8_t *__restrict__ paths, RankLut lut)
{
    constexpr int T = 32 * G;
    const int group = threadIdx.x / T, tid = threadIdx.x % T;
    const int sc = blockIdx.x * (blockDim.x / T) + group;
    if (sc >= n_sc) return;
    select_group_body<QAM, G, kSelLut>(sc, nt, n_pe, sigma2, Rp, paths,
                                       group * (int)sel_group_bytes(n_pe), group, tid, lut);
}

// The 2 nt real levels of the real-valued decomposition (nt here: 2 nt).
template <int QAM, int G>
__global__ void __launch_bounds__(kSelMaxWarps * 32)
select_paths_pam_kernel(int n_sc, int nt, int n_pe, float sigma2, const float2 *__restrict__ Rp,
                        uint8_t *__restrict__ paths)
{
    constexpr int T = 32 * G;
    const int group = threadIdx.x / T, tid = threadIdx.x % T;
    const int sc = blockIdx.x * (blockDim.x / T) + group;
    if (sc >= n_sc) return;
    select_group_body<QAM, G, kSelPam>(sc, nt, n_pe, sigma2, Rp, paths,
                                       group * (int)sel_group_bytes(n_pe), group, tid);
}

// Persistent variant over a batch of radio units of mixed sizes: every
// group takes (unit, subcarrier) work items from a global counter.
template <int G>
__global__ void __launch_bounds__(kSelMaxWarps * 32)
select_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ start,
                    int n_items, int *__restrict__ counter, int group_bytes)
{
    __shared__ int s_w[kSelMaxWarps];
    constexpr int T = 32 * G;
    const int group = threadIdx.x / T, tid = threadIdx.x % T;
    const int base = group * group_bytes;
    const int total = start[n_items];
    for (;;) {
        if (tid == 0) s_w[group] = atomicAdd(counter, 1);
        group_sync<G>(group);
        const int w = s_w[group];
        group_sync<G>(group);  // every thread has read the item before the next fetch
        if (w >= total) break;
        const int i = find_item(start, n_items, w);
        const BatchItem &it = items[i];
        const int sc = w - start[i];
        switch (it.qam) {
        case 4: select_group_body<4, G>(sc, it.nt, it.n_pe, it.sigma2, it.R, it.paths, base, group, tid); break;
        case 16: select_group_body<16, G>(sc, it.nt, it.n_pe, it.sigma2, it.R, it.paths, base, group, tid); break;
        default: select_group_body<64, G>(sc, it.nt, it.n_pe, it.sigma2, it.R, it.paths, base, group, tid); break;
        }
    }
}

template <int QAM, int G>
cudaError_t launch_group_lut(int n_sc, int nt, int n_pe, float sigma2, const float2 *R,
                             uint8_t *paths, RankLut lut, cudaStream_t stream)
{
    const size_t per = sel_group_bytes(n_pe);
    int groups = (int)((100 * 1024) / per);
    groups = groups < 1 ? 1 : (groups > kSelMaxWarps / G ? kSelMaxWarps / G : groups);
    const size_t smem = per * groups;
    cudaError_t e = allow_dynamic_smem(select_paths_lut_kernel<QAM, G>, smem);
    if (e != cudaSuccess) return e;
    const int grid = (n_sc + groups - 1) / groups;
    select_paths_lut_kernel<QAM, G><<<grid, groups * G * 32, smem, stream>>>(n_sc, nt, n_pe,
                                                                            sigma2, R, paths, lut);
    return cudaGetLastError();
}

template <int QAM, int G>
cudaError_t launch_group_pam(int n_sc, int ntr, int n_pe, float sigma2, const float2 *R,
                             uint8_t *paths, cudaStream_t stream)
{
    const size_t per = sel_group_bytes(n_pe);
    int groups = (int)((100 * 1024) / per);
    groups = groups < 1 ? 1 : (groups > kSelMaxWarps / G ? kSelMaxWarps / G : groups);
    const size_t smem = per * groups;
    cudaError_t e = allow_dynamic_smem(select_paths_pam_kernel<QAM, G>, smem);
    if (e != cudaSuccess) return e;
    const int grid = (n_sc + groups - 1) / groups;
    select_paths_pam_kernel<QAM, G><<<grid, groups * G * 32, smem, stream>>>(n_sc, ntr, n_pe,
                                                                            sigma2, R, paths);
    return cudaGetLastError();
}

template <int QAM, int G>
cudaError_t launch_group_narrow(int n_sc, int nt, int n_pe, float sigma2, const float2 *R,
                                uint8_t *paths, cudaStream_t stream)
{
    // narrow keys, a CTA of kSelMaxWarps warps (kSelMaxWarps / G subcarriers)
    {
        const int groups = kSelMaxWarps / G;
        const size_t smem = narrow_group_bytes(n_pe) * groups;
        cudaError_t e = allow_dynamic_smem(select_paths_narrow_kernel<QAM, G>, smem);
        if (e != cudaSuccess) return e;
        const int grid = (n_sc + groups - 1) / groups;
        select_paths_narrow_kernel<QAM, G><<<grid, groups * G * 32, smem, stream>>>(
            n_sc, nt, n_pe, sigma2, R, paths);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // the subcarriers it left, by the general body
    const size_t per = sel_group_bytes(n_pe);
    int groups = (int)((100 * 1024) / per);
    groups = groups < 1 ? 1 : (groups > kSelMaxWarps / G ? kSelMaxWarps / G : groups);
    const size_t smem = per * groups;
    cudaError_t e = allow_dynamic_smem(select_paths_rest_kernel<QAM, G>, smem);
    if (e != cudaSuccess) return e;
    const int grid = min((n_sc + groups - 1) / groups, 128);
    select_paths_rest_kernel<QAM, G><<<grid, groups * G * 32, smem, stream>>>(n_sc, nt, n_pe,
                                                                             sigma2, R, paths);
    return cudaGetLastError();
}

template <int QAM, int G>
cudaError_t launch_group(int n_sc, int nt, int n_pe, float sigma2, const float2 *R,
                         uint8_t *paths, cudaStream_t stream)
{
    if (n_pe >= kNarrowMinPe)
        return launch_group_narrow<QAM, G>(n_sc, nt, n_pe, sigma2, R, paths, stream);
    // as many groups (subcarriers) per CTA as fit in about 100 KB of shared
    // memory, at most kSelMaxWarps warps
    const size_t per = sel_group_bytes(n_pe);
    int groups = (int)((100 * 1024) / per);
    groups = groups < 1 ? 1 : (groups > kSelMaxWarps / G ? kSelMaxWarps / G : groups);
    const size_t smem = per * groups;
    {
        cudaError_t e = allow_dynamic_smem(select_paths_kernel<QAM, G>, smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = (n_sc + groups - 1) / groups;
    select_paths_kernel<QAM, G><<<grid, groups * G * 32, smem, stream>>>(n_sc, nt, n_pe, sigma2, R,
                                                                        paths);
    return cudaGetLastError();
}

template <int QAM>
cudaError_t launch_tpl(int n_sc, int nt, int n_pe, float sigma2, const float2 *R,
                       uint8_t *paths, int warps, cudaStream_t stream)
{
    if (warps == 4) return launch_group<QAM, 4>(n_sc, nt, n_pe, sigma2, R, paths, stream);
    if (warps == 2) return launch_group<QAM, 2>(n_sc, nt, n_pe, sigma2, R, paths, stream);
    return launch_group<QAM, 1>(n_sc, nt, n_pe, sigma2, R, paths, stream);
}

template <int G>
cudaError_t launch_select_batch_g(const BatchItem *items, const int *start, int n_items,
                                  int *counter, int group_bytes, int grid, cudaStream_t stream)
{
    const int groups = kSelMaxWarps / G;
    const size_t smem = (size_t)group_bytes * groups;
    cudaError_t e = allow_dynamic_smem(select_batch_kernel<G>, smem);
    if (e != cudaSuccess) return e;
    select_batch_kernel<G><<<grid, kSelMaxWarps * 32, smem, stream>>>(items, start, n_items,
                                                                     counter, group_bytes);
    return cudaGetLastError();
}

}  // namespace

size_t select_group_bytes(int n_pe) { return sel_group_bytes(n_pe); }

cudaError_t launch_select_batch(const BatchItem *items, const int *start, int n_items,
                                int *counter, int group_bytes, int warps, int grid,
                                cudaStream_t stream)
{
    if (warps == 4) return launch_select_batch_g<4>(items, start, n_items, counter, group_bytes, grid, stream);
    if (warps == 2) return launch_select_batch_g<2>(items, start, n_items, counter, group_bytes, grid, stream);
    return launch_select_batch_g<1>(items, start, n_items, counter, group_bytes, grid, stream);
}

cudaError_t launch_select_paths_lut(int n_sc, int nt, int qam, int n_pe, float sigma2,
                                    const float2 *R, const float *edges, const float *cost,
                                    int n_bins, uint8_t *paths, int warps, cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    const RankLut lut{edges, cost, n_bins};
    const int g = warps == 4 ? 4 : (warps == 2 ? 2 : 1);
#define MPNL_SEL_LUT(Q)                                                                     \
    return g == 4 ? launch_group_lut<Q, 4>(n_sc, nt, n_pe, sigma2, R, paths, lut, stream)   \
         : g == 2 ? launch_group_lut<Q, 2>(n_sc, nt, n_pe, sigma2, R, paths, lut, stream)   \
                  : launch_group_lut<Q, 1>(n_sc, nt, n_pe, sigma2, R, paths, lut, stream)
    switch (qam) {
    case 4: MPNL_SEL_LUT(4);
    case 16: MPNL_SEL_LUT(16);
    default: MPNL_SEL_LUT(64);
    }
#undef MPNL_SEL_LUT
}

cudaError_t launch_select_paths_pam(int n_sc, int ntr, int qam, int n_pe, float sigma2,
                                    const float2 *R, uint8_t *paths, int warps,
                                    cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    const int g = warps == 4 ? 4 : (warps == 2 ? 2 : 1);
#define MPNL_SEL_PAM(Q)                                                                     \
    return g == 4 ? launch_group_pam<Q, 4>(n_sc, ntr, n_pe, sigma2, R, paths, stream)       \
         : g == 2 ? launch_group_pam<Q, 2>(n_sc, ntr, n_pe, sigma2, R, paths, stream)       \
                  : launch_group_pam<Q, 1>(n_sc, ntr, n_pe, sigma2, R, paths, stream)
    switch (qam) {
    case 4: MPNL_SEL_PAM(4);
    case 16: MPNL_SEL_PAM(16);
    default: MPNL_SEL_PAM(64);
    }
#undef MPNL_SEL_PAM
}

cudaError_t launch_select_paths(int n_sc, int nt, int qam, int n_pe, float sigma2,
                                const float2 *R, uint8_t *paths, int warps, cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    switch (qam) {
    case 4: return launch_tpl<4>(n_sc, nt, n_pe, sigma2, R, paths, warps, stream);
    case 16: return launch_tpl<16>(n_sc, nt, n_pe, sigma2, R, paths, warps, stream);
    default: return launch_tpl<64>(n_sc, nt, n_pe, sigma2, R, paths, warps, stream);
    }
}

}  // namespace mpnl
