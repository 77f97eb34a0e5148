// Real-valued decomposition (RVD) variant of the walks (mpnl_rvd_embed,
// mpnl_detect_rvd).  The paper's levels are complex; in the RVD
//   [Re y; Im y] = [[Re H, -Im H]; [Im H, Re H]] [Re s; Im s] + noise,
// the 2 nt real columns are the users' real (column u) and imaginary
// (column nt + u) parts, each an L-PAM axis of the square QAM (L = sqrt M)
// with the axis's Gray labels.  The sorted QR of the real matrix is
// mpnl_preprocess run on the embedded matrix (imaginary parts zero, so every
// product and sum stays real); the position vectors come from
// mpnl_select_paths_pam; this file holds the embedding and the walks.
//
// A walk visits the 2 nt real levels top-down: e_l = z_l - sum_{j>l} R_lj
// s_j, b = e_l / R_ll, s_l = the p_l-th closest PAM point by (distance,
// axis label), d += R_ll^2 (b - s_l)^2.  One CTA per subcarrier, a lane per
// table row and symbol; the residuals are a real shift-register file (one
// FFMA per term).  On a line the p-th closest point is closed-form: the
// nearest point, then alternately one step towards b and one away
// (AxisOrder), with an exact distance tie -- at most two points share a
// distance -- resolved by label against the neighbour in that sequence; so
// every rank costs the same and no row ordering is needed.  The argmin, the
// runner-up and the per-(level, axis bit) LLR minima use the warp reduction
// of the complex walks over B/2-bit labels; the results join each user's
// two axes (bits b0 b2 .. from the real part, b1 b3 .. from the imaginary).
#include "detect_impl.cuh"

namespace mpnl {
namespace {

struct RvdSmem {
    int off_rc, off_r2, off_invd, off_perm, off_z, off_tab, off_m, off_best, off_wmin, off_second,
        off_blab, bytes;
};

__host__ __device__ inline RvdSmem rvd_layout(int NTR, int BH, int n_pe, int n_sym, int WORDS)
{
    const int chunks = (n_pe + 31) / 32;
    RvdSmem s;
    int o = 0;
    s.off_rc = o;
    o = a16(o + NTR * NTR * 4);
    s.off_r2 = o;
    o = a16(o + NTR * 4);
    s.off_invd = o;
    o = a16(o + NTR * 4);
    s.off_perm = o;
    o = a16(o + NTR * 4);
    s.off_z = o;
    o = a16(o + n_sym * NTR * 4);
    s.off_tab = o;
    o = a16(o + chunks * 32 * NTR);
    s.off_m = o;
    o = a16(o + n_sym * NTR * BH * 2 * 4);
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

// The p-th closest PAM point to b (grid index), by (distance, axis label);
// dist receives its squared distance.
template <int QAM>
__device__ __forceinline__ int pam_kth(float b, int p, float &dist)
{
    constexpr int L = Qam<QAM>::L;
    float d0, pos0;
    const int i0 = axis_round<QAM>(b, d0, pos0);
    if (p <= 1) {
        dist = d0;
        return i0;
    }
    const AxisOrder<QAM> o(b, i0);
    auto sq = [&](int i) {
        const float t = b - axis_pos<QAM>(i);
        return t * t;
    };
    int c = o.idx(p - 1);
    float dc = sq(c);
    const int a = o.idx(p - 2);
    const float da = sq(a);
    if (da == dc && Qam<QAM>::axis_label(a) > Qam<QAM>::axis_label(c)) {
        c = a;
        dc = da;
    } else if (p < L) {
        const int n = o.idx(p);
        const float dn = sq(n);
        if (dn == dc && Qam<QAM>::axis_label(n) < Qam<QAM>::axis_label(c)) {
            c = n;
            dc = dn;
        }
    }
    dist = dc;
    return c;
}

// e'[i] = e[i+1] - R_{l-1-i, l} s for i < W (W >= l), col = column l of R
// above the diagonal, bottom-up, four terms per 16-byte broadcast load.
template <int W, int NTR>
__device__ __forceinline__ void cancel_shift_r(float (&e)[NTR], const float *col, float s)
{
    static_assert(W < NTR, "the shift reads entry W");
    const float4 *c4 = reinterpret_cast<const float4 *>(col);
#pragma unroll
    for (int i4 = 0; i4 < (W + 3) / 4; ++i4) {
        const float4 r = c4[i4];
        const float rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = 4 * i4 + t;
            if (i < W) e[i] = fmaf(-rv[t], s, e[i + 1]);
        }
    }
}

template <int NTR>
__device__ __forceinline__ void cancel_level_r(int l, float (&e)[NTR], const float *col, float s)
{
    if constexpr (NTR == 16) {
        if (l > 11) cancel_shift_r<15>(e, col, s);
        else if (l > 7) cancel_shift_r<11>(e, col, s);
        else if (l > 3) cancel_shift_r<7>(e, col, s);
        else if (l > 0) cancel_shift_r<3>(e, col, s);
    } else if constexpr (NTR == 8) {
        if (l > 3) cancel_shift_r<7>(e, col, s);
        else if (l > 0) cancel_shift_r<3>(e, col, s);
    } else {
        if (l > 0) cancel_shift_r<3>(e, col, s);
    }
}

struct RvdArgs {
    int n_sym, nt, n_pe;  // nt: users (complex); 2 nt real levels
    float sigma2;
    const float2 *Rp;     // [n_sc][ntr (ntr + 1) / 2], imaginary parts zero
    const float *inv_diag;
    const uint8_t *perm;  // real columns
    const uint8_t *paths; // [n_sc][n_pe][ntr], ranks 1..L
    const float2 *Z;      // [n_sc][n_sym][ntr]
    uint8_t *hard;        // [n_sc][n_sym][nt]
    float *llr;           // [n_sc][n_sym][nt][B]
    float *ped2;
    unsigned *status;
};

template <int NTR, int QAM>
__global__ void __launch_bounds__(kThreads, 3) detect_rvd_kernel(RvdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int B = Qam<QAM>::B, BH = B / 2, L = Qam<QAM>::L;
    using Lab = Labels<NTR, BH>;
    constexpr int WORDS = Lab::WORDS;
    const int sc = blockIdx.x;
    const int n_sym = a.n_sym, nt = a.nt, ntr = 2 * a.nt, n_pe = a.n_pe;
    const int chunks = (n_pe + 31) / 32, nrows = chunks * 32;
    const RvdSmem S = rvd_layout(NTR, BH, n_pe, n_sym, WORDS);
    float *sRr = reinterpret_cast<float *>(smem + S.off_rc);
    float *sR2 = reinterpret_cast<float *>(smem + S.off_r2);
    float *sInvd = reinterpret_cast<float *>(smem + S.off_invd);
    int *sPerm = reinterpret_cast<int *>(smem + S.off_perm);
    float *sZ = reinterpret_cast<float *>(smem + S.off_z);
    uint8_t *sTab = smem + S.off_tab;
    unsigned *sM = reinterpret_cast<unsigned *>(smem + S.off_m);
    unsigned long long *sBest = reinterpret_cast<unsigned long long *>(smem + S.off_best);
    unsigned *sWmin = reinterpret_cast<unsigned *>(smem + S.off_wmin);
    unsigned *sSecond = reinterpret_cast<unsigned *>(smem + S.off_second);
    uint32_t *sBlab = reinterpret_cast<uint32_t *>(smem + S.off_blab);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- stage the subcarrier
    const int P = ntr * (ntr + 1) / 2;
    const float2 *gR = a.Rp + (size_t)sc * P;
    for (int k = tid; k < NTR * NTR; k += kThreads) {
        const int l = k / NTR, i = k - l * NTR;
        float v = 0.f;
        if (l < ntr && i < l) {
            const int r = l - 1 - i;
            v = gR[r * ntr - (r * (r - 1)) / 2 + (l - r)].x;
        }
        sRr[k] = v;
    }
    for (int l = tid; l < NTR; l += kThreads) {
        if (l < ntr) {
            const float v = gR[l * ntr - (l * (l - 1)) / 2].x;
            sR2[l] = v * v;
            sInvd[l] = a.inv_diag[(size_t)sc * ntr + l];
            sPerm[l] = a.perm[(size_t)sc * ntr + l];
        }
    }
    for (int k = tid; k < n_sym * NTR; k += kThreads) {
        const int s = k / NTR, l = k - s * NTR;
        sZ[k] = l < ntr ? a.Z[((size_t)sc * n_sym + s) * ntr + l].x : 0.f;
    }
    for (int k = tid; k < nrows * NTR; k += kThreads) {
        const int r = k / NTR, l = k - r * NTR;
        int v = 1;  // padding rows and levels: rank 1
        if (r < n_pe && l < ntr) {
            v = a.paths[((size_t)sc * n_pe + r) * ntr + l];
            if (v < 1 || v > L) {
                atomicOr(a.status, kStatusBadPathEntry);
                v = v < 1 ? 1 : L;
            }
        }
        sTab[k] = (uint8_t)v;
    }
    for (int k = tid; k < n_sym * NTR * BH * 2; k += kThreads) sM[k] = kInfBits;
    for (int k = tid; k < n_sym; k += kThreads) sBest[k] = ~0ull;
    __syncthreads();

    // ---- walks: warp item = (chunk of 32 rows, symbol)
    for (int item = warp; item < chunks * n_sym; item += kWarps) {
        const int chunk = item / n_sym, s = item - chunk * n_sym;
        const int row = chunk * 32 + lane;
        const bool active = row < n_pe;
        const uint8_t *trow = sTab + row * NTR;
        float e[NTR];
#pragma unroll
        for (int i = 0; i < NTR; ++i) {
            const int lz = ntr - 1 - i;
            e[i] = lz >= 0 ? sZ[s * NTR + lz] : 0.f;
        }
        Lab lab;
        lab.clear();
        float d = 0.f;
#pragma unroll 1
        for (int l = ntr - 1; l >= 0; --l) {
            const int p = trow[l];
            const float b = e[0] * sInvd[l];
            float dist;
            const int idx = pam_kth<QAM>(b, p, dist);
            d = fmaf(sR2[l], dist, d);
            lab.push(Qam<QAM>::axis_label(idx));
            cancel_level_r<NTR>(l, e, sRr + l * NTR, axis_pos<QAM>(idx));
        }
        warp_reduce_symbol<NTR, BH>(true, active, row, chunk, chunks, ntr, d, lab, s, sBest,
                                    sWmin, sSecond, sBlab, sM, a.llr != nullptr);
    }
    __syncthreads();

    // ---- per-symbol results, each user's two axes joined; the level of a
    // real column is found in the permutation
    auto level_of = [&](int col) {
        int lv = 0;
        for (int l = 0; l < ntr; ++l)
            if (sPerm[l] == col) lv = l;
        return lv;
    };
    for (int s = warp; s < n_sym; s += kWarps) {
        const size_t det = (size_t)sc * n_sym + s;
        const unsigned long long key = sBest[s];
        const unsigned bd = (unsigned)(key >> 32);
        int bc = (int)((key & 0xffffu) >> 5);
        if (bc >= chunks) bc = 0;
        const uint32_t *wb = sBlab + (s * chunks + bc) * WORDS;
        if (lane < nt) {
            const int lre = label_at<BH>(wb, level_of(lane));
            const int lim = label_at<BH>(wb, level_of(nt + lane));
            a.hard[det * nt + lane] = (uint8_t)join_label<QAM>(lre, lim);
        }
        if (a.ped2 != nullptr) {
            unsigned sec = kInfBits;
            for (int c = lane; c < chunks; c += 32)
                sec = min(sec, c == bc ? sSecond[s * chunks + c] : sWmin[s * chunks + c]);
            sec = __reduce_min_sync(0xffffffffu, sec);
            if (lane == 0) {
                a.ped2[det * 2] = __uint_as_float(bd);
                a.ped2[det * 2 + 1] = __uint_as_float(sec);
            }
        }
        if (a.llr != nullptr) {
            for (int slot = lane; slot < nt * B; slot += 32) {
                const int u = slot / B, bit = slot - u * B;
                const int l = level_of((bit & 1) * nt + u);  // even bits: real axis, odd: imaginary
                const unsigned *mm = sM + (s * NTR * BH + l * BH + (bit >> 1)) * 2;
                float v;
                if (mm[1] == kInfBits) v = kLlrMax;
                else if (mm[0] == kInfBits) v = -kLlrMax;
                else v = (__uint_as_float(mm[1]) - __uint_as_float(mm[0])) / a.sigma2;
                a.llr[(det * nt + u) * B + bit] = v;
            }
        }
    }
}

template <int NTR, int QAM>
cudaError_t launch_rvd_tpl(int n_sc, const RvdArgs &a, cudaStream_t stream)
{
    constexpr int BH = Qam<QAM>::B / 2;
    const size_t smem = rvd_layout(NTR, BH, a.n_pe, a.n_sym, Labels<NTR, BH>::WORDS).bytes;
    cudaError_t e = allow_dynamic_smem(detect_rvd_kernel<NTR, QAM>, smem);
    if (e != cudaSuccess) return e;
    detect_rvd_kernel<NTR, QAM><<<n_sc, kThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int NTR>
cudaError_t launch_rvd_q(int n_sc, int qam, const RvdArgs &a, cudaStream_t stream)
{
    switch (qam) {
    case 4: return launch_rvd_tpl<NTR, 4>(n_sc, a, stream);
    case 16: return launch_rvd_tpl<NTR, 16>(n_sc, a, stream);
    default: return launch_rvd_tpl<NTR, 64>(n_sc, a, stream);
    }
}

// Hr [n_sc][2nr][2nt] and Yr [n_sc][n_sym][2nr] (complex, imaginary parts
// zero) from H and Y; one thread per output element.
__global__ void rvd_embed_kernel(int n_sc, int n_sym, int nr, int nt, const float2 *__restrict__ H,
                                 const float2 *__restrict__ Y, float2 *__restrict__ Hr,
                                 float2 *__restrict__ Yr)
{
    const long long nh = (long long)n_sc * 4 * nr * nt;
    const long long ny = (long long)n_sc * n_sym * 2 * nr;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nh + ny; k += stride) {
        if (k < nh) {
            const int c = (int)(k % (2 * nt));
            const int r = (int)((k / (2 * nt)) % (2 * nr));
            const long long sc = k / (4LL * nr * nt);
            const float2 h = H[(sc * nr + (r % nr)) * nt + (c % nt)];
            // [[Re H, -Im H]; [Im H, Re H]]
            float v;
            if (r < nr) v = c < nt ? h.x : -h.y;
            else v = c < nt ? h.y : h.x;
            Hr[k] = make_float2(v, 0.f);
        } else {
            const long long j = k - nh;
            const int r = (int)(j % (2 * nr));
            const long long q = j / (2 * nr);  // (sc, symbol)
            const float2 y = Y[q * nr + (r % nr)];
            Yr[j] = make_float2(r < nr ? y.x : y.y, 0.f);
        }
    }
}

}  // namespace

size_t rvd_smem_bytes(int nt, int qam, int n_pe, int n_sym)
{
    const int ntr = 2 * nt;
    const int NTR = ntr <= 4 ? 4 : (ntr <= 8 ? 8 : 16);
    const int BH = (qam == 4 ? 2 : (qam == 16 ? 4 : 6)) / 2;
    return rvd_layout(NTR, BH, n_pe, n_sym, (NTR * BH + 31) / 32).bytes;
}

cudaError_t launch_rvd_embed(int n_sc, int n_sym, int nr, int nt, const float2 *H, const float2 *Y,
                             float2 *Hr, float2 *Yr, cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    const long long total = (long long)n_sc * (4LL * nr * nt + 2LL * n_sym * nr);
    long long grid = (total + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    rvd_embed_kernel<<<(unsigned)grid, 256, 0, stream>>>(n_sc, n_sym, nr, nt, H, Y, Hr, Yr);
    return cudaGetLastError();
}

cudaError_t launch_detect_rvd(int n_sc, int n_sym, int nt, int qam, int n_pe, float sigma2,
                              const float2 *R, const float *inv_diag, const uint8_t *perm,
                              const uint8_t *paths, const float2 *Z, uint8_t *hard, float *llr,
                              float *ped2, unsigned *status, cudaStream_t stream)
{
    if (n_sc == 0) return cudaSuccess;
    const RvdArgs a{n_sym, nt, n_pe, sigma2, R, inv_diag, perm, paths, Z, hard, llr, ped2, status};
    const int ntr = 2 * nt;
    if (ntr <= 4) return launch_rvd_q<4>(n_sc, qam, a, stream);
    if (ntr <= 8) return launch_rvd_q<8>(n_sc, qam, a, stream);
    return launch_rvd_q<16>(n_sc, qam, a, stream);
}

}  // namespace mpnl
