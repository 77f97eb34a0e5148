// Table-driven rank model, offline part: the rank-probability histogram of
// the sent symbol per SNR by Monte-Carlo, and the rank costs derived from it
// (mpnl_rank_counts, mpnl_rank_costs).  The per-level model is a reading:
// the paper gives none; this is the FlexCore-style alternative to the
// geometric model, with the probability of each rank estimated once per SNR
// and looked up per level by mpnl_select_paths_lut.
//
// Per SNR gamma_b, every trial draws a label s uniformly and complex
// Gaussian noise n of total variance 1/gamma_b -- the law of
// b_l = s + n_l / R_ll in the walks when gamma = R_ll^2 / sigma2 and
// E_s = 1 -- and counts the rank of s among all M points ordered by
// (|b - q|^2, label).  Arithmetic in double (an offline table; GB300's FP64
// rate is ample for millions of trials).
//
// Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a
// counter-based generator.  Draw n is
//   z = seed + n * 0x9E3779B97F4A7C15,
//   z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9,
//   z = (z ^ (z >> 27)) * 0x94D049BB133111EB,  out = z ^ (z >> 31),
// with n = 1 + (b << 40) + (t << 2) + i for draw i of trial t.  Draw 0 gives
// the label (its top B bits); draws 1 and 2 give u = ((out >> 11) + 0.5)
// 2^-53 in (0, 1), and Box-Muller gives the noise:
// r = sqrt(-2 ln u1 / (2 gamma)), n = r (cos 2 pi u2, sin 2 pi u2).
#include "mpnl_common.cuh"
#include "mpnl_internal.h"

namespace mpnl {
namespace {

constexpr int kLutThreads = 256;
constexpr double kTwoPi = 6.283185307179586476925;
constexpr double kLn2 = 0.69314718055994530942;

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long n)
{
    unsigned long long z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double unit_open(unsigned long long x)
{
    return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

// grid: (chunks of trials, bins); a CTA histograms its trials in shared
// memory and adds them to the bin's global counters once.
template <int QAM>
__global__ void __launch_bounds__(kLutThreads)
rank_counts_kernel(const double *__restrict__ gamma, long long n_trials, unsigned long long seed,
                   unsigned long long *__restrict__ counts)
{
    constexpr int M = QAM, B = Qam<QAM>::B, L = Qam<QAM>::L;
    __shared__ double2 pts[M];
    __shared__ unsigned hist[M];
    const int bin = blockIdx.y;
    if (threadIdx.x < M) {
        const int ire = threadIdx.x / L, iim = threadIdx.x % L;
        const double inv = 1.0 / sqrt(QAM == 4 ? 2.0 : (QAM == 16 ? 10.0 : 42.0));
        const int lab = join_label<QAM>(Qam<QAM>::axis_label(ire), Qam<QAM>::axis_label(iim));
        pts[lab] = make_double2((double)(2 * ire - (L - 1)) * inv, (double)(2 * iim - (L - 1)) * inv);
        hist[threadIdx.x] = 0u;
    }
    __syncthreads();
    const double sd = sqrt(1.0 / (2.0 * gamma[bin]));
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_trials; t += stride) {
        const unsigned long long base =
            1ull + ((unsigned long long)bin << 40) + ((unsigned long long)t << 2);
        const int s = (int)(splitmix64_at(seed, base) >> (64 - B));
        const double u1 = unit_open(splitmix64_at(seed, base + 1));
        const double u2 = unit_open(splitmix64_at(seed, base + 2));
        const double r = sqrt(-2.0 * log(u1)) * sd;
        double sn, cs;
        sincos(kTwoPi * u2, &sn, &cs);
        const double2 ps = pts[s];
        const double yx = ps.x + r * cs, yy = ps.y + r * sn;
        const double ex = yx - ps.x, ey = yy - ps.y;
        const double ds = ex * ex + ey * ey;
        int rank = 1;
        for (int q = 0; q < M; ++q) {
            const double dx = yx - pts[q].x, dy = yy - pts[q].y;
            const double dq = dx * dx + dy * dy;
            rank += (q != s && (dq < ds || (dq == ds && q < s))) ? 1 : 0;
        }
        atomicAdd(&hist[rank - 1], 1u);
    }
    __syncthreads();
    if (threadIdx.x < M && hist[threadIdx.x] != 0u)
        atomicAdd(counts + (size_t)bin * M + threadIdx.x, (unsigned long long)hist[threadIdx.x]);
}

// Costs (a reading): c(k) = log P(1) - log P(k) with P(k) = count_k /
// n_trials for the ranks seen; a rank never seen is taken as half as likely
// as the rank before it (c(k) = c(k-1) + ln 2: every cost finite, the unseen
// ranks still ordered); rank 1 never seen counts as half a trial.  Made
// nondecreasing in k by a running maximum; c(1) = 0.  One thread per bin.
__global__ void rank_costs_kernel(int qam, int n_bins, const unsigned long long *__restrict__ counts,
                                  long long n_trials, float *__restrict__ cost)
{
    const int bin = blockIdx.x * blockDim.x + threadIdx.x;
    if (bin >= n_bins) return;
    const unsigned long long *cnt = counts + (size_t)bin * qam;
    float *c = cost + (size_t)bin * qam;
    const double n = (double)n_trials;
    const double lp1 = log((cnt[0] > 0 ? (double)cnt[0] : 0.5) / n);
    double run = 0.0;
    c[0] = 0.f;
    for (int k = 1; k < qam; ++k) {
        const double v = cnt[k] > 0 ? lp1 - log((double)cnt[k] / n) : run + kLn2;
        run = v > run ? v : run;
        c[k] = (float)run;
    }
}

template <int QAM>
cudaError_t launch_counts_tpl(int n_bins, const double *gamma, long long n_trials,
                              unsigned long long seed, unsigned long long *counts,
                              cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)n_bins * QAM,
                                    stream);
    if (e != cudaSuccess) return e;
    long long chunks = (n_trials + (long long)kLutThreads * 64 - 1) / ((long long)kLutThreads * 64);
    if (chunks > 1024) chunks = 1024;
    if (chunks < 1) chunks = 1;
    const dim3 grid((unsigned)chunks, (unsigned)n_bins);
    rank_counts_kernel<QAM><<<grid, kLutThreads, 0, stream>>>(gamma, n_trials, seed, counts);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rank_counts(int qam, int n_bins, const double *gamma, long long n_trials,
                               unsigned long long seed, unsigned long long *counts,
                               cudaStream_t stream)
{
    switch (qam) {
    case 4: return launch_counts_tpl<4>(n_bins, gamma, n_trials, seed, counts, stream);
    case 16: return launch_counts_tpl<16>(n_bins, gamma, n_trials, seed, counts, stream);
    default: return launch_counts_tpl<64>(n_bins, gamma, n_trials, seed, counts, stream);
    }
}

cudaError_t launch_rank_costs(int qam, int n_bins, const unsigned long long *counts,
                              long long n_trials, float *cost, cudaStream_t stream)
{
    rank_costs_kernel<<<(n_bins + 127) / 128, 128, 0, stream>>>(qam, n_bins, counts, n_trials,
                                                                cost);
    return cudaGetLastError();
}

}  // namespace mpnl
