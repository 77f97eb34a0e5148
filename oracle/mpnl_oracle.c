/*
 * FP64 CPU oracle of the MPNL uplink detection path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may build, load or call it; the product
 * library never links it and shares no code, header or table with it.
 *
 * What it computes (Katsaros & Nikitopoulos, "Enabling Ultra-Dense, Open-RAN,
 * Vehicular Networks with Non-Linear MIMO Processing", arXiv 2409.14355):
 *   §II (Background) describes MPNL only in words: the position of the most
 *   promising solutions relative to any transmit vector is found from the
 *   channel alone, before data arrives, and during transmission the N_p most
 *   promising candidate vectors are evaluated in parallel.  §III-B fixes
 *   N_p <= 32 for the link simulations and the 14-symbol slot (12 data +
 *   2 DMRS) over which the channel is constant; §III-B also names the linear
 *   MMSE detector as the baseline.  Everything below that the paper leaves
 *   open is a stated reading (each marked "Reading:"):
 *
 *   1. sorted QR (SQRD, Wuebben et al. 2001) of H by modified Gram-Schmidt with
 *      the minimum-residual-norm column picked first;
 *   2. z = Q^H y per OFDM symbol;
 *   3. per-level error model and best-first selection of the N_pe most
 *      probable position vectors (rank of the chosen symbol at each level);
 *   4. the N_pe walks: interference cancellation, p_l-th nearest symbol,
 *      partial Euclidean distance (PED);
 *   5. argmin over the list -> hard decisions, un-permuted to user order;
 *   6. max-log LLRs over the list;
 *   7. linear MMSE baseline with 1-D max-log LLRs.
 *
 * Precision: double throughout.  Complex values cross the interface as
 * interleaved (re, im) doubles.  No blocking, fusion or reordering beyond
 * what the definitions state.  Build flags keep FMA contraction off so that
 * x86 and Arm hosts round identically.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef double complex cplx;

#define ORC_MAX_NT 16
#define ORC_MAX_NR 32
#define ORC_MAX_M 64
#define ORC_MAX_NPE 1024
/* Reading: LLR magnitude used when the list holds no candidate with the
 * opposite bit value (max-log has no finite value then). */
#define ORC_LLR_MAX 20.0
/* Reading: the per-level symbol-error probability is floored at this value so
 * that no level is ever treated as error-free (keeps every log finite). */
#define ORC_PE_FLOOR 1e-12
#define ORC_PI 3.14159265358979323846
#define ORC_LN2 0.69314718055994530942

static int bits_of(int qam)
{
    switch (qam) {
    case 4: return 2;
    case 16: return 4;
    case 64: return 6;
    default: return 0;
    }
}

/* ---------------------------------------------------------------------------
 * Constellation: 3GPP TS 38.211 §5.1.3 (QPSK), §5.1.4 (16QAM), §5.1.5 (64QAM).
 * Bits b0..b{B-1}; the label is the integer with b0 as its most significant
 * bit.  Unit average energy.
 * ------------------------------------------------------------------------- */
static cplx qam_point(int qam, int label)
{
    int B = bits_of(qam);
    int b[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < B; i++)
        b[i] = (label >> (B - 1 - i)) & 1;
    double re, im;
    if (qam == 4) {
        re = (1 - 2 * b[0]) / sqrt(2.0);
        im = (1 - 2 * b[1]) / sqrt(2.0);
    } else if (qam == 16) {
        re = (1 - 2 * b[0]) * (2 - (1 - 2 * b[2])) / sqrt(10.0);
        im = (1 - 2 * b[1]) * (2 - (1 - 2 * b[3])) / sqrt(10.0);
    } else {
        re = (1 - 2 * b[0]) * (4 - (1 - 2 * b[2]) * (2 - (1 - 2 * b[4]))) / sqrt(42.0);
        im = (1 - 2 * b[1]) * (4 - (1 - 2 * b[3]) * (2 - (1 - 2 * b[5]))) / sqrt(42.0);
    }
    return re + I * im;
}

int orc_constellation(int qam, double *pts)
{
    if (!bits_of(qam)) return -1;
    for (int l = 0; l < qam; l++) {
        cplx q = qam_point(qam, l);
        pts[2 * l] = creal(q);
        pts[2 * l + 1] = cimag(q);
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Step 1: sorted QR decomposition H P = Q R (SQRD, Wuebben et al. 2001), the
 * channel pre-processing of §II ("observing the MIMO channel").
 * Modified Gram-Schmidt; at step i the remaining column with the smallest
 * residual norm becomes column i (tie -> smaller original column index).
 * R is upper triangular with a real, positive diagonal.  Detection later
 * starts at the last level (index nt-1), the column picked last.
 *
 * H: [nr][nt] row-major complex.  Q: [nr][nt].  R: [nt][nt] (full, zero below
 * the diagonal).  perm[i] = original column (user) that became column i.
 * gap[i] (optional): relative gap between the smallest and second smallest
 * candidate norm at step i (+inf when only one candidate is left); used by
 * the tests to spot ordering near-ties.
 * ------------------------------------------------------------------------- */
static void sqrd(int nr, int nt, const cplx *H, cplx *Q, cplx *R, int *perm, double *gap)
{
    for (int r = 0; r < nr; r++)
        for (int c = 0; c < nt; c++)
            Q[r * nt + c] = H[r * nt + c];
    for (int i = 0; i < nt * nt; i++)
        R[i] = 0.0;
    for (int c = 0; c < nt; c++)
        perm[c] = c;

    for (int i = 0; i < nt; i++) {
        /* residual norms of the columns not yet placed */
        double norm[ORC_MAX_NT];
        for (int k = i; k < nt; k++) {
            double s = 0.0;
            for (int r = 0; r < nr; r++) {
                cplx v = Q[r * nt + k];
                s += creal(v) * creal(v) + cimag(v) * cimag(v);
            }
            norm[k] = s;
        }
        int kmin = i;
        for (int k = i + 1; k < nt; k++) {
            if (norm[k] < norm[kmin] || (norm[k] == norm[kmin] && perm[k] < perm[kmin]))
                kmin = k;
        }
        if (gap) {
            double second = INFINITY;
            for (int k = i; k < nt; k++)
                if (k != kmin && norm[k] < second) second = norm[k];
            gap[i] = isinf(second) ? INFINITY : (second - norm[kmin]) / norm[kmin];
        }
        /* swap column i and kmin in Q, in the already computed rows of R, and in perm */
        if (kmin != i) {
            for (int r = 0; r < nr; r++) {
                cplx t = Q[r * nt + i];
                Q[r * nt + i] = Q[r * nt + kmin];
                Q[r * nt + kmin] = t;
            }
            for (int r = 0; r < i; r++) {
                cplx t = R[r * nt + i];
                R[r * nt + i] = R[r * nt + kmin];
                R[r * nt + kmin] = t;
            }
            int t = perm[i];
            perm[i] = perm[kmin];
            perm[kmin] = t;
        }
        double rii = sqrt(norm[kmin]);
        R[i * nt + i] = rii;
        for (int r = 0; r < nr; r++)
            Q[r * nt + i] /= rii;
        for (int j = i + 1; j < nt; j++) {
            cplx rij = 0.0;
            for (int r = 0; r < nr; r++)
                rij += conj(Q[r * nt + i]) * Q[r * nt + j];
            R[i * nt + j] = rij;
            for (int r = 0; r < nr; r++)
                Q[r * nt + j] -= rij * Q[r * nt + i];
        }
    }
}

int orc_sqrd(int nr, int nt, const double *H, double *Q, double *R, int *perm, double *gap)
{
    if (nt < 1 || nt > ORC_MAX_NT || nr < nt || nr > ORC_MAX_NR) return -1;
    sqrd(nr, nt, (const cplx *)H, (cplx *)Q, (cplx *)R, perm, gap);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Step 1 for more users than antennas (Nt > Nr, the regime of §III-IV where
 * MPNL serves e.g. 12 streams on 7 antennas).  Reading: the MMSE-extended
 * sorted QR (Wuebben et al. 2003): the SQRD above applied to the augmented
 * channel H_a = [H; sigma I] ((nr + nt) x nt) and y_a = [y; 0].  Then
 * ||y_a - H_a s||^2 = ||y - H s||^2 + sigma2 ||s||^2, R is nt x nt and
 * regular for any nr, and z = Q_a^H y_a uses only the top nr rows of Q_a.
 * Q: [(nr + nt)][nt].
 * ------------------------------------------------------------------------- */
static void augment(int nr, int nt, const cplx *H, double sigma2, cplx *Ha)
{
    double sg = sqrt(sigma2);
    for (int r = 0; r < nr + nt; r++)
        for (int c = 0; c < nt; c++)
            Ha[r * nt + c] = r < nr ? H[r * nt + c] : (r - nr == c ? sg : 0.0);
}

int orc_sqrd_mmse(int nr, int nt, const double *H, double sigma2, double *Q, double *R, int *perm,
                  double *gap)
{
    if (nt < 1 || nt > ORC_MAX_NT || nr < 1 || nr + nt > ORC_MAX_NR || !(sigma2 > 0.0)) return -1;
    cplx Ha[ORC_MAX_NR * ORC_MAX_NT];
    augment(nr, nt, (const cplx *)H, sigma2, Ha);
    sqrd(nr + nt, nt, Ha, (cplx *)Q, (cplx *)R, perm, gap);
    return 0;
}

/* Step 2: z = Q^H y for each OFDM symbol.  Y: [n_sym][nr], Z: [n_sym][nt]. */
static void qhy(int nr, int nt, int n_sym, const cplx *Q, const cplx *Y, cplx *Z)
{
    for (int s = 0; s < n_sym; s++)
        for (int i = 0; i < nt; i++) {
            cplx acc = 0.0;
            for (int r = 0; r < nr; r++)
                acc += conj(Q[r * nt + i]) * Y[s * nr + r];
            Z[s * nt + i] = acc;
        }
}

int orc_qhy(int nr, int nt, int n_sym, const double *Q, const double *Y, double *Z)
{
    if (nt < 1 || nt > ORC_MAX_NT || nr < nt || nr > ORC_MAX_NR) return -1;
    qhy(nr, nt, n_sym, (const cplx *)Q, (const cplx *)Y, (cplx *)Z);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Step 3: selection of the N_pe most promising position vectors (§II: found
 * "before any transmission begins", from the channel only; §III-B: N_p).
 *
 * A position vector p has one entry per level, p_l in 1..M: the rank (by
 * distance to the level's unconstrained estimate) of the symbol taken at that
 * level.  Reading of the error model (the paper gives none):
 *   gamma_l = R_ll^2 / sigma2                    (unit-energy symbols)
 *   Pe_l    = 1 - (1 - c Qf(sqrt(3 gamma_l / (M - 1))))^2, c = 2 (1 - 1/sqrt(M)),
 *             the nearest-neighbour symbol-error rate of square M-QAM,
 *             floored at ORC_PE_FLOOR; Qf(x) = erfc(x / sqrt 2) / 2
 *   P_l(k)  = (1 - Pe_l) Pe_l^(k-1)              (geometric rank model)
 *   score(p) = sum_l log P_l(p_l)
 * The N_pe vectors of largest score are enumerated best-first from the
 * all-ones vector (the plain SIC path).  Order: larger score first; equal
 * scores -> lexicographically smaller vector first, comparing from the top
 * level (index nt-1) down.  Children of p: p + e_l for every level
 * l >= h(p), where h(p) is the highest level with p_l > 1 (h = 0 for the
 * all-ones vector); this reaches every vector exactly once, and a child never
 * precedes its parent.
 * The frontier is a plain array scanned linearly for its best entry.
 *
 * rdiag[nt]: R_ll.  paths: [n_pe][nt] ranks (1-based), rows in pop order.
 * score[n_pe] (optional), level_pe[nt] (optional).
 * ------------------------------------------------------------------------- */
static double level_pe(double rll, double sigma2, int M)
{
    double gamma = rll * rll / sigma2;
    double x = sqrt(3.0 * gamma / (double)(M - 1));
    double qf = 0.5 * erfc(x / sqrt(2.0));
    double cq = 2.0 * (1.0 - 1.0 / sqrt((double)M)) * qf;
    /* 1 - (1 - cq)^2 written as cq (2 - cq): same value, no cancellation when
     * cq is tiny (high SNR) */
    double pe = cq * (2.0 - cq);
    if (pe < ORC_PE_FLOOR) pe = ORC_PE_FLOOR;
    return pe;
}

typedef struct {
    unsigned char p[ORC_MAX_NT];
    double score;
} orc_cand;

/* 1 if a precedes b in the selection order */
static int cand_before(const orc_cand *a, const orc_cand *b, int nt)
{
    if (a->score > b->score) return 1;
    if (a->score < b->score) return 0;
    for (int l = nt - 1; l >= 0; l--) {
        if (a->p[l] < b->p[l]) return 1;
        if (a->p[l] > b->p[l]) return 0;
    }
    return 0;
}

/* Best-first enumeration over per-level log-probabilities logp[l][k] (rank
 * k = 1..M at level l), nonincreasing in k so that a child never precedes
 * its parent.  Shared by the geometric model and the table-driven model. */
static int select_best_first(int nt, int qam, double logp[ORC_MAX_NT][ORC_MAX_M + 1], int n_pe,
                             unsigned char *paths, double *score_out)
{
    int M = qam;
    size_t cap = 1 + (size_t)n_pe * (size_t)nt;
    orc_cand *front = (orc_cand *)malloc(cap * sizeof(orc_cand));
    if (!front) return -2;
    size_t nf = 0;
    orc_cand root;
    memset(&root, 0, sizeof root);
    root.score = 0.0;
    for (int l = 0; l < nt; l++) {
        root.p[l] = 1;
        root.score += logp[l][1];
    }
    front[nf++] = root;
    for (int n = 0; n < n_pe; n++) {
        if (nf == 0) {
            free(front);
            return -3; /* fewer than n_pe vectors exist */
        }
        size_t best = 0;
        for (size_t f = 1; f < nf; f++)
            if (cand_before(&front[f], &front[best], nt)) best = f;
        orc_cand c = front[best];
        front[best] = front[--nf];
        memcpy(paths + (size_t)n * nt, c.p, (size_t)nt);
        if (score_out) score_out[n] = c.score;
        int h = 0;
        for (int l = nt - 1; l >= 0; l--)
            if (c.p[l] > 1) {
                h = l;
                break;
            }
        for (int l = h; l < nt; l++) {
            if (c.p[l] >= M) continue;
            orc_cand ch = c;
            ch.p[l] += 1;
            ch.score = 0.0;
            for (int m = 0; m < nt; m++)
                ch.score += logp[m][ch.p[m]];
            front[nf++] = ch;
        }
    }
    free(front);
    return 0;
}

static int select_paths(int nt, int qam, const double *rdiag, double sigma2, int n_pe,
                        unsigned char *paths, double *score_out, double *pe_out)
{
    int M = qam;
    double logp[ORC_MAX_NT][ORC_MAX_M + 1];
    for (int l = 0; l < nt; l++) {
        double pe = level_pe(rdiag[l], sigma2, M);
        if (pe_out) pe_out[l] = pe;
        for (int k = 1; k <= M; k++)
            logp[l][k] = log(1.0 - pe) + (double)(k - 1) * log(pe);
    }
    return select_best_first(nt, qam, logp, n_pe, paths, score_out);
}

static double ipow(double b, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; i++) r *= b;
    return r;
}

int orc_select_paths(int nt, int qam, const double *rdiag, double sigma2, int n_pe,
                     unsigned char *paths, double *score, double *pe)
{
    if (nt < 1 || nt > ORC_MAX_NT || !bits_of(qam) || n_pe < 1 || n_pe > ORC_MAX_NPE) return -1;
    if ((double)n_pe > ipow((double)qam, nt)) return -1;
    if (!(sigma2 > 0.0)) return -1;
    return select_paths(nt, qam, rdiag, sigma2, n_pe, paths, score, pe);
}

/* ---------------------------------------------------------------------------
 * Table-driven rank model (Reading: the paper gives no model; this is the
 * alternative to the geometric model above in which the probability of each
 * rank is estimated once, offline, per SNR, and looked up per level).
 *
 * Estimation by Monte-Carlo, per SNR gamma_b (b = 0..n_bins-1): n_trials
 * draws of a uniformly chosen constellation label s and of complex Gaussian
 * noise n of total variance 1/gamma_b -- the law of b_l = s + n_l / R_ll in
 * step 4 when gamma = R_ll^2 / sigma2 and E_s = 1 -- and the rank of s among
 * all M points ordered by (|b - q|^2, label) is counted: counts[b][k-1].
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
 * counter-based generator.  Draw number n gives
 *   z = seed + n * 0x9E3779B97F4A7C15;
 *   z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
 *   z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
 *   out = z ^ (z >> 31)
 * with n = 1 + (b << 40) + (t << 2) + i for draw i (0..2) of trial t (t < 2^38).
 * Draw 0: the label, its top B bits.  Draws 1, 2: u = ((out >> 11) + 0.5)
 * 2^-53, in (0, 1).  Noise by Box-Muller: r = sqrt(-2 ln u1 / (2 gamma)),
 * n = r (cos 2 pi u2, sin 2 pi u2).
 *
 * Costs (Reading): P(k) = counts[k-1] / n_trials, c(k) = log P(1) - log P(k)
 * for the ranks seen; a rank never seen is taken as half as likely as the
 * rank before it (c(k) = c(k-1) + ln 2, a geometric tail: every cost finite
 * and the unseen ranks still ordered); rank 1 never seen counts as half a
 * trial.  The costs are then made nondecreasing in k by a running maximum
 * (so the top-N set stays downward-closed); c(1) = 0.  Selection then
 * maximises -sum_l c_l(p_l), which orders vectors as sum_l log P_l(p_l)
 * does wherever P is nonincreasing.
 *
 * Lookup: the bin of a level is the number of edges e (ascending, n_bins - 1
 * of them) with gamma >= e, where gamma = R_ll^2 / sigma2 is formed in
 * float (R_ll and sigma2 rounded to float first): a float decides the bin, in
 * the precision the GPU path uses.
 * ------------------------------------------------------------------------- */
static uint64_t splitmix64_at(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double unit_open(uint64_t x)
{
    return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

int orc_rank_counts_mc(int qam, int n_bins, const double *gamma, long long n_trials,
                       unsigned long long seed, long long *counts)
{
    int M = qam, B = bits_of(qam);
    if (!B || n_bins < 1 || n_trials < 1 || n_trials >= (1ll << 38)) return -1;
    cplx pts[ORC_MAX_M];
    for (int q = 0; q < M; q++) pts[q] = qam_point(qam, q);
    for (int b = 0; b < n_bins; b++) {
        if (!(gamma[b] > 0.0)) return -1;
        long long *cnt = counts + (size_t)b * M;
        for (int k = 0; k < M; k++) cnt[k] = 0;
        double sd = sqrt(1.0 / (2.0 * gamma[b]));
        for (long long t = 0; t < n_trials; t++) {
            uint64_t base = 1ull + ((uint64_t)b << 40) + ((uint64_t)t << 2);
            int s = (int)(splitmix64_at(seed, base) >> (64 - B));
            double u1 = unit_open(splitmix64_at(seed, base + 1));
            double u2 = unit_open(splitmix64_at(seed, base + 2));
            double r = sqrt(-2.0 * log(u1)) * sd;
            double th = 2.0 * ORC_PI * u2;
            cplx y = pts[s] + r * cos(th) + I * (r * sin(th));
            cplx df = y - pts[s];
            double ds = creal(df) * creal(df) + cimag(df) * cimag(df);
            int rank = 1;
            for (int q = 0; q < M; q++) {
                if (q == s) continue;
                cplx e = y - pts[q];
                double dq = creal(e) * creal(e) + cimag(e) * cimag(e);
                if (dq < ds || (dq == ds && q < s)) rank++;
            }
            cnt[rank - 1]++;
        }
    }
    return 0;
}

int orc_rank_costs(int qam, int n_bins, const long long *counts, long long n_trials, double *cost)
{
    int M = qam;
    if (!bits_of(qam) || n_bins < 1 || n_trials < 1) return -1;
    for (int b = 0; b < n_bins; b++) {
        const long long *cnt = counts + (size_t)b * M;
        double *c = cost + (size_t)b * M;
        double lp1 = log((cnt[0] > 0 ? (double)cnt[0] : 0.5) / (double)n_trials);
        c[0] = 0.0;
        for (int k = 1; k < M; k++) {
            double v = cnt[k] > 0 ? lp1 - log((double)cnt[k] / (double)n_trials)
                                  : c[k - 1] + ORC_LN2;
            c[k] = v > c[k - 1] ? v : c[k - 1];
        }
    }
    return 0;
}

static int lut_bin(double rll, double sigma2, int n_bins, const float *edges)
{
    float rf = (float)rll, s2 = (float)sigma2;
    float sq = rf * rf;
    float g = sq / s2;
    int b = 0;
    for (int e = 0; e < n_bins - 1; e++)
        if (g >= edges[e]) b = e + 1;
    return b;
}

int orc_select_paths_lut(int nt, int qam, const double *rdiag, double sigma2, int n_bins,
                         const float *edges, const float *cost, int n_pe, unsigned char *paths,
                         double *score, int *bins)
{
    if (nt < 1 || nt > ORC_MAX_NT || !bits_of(qam) || n_pe < 1 || n_pe > ORC_MAX_NPE) return -1;
    if ((double)n_pe > ipow((double)qam, nt)) return -1;
    if (!(sigma2 > 0.0) || n_bins < 1) return -1;
    int M = qam;
    double logp[ORC_MAX_NT][ORC_MAX_M + 1];
    for (int l = 0; l < nt; l++) {
        int b = lut_bin(rdiag[l], sigma2, n_bins, edges);
        if (bins) bins[l] = b;
        for (int k = 1; k <= M; k++)
            logp[l][k] = -(double)cost[(size_t)b * M + (k - 1)];
    }
    return select_best_first(nt, qam, logp, n_pe, paths, score);
}

/* ---------------------------------------------------------------------------
 * Step 4-6: evaluation of the N_pe position vectors for one subcarrier
 * (§II: the most promising solutions "processed in parallel").
 *
 * For every symbol and every row p of the table, independently:
 *   for l = nt-1 down to 0:
 *     e_l = z_l - sum_{j>l} R_lj s_j
 *     b_l = e_l / R_ll
 *     s_l = the p_l-th closest constellation point to b_l; closeness is
 *           ordered by (|b_l - q|^2, label) ascending (Reading: lower label
 *           wins an exact distance tie)
 *     d  += R_ll^2 |b_l - s_l|^2
 * so that d = ||z - R s||^2 at the end.  The hard decision is the row with
 * the smallest d (tie -> lower row index); user perm[l] receives s_l.
 * Max-log LLR of bit b of user k (Reading: positive means bit 0):
 *   (min_{rows with bit 1} d - min_{rows with bit 0} d) / sigma2,
 *   +ORC_LLR_MAX when no row has the bit at 1, -ORC_LLR_MAX when none has 0.
 *
 * R: [nt][nt] full upper triangular, real positive diagonal.  Z: [n_sym][nt].
 * paths: [n_pe][nt].  Outputs: hard [n_sym][nt] labels in user order,
 * llr [n_sym][nt][B] (user order, bit b0 first), ped2 [n_sym][2] (best and
 * runner-up d; runner-up +inf when n_pe == 1), margin [n_sym] (optional:
 * smallest gap, in constellation distance units, between the chosen point
 * and its neighbours in any ranking of that symbol), ped_all [n_sym][n_pe]
 * (optional), sym_all [n_sym][n_pe][nt] (optional: labels of every walk,
 * detection order), flip_floor [n_sym] (optional: over all rankings whose
 * neighbour gap is below tie_eps, the smallest partial PED through that
 * level; +inf if none).  margin and flip_floor are diagnostics for the tests:
 * they do not change any result.
 * ------------------------------------------------------------------------- */
/* The walks, argmin and LLRs over a constellation given as its M points
 * (label-indexed) with B bits per label: the square QAM of the complex model
 * (detect_sc), or one PAM axis of it in the real-valued decomposition. */
static int detect_pts(int nt, const cplx *pts, int M, int B, int n_sym, const cplx *R,
                      const cplx *Z, const int *perm, int n_pe, const unsigned char *paths,
                      double sigma2, unsigned char *hard, double *llr, double *ped2,
                      double *margin, double *ped_all, unsigned char *sym_all, double tie_eps,
                      double *flip_floor)
{

    double *d = (double *)malloc((size_t)n_pe * sizeof(double));
    unsigned char *lab = (unsigned char *)malloc((size_t)n_pe * nt);
    if (!d || !lab) {
        free(d);
        free(lab);
        return -2;
    }
    for (int s = 0; s < n_sym; s++) {
        const cplx *z = Z + (size_t)s * nt;
        double mg = INFINITY, ff = INFINITY;
        for (int row = 0; row < n_pe; row++) {
            const unsigned char *p = paths + (size_t)row * nt;
            cplx sv[ORC_MAX_NT];
            double dd = 0.0;
            for (int l = nt - 1; l >= 0; l--) {
                cplx e = z[l];
                for (int j = l + 1; j < nt; j++)
                    e -= R[l * nt + j] * sv[j];
                double rll = creal(R[l * nt + l]);
                cplx b = e / rll;
                /* rank all M points by (distance, label) */
                int order[ORC_MAX_M] = {0};
                double dist[ORC_MAX_M] = {0.0};
                for (int q = 0; q < M; q++) {
                    cplx df = b - pts[q];
                    dist[q] = creal(df) * creal(df) + cimag(df) * cimag(df);
                    order[q] = q;
                }
                for (int a = 1; a < M; a++) { /* insertion sort, stable in label */
                    int key = order[a];
                    int c = a - 1;
                    while (c >= 0 && (dist[order[c]] > dist[key] ||
                                      (dist[order[c]] == dist[key] && order[c] > key))) {
                        order[c + 1] = order[c];
                        c--;
                    }
                    order[c + 1] = key;
                }
                int k = p[l] - 1;
                int q = order[k];
                double gk = INFINITY;
                if (k > 0) {
                    double g = sqrt(dist[q]) - sqrt(dist[order[k - 1]]);
                    if (g < gk) gk = g;
                }
                if (k + 1 < M) {
                    double g = sqrt(dist[order[k + 1]]) - sqrt(dist[q]);
                    if (g < gk) gk = g;
                }
                if (gk < mg) mg = gk;
                /* a ranking this close to a tie may resolve the other way in
                 * lower precision; such a walk keeps at least its PED up to
                 * and including this level (the nearer candidate's term) */
                if (gk < tie_eps) {
                    double dn = dist[q];
                    if (k > 0 && dist[order[k - 1]] < dn) dn = dist[order[k - 1]];
                    double part = dd + rll * rll * dn;
                    if (part < ff) ff = part;
                }
                sv[l] = pts[q];
                lab[(size_t)row * nt + l] = (unsigned char)q;
                dd += rll * rll * dist[q];
            }
            d[row] = dd;
        }
        if (margin) margin[s] = mg;
        if (flip_floor) flip_floor[s] = ff;
        if (ped_all) memcpy(ped_all + (size_t)s * n_pe, d, (size_t)n_pe * sizeof(double));
        if (sym_all) memcpy(sym_all + (size_t)s * n_pe * nt, lab, (size_t)n_pe * nt);

        int best = 0;
        for (int row = 1; row < n_pe; row++)
            if (d[row] < d[best]) best = row;
        double second = INFINITY;
        for (int row = 0; row < n_pe; row++)
            if (row != best && d[row] < second) second = d[row];
        ped2[2 * s] = d[best];
        ped2[2 * s + 1] = second;
        for (int l = 0; l < nt; l++)
            hard[(size_t)s * nt + perm[l]] = lab[(size_t)best * nt + l];

        for (int l = 0; l < nt; l++) {
            for (int bit = 0; bit < B; bit++) {
                double m0 = INFINITY, m1 = INFINITY;
                for (int row = 0; row < n_pe; row++) {
                    int v = (lab[(size_t)row * nt + l] >> (B - 1 - bit)) & 1;
                    if (v) {
                        if (d[row] < m1) m1 = d[row];
                    } else {
                        if (d[row] < m0) m0 = d[row];
                    }
                }
                double val;
                if (isinf(m1)) val = ORC_LLR_MAX;
                else if (isinf(m0)) val = -ORC_LLR_MAX;
                else val = (m1 - m0) / sigma2;
                llr[((size_t)s * nt + perm[l]) * B + bit] = val;
            }
        }
    }
    free(d);
    free(lab);
    return 0;
}

static int detect_sc(int nt, int qam, int n_sym, const cplx *R, const cplx *Z, const int *perm,
                     int n_pe, const unsigned char *paths, double sigma2, unsigned char *hard,
                     double *llr, double *ped2, double *margin, double *ped_all,
                     unsigned char *sym_all, double tie_eps, double *flip_floor)
{
    cplx pts[ORC_MAX_M];
    for (int q = 0; q < qam; q++) pts[q] = qam_point(qam, q);
    return detect_pts(nt, pts, qam, bits_of(qam), n_sym, R, Z, perm, n_pe, paths, sigma2, hard,
                      llr, ped2, margin, ped_all, sym_all, tie_eps, flip_floor);
}

int orc_detect(int nt, int qam, int n_sym, const double *R, const double *Z, const int *perm,
               int n_pe, const unsigned char *paths, double sigma2, unsigned char *hard, double *llr,
               double *ped2, double *margin, double *ped_all, unsigned char *sym_all,
               double tie_eps, double *flip_floor)
{
    if (nt < 1 || nt > ORC_MAX_NT || !bits_of(qam) || n_pe < 1 || n_pe > ORC_MAX_NPE) return -1;
    for (int row = 0; row < n_pe; row++)
        for (int l = 0; l < nt; l++) {
            int v = paths[(size_t)row * nt + l];
            if (v < 1 || v > qam) return -1;
        }
    return detect_sc(nt, qam, n_sym, (const cplx *)R, (const cplx *)Z, perm, n_pe, paths, sigma2,
                     hard, llr, ped2, margin, ped_all, sym_all, tie_eps, flip_floor);
}

/* ---------------------------------------------------------------------------
 * Real-valued decomposition (RVD; a variant, the paper uses complex levels):
 *   [Re y; Im y] = [[Re H, -Im H]; [Im H, Re H]] [Re s; Im s] + [Re n; Im n],
 * 2 nt real levels, real column c < nt carrying the real part of user c and
 * column nt + c its imaginary part.  Each real level is one axis of the
 * square QAM: an L-PAM (L = sqrt M) whose points, indexed by the axis label
 * (the label's real-axis bits b0 b2 b4 .. read as an integer, MSB first),
 * are the real parts of the QAM points with those bits and all imaginary-axis
 * bits 0 (TS 38.211 §5.1 maps the two axes by the same rule).  The sorted QR
 * of the real matrix is the complex routine on a matrix with zero imaginary
 * parts (every product and sum stays real).
 *
 * Per-level model for a real level: noise variance sigma2/2 per real
 * dimension, so with gamma_l = R_ll^2 / sigma2 an L-PAM level errs with
 * Pe_l = 2 (1 - 1/L) Q(sqrt(3 gamma_l / (M - 1))) (the same Q argument as the
 * square QAM's), floored as before; P_l(k) geometric over k = 1..L.
 *
 * orc_detect_pam returns, per real level in column order, the chosen axis
 * labels (hard [n_sym][2nt]) and the LLRs of their B/2 bits
 * (llr [n_sym][2nt][B/2]); joining the two axes of each user is left to the
 * caller (bits b0 b2 .. from column u, b1 b3 .. from column nt + u).
 * ------------------------------------------------------------------------- */
static void pam_points(int qam, cplx *pts)
{
    int B = bits_of(qam), H = B / 2, L = 1 << H;
    for (int a = 0; a < L; a++) {
        int lab = 0;
        for (int t = 0; t < H; t++)
            lab |= ((a >> (H - 1 - t)) & 1) << (B - 1 - 2 * t);
        pts[a] = creal(qam_point(qam, lab));
    }
}

int orc_pam_points(int qam, double *pos)
{
    if (!bits_of(qam)) return -1;
    cplx pts[8];
    pam_points(qam, pts);
    for (int a = 0; a < (1 << (bits_of(qam) / 2)); a++) pos[a] = creal(pts[a]);
    return 0;
}

int orc_select_paths_pam(int ntr, int qam, const double *rdiag, double sigma2, int n_pe,
                         unsigned char *paths, double *score, double *pe_out)
{
    int L = 1 << (bits_of(qam) / 2);
    if (ntr < 1 || ntr > ORC_MAX_NT || !bits_of(qam) || n_pe < 1 || n_pe > ORC_MAX_NPE) return -1;
    if ((double)n_pe > ipow((double)L, ntr)) return -1;
    if (!(sigma2 > 0.0)) return -1;
    double logp[ORC_MAX_NT][ORC_MAX_M + 1];
    for (int l = 0; l < ntr; l++) {
        double gamma = rdiag[l] * rdiag[l] / sigma2;
        double x = sqrt(3.0 * gamma / (double)(qam - 1));
        double pe = 2.0 * (1.0 - 1.0 / (double)L) * 0.5 * erfc(x / sqrt(2.0));
        if (pe < ORC_PE_FLOOR) pe = ORC_PE_FLOOR;
        if (pe_out) pe_out[l] = pe;
        for (int k = 1; k <= L; k++)
            logp[l][k] = log(1.0 - pe) + (double)(k - 1) * log(pe);
    }
    return select_best_first(ntr, L, logp, n_pe, paths, score);
}

int orc_detect_pam(int ntr, int qam, int n_sym, const double *R, const double *Z, const int *perm,
                   int n_pe, const unsigned char *paths, double sigma2, unsigned char *hard,
                   double *llr, double *ped2, double *margin, double tie_eps, double *flip_floor)
{
    int B = bits_of(qam), L = 1 << (B / 2);
    if (ntr < 1 || ntr > ORC_MAX_NT || !B || n_pe < 1 || n_pe > ORC_MAX_NPE) return -1;
    for (int row = 0; row < n_pe; row++)
        for (int l = 0; l < ntr; l++) {
            int v = paths[(size_t)row * ntr + l];
            if (v < 1 || v > L) return -1;
        }
    cplx pts[8];
    pam_points(qam, pts);
    return detect_pts(ntr, pts, L, B / 2, n_sym, (const cplx *)R, (const cplx *)Z, perm, n_pe,
                      paths, sigma2, hard, llr, ped2, margin, NULL, NULL, tie_eps, flip_floor);
}

/* ---------------------------------------------------------------------------
 * Step 7: linear MMSE baseline (§I and §III-B: "de facto standard linear
 * MMSE").  A = H^H H + sigma2 I, factored A = L L^H (Cholesky);
 * W = A^{-1} H^H; for each symbol x = W y; mu_k = Re (W H)_kk;
 * x~_k = x_k / mu_k; nu_k = (1 - mu_k) / mu_k (post-detection noise variance
 * for unit-energy symbols).  Hard decision: nearest point to x~_k (tie ->
 * lower label).  LLR of bit b: (min_{q: bit 1} |x~ - q|^2 -
 * min_{q: bit 0} |x~ - q|^2) / nu_k.
 * H: [nr][nt], Y: [n_sym][nr]; outputs in user order: hard [n_sym][nt],
 * llr [n_sym][nt][B], xt [n_sym][nt] complex (optional), nu [nt] (optional).
 * ------------------------------------------------------------------------- */
static int mmse_sc(int nr, int nt, int qam, int n_sym, const cplx *H, const cplx *Y, double sigma2,
                   unsigned char *hard, double *llr, cplx *xt_out, double *nu_out)
{
    int M = qam, B = bits_of(qam);
    cplx pts[ORC_MAX_M];
    for (int q = 0; q < M; q++) pts[q] = qam_point(qam, q);

    cplx A[ORC_MAX_NT * ORC_MAX_NT], L[ORC_MAX_NT * ORC_MAX_NT];
    for (int i = 0; i < nt; i++)
        for (int j = 0; j < nt; j++) {
            cplx acc = 0.0;
            for (int r = 0; r < nr; r++)
                acc += conj(H[r * nt + i]) * H[r * nt + j];
            if (i == j) acc += sigma2;
            A[i * nt + j] = acc;
        }
    /* Cholesky A = L L^H, L lower triangular with real positive diagonal */
    for (int i = 0; i < nt * nt; i++) L[i] = 0.0;
    for (int j = 0; j < nt; j++) {
        double s = creal(A[j * nt + j]);
        for (int k = 0; k < j; k++)
            s -= creal(L[j * nt + k] * conj(L[j * nt + k]));
        if (!(s > 0.0)) return -4;
        double ljj = sqrt(s);
        L[j * nt + j] = ljj;
        for (int i = j + 1; i < nt; i++) {
            cplx t = A[i * nt + j];
            for (int k = 0; k < j; k++)
                t -= L[i * nt + k] * conj(L[j * nt + k]);
            L[i * nt + j] = t / ljj;
        }
    }
    /* W = A^{-1} H^H, one column of H^H (= one receive antenna) at a time */
    cplx W[ORC_MAX_NT * ORC_MAX_NR];
    for (int r = 0; r < nr; r++) {
        cplx u[ORC_MAX_NT], v[ORC_MAX_NT];
        for (int i = 0; i < nt; i++) { /* L u = h_r^* */
            cplx t = conj(H[r * nt + i]);
            for (int k = 0; k < i; k++) t -= L[i * nt + k] * u[k];
            u[i] = t / creal(L[i * nt + i]);
        }
        for (int i = nt - 1; i >= 0; i--) { /* L^H v = u */
            cplx t = u[i];
            for (int k = i + 1; k < nt; k++) t -= conj(L[k * nt + i]) * v[k];
            v[i] = t / creal(L[i * nt + i]);
        }
        for (int i = 0; i < nt; i++) W[i * nr + r] = v[i];
    }
    double mu[ORC_MAX_NT], nu[ORC_MAX_NT];
    for (int k = 0; k < nt; k++) {
        cplx acc = 0.0;
        for (int r = 0; r < nr; r++) acc += W[k * nr + r] * H[r * nt + k];
        mu[k] = creal(acc);
        nu[k] = (1.0 - mu[k]) / mu[k];
        if (nu_out) nu_out[k] = nu[k];
    }
    for (int s = 0; s < n_sym; s++) {
        const cplx *y = Y + (size_t)s * nr;
        for (int k = 0; k < nt; k++) {
            cplx x = 0.0;
            for (int r = 0; r < nr; r++) x += W[k * nr + r] * y[r];
            cplx xk = x / mu[k];
            if (xt_out) xt_out[(size_t)s * nt + k] = xk;
            double dist[ORC_MAX_M];
            int best = 0;
            for (int q = 0; q < M; q++) {
                cplx df = xk - pts[q];
                dist[q] = creal(df) * creal(df) + cimag(df) * cimag(df);
                if (dist[q] < dist[best]) best = q;
            }
            hard[(size_t)s * nt + k] = (unsigned char)best;
            for (int bit = 0; bit < B; bit++) {
                double m0 = INFINITY, m1 = INFINITY;
                for (int q = 0; q < M; q++) {
                    if ((q >> (B - 1 - bit)) & 1) {
                        if (dist[q] < m1) m1 = dist[q];
                    } else {
                        if (dist[q] < m0) m0 = dist[q];
                    }
                }
                llr[((size_t)s * nt + k) * B + bit] = (m1 - m0) / nu[k];
            }
        }
    }
    return 0;
}

int orc_mmse(int nr, int nt, int qam, int n_sym, const double *H, const double *Y, double sigma2,
             unsigned char *hard, double *llr, double *xt, double *nu)
{
    /* A = H^H H + sigma2 I is positive definite for any nr, so nt > nr is fine */
    if (nt < 1 || nt > ORC_MAX_NT || nr < 1 || nr > ORC_MAX_NR || !bits_of(qam)) return -1;
    if (!(sigma2 > 0.0)) return -1;
    return mmse_sc(nr, nt, qam, n_sym, (const cplx *)H, (const cplx *)Y, sigma2, hard, llr,
                   (cplx *)xt, nu);
}

/* ---------------------------------------------------------------------------
 * Whole slot: steps 1-6 (and optionally 7) for n_sc independent subcarriers,
 * split across host threads in contiguous blocks.  The subcarriers share
 * nothing, so the split changes no result.
 * H: [n_sc][nr][nt], Y: [n_sc][n_sym][nr] complex.  If paths_in is non-NULL
 * it replaces step 3 ([n_sc][n_pe][nt]).  Outputs (all optional except hard,
 * llr, ped2): R [n_sc][nt][nt], perm [n_sc][nt], Z [n_sc][n_sym][nt],
 * paths_out [n_sc][n_pe][nt], sqrd_gap [n_sc][nt], margin [n_sc][n_sym],
 * mmse_hard [n_sc][n_sym][nt], mmse_llr [n_sc][n_sym][nt][B],
 * flip_floor [n_sc][n_sym] (with tie_eps, as for orc_detect).  mmse_qr != 0
 * replaces step 1 by the MMSE-extended sorted QR (orc_sqrd_mmse), which also
 * allows nt > nr.
 * Returns the number of threads used (>0) or a negative error.
 * ------------------------------------------------------------------------- */
typedef struct {
    int n_sc, n_sym, nr, nt, qam, n_pe;
    double sigma2;
    const double *H, *Y;
    const unsigned char *paths_in;
    double *R, *Z, *ped2, *llr, *sqrd_gap, *margin, *mmse_llr, *flip_floor;
    double tie_eps;
    int mmse_qr;
    int *perm;
    unsigned char *paths_out, *hard, *mmse_hard;
    int sc_begin, sc_end;
    int status;
} orc_job;

static void *slot_worker(void *arg)
{
    orc_job *j = (orc_job *)arg;
    int nr = j->nr, nt = j->nt, ns = j->n_sym, npe = j->n_pe, B = bits_of(j->qam);
    cplx *Q = (cplx *)malloc(sizeof(cplx) * (nr + nt) * nt);
    cplx *R = (cplx *)malloc(sizeof(cplx) * nt * nt);
    cplx *Z = (cplx *)malloc(sizeof(cplx) * ns * nt);
    unsigned char *paths = (unsigned char *)malloc((size_t)npe * nt);
    j->status = 0;
    if (!Q || !R || !Z || !paths) {
        j->status = -2;
        goto out;
    }
    for (int sc = j->sc_begin; sc < j->sc_end; sc++) {
        const cplx *H = (const cplx *)j->H + (size_t)sc * nr * nt;
        const cplx *Y = (const cplx *)j->Y + (size_t)sc * ns * nr;
        int perm[ORC_MAX_NT];
        double gap[ORC_MAX_NT];
        if (j->mmse_qr) {
            /* Q_a is (nr + nt) x nt; z = Q_a^H [y; 0] reads its top nr rows,
             * which with row stride nt are Q_a's first nr rows */
            cplx Ha[ORC_MAX_NR * ORC_MAX_NT];
            augment(nr, nt, H, j->sigma2, Ha);
            sqrd(nr + nt, nt, Ha, Q, R, perm, gap);
        } else {
            sqrd(nr, nt, H, Q, R, perm, gap);
        }
        qhy(nr, nt, ns, Q, Y, Z);
        const unsigned char *pt;
        if (j->paths_in) {
            pt = j->paths_in + (size_t)sc * npe * nt;
        } else {
            double rdiag[ORC_MAX_NT];
            for (int l = 0; l < nt; l++) rdiag[l] = creal(R[l * nt + l]);
            int st = select_paths(nt, j->qam, rdiag, j->sigma2, npe, paths, NULL, NULL);
            if (st) {
                j->status = st;
                goto out;
            }
            pt = paths;
        }
        int st = detect_sc(nt, j->qam, ns, R, Z, perm, npe, pt, j->sigma2,
                           j->hard + (size_t)sc * ns * nt, j->llr + (size_t)sc * ns * nt * B,
                           j->ped2 + (size_t)sc * ns * 2,
                           j->margin ? j->margin + (size_t)sc * ns : NULL, NULL, NULL,
                           j->tie_eps, j->flip_floor ? j->flip_floor + (size_t)sc * ns : NULL);
        if (st) {
            j->status = st;
            goto out;
        }
        if (j->mmse_hard && j->mmse_llr) {
            st = mmse_sc(nr, nt, j->qam, ns, H, Y, j->sigma2, j->mmse_hard + (size_t)sc * ns * nt,
                         j->mmse_llr + (size_t)sc * ns * nt * B, NULL, NULL);
            if (st) {
                j->status = st;
                goto out;
            }
        }
        if (j->R) memcpy(j->R + (size_t)sc * nt * nt * 2, R, sizeof(cplx) * nt * nt);
        if (j->Z) memcpy(j->Z + (size_t)sc * ns * nt * 2, Z, sizeof(cplx) * ns * nt);
        if (j->perm) memcpy(j->perm + (size_t)sc * nt, perm, sizeof(int) * nt);
        if (j->sqrd_gap) memcpy(j->sqrd_gap + (size_t)sc * nt, gap, sizeof(double) * nt);
        if (j->paths_out) memcpy(j->paths_out + (size_t)sc * npe * nt, pt, (size_t)npe * nt);
    }
out:
    free(Q);
    free(R);
    free(Z);
    free(paths);
    return NULL;
}

int orc_detect_slot(int n_sc, int n_sym, int nr, int nt, int qam, int n_pe, double sigma2,
                    const double *H, const double *Y, const unsigned char *paths_in,
                    unsigned char *hard, double *llr, double *ped2, double *R, int *perm, double *Z,
                    unsigned char *paths_out, double *sqrd_gap, double *margin,
                    unsigned char *mmse_hard, double *mmse_llr, int n_threads, double tie_eps,
                    double *flip_floor, int mmse_qr)
{
    if (n_sc < 0 || n_sym < 1 || nt < 1 || nt > ORC_MAX_NT || nr < 1 || !bits_of(qam) ||
        n_pe < 1 || n_pe > ORC_MAX_NPE || !(sigma2 > 0.0))
        return -1;
    if (mmse_qr ? nr + nt > ORC_MAX_NR : (nr < nt || nr > ORC_MAX_NR)) return -1;
    if ((double)n_pe > ipow((double)qam, nt)) return -1;
    if (n_threads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        n_threads = c > 0 ? (int)c : 1;
    }
    if (n_threads > n_sc) n_threads = n_sc > 0 ? n_sc : 1;
    orc_job *jobs = (orc_job *)calloc((size_t)n_threads, sizeof(orc_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !tids) {
        free(jobs);
        free(tids);
        return -2;
    }
    for (int t = 0; t < n_threads; t++) {
        orc_job *j = &jobs[t];
        j->n_sc = n_sc;
        j->n_sym = n_sym;
        j->nr = nr;
        j->nt = nt;
        j->qam = qam;
        j->n_pe = n_pe;
        j->sigma2 = sigma2;
        j->H = H;
        j->Y = Y;
        j->paths_in = paths_in;
        j->R = R;
        j->Z = Z;
        j->ped2 = ped2;
        j->llr = llr;
        j->sqrd_gap = sqrd_gap;
        j->margin = margin;
        j->mmse_llr = mmse_llr;
        j->perm = perm;
        j->paths_out = paths_out;
        j->hard = hard;
        j->mmse_hard = mmse_hard;
        j->tie_eps = tie_eps;
        j->flip_floor = flip_floor;
        j->mmse_qr = mmse_qr;
        j->sc_begin = (int)((long)n_sc * t / n_threads);
        j->sc_end = (int)((long)n_sc * (t + 1) / n_threads);
    }
    int started = 0;
    for (int t = 1; t < n_threads; t++) {
        if (pthread_create(&tids[t], NULL, slot_worker, &jobs[t]) != 0) break;
        started = t;
    }
    slot_worker(&jobs[0]);
    /* threads that failed to start are run here, in order */
    for (int t = started + 1; t < n_threads; t++) slot_worker(&jobs[t]);
    for (int t = 1; t <= started; t++) pthread_join(tids[t], NULL);
    int status = 0;
    for (int t = 0; t < n_threads; t++)
        if (jobs[t].status) status = jobs[t].status;
    free(jobs);
    free(tids);
    return status ? status : n_threads;
}
