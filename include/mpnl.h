/*
 * mpnl.h -- C ABI of the GB300 MPNL uplink MIMO detection path.
 *
 * Katsaros & Nikitopoulos, "Enabling Ultra-Dense, Open-RAN, Vehicular
 * Networks with Non-Linear MIMO Processing" (arXiv 2409.14355).  §II
 * (Background) describes the Massively Parallelizable Non-Linear (MPNL)
 * detector: the position of the most promising candidate transmit vectors is
 * found from the channel alone, before data arrives; during transmission
 * those N_p candidates are evaluated in parallel.  §III-B uses N_p <= 32,
 * 14-symbol slots with the channel constant over the slot, and the linear
 * MMSE detector as the baseline.
 *
 * The path, per subcarrier (sc) and OFDM symbol, with y = H s + n:
 *   mpnl_preprocess    sorted QR  H P = Q R  and  z = Q^H y
 *   mpnl_select_paths  the N_pe most probable position vectors per sc
 *                      (mpnl_select_paths_lut: with a table of rank costs)
 *   mpnl_detect        N_pe SIC / partial-Euclidean-distance walks, argmin
 *                      -> hard decisions, max-log LLRs over the list
 *   mpnl_linear_mmse   linear MMSE baseline (hard decisions + LLRs)
 * Variants: mpnl_preprocess_mmse (more users than antennas), mpnl_detect_mixed
 * and mpnl_qhy_mixed (FP16), mpnl_refine_qr (FP64 re-factorisation), the
 * rank-cost table (mpnl_rank_counts, mpnl_rank_costs), the real-valued
 * decomposition (mpnl_rvd_embed, mpnl_select_paths_pam, mpnl_detect_rvd);
 * for serving: mpnl_factor, mpnl_qhy and the batch calls (mpnl_batch_*).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every data pointer is DEVICE memory (or host memory registered with /
 *   allocated by CUDA) owned by the caller; the library never allocates on
 *   these calls and keeps no pointer after returning.
 * - Complex values are interleaved (re, im) float32 pairs ("c64"), 8-byte
 *   aligned.  Real arrays are float32, 4-byte aligned.
 * - Symbol labels are the TS 38.211 §5.1 Gray bit labels as integers, bit b0
 *   (the most significant) first; constellations have unit average energy.
 * - Level index l = 0..nt-1 is the row of R; detection runs from level nt-1
 *   (the column the sorted QR picked last) down to level 0.
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *   only enqueues work on it and returns; nothing synchronises.
 * - Return value: MPNL_OK (0) or a negative MPNL_ERR_*.  On error nothing was
 *   enqueued, except MPNL_ERR_CUDA from a failed launch; mpnl_last_error()
 *   returns the message.  No call prints, aborts or traps.
 * - Limits: 1 <= nt <= 16, 1 <= nr <= 32 (nt <= nr for mpnl_preprocess,
 *   nr + nt <= 32 for mpnl_preprocess_mmse), qam in {4, 16, 64},
 *   1 <= n_sym <= 32, 1 <= n_pe <= min(1024, qam^nt), n_sc >= 0 (0 is a
 *   no-op), sigma2 > 0 and finite.
 */
#ifndef MPNL_H
#define MPNL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPNL_OK 0
#define MPNL_ERR_INVALID_ARG (-1) /* bad size, null or misaligned pointer, bad value */
#define MPNL_ERR_UNSUPPORTED (-2) /* valid request outside what this build implements */
#define MPNL_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define MPNL_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up */

#define MPNL_MAX_NT 16
#define MPNL_MAX_NR 32
#define MPNL_MAX_NSYM 32
#define MPNL_MAX_NPE 1024
/* |LLR| written when the list holds no candidate with the opposite bit. */
#define MPNL_LLR_MAX 20.0f

typedef struct mpnl_ctx mpnl_ctx;

/* Problem sizes of one slot: n_sc subcarriers x n_sym OFDM symbols, nr
 * receive antennas, nt single-antenna users (streams), QAM order, and the
 * number N_pe of position vectors evaluated per detection. */
typedef struct {
    int n_sc;
    int n_sym;
    int nr;
    int nt;
    int qam;
    int n_pe;
} mpnl_dims;

/* Create a context bound to CUDA device `device` (made current on the calling
 * thread).  *ctx receives the handle; release it with mpnl_destroy.
 * Errors: MPNL_ERR_INVALID_ARG (ctx NULL), MPNL_ERR_CUDA (no such device). */
int mpnl_create(mpnl_ctx **ctx, int device);

/* Release a context (NULL is ignored).  Does not synchronise any stream. */
void mpnl_destroy(mpnl_ctx *ctx);

/* Message of the last error on this context ("" if none).  The string is
 * owned by the context and valid until the next call on it. */
const char *mpnl_last_error(const mpnl_ctx *ctx);

/* Device scratch bytes the calls below need for `dims` (0: the kernels keep
 * all intermediates on chip).  `ws` arguments below may then be NULL. */
size_t mpnl_workspace_bytes(const mpnl_dims *dims);

/* Channel pre-processing (§II: "observing the MIMO channel"): sorted QR
 * H P = Q R with the smallest-residual-norm column first (SQRD) and
 * z = Q^H y for every symbol, per subcarrier.
 *   H        in  c64 [n_sc][nr][nt]          channel, row-major
 *   Y        in  c64 [n_sc][n_sym][nr]       received symbols
 *   R        out c64 [n_sc][nt(nt+1)/2]      upper triangle, packed row by
 *                row: entry (i, j >= i) at i*nt - i(i-1)/2 + (j - i); the
 *                diagonal is real and positive (imaginary part 0)
 *   inv_diag out f32 [n_sc][nt]              1 / R_ll
 *   perm     out u8  [n_sc][nt]              perm[l] = user in column l of HP
 *   Z        out c64 [n_sc][n_sym][nt]       z = Q^H y  (Q is not stored) */
int mpnl_preprocess(mpnl_ctx *ctx, const mpnl_dims *dims, const void *H, const void *Y, void *R,
                    float *inv_diag, uint8_t *perm, void *Z, void *ws, void *stream);

/* MMSE-extended pre-processing, for more users than antennas (the regime of
 * §III-IV where MPNL serves e.g. 12 streams on 7 antennas) and usable for any
 * nt: the sorted QR of the augmented channel [H; sqrt(sigma2) I] and
 * z = Q_a^H [y; 0] (Wuebben et al. 2003's MMSE-SQRD).  The walks of
 * mpnl_detect then minimise ||y - H s||^2 + sigma2 ||s||^2 instead of
 * ||y - H s||^2.  Same outputs and layouts as mpnl_preprocess; requires
 * nr + nt <= MPNL_MAX_NR (nt > nr allowed) and sigma2 > 0. */
int mpnl_preprocess_mmse(mpnl_ctx *ctx, const mpnl_dims *dims, const void *H, const void *Y,
                         float sigma2, void *R, float *inv_diag, uint8_t *perm, void *Z, void *ws,
                         void *stream);

/* Sorted QR keeping Q: the per-unit state a serving loop holds while the
 * channel stays the same over several slots (§III-B: H constant over a
 * slot; the channel changes slowly at vehicular speeds).  sigma2 = 0: plain
 * sorted QR (nt <= nr); sigma2 > 0: MMSE-extended (as mpnl_preprocess_mmse).
 *   H               in   c64 [n_sc][nr][nt]
 *   Q               out  c64 [n_sc][nr][nt]  antenna rows of Q, column l
 *                        belongs to level l (the sorted order)
 *   R, inv_diag, perm out as mpnl_preprocess (dims.n_sym is not used) */
int mpnl_factor(mpnl_ctx *ctx, const mpnl_dims *dims, const void *H, float sigma2, void *Q,
                void *R, float *inv_diag, uint8_t *perm, void *ws, void *stream);

/* z = Q^H y for every symbol, from a stored Q (mpnl_factor); for the
 * MMSE-extended factor this is Q_a^H [y; 0].
 *   Q  in   c64 [n_sc][nr][nt];  Y  in  c64 [n_sc][n_sym][nr]
 *   Z  out  c64 [n_sc][n_sym][nt] */
int mpnl_qhy(mpnl_ctx *ctx, const mpnl_dims *dims, const void *Q, const void *Y, void *Z,
             void *ws, void *stream);

/* z = Q^H y as mpnl_qhy, on the tensor cores with FP16 operands and FP32
 * accumulation (the Q^H y of the mixed-precision path): per subcarrier the
 * symbols form one small real GEMM [Re y | Im y] [[Re Q, -Im Q]; [Im Q,
 * Re Q]] = [Re z | Im z] (mma.sync m16n8k16).  Q and y are rounded to FP16
 * (11-bit significand) after each subcarrier's y is scaled by the power of
 * two that brings its largest component into [0.5, 1) (undone on z, so any
 * input scale is exact): each z_j is off by about 2^-11 sum_i |Q_ij| |y_i|.
 * Arguments and errors as mpnl_qhy. */
int mpnl_qhy_mixed(mpnl_ctx *ctx, const mpnl_dims *dims, const void *Q, const void *Y, void *Z,
                   void *ws, void *stream);

/* FP64 re-factorisation of ill-conditioned channels.  Run after
 * mpnl_preprocess / mpnl_preprocess_mmse (sigma2 > 0 selects the latter's
 * augmented matrix, 0 the plain one) or mpnl_factor (Y and Z NULL, Q not
 * NULL): for every subcarrier whose FP32 R has max R_ll / min R_ll >
 * cond_threshold (a lower bound on the condition number; NaN or zero
 * diagonals count as above), the sorted QR, z and Q are recomputed in FP64
 * from H and Y and overwrite R, inv_diag, perm, Z and Q (rounded to FP32);
 * the other subcarriers are left untouched.  The FP16 walk path is stated
 * for cond_threshold = 1e3.
 *   n_refined  device int (nullable): incremented once per subcarrier redone
 * Errors: as mpnl_preprocess; cond_threshold must be >= 1. */
int mpnl_refine_qr(mpnl_ctx *ctx, const mpnl_dims *dims, const void *H, const void *Y,
                   float sigma2, float cond_threshold, void *R, float *inv_diag, uint8_t *perm,
                   void *Z, void *Q, int *n_refined, void *ws, void *stream);

/* Position-vector pre-selection (§II: found "before any transmission
 * begins" from the channel; §III-B: N_p).  Per level, gamma_l = R_ll^2 /
 * sigma2 gives the square-QAM symbol-error probability Pe_l (floored at
 * 1e-12), and P_l(k) = (1 - Pe_l) Pe_l^(k-1) the chance that the transmitted
 * symbol is the k-th closest.  The N_pe vectors of largest prod_l P_l(p_l)
 * are written best first (ties: lexicographically smaller from level nt-1
 * down); row 0 is the all-ones vector (plain SIC).  The ranking uses the
 * cost -log of that product relative to all-ones, sum_l (p_l - 1)(-log Pe_l):
 * each level's term in float, the sum exact (64-bit fixed point, units of
 * 2^-32).
 *   R      in  c64 [n_sc][nt(nt+1)/2]  as written by mpnl_preprocess (only
 *              the diagonal is read)
 *   paths  out u8  [n_sc][n_pe][nt]     ranks 1..qam, level index last */
int mpnl_select_paths(mpnl_ctx *ctx, const mpnl_dims *dims, const void *R, float sigma2,
                      uint8_t *paths, void *ws, void *stream);

/* Table-driven rank model (a reading: the paper gives no per-level model;
 * this is the FlexCore-style alternative to the geometric model above).  The
 * chance that the transmitted symbol is the k-th closest is estimated once
 * per SNR, offline, and looked up per level: the table's bin for level l is
 * the number of edges e with gamma_l = R_ll^2 / sigma2 >= e (float), and the
 * N_pe vectors of smallest sum_l cost[bin_l][p_l - 1] are written in the
 * order and with the tie rule of mpnl_select_paths.
 *   qam, n_bins  the table's constellation (must equal dims->qam) and bins
 *   edges  in  f32 [n_bins - 1]     ascending linear SNRs (device)
 *   cost   in  f32 [n_bins][qam]    c(k) at k - 1: c(1) = 0, nondecreasing in
 *                                   k, finite (device; mpnl_rank_costs);
 *                                   costs above 2^20 are taken as 2^20, and
 *                                   the terms are summed as in
 *                                   mpnl_select_paths  */
typedef struct {
    int qam, n_bins;
    const float *edges;
    const float *cost;
} mpnl_rank_lut;

/* Errors: as mpnl_select_paths; a table whose qam differs from dims->qam,
 * n_bins < 1 or NULL arrays.  Rows that break the cost rules (decreasing,
 * NaN) are the caller's error: the position-vector table is then
 * unspecified, though every access stays within its buffers, and
 * mpnl_detect clamps ranks outside 1..qam and reports them through
 * mpnl_check_status. */
int mpnl_select_paths_lut(mpnl_ctx *ctx, const mpnl_dims *dims, const void *R, float sigma2,
                          const mpnl_rank_lut *lut, uint8_t *paths, void *ws, void *stream);

/* Real-valued decomposition (RVD; a variant: the paper's levels are
 * complex).  [Re y; Im y] = [[Re H, -Im H]; [Im H, Re H]] [Re s; Im s] +
 * noise: 2 nt real levels, real column u the real part of user u and column
 * nt + u its imaginary part, each an L-PAM axis (L = sqrt qam) of the square
 * QAM labelled by that axis's Gray bits.  The path: mpnl_rvd_embed, then
 * mpnl_preprocess with nr' = 2 nr, nt' = 2 nt on the embedded arrays (its R
 * and z come out real), mpnl_select_paths_pam, mpnl_detect_rvd.  In these
 * three calls dims describe the complex problem: nt <= 8 users (2 nt real
 * levels <= 16), and for the embedding nr <= 16.
 *   mpnl_rvd_embed:  H in c64 [n_sc][nr][nt], Y in c64 [n_sc][n_sym][nr];
 *                    Hr out c64 [n_sc][2nr][2nt], Yr out c64 [n_sc][n_sym][2nr]
 *                    (imaginary parts zero)
 *   mpnl_select_paths_pam:  per real level the L-PAM error probability
 *                    Pe_l = 2 (1 - 1/L) Q(sqrt(3 gamma_l / (qam - 1))),
 *                    gamma_l = R_ll^2 / sigma2 (noise sigma2/2 per real
 *                    dimension), geometric over ranks 1..L; order and ties as
 *                    mpnl_select_paths.  R in c64 [n_sc][2nt(2nt+1)/2];
 *                    paths out u8 [n_sc][n_pe][2nt]; n_pe <= min(1024, L^(2nt))
 *   mpnl_detect_rvd: the walks over the real levels (p-th closest PAM point
 *                    by (distance, axis label)); hard decisions, LLRs and PED
 *                    pairs in the layouts of mpnl_detect, each user's label
 *                    joining its two axes (bits b0 b2 .. from the real part,
 *                    b1 b3 .. from the imaginary part, TS 38.211 §5.1).
 *                    R, inv_diag, perm, Z over the 2 nt real levels.
 * Errors: as the complex calls, and nt > 8, 2 nr > MPNL_MAX_NR (embedding). */
int mpnl_rvd_embed(mpnl_ctx *ctx, const mpnl_dims *dims, const void *H, const void *Y, void *Hr,
                   void *Yr, void *stream);
int mpnl_select_paths_pam(mpnl_ctx *ctx, const mpnl_dims *dims, const void *R, float sigma2,
                          uint8_t *paths, void *ws, void *stream);
int mpnl_detect_rvd(mpnl_ctx *ctx, const mpnl_dims *dims, const void *R, const float *inv_diag,
                    const uint8_t *perm, const uint8_t *paths, const void *Z, float sigma2,
                    uint8_t *hard, float *llr, float *ped2, void *ws, void *stream);

/* Monte-Carlo rank histogram for the table: for each of n_bins SNRs
 * gamma[b] (linear), n_trials draws of a uniform symbol and of complex
 * Gaussian noise of variance 1/gamma[b] (the law of b_l = s + n_l / R_ll),
 * counting the rank of the sent symbol among all qam points by (distance,
 * label).  Random numbers: SplitMix64 used as a counter-based generator
 * keyed by (seed, bin, trial), so the table depends only on its arguments.
 *   gamma   in   f64 [n_bins]        (device), all > 0
 *   counts  out  u64 [n_bins][qam]   (device), zeroed first
 * Errors: qam not 4/16/64, n_bins < 1 or > 65535, n_trials < 1 or >= 2^38,
 * NULL or host pointers. */
int mpnl_rank_counts(mpnl_ctx *ctx, int qam, int n_bins, const double *gamma, long long n_trials,
                     unsigned long long seed, unsigned long long *counts, void *stream);

/* Rank costs from the histogram (a reading): c(k) = log P(1) - log P(k)
 * with P(k) = counts / n_trials for the ranks seen; a rank never seen is
 * taken as half as likely as the rank before it (c(k) = c(k-1) + ln 2), rank
 * 1 never seen as half a trial; then made nondecreasing in k by a running
 * maximum, c(1) = 0 -- the cost table of mpnl_select_paths_lut.
 *   counts  in   u64 [n_bins][qam];  cost  out  f32 [n_bins][qam]  (device)
 * Errors: as mpnl_rank_counts. */
int mpnl_rank_costs(mpnl_ctx *ctx, int qam, int n_bins, const unsigned long long *counts,
                    long long n_trials, float *cost, void *stream);

/* Evaluation of the position vectors (§II: the most promising solutions
 * "processed in parallel").  For every (sc, symbol) and every row p of the
 * table, independently: for l = nt-1..0, e_l = z_l - sum_{j>l} R_lj s_j,
 * b_l = e_l / R_ll, s_l = the p_l-th closest constellation point to b_l
 * (ordered by distance, then label), d += R_ll^2 |b_l - s_l|^2.  The row
 * with the smallest d (tie: lower row) gives the hard decisions; user
 * perm[l] receives s_l.  Max-log LLR of bit b of user k:
 * (min_{rows, bit=1} d - min_{rows, bit=0} d) / sigma2 (positive: bit 0),
 * +-MPNL_LLR_MAX when one side is empty.
 *   R, inv_diag, perm, Z   in   as written by mpnl_preprocess
 *   paths                  in   u8 [n_sc][n_pe][nt], entries 1..qam
 *                               (checked on the device: a bad entry is
 *                               clamped and reported as MPNL_ERR_INVALID_ARG
 *                               by mpnl_check_status)
 *   hard                   out  u8  [n_sc][n_sym][nt]      labels, user order
 *   llr                    out  f32 [n_sc][n_sym][nt][log2 qam] (NULL: skip)
 *   ped2                   out  f32 [n_sc][n_sym][2] best and runner-up d
 *                               (+inf runner-up when n_pe == 1; NULL: skip) */
int mpnl_detect(mpnl_ctx *ctx, const mpnl_dims *dims, const void *R, const float *inv_diag,
                const uint8_t *perm, const uint8_t *paths, const void *Z, float sigma2,
                uint8_t *hard, float *llr, float *ped2, void *ws, void *stream);

/* Mixed-precision variant of mpnl_detect (same arguments, same layouts).
 * The walks choose their vectors with the interference-cancelled residuals
 * e in FP16 (half2, packed half-precision FMAs); b = e_l / R_ll, the ranking
 * and the PED accumulation of the walk stay in FP32.  Every metric the call
 * reports is then recomputed in FP32 from the chosen vector -- the re-check
 * covers every row, not only the best and runner-up: d = ||z - R s||^2
 * replayed level by level -- so the hard decisions are the argmin of FP32
 * metrics over the FP16 walks' list, ped2 holds the best and runner-up of
 * those metrics, and each LLR is a difference of two of them (its sign agrees
 * with the decided bit).  R and z are scaled per subcarrier by a power of
 * two before the conversion to FP16, so any input scale is handled exactly.
 * Decisions can differ from mpnl_detect's where FP16 rounding changes a
 * ranking and so the list; the decision-mismatch rate and BER delta against
 * the FP64 oracle are reported by the tests and the benchmark. */
int mpnl_detect_mixed(mpnl_ctx *ctx, const mpnl_dims *dims, const void *R, const float *inv_diag,
                      const uint8_t *perm, const uint8_t *paths, const void *Z, float sigma2,
                      uint8_t *hard, float *llr, float *ped2, void *ws, void *stream);

/* End-to-end detection of one slot held in the caller's buffers (the whole
 * path of §II and the MMSE baseline of §III-B in one call): H and Y are
 * copied into the workspace, the sorted QR + z, the path selection, the
 * walks and, with MPNL_SLOT_MMSE, the linear MMSE baseline run there, and the
 * hard decisions, LLRs and PED pairs (and the baseline's outputs) are copied
 * back -- all enqueued on `stream` in that order, so the results are in the
 * caller's buffers once the stream has reached the end of the call.  The
 * baseline (it needs only H and Y) runs beside the path on a side stream of
 * the context, forked from `stream` after the input copies and joined back
 * before its outputs are copied; the context makes that stream on first use
 * and serialises the fork and join of concurrent callers.  A call made while
 * `stream` is being captured into a CUDA graph draws the side stream into
 * that capture until the capture ends, so no other call with MPNL_SLOT_MMSE
 * may use the same context in between (a capturing thread takes a context
 * of its own).  The
 * buffers may be host memory (pinned lets the copies run asynchronously;
 * pageable makes CUDA copy them synchronously) or device memory.
 *   H, Y                 in   as mpnl_preprocess (nt <= nr, or nr + nt <= MPNL_MAX_NR
 *                             with MPNL_SLOT_MMSE_QR)
 *   hard, llr, ped2      out  as mpnl_detect (llr, ped2 nullable)
 *   mmse_hard, mmse_llr  out  as mpnl_linear_mmse (MPNL_SLOT_MMSE; mmse_llr nullable)
 *   flags                MPNL_SLOT_MMSE, MPNL_SLOT_FP16 (the walks of mpnl_detect_mixed),
 *                        MPNL_SLOT_MMSE_QR (the pre-processing of mpnl_preprocess_mmse)
 *   ws, ws_bytes         device workspace of at least mpnl_slot_workspace_bytes(dims,
 *                        flags) bytes, 256-byte aligned, owned by the caller; it holds
 *                        the slot's intermediates until the stream passes the call, so
 *                        one call in flight per workspace
 * Errors: as the per-call steps; a workspace too small or misaligned. */
#define MPNL_SLOT_MMSE 1
#define MPNL_SLOT_FP16 2
#define MPNL_SLOT_MMSE_QR 4
size_t mpnl_slot_workspace_bytes(const mpnl_dims *dims, int flags);
int mpnl_detect_slot(mpnl_ctx *ctx, const mpnl_dims *dims, float sigma2, const void *H,
                     const void *Y, uint8_t *hard, float *llr, float *ped2, uint8_t *mmse_hard,
                     float *mmse_llr, int flags, void *ws, size_t ws_bytes, void *stream);

/* Linear MMSE baseline (§I, §III-B: "de facto standard linear MMSE"):
 * W = (H^H H + sigma2 I)^{-1} H^H; x = W y; mu_k = (W H)_kk;
 * x~_k = x_k / mu_k, nu_k = (1 - mu_k) / mu_k; hard = nearest point to x~_k;
 * LLR_b = (min_{q: bit b = 1} |x~ - q|^2 - min_{q: bit b = 0} |x~ - q|^2) / nu_k.
 *   H, Y  in   as for mpnl_preprocess
 *   hard  out  u8  [n_sc][n_sym][nt]
 *   llr   out  f32 [n_sc][n_sym][nt][log2 qam]   (NULL: skip) */
int mpnl_linear_mmse(mpnl_ctx *ctx, const mpnl_dims *dims, const void *H, const void *Y,
                     float sigma2, uint8_t *hard, float *llr, void *ws, void *stream);

/* Synchronise `stream` and report device-side argument errors recorded by
 * the calls enqueued on this context since the previous check (currently: a
 * position-vector entry outside 1..qam seen by mpnl_detect).  Returns MPNL_OK,
 * MPNL_ERR_INVALID_ARG (with a message) or MPNL_ERR_CUDA. */
int mpnl_check_status(mpnl_ctx *ctx, void *stream);

/* Mixed-size batches in persistent launches ---------------------------------
 *
 * A batch holds the slots of many radio units with different sizes.  Each
 * stage (sorted QR + z, selection, walks, MMSE baseline) is ONE persistent
 * launch for the whole batch: its workers (a warp, a group of warps or a
 * CTA) take (unit, subcarrier) items from a device counter, largest units
 * first, and run the kernel instance that fits each unit.  With
 * MPNL_RUN_GRAPH the stages are captured once into a CUDA graph and replayed.
 * The results are those of the per-call API on each unit alone. */
typedef struct {
    mpnl_dims dims;
    float sigma2;
    int flags;            /* MPNL_ITEM_MMSE_QR, MPNL_ITEM_LINEAR_MMSE, MPNL_ITEM_FP16 */
    int stages;           /* MPNL_STAGE_* bits this unit takes part in; 0 = the whole path
                             (sorted QR + z, selection, walks, and MMSE with the flag) */
    void *Q;              /* c64 [n_sc][nr][nt]: written by the QR stage if not NULL,
                             read by the MPNL_STAGE_QHY stage */
    const void *H;        /* in  c64 [n_sc][nr][nt] */
    const void *Y;        /* in  c64 [n_sc][n_sym][nr] */
    void *R;              /* out c64 [n_sc][nt(nt+1)/2]  (unit state, as mpnl_preprocess) */
    float *inv_diag;      /* out f32 [n_sc][nt] */
    uint8_t *perm;        /* out u8  [n_sc][nt] */
    void *Z;              /* out c64 [n_sc][n_sym][nt] */
    uint8_t *paths;       /* out u8  [n_sc][n_pe][nt]    (as mpnl_select_paths) */
    uint8_t *hard;        /* out u8  [n_sc][n_sym][nt]   (as mpnl_detect) */
    float *llr;           /* out f32 [n_sc][n_sym][nt][log2 qam] (NULL: skip) */
    float *ped2;          /* out f32 [n_sc][n_sym][2]    (NULL: skip) */
    uint8_t *mmse_hard;   /* out u8  [n_sc][n_sym][nt]   with MPNL_ITEM_LINEAR_MMSE */
    float *mmse_llr;      /* out f32 [n_sc][n_sym][nt][log2 qam] (NULL: skip) */
} mpnl_batch_item;

#define MPNL_ITEM_MMSE_QR 1      /* MMSE-extended QR (mpnl_preprocess_mmse); allows nt > nr */
#define MPNL_ITEM_LINEAR_MMSE 2  /* also run the linear MMSE baseline */
#define MPNL_ITEM_FP16 4         /* the mixed-precision path: walks as mpnl_detect_mixed and,
                                    in the Q^H y stage, z as mpnl_qhy_mixed */
#define MPNL_ITEM_REFINE_QR 8    /* right after the QR stage, the FP64 re-factorisation of
                                    mpnl_refine_qr with cond_threshold 1e3 (R, 1/R_ll, perm,
                                    Q if given, and z where the QR stage formed it) */

/* Stages run in the order QR, selection, Q^H y, walks, MMSE.  A unit whose
 * stages include MPNL_STAGE_QHY gets z from its stored Q; otherwise, if its
 * stages include the walks, its QR stage also forms z; else (a channel
 * update: QR and selection only) the QR stage only factors. */
#define MPNL_STAGE_PREPROCESS 1
#define MPNL_STAGE_SELECT 2
#define MPNL_STAGE_DETECT 4
#define MPNL_STAGE_MMSE 8
#define MPNL_RUN_GRAPH 16  /* capture the stages into a CUDA graph once, then replay it */
/* leave room on every SM for other work (e.g. a higher-priority stream's
 * launches): the walk stage runs one CTA per SM fewer than tuned (at least
 * one), the other stages half their workers; results are unchanged */
#define MPNL_RUN_SHARE_SMS 64
/* every CTA of every stage takes one work item (as many CTAs as items)
 * instead of a persistent grid drawing items until they run out: short CTAs
 * that the hardware spreads over whatever SMs free up, for a latency-bound
 * batch that shares the GPU with longer work (a serving loop's small units
 * beside a large unit's walks); results are unchanged */
#define MPNL_RUN_SHORT_CTAS 128
#define MPNL_STAGE_QHY 32
#define MPNL_STAGES_ALL 47

typedef struct mpnl_batch mpnl_batch;

/* Validate `n_items` items (each as the per-call API would), order them
 * largest first and copy their descriptors to the device.  The batch keeps
 * the items' pointers (not the host array); it allocates its descriptor
 * table and counters here, never when it runs.  Errors: as the per-call
 * checks (MPNL_ERR_INVALID_ARG with the item index in the message),
 * MPNL_ERR_UNSUPPORTED if a unit needs more shared memory than an SM has,
 * MPNL_ERR_CUDA. */
int mpnl_batch_create(mpnl_ctx *ctx, const mpnl_batch_item *items, int n_items,
                      mpnl_batch **batch);

/* Replace the batch's units by `n_items` new ones (n_items <= the count it
 * was created with), validated and ordered as by mpnl_batch_create, reusing
 * its allocations; cached graphs are dropped.  The new descriptors go to
 * the device with the next mpnl_batch_run, asynchronously on its stream (a
 * reset waits only until the previous upload has been read).  The previous
 * runs' kernels may still be in flight only if they have finished reading
 * nothing the new items change -- in practice: reset after the previous run
 * of this batch completed.  flags: MPNL_RESET_TRUSTED_POINTERS skips the
 * per-pointer CUDA attribute queries (null and alignment are still checked;
 * for callers that draw every buffer from their own device pools). */
#define MPNL_RESET_TRUSTED_POINTERS 1
int mpnl_batch_reset(mpnl_ctx *ctx, mpnl_batch *batch, const mpnl_batch_item *items,
                     int n_items, int flags);

/* Enqueue the stages in `stages` (MPNL_STAGE_* bits, in pipeline order,
 * optionally with MPNL_RUN_GRAPH, MPNL_RUN_SHARE_SMS, MPNL_RUN_SHORT_CTAS) on `stream`; with
 * MPNL_RUN_GRAPH the stream must not be the legacy default stream (NULL).  Device-side argument errors go to mpnl_check_status. */
int mpnl_batch_run(mpnl_ctx *ctx, mpnl_batch *batch, int stages, void *stream);

/* One round of a serving loop in one call (a DU serving many RUs, §I and
 * §IV): the requests' inputs copied from host buffers into device staging,
 * the batch reset with one item per request (trusted pointers, as
 * MPNL_RESET_TRUSTED_POINTERS), the stages run, and the slots' decisions and
 * LLRs copied back to host buffers -- all enqueued on `stream`.  A request
 * refers to its unit's resident state through `unit` (an mpnl_batch_item
 * with dims, sigma2, flags and the device arrays Q, R, inv_diag, perm,
 * paths; its other fields are ignored).  A channel update runs the sorted QR
 * (keeping Q; with MPNL_ITEM_REFINE_QR in the unit's flags also the FP64
 * re-factorisation) and the selection from H; a slot runs Q^H y and the
 * walks on Y.  Channel updates are ordered before slots, so a slot of the
 * same unit in the round sees the new state.  The batch must have room for
 * n_reqs items and its previous round must have completed (as
 * mpnl_batch_reset).  run_flags: 0, MPNL_RUN_SHARE_SMS, MPNL_RUN_SHORT_CTAS.
 * Errors: as mpnl_batch_reset / mpnl_batch_run; a request without a unit,
 * a bad kind, or a slot without its buffers. */
#define MPNL_ROUND_SLOT 0
#define MPNL_ROUND_CHANNEL 1
typedef struct {
    const mpnl_batch_item *unit;  /* the unit's state (device arrays) and sizes */
    int kind;                     /* MPNL_ROUND_SLOT or MPNL_ROUND_CHANNEL */
    const void *payload;          /* host (pinned) Y [n_sc][n_sym][nr], or H [n_sc][nr][nt] */
    void *staging;                /* device buffer the payload is copied to */
    void *Z;                      /* device c64 [n_sc][n_sym][nt] (slots) */
    uint8_t *hard;                /* device u8 [n_sc][n_sym][nt] (slots) */
    float *llr;                   /* device f32 [n_sc][n_sym][nt][log2 qam] (slots; nullable) */
    uint8_t *hard_host;           /* host copy of hard (slots) */
    float *llr_host;              /* host copy of llr (slots; nullable) */
} mpnl_round_req;
int mpnl_serve_round(mpnl_ctx *ctx, mpnl_batch *batch, const mpnl_round_req *reqs, int n_reqs,
                     int run_flags, void *stream);

/* Release a batch (NULL is ignored); its work must have completed. */
void mpnl_batch_destroy(mpnl_batch *batch);

/* SM partition for serving (§I, §IV: a distributed unit allocates its
 * compute to the radio units where the load is).  Splits the SMs of the
 * context's device into two disjoint groups with CUDA green contexts: group
 * 0 of at least sms_first SMs (rounded up to the device's partition
 * granularity, 8 SMs on this GPU), group 1 the rest.  Kernels enqueued on a
 * stream of a group run on that group's SMs only; everything else about the
 * stream is as for any stream of the device (a green context is the primary
 * context with fewer SMs): device memory, every call of this library,
 * events, CUDA graphs.  The serving loop puts its small radio units' rounds
 * on group 0, so they never wait for an SM behind a large unit's walks.
 *   sms    out int[2]: the SMs of group 0 and group 1
 * Errors: MPNL_ERR_INVALID_ARG for a NULL pointer or sms_first outside
 * 1..SMs-1 (or a split the device cannot make), MPNL_ERR_UNSUPPORTED when
 * the driver has no green contexts, MPNL_ERR_CUDA. */
typedef struct mpnl_sm_split mpnl_sm_split;
int mpnl_sm_split_create(mpnl_ctx *ctx, int sms_first, mpnl_sm_split **split, int *sms);

/* A new non-blocking stream (a cudaStream_t) in group `part` (0 or 1), at
 * `priority` as for cudaStreamCreateWithPriority.  The split owns it:
 * mpnl_sm_split_destroy destroys it. */
int mpnl_sm_split_stream(mpnl_ctx *ctx, mpnl_sm_split *split, int part, int priority,
                         void **stream);

/* Waits for the work queued on the split's streams, destroys them and the
 * green contexts, frees the split.  NULL is a no-op.  Destroy only a split
 * whose streams nothing will touch again: events that other code recorded
 * on them (a framework's caching allocators do, for the copies and
 * allocations they see on a stream) stay bound to the green contexts, and
 * using them afterwards is undefined.  A split can instead be kept for the
 * life of the process, as frameworks keep their own streams. */
int mpnl_sm_split_destroy(mpnl_ctx *ctx, mpnl_sm_split *split);

/* Walks of up to MPNL_NOALLOC_MAX_UNITS radio units in one persistent launch,
 * without allocating anything.  The paper has no counterpart: this is an
 * interface for callers that must not allocate device memory once they are
 * running -- a distributed unit's real-time threads, where cudaMalloc and
 * cudaFree can block or synchronise the device and so cost a slot deadline,
 * and host frameworks that hand out all device memory from their own pool
 * and forbid libraries to allocate behind their back.  Those callers cannot
 * create an mpnl_batch (its creation allocates the descriptor table and work
 * counters) or even an mpnl_ctx (which allocates a status word).
 *
 * Each item is as for the batch calls, restricted to the walk stage: dims,
 * sigma2, flags (0 or MPNL_ITEM_FP16, the arithmetic of mpnl_detect_mixed),
 * stages (0 or MPNL_STAGE_DETECT), and the device arrays R, inv_diag, perm,
 * Z, paths (inputs, as mpnl_preprocess and mpnl_select_paths write them) and
 * hard, llr, ped2 (outputs; llr and ped2 nullable).  The other fields are
 * ignored.  Results equal those of mpnl_detect / mpnl_detect_mixed on each
 * unit alone.  Runs on the calling thread's current device; every array must
 * be reachable from it.
 *
 * The scratch the persistent kernel needs (the units' descriptors, the
 * prefix sums of their subcarrier counts, its work counter and a status
 * word; about 10 KB for 64 units) is one fixed array in the library's device
 * code, held by every device that loads the library until the process exits.
 * The first call on a device looks up that array's device address (and the
 * SM count); make that first call before capturing any stream into a graph.
 * Every call reuses the same array: the work counter and status word are
 * cleared at the start of each call, and two calls whose work overlaps on
 * the device (on different streams, or from different threads without
 * ordering) race on the array and give wrong results.  Calls on one stream
 * are ordered and safe.  The host copies the descriptors from the caller's
 * stack (pageable memory), so the call returns once they have been staged.
 * Table entries outside 1..qam are clamped as by mpnl_detect but not
 * reported (there is no context to hold the status).
 *
 * Returns MPNL_OK; MPNL_ERR_INVALID_ARG (NULL items, n_items < 1, a bad size,
 * flag, stage, sigma2 or pointer in some item); MPNL_ERR_UNSUPPORTED (n_items
 * > MPNL_NOALLOC_MAX_UNITS, or a unit needing more shared memory than an SM
 * has); MPNL_ERR_CUDA (no current device, set-up or launch failed).  There
 * is no context, so no message: the code is the whole report. */
#define MPNL_NOALLOC_MAX_UNITS 64
int mpnl_detect_units_noalloc(const mpnl_batch_item *items, int n_items, void *stream);

/* Launch-shape knobs.  They change how the work is spread over threads,
 * never the results.  Indexed by problem class: nt class (0: nt <= 4,
 * 1: nt <= 8, 2: nt <= 16), qam class (0: 4, 1: 16, 2: 64) and N_pe class
 * (0: n_pe < 256, 1: n_pe >= 256).  An entry of 0 means the built-in choice.
 * The package's autotuner measures the candidates and sets them. */
typedef struct {
    uint8_t detect_sym[3][3][2];    /* symbols per lane in the walk kernel: 1 or 2
                                       (built-in: 1 for nt > 8, else 2) */
    uint8_t select_warps[3][3][2];  /* warps per subcarrier in the selection: 1, 2 or 4
                                       (built-in: 2 for n_pe >= 256, else 1) */
    uint8_t persistent_ctas_per_sm; /* CTAs per SM of the batch (persistent) walk launch: 1, 2
                                       or 3 (built-in 3; fewer when shared memory is short) */
    uint8_t persistent_select_warps; /* warps per subcarrier of the batch selection launch:
                                        1, 2 or 4 (built-in 2) */
} mpnl_tuning;

/* Set the knobs of this context (NULL restores the built-in choices);
 * values outside the ranges above are rejected (MPNL_ERR_INVALID_ARG). */
int mpnl_set_tuning(mpnl_ctx *ctx, const mpnl_tuning *tuning);

/* Copy this context's knobs to *tuning (zeros for built-in choices). */
int mpnl_get_tuning(mpnl_ctx *ctx, mpnl_tuning *tuning);

#ifdef __cplusplus
}
#endif

#endif /* MPNL_H */
