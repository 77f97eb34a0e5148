// C ABI of the MPNL detection path (declared in include/mpnl.h): context,
// host-side validation of every argument, dispatch to the kernel launchers.
// Validation happens before anything is enqueued, so a rejected call leaves
// the stream untouched; no call prints, aborts or traps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "mpnl.h"
#include "mpnl_internal.h"

struct mpnl_ctx {
    int device = 0;
    unsigned *status = nullptr;  // device word of kStatus* bits, cleared by mpnl_check_status
    mpnl_tuning tuning{};
    char err[512] = {};
    // mpnl_detect_slot runs the MMSE baseline on a side stream of the
    // context (made on first use), forked from and joined back into the
    // caller's stream with these events; the mutex keeps a fork/join pair
    // whole when several threads share the context
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    std::mutex side_mu;
};

namespace {

int fail(mpnl_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(mpnl_ctx *ctx, const char *what, cudaError_t e)
{
    return fail(ctx, MPNL_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int bits_of(int qam) { return qam == 4 ? 2 : qam == 16 ? 4 : qam == 64 ? 6 : 0; }

int nt_class(int nt) { return nt <= 4 ? 0 : (nt <= 8 ? 1 : 2); }
int qam_class(int qam) { return qam == 4 ? 0 : (qam == 16 ? 1 : 2); }
int pe_class(int n_pe) { return n_pe >= 256 ? 1 : 0; }

int tuned_sym(const mpnl_ctx *ctx, const mpnl_dims *d)
{
    const int v = ctx->tuning.detect_sym[nt_class(d->nt)][qam_class(d->qam)][pe_class(d->n_pe)];
    if (v) return v;
    return d->nt > 8 ? 1 : 2;  // measured: one symbol per lane is faster at nt 9..16
}

int tuned_select_warps(const mpnl_ctx *ctx, const mpnl_dims *d)
{
    const int v = ctx->tuning.select_warps[nt_class(d->nt)][qam_class(d->qam)][pe_class(d->n_pe)];
    return v ? v : (d->n_pe >= 256 ? 2 : 1);
}

// Rules for nr: the plain sorted QR needs nt <= nr <= MPNL_MAX_NR (a square
// or tall channel); the MMSE-extended one factors nr + nt rows and needs
// nr + nt <= MPNL_MAX_NR; the other calls take nr from the caller's buffers
// (MMSE baseline) or ignore it (selection, walks) and need 1 <= nr <= MAX.
enum NrRule { kNrTall, kNrAugmented, kNrAny };

int check_dims(mpnl_ctx *ctx, const mpnl_dims *d, bool need_pe, NrRule nr_rule = kNrAny)
{
    if (!d) return fail(ctx, MPNL_ERR_INVALID_ARG, "dims is NULL");
    if (d->n_sc < 0) return fail(ctx, MPNL_ERR_INVALID_ARG, "n_sc=%d < 0", d->n_sc);
    if (d->nt < 1 || d->nt > MPNL_MAX_NT)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "nt=%d outside 1..%d", d->nt, MPNL_MAX_NT);
    if (d->nr < 1 || d->nr > MPNL_MAX_NR)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "nr=%d outside 1..%d", d->nr, MPNL_MAX_NR);
    if (nr_rule == kNrTall && d->nr < d->nt)
        return fail(ctx, MPNL_ERR_INVALID_ARG,
                    "nr=%d < nt=%d: use mpnl_preprocess_mmse for more users than antennas", d->nr,
                    d->nt);
    if (nr_rule == kNrAugmented && d->nr + d->nt > MPNL_MAX_NR)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "nr + nt = %d exceeds %d", d->nr + d->nt,
                    MPNL_MAX_NR);
    if (d->n_sym < 1 || d->n_sym > MPNL_MAX_NSYM)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "n_sym=%d outside 1..%d", d->n_sym, MPNL_MAX_NSYM);
    if (!bits_of(d->qam)) return fail(ctx, MPNL_ERR_INVALID_ARG, "qam=%d not in {4,16,64}", d->qam);
    if (need_pe) {
        double cap = pow((double)d->qam, (double)d->nt);
        if (d->n_pe < 1 || d->n_pe > MPNL_MAX_NPE || (double)d->n_pe > cap)
            return fail(ctx, MPNL_ERR_INVALID_ARG, "n_pe=%d outside 1..min(%d, qam^nt)", d->n_pe,
                        MPNL_MAX_NPE);
    }
    return MPNL_OK;
}

int check_sigma2(mpnl_ctx *ctx, float s)
{
    if (!(s > 0.0f) || isinf(s)) return fail(ctx, MPNL_ERR_INVALID_ARG, "sigma2=%g must be > 0 and finite", (double)s);
    return MPNL_OK;
}

// Non-NULL, aligned, and reachable from the context's device (device,
// managed or CUDA-registered host memory).  Plain pageable host memory is
// rejected: a kernel reading it would fault.
int check_ptr(mpnl_ctx *ctx, const void *p, size_t align, const char *name, bool nullable)
{
    if (!p) {
        if (nullable) return MPNL_OK;
        return fail(ctx, MPNL_ERR_INVALID_ARG, "%s is NULL", name);
    }
    if ((uintptr_t)p % align)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "%s is not %zu-byte aligned", name, align);
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, MPNL_ERR_INVALID_ARG, "%s: not a CUDA pointer (%s)", name, cudaGetErrorName(e));
    }
    if (a.type == cudaMemoryTypeUnregistered)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "%s is unregistered host memory", name);
    if (a.type == cudaMemoryTypeDevice && a.device != ctx->device)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "%s lives on device %d, context is on device %d", name,
                    a.device, ctx->device);
    return MPNL_OK;
}

int begin(mpnl_ctx *ctx)
{
    if (!ctx) return MPNL_ERR_INVALID_ARG;
    ctx->err[0] = '\0';
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, "cudaSetDevice", e);
    return MPNL_OK;
}

#define MPNL_TRY(x)            \
    do {                       \
        int _st = (x);         \
        if (_st) return _st;   \
    } while (0)

}  // namespace

// Stage slots of a batch, in execution order.
// The FP64 refinement (units with MPNL_ITEM_REFINE_QR) runs with the QR stage.
enum BatchStage { kBPre, kBRef, kBSel, kBQhy, kBDet, kBMmse, kBStages };
constexpr int kGraphSlots = 4 * (MPNL_STAGES_ALL + 1);
static const int kStageBit[kBStages] = {MPNL_STAGE_PREPROCESS, MPNL_STAGE_PREPROCESS,
                                        MPNL_STAGE_SELECT,     MPNL_STAGE_QHY,
                                        MPNL_STAGE_DETECT,     MPNL_STAGE_MMSE};
// the condition-estimate threshold of the batch refinement (the one the
// mixed-precision path is stated for)
constexpr float kBatchRefineThreshold = 1e3f;

struct mpnl_batch {
    int device;
    int capacity;
    int n_items;
    mpnl::BatchItem *h_items;  // pinned staging of the descriptors (schedule order)
    int *h_start;              // pinned staging of the prefix sums
    bool dirty;                // staging newer than the device copy
    cudaEvent_t copied;        // the last upload has been read
    mpnl::BatchItem *d_items;  // schedule order
    int *d_start;              // kBStages x (capacity + 1) prefix sums of n_sc per stage
    int *d_counters;           // one per stage
    int stage_units[kBStages];
    int pre_warp_bytes, ref_warp_bytes, sel_group_bytes, qhy_warp_bytes, mmse_warp_bytes;
    size_t det_smem;
    int sel_warps, det_ctas;
    int sms;
    cudaGraphExec_t graph[kGraphSlots];  // by stage mask, MPNL_RUN_SHARE_SMS, MPNL_RUN_SHORT_CTAS
};

namespace {

// Rough per-subcarrier cost of a unit's walks, for largest-first ordering.
double unit_cost(const mpnl_dims &d) { return (double)d.n_pe * d.nt * (d.nt + 4) * d.n_sym; }

int item_stages(const mpnl_batch_item &it)
{
    if (it.stages) return it.stages;
    return MPNL_STAGE_PREPROCESS | MPNL_STAGE_SELECT | MPNL_STAGE_DETECT |
           ((it.flags & MPNL_ITEM_LINEAR_MMSE) ? MPNL_STAGE_MMSE : 0);
}

// Validate the items, order them largest first, and write the descriptors
// and per-stage prefix sums into the batch's device arrays.
int fill_batch(mpnl_ctx *ctx, mpnl_batch *b, const mpnl_batch_item *items, int n_items,
               bool check_pointers = true)
{
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    std::vector<mpnl::BatchItem> host(n_items);
    std::vector<int> order(n_items), stg(n_items);
    size_t pre = 16, ref = 16, sel = 16, qhy = 16, mm = 16, det = 16;
    std::vector<char> refine(n_items);
    for (int i = 0; i < n_items; ++i) {
        const mpnl_batch_item &it = items[i];
        const mpnl_dims *d = &it.dims;
        const bool mqr = it.flags & MPNL_ITEM_MMSE_QR, lin = it.flags & MPNL_ITEM_LINEAR_MMSE;
        const int st_bits = item_stages(it);
        stg[i] = st_bits;
        const bool pre_on = st_bits & MPNL_STAGE_PREPROCESS, qhy_on = st_bits & MPNL_STAGE_QHY;
        // the QR stage also forms z when the walks follow and no Q^H y stage does
        const bool carry_y = pre_on && (st_bits & MPNL_STAGE_DETECT) && !qhy_on;
        int st = check_dims(ctx, d, true, mqr ? kNrAugmented : kNrTall);
        if (st == MPNL_OK) st = check_sigma2(ctx, it.sigma2);
        if (st == MPNL_OK && (it.flags & ~(MPNL_ITEM_MMSE_QR | MPNL_ITEM_LINEAR_MMSE |
                                           MPNL_ITEM_FP16 | MPNL_ITEM_REFINE_QR)))
            st = fail(ctx, MPNL_ERR_INVALID_ARG, "unknown flags 0x%x", it.flags);
        if (st == MPNL_OK && (st_bits & ~(MPNL_STAGES_ALL)))
            st = fail(ctx, MPNL_ERR_INVALID_ARG, "unknown stage bits 0x%x", st_bits);
        if (st == MPNL_OK && (st_bits & MPNL_STAGE_MMSE) && !lin)
            st = fail(ctx, MPNL_ERR_INVALID_ARG, "MMSE stage without MPNL_ITEM_LINEAR_MMSE");
        if (st == MPNL_OK && d->n_sc > 0) {
            struct Need {
                const void *p;
                const char *name;
                size_t align;
                bool need;
            } need[] = {
                {it.H, "H", 8, pre_on || (st_bits & MPNL_STAGE_MMSE)},
                {it.Y, "Y", 8, carry_y || qhy_on || (st_bits & MPNL_STAGE_MMSE)},
                {it.Q, "Q", 8, qhy_on},
                {it.R, "R", 8, pre_on || (st_bits & (MPNL_STAGE_SELECT | MPNL_STAGE_DETECT))},
                {it.inv_diag, "inv_diag", 4, pre_on || (st_bits & MPNL_STAGE_DETECT)},
                {it.perm, "perm", 1, pre_on || (st_bits & MPNL_STAGE_DETECT)},
                {it.Z, "Z", 8, carry_y || qhy_on || (st_bits & MPNL_STAGE_DETECT)},
                {it.paths, "paths", 1, (st_bits & (MPNL_STAGE_SELECT | MPNL_STAGE_DETECT)) != 0},
                {it.hard, "hard", 1, (st_bits & MPNL_STAGE_DETECT) != 0},
                {it.mmse_hard, "mmse_hard", 1, (st_bits & MPNL_STAGE_MMSE) != 0},
            };
            for (const Need &n : need)
                if (st == MPNL_OK && n.need) {
                    if (check_pointers) st = check_ptr(ctx, n.p, n.align, n.name, false);
                    else if (!n.p || (uintptr_t)n.p % n.align)
                        st = fail(ctx, MPNL_ERR_INVALID_ARG, "%s is NULL or misaligned", n.name);
                }
            if (check_pointers) {
                if (st == MPNL_OK) st = check_ptr(ctx, it.Q, 8, "Q", true);
                if (st == MPNL_OK) st = check_ptr(ctx, it.llr, 4, "llr", true);
                if (st == MPNL_OK) st = check_ptr(ctx, it.ped2, 4, "ped2", true);
                if (st == MPNL_OK) st = check_ptr(ctx, it.mmse_llr, 4, "mmse_llr", true);
            }
        }
        if (st != MPNL_OK) {
            char msg[sizeof ctx->err];
            snprintf(msg, sizeof msg, "item %d: %s", i, ctx->err);
            return fail(ctx, st, "%s", msg);
        }
        mpnl::BatchItem &h = host[i];
        h.n_sc = d->n_sc;
        h.n_sym = d->n_sym;
        h.nr = d->nr;
        h.nt = d->nt;
        h.qam = d->qam;
        h.n_pe = d->n_pe;
        h.sigma2 = it.sigma2;
        h.sigma = mqr ? sqrtf(it.sigma2) : 0.f;
        h.sym = tuned_sym(ctx, d);
        h.mmse = (st_bits & MPNL_STAGE_MMSE) ? 1 : 0;
        h.f16 = (it.flags & MPNL_ITEM_FP16) ? 1 : 0;
        h.factor_sym = carry_y ? d->n_sym : 0;
        refine[i] = pre_on && (it.flags & MPNL_ITEM_REFINE_QR) ? 1 : 0;
        h.refine_threshold = refine[i] ? kBatchRefineThreshold : 0.f;
        h.Q = (float2 *)it.Q;
        h.H = (const float2 *)it.H;
        h.Y = (const float2 *)it.Y;
        h.R = (float2 *)it.R;
        h.inv_diag = it.inv_diag;
        h.perm = it.perm;
        h.Z = (float2 *)it.Z;
        h.paths = it.paths;
        h.hard = it.hard;
        h.llr = it.llr;
        h.ped2 = it.ped2;
        h.mmse_hard = lin ? it.mmse_hard : nullptr;
        h.mmse_llr = lin ? it.mmse_llr : nullptr;
        if (pre_on) {
            const int rows = mqr ? d->nr + d->nt : d->nr;
            pre = std::max(pre, mpnl::preprocess_warp_bytes(h.factor_sym, rows, d->nt));
            if (refine[i]) ref = std::max(ref, mpnl::refine_warp_bytes(rows, d->nt, h.factor_sym));
        }
        if (st_bits & MPNL_STAGE_SELECT) sel = std::max(sel, mpnl::select_group_bytes(d->n_pe));
        if (qhy_on) qhy = std::max(qhy, mpnl::qhy_warp_bytes(d->n_sym, d->nr, d->nt));
        if (qhy_on && (it.flags & MPNL_ITEM_FP16))
            qhy = std::max(qhy, mpnl::qhy_mma_warp_bytes(d->n_sym, d->nr, d->nt));
        if (st_bits & MPNL_STAGE_DETECT)
            det = std::max(det, mpnl::detect_smem_bytes(d->nt, d->qam, d->n_pe, d->n_sym));
        if (st_bits & MPNL_STAGE_MMSE) mm = std::max(mm, mpnl::mmse_warp_bytes(d->n_sym, d->nr, d->nt));
        order[i] = i;
    }
    // the persistent selection uses one group shape for every unit
    const int sel_warps =
        ctx->tuning.persistent_select_warps ? ctx->tuning.persistent_select_warps : 2;
    int det_ctas = ctx->tuning.persistent_ctas_per_sm ? ctx->tuning.persistent_ctas_per_sm : 3;
    while (det_ctas > 1 && (size_t)det_ctas * det > (size_t)dev_smem) --det_ctas;
    if (det > (size_t)dev_smem || pre * 4 > (size_t)dev_smem || mm * 4 > (size_t)dev_smem ||
        ref * 2 > (size_t)dev_smem ||
        qhy * 4 > (size_t)dev_smem || sel * (4 / sel_warps) > (size_t)dev_smem)
        return fail(ctx, MPNL_ERR_UNSUPPORTED, "a unit needs more shared memory than one SM has");
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return unit_cost(items[a].dims) > unit_cost(items[c].dims);
    });
    // the previous upload must have been read before the staging is rewritten
    cudaError_t ce = cudaEventSynchronize(b->copied);
    if (ce != cudaSuccess) return cuda_fail(ctx, "batch staging", ce);
    const int cap1 = b->capacity + 1;
    mpnl::BatchItem *sorted = b->h_items;
    int *start = b->h_start;
    for (int k = 0; k < kBStages * cap1; ++k) start[k] = 0;
    for (int k = 0; k < n_items; ++k) {
        sorted[k] = host[order[k]];
        const int bits = stg[order[k]];
        for (int q = 0; q < kBStages; ++q) {
            const bool in = (bits & kStageBit[q]) && (q != kBRef || refine[order[k]]);
            start[q * cap1 + k + 1] = start[q * cap1 + k] + (in ? sorted[k].n_sc : 0);
        }
    }
    for (int q = 0; q < kBStages; ++q) {
        b->stage_units[q] = start[q * cap1 + n_items];
        // entries past n_items repeat the total (the kernels read start[n_items])
        for (int k = n_items + 1; k < cap1; ++k) start[q * cap1 + k] = start[q * cap1 + n_items];
    }
    b->dirty = true;  // uploaded by the next run, on its stream
    b->n_items = n_items;
    b->pre_warp_bytes = (int)pre;
    b->ref_warp_bytes = (int)ref;
    b->sel_group_bytes = (int)sel;
    b->qhy_warp_bytes = (int)qhy;
    b->mmse_warp_bytes = (int)mm;
    b->det_smem = det;
    b->sel_warps = sel_warps;
    b->det_ctas = det_ctas;
    for (int k = 0; k < kGraphSlots; ++k)
        if (b->graph[k]) {
            cudaGraphExecDestroy(b->graph[k]);
            b->graph[k] = nullptr;
        }
    return MPNL_OK;
}

int upload_batch(mpnl_ctx *ctx, mpnl_batch *b, cudaStream_t st)
{
    if (!b->dirty) return MPNL_OK;
    const int cap1 = b->capacity + 1;
    cudaError_t e = cudaMemcpyAsync(b->d_items, b->h_items, sizeof(mpnl::BatchItem) * b->n_items,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_start, b->h_start, sizeof(int) * kBStages * cap1,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->copied, st);
    if (e != cudaSuccess) return cuda_fail(ctx, "batch descriptors", e);
    b->dirty = false;
    return MPNL_OK;
}

// share: leave room on every SM for other work (MPNL_RUN_SHARE_SMS): the walk
// stage runs one CTA per SM fewer than tuned (at least one), the warp- and
// group-worker stages half their workers.
// shorts: one item per walk CTA and per warp worker (MPNL_RUN_SHORT_CTAS).
int enqueue_batch(mpnl_ctx *ctx, mpnl_batch *b, int stages, cudaStream_t st, bool share,
                  bool shorts = false)
{
    const int workers = share ? b->sms * 2 : b->sms * 4;
    const int det_ctas = share && b->det_ctas > 1 ? b->det_ctas - 1 : b->det_ctas;
    // CTAs of each stage: persistent (a fixed number per SM, drawing items
    // from the counter until it runs out), or with MPNL_RUN_SHORT_CTAS as many
    // as the stage has items (warp stages: 4 warps per CTA), so that every
    // CTA is short and the hardware spreads them over whatever SMs free up
    auto grid_of = [&](int q, int persistent, int per_cta) {
        if (!shorts) return persistent;
        const long long g = ((long long)b->stage_units[q] + per_cta - 1) / per_cta;
        return (int)std::min<long long>(std::max<long long>(g, 1), 1 << 24);
    };
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, kBStages * sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(ctx, "batch counter reset", e);
    const int cap1 = b->capacity + 1;
    const int *start[kBStages];
    for (int q = 0; q < kBStages; ++q) start[q] = b->d_start + q * cap1;
    const int n = b->n_items;
    if ((stages & MPNL_STAGE_PREPROCESS) && b->stage_units[kBPre]) {
        e = mpnl::launch_preprocess_batch(b->d_items, start[kBPre], n, b->d_counters + kBPre,
                                          b->pre_warp_bytes, grid_of(kBPre, workers, 4), st);
        if (e != cudaSuccess) return cuda_fail(ctx, "batch preprocess launch", e);
    }
    if ((stages & MPNL_STAGE_PREPROCESS) && b->stage_units[kBRef]) {
        e = mpnl::launch_refine_batch(b->d_items, start[kBRef], n, b->d_counters + kBRef,
                                      b->ref_warp_bytes, grid_of(kBRef, workers, 2), st);
        if (e != cudaSuccess) return cuda_fail(ctx, "batch refine launch", e);
    }
    if ((stages & MPNL_STAGE_SELECT) && b->stage_units[kBSel]) {
        e = mpnl::launch_select_batch(b->d_items, start[kBSel], n, b->d_counters + kBSel,
                                      b->sel_group_bytes, b->sel_warps,
                                      grid_of(kBSel, workers, 4 / b->sel_warps), st);
        if (e != cudaSuccess) return cuda_fail(ctx, "batch select launch", e);
    }
    if ((stages & MPNL_STAGE_QHY) && b->stage_units[kBQhy]) {
        e = mpnl::launch_qhy_batch(b->d_items, start[kBQhy], n, b->d_counters + kBQhy,
                                   b->qhy_warp_bytes, grid_of(kBQhy, workers, 4), st);
        if (e != cudaSuccess) return cuda_fail(ctx, "batch qhy launch", e);
    }
    if ((stages & MPNL_STAGE_DETECT) && b->stage_units[kBDet]) {
        e = mpnl::launch_detect_batch(b->d_items, start[kBDet], n, b->d_counters + kBDet,
                                      ctx->status, b->det_smem, grid_of(kBDet, b->sms * det_ctas, 1),
                                      st);
        if (e != cudaSuccess) return cuda_fail(ctx, "batch detect launch", e);
    }
    if ((stages & MPNL_STAGE_MMSE) && b->stage_units[kBMmse]) {
        e = mpnl::launch_mmse_batch(b->d_items, start[kBMmse], n, b->d_counters + kBMmse,
                                    b->mmse_warp_bytes, grid_of(kBMmse, workers, 4), st);
        if (e != cudaSuccess) return cuda_fail(ctx, "batch mmse launch", e);
    }
    return MPNL_OK;
}

}  // namespace

// for the calls defined in other translation units (sm_split.cu)
namespace mpnl {
int api_begin(mpnl_ctx *ctx) { return begin(ctx); }
int api_device(const mpnl_ctx *ctx) { return ctx->device; }
int api_fail(mpnl_ctx *ctx, int code, const char *what, const char *detail)
{
    return detail && detail[0] ? fail(ctx, code, "%s: %s", what, detail) : fail(ctx, code, "%s", what);
}
}  // namespace mpnl

extern "C" {

int mpnl_batch_create(mpnl_ctx *ctx, const mpnl_batch_item *items, int n_items,
                      mpnl_batch **out)
{
    MPNL_TRY(begin(ctx));
    if (!out) return fail(ctx, MPNL_ERR_INVALID_ARG, "batch is NULL");
    *out = nullptr;
    if (n_items < 1 || !items) return fail(ctx, MPNL_ERR_INVALID_ARG, "need at least one item");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    mpnl_batch *b = (mpnl_batch *)calloc(1, sizeof(mpnl_batch));
    if (!b) return fail(ctx, MPNL_ERR_CUDA, "out of host memory");
    b->device = ctx->device;
    b->capacity = n_items;
    b->sms = sms > 0 ? sms : 1;
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(mpnl::BatchItem) * n_items);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_start, sizeof(int) * kBStages * (n_items + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(int) * kBStages);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_items, sizeof(mpnl::BatchItem) * n_items);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_start, sizeof(int) * kBStages * (n_items + 1));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        mpnl_batch_destroy(b);
        return cuda_fail(ctx, "batch create", e);
    }
    const int rc = fill_batch(ctx, b, items, n_items);
    if (rc != MPNL_OK) {
        mpnl_batch_destroy(b);
        return rc;
    }
    *out = b;
    return MPNL_OK;
}

int mpnl_batch_reset(mpnl_ctx *ctx, mpnl_batch *b, const mpnl_batch_item *items, int n_items,
                     int flags)
{
    MPNL_TRY(begin(ctx));
    if (!b) return fail(ctx, MPNL_ERR_INVALID_ARG, "batch is NULL");
    if (b->device != ctx->device)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "batch lives on device %d, context on %d", b->device,
                    ctx->device);
    if (n_items < 1 || n_items > b->capacity || !items)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "n_items=%d outside 1..%d", n_items, b->capacity);
    if (flags & ~MPNL_RESET_TRUSTED_POINTERS)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "unknown reset flags 0x%x", flags);
    return fill_batch(ctx, b, items, n_items, !(flags & MPNL_RESET_TRUSTED_POINTERS));
}

int mpnl_batch_run(mpnl_ctx *ctx, mpnl_batch *b, int stages, void *stream)
{
    MPNL_TRY(begin(ctx));
    if (!b) return fail(ctx, MPNL_ERR_INVALID_ARG, "batch is NULL");
    if (b->device != ctx->device)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "batch lives on device %d, context on %d", b->device,
                    ctx->device);
    if (stages & ~(MPNL_STAGES_ALL | MPNL_RUN_GRAPH | MPNL_RUN_SHARE_SMS | MPNL_RUN_SHORT_CTAS))
        return fail(ctx, MPNL_ERR_INVALID_ARG, "unknown stage bits 0x%x", stages);
    const int mask = stages & MPNL_STAGES_ALL;
    const bool share = (stages & MPNL_RUN_SHARE_SMS) != 0;
    const bool shorts = (stages & MPNL_RUN_SHORT_CTAS) != 0;
    const int slot = mask + (share ? MPNL_STAGES_ALL + 1 : 0) + (shorts ? 2 * (MPNL_STAGES_ALL + 1) : 0);
    cudaStream_t st = (cudaStream_t)stream;
    MPNL_TRY(upload_batch(ctx, b, st));
    if (!(stages & MPNL_RUN_GRAPH)) return enqueue_batch(ctx, b, mask, st, share, shorts);
    if (!st) return fail(ctx, MPNL_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    if (!b->graph[slot]) {
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(ctx, "graph capture begin", e);
        const int rc = enqueue_batch(ctx, b, mask, st, share, shorts);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (rc != MPNL_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, "graph capture end", e);
        e = cudaGraphInstantiate(&b->graph[slot], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph[slot] = nullptr;
            return cuda_fail(ctx, "graph instantiate", e);
        }
    }
    cudaError_t e = cudaGraphLaunch(b->graph[slot], st);
    if (e != cudaSuccess) return cuda_fail(ctx, "graph launch", e);
    return MPNL_OK;
}

int mpnl_serve_round(mpnl_ctx *ctx, mpnl_batch *b, const mpnl_round_req *reqs, int n_reqs,
                     int run_flags, void *stream)
{
    MPNL_TRY(begin(ctx));
    if (!b) return fail(ctx, MPNL_ERR_INVALID_ARG, "batch is NULL");
    if (b->device != ctx->device)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "batch lives on device %d, context on %d", b->device,
                    ctx->device);
    if (!reqs || n_reqs < 1 || n_reqs > b->capacity)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "n_reqs=%d outside 1..%d", n_reqs, b->capacity);
    if (run_flags & ~(MPNL_RUN_SHARE_SMS | MPNL_RUN_SHORT_CTAS))
        return fail(ctx, MPNL_ERR_INVALID_ARG, "unknown run flags 0x%x", run_flags);
    // channel updates first (stable): the stages run in order, so a slot of
    // the same unit in this round reads the new state
    std::vector<int> order;
    order.reserve(n_reqs);
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < n_reqs; ++i)
            if ((reqs[i].kind == MPNL_ROUND_CHANNEL) == (pass == 0)) order.push_back(i);
    std::vector<mpnl_batch_item> items(n_reqs);
    cudaStream_t st = (cudaStream_t)stream;
    for (int k = 0; k < n_reqs; ++k) {
        const mpnl_round_req &q = reqs[order[k]];
        if (!q.unit || (q.kind != MPNL_ROUND_SLOT && q.kind != MPNL_ROUND_CHANNEL) || !q.payload ||
            !q.staging)
            return fail(ctx, MPNL_ERR_INVALID_ARG, "request %d: bad unit, kind or buffers",
                        order[k]);
        const mpnl_dims &d = q.unit->dims;
        if (d.n_sc < 0 || d.n_sym < 0 || d.nr < 1 || d.nt < 1)
            return fail(ctx, MPNL_ERR_INVALID_ARG, "request %d: bad sizes", order[k]);
        mpnl_batch_item it = *q.unit;
        it.H = it.Y = nullptr;
        it.Z = nullptr;
        it.hard = it.mmse_hard = nullptr;
        it.llr = it.ped2 = it.mmse_llr = nullptr;
        if (q.kind == MPNL_ROUND_CHANNEL) {
            it.stages = MPNL_STAGE_PREPROCESS | MPNL_STAGE_SELECT;
            it.H = q.staging;
        } else {
            if (!q.Z || !q.hard || !q.hard_host || (q.llr_host && !q.llr))
                return fail(ctx, MPNL_ERR_INVALID_ARG, "request %d: slot buffers missing",
                            order[k]);
            it.stages = MPNL_STAGE_QHY | MPNL_STAGE_DETECT;
            it.Y = q.staging;
            it.Z = q.Z;
            it.hard = q.hard;
            it.llr = q.llr;
        }
        items[k] = it;
    }
    // everything validated: now enqueue (inputs in, the stages, results out)
    MPNL_TRY(fill_batch(ctx, b, items.data(), n_reqs, false));
    for (int k = 0; k < n_reqs; ++k) {
        const mpnl_round_req &q = reqs[order[k]];
        const mpnl_dims &d = q.unit->dims;
        const size_t bytes = q.kind == MPNL_ROUND_CHANNEL
                                 ? (size_t)d.n_sc * d.nr * d.nt * 8
                                 : (size_t)d.n_sc * d.n_sym * d.nr * 8;
        cudaError_t e = cudaMemcpyAsync(q.staging, q.payload, bytes, cudaMemcpyDefault, st);
        if (e != cudaSuccess) return cuda_fail(ctx, "round input copy", e);
    }
    MPNL_TRY(upload_batch(ctx, b, st));
    MPNL_TRY(enqueue_batch(ctx, b, MPNL_STAGES_ALL, st, (run_flags & MPNL_RUN_SHARE_SMS) != 0,
                           (run_flags & MPNL_RUN_SHORT_CTAS) != 0));
    for (int k = 0; k < n_reqs; ++k) {
        const mpnl_round_req &q = reqs[order[k]];
        if (q.kind != MPNL_ROUND_SLOT) continue;
        const mpnl_dims &d = q.unit->dims;
        const size_t det = (size_t)d.n_sc * d.n_sym;
        cudaError_t e = cudaMemcpyAsync(q.hard_host, q.hard, det * d.nt, cudaMemcpyDefault, st);
        if (e == cudaSuccess && q.llr_host)
            e = cudaMemcpyAsync(q.llr_host, q.llr, det * d.nt * bits_of(d.qam) * 4,
                                cudaMemcpyDefault, st);
        if (e != cudaSuccess) return cuda_fail(ctx, "round output copy", e);
    }
    return MPNL_OK;
}

void mpnl_batch_destroy(mpnl_batch *b)
{
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    for (int k = 0; k < kGraphSlots; ++k)
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_start) cudaFree(b->d_start);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->h_items) cudaFreeHost(b->h_items);
    if (b->h_start) cudaFreeHost(b->h_start);
    if (b->copied) {
        cudaEventSynchronize(b->copied);
        cudaEventDestroy(b->copied);
    }
    free(b);
    if (prev >= 0) cudaSetDevice(prev);
}


int mpnl_create(mpnl_ctx **out, int device)
{
    if (!out) return MPNL_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return MPNL_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return MPNL_ERR_CUDA;
    mpnl_ctx *ctx = new (std::nothrow) mpnl_ctx;
    if (!ctx) return MPNL_ERR_CUDA;
    ctx->device = device;
    if (cudaMalloc(&ctx->status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(ctx->status, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->status) cudaFree(ctx->status);
        delete ctx;
        return MPNL_ERR_CUDA;
    }
    *out = ctx;
    return MPNL_OK;
}

void mpnl_destroy(mpnl_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
    }
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->join) cudaEventDestroy(ctx->join);
    cudaFree(ctx->status);
    delete ctx;
}

const char *mpnl_last_error(const mpnl_ctx *ctx) { return ctx ? ctx->err : "context is NULL"; }


size_t mpnl_workspace_bytes(const mpnl_dims *dims)
{
    (void)dims;
    return 0;
}

static int preprocess_impl(mpnl_ctx *ctx, const mpnl_dims *d, const void *H, const void *Y,
                           float sigma, void *R, float *inv_diag, uint8_t *perm, void *Z,
                           void *stream)
{
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, H, 8, "H", false));
    MPNL_TRY(check_ptr(ctx, Y, 8, "Y", false));
    MPNL_TRY(check_ptr(ctx, R, 8, "R", false));
    MPNL_TRY(check_ptr(ctx, inv_diag, 4, "inv_diag", false));
    MPNL_TRY(check_ptr(ctx, perm, 1, "perm", false));
    MPNL_TRY(check_ptr(ctx, Z, 8, "Z", false));
    cudaError_t e = mpnl::launch_preprocess(d->n_sc, d->n_sym, d->nr, d->nt, sigma,
                                            (const float2 *)H, (const float2 *)Y, (float2 *)R,
                                            inv_diag, perm, (float2 *)Z, nullptr,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "preprocess launch", e);
    return MPNL_OK;
}

int mpnl_preprocess(mpnl_ctx *ctx, const mpnl_dims *d, const void *H, const void *Y, void *R,
                    float *inv_diag, uint8_t *perm, void *Z, void *ws, void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_dims(ctx, d, false, kNrTall));
    return preprocess_impl(ctx, d, H, Y, 0.f, R, inv_diag, perm, Z, stream);
}

int mpnl_preprocess_mmse(mpnl_ctx *ctx, const mpnl_dims *d, const void *H, const void *Y,
                         float sigma2, void *R, float *inv_diag, uint8_t *perm, void *Z, void *ws,
                         void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_dims(ctx, d, false, kNrAugmented));
    MPNL_TRY(check_sigma2(ctx, sigma2));
    return preprocess_impl(ctx, d, H, Y, sqrtf(sigma2), R, inv_diag, perm, Z, stream);
}

int mpnl_factor(mpnl_ctx *ctx, const mpnl_dims *d, const void *H, float sigma2, void *Q, void *R,
                float *inv_diag, uint8_t *perm, void *ws, void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    const bool mmse = sigma2 != 0.0f;
    MPNL_TRY(check_dims(ctx, d, false, mmse ? kNrAugmented : kNrTall));
    if (mmse) MPNL_TRY(check_sigma2(ctx, sigma2));
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, H, 8, "H", false));
    MPNL_TRY(check_ptr(ctx, Q, 8, "Q", false));
    MPNL_TRY(check_ptr(ctx, R, 8, "R", false));
    MPNL_TRY(check_ptr(ctx, inv_diag, 4, "inv_diag", false));
    MPNL_TRY(check_ptr(ctx, perm, 1, "perm", false));
    cudaError_t e = mpnl::launch_preprocess(d->n_sc, 0, d->nr, d->nt, mmse ? sqrtf(sigma2) : 0.f,
                                            (const float2 *)H, nullptr, (float2 *)R, inv_diag, perm,
                                            nullptr, (float2 *)Q, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "factor launch", e);
    return MPNL_OK;
}

int mpnl_refine_qr(mpnl_ctx *ctx, const mpnl_dims *d, const void *H, const void *Y, float sigma2,
                   float cond_threshold, void *R, float *inv_diag, uint8_t *perm, void *Z,
                   void *Q, int *n_refined, void *ws, void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    const bool mmse = sigma2 != 0.0f;
    MPNL_TRY(check_dims(ctx, d, false, mmse ? kNrAugmented : kNrTall));
    if (mmse) MPNL_TRY(check_sigma2(ctx, sigma2));
    if (!(cond_threshold >= 1.0f))
        return fail(ctx, MPNL_ERR_INVALID_ARG, "cond_threshold=%g must be >= 1", (double)cond_threshold);
    if (d->n_sc == 0) return MPNL_OK;
    const bool with_z = Z != nullptr || Y != nullptr;
    MPNL_TRY(check_ptr(ctx, H, 8, "H", false));
    MPNL_TRY(check_ptr(ctx, Y, 8, "Y", !with_z));
    MPNL_TRY(check_ptr(ctx, Z, 8, "Z", !with_z));
    MPNL_TRY(check_ptr(ctx, R, 8, "R", false));
    MPNL_TRY(check_ptr(ctx, inv_diag, 4, "inv_diag", false));
    MPNL_TRY(check_ptr(ctx, perm, 1, "perm", false));
    MPNL_TRY(check_ptr(ctx, Q, 8, "Q", true));
    MPNL_TRY(check_ptr(ctx, n_refined, 4, "n_refined", true));
    cudaError_t e = mpnl::launch_refine(d->n_sc, with_z ? d->n_sym : 0, d->nr, d->nt,
                                        mmse ? sqrtf(sigma2) : 0.f, cond_threshold,
                                        (const float2 *)H, (const float2 *)Y, (float2 *)R, inv_diag,
                                        perm, (float2 *)Z, (float2 *)Q, n_refined,
                                        (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "refine launch", e);
    return MPNL_OK;
}

int mpnl_qhy(mpnl_ctx *ctx, const mpnl_dims *d, const void *Q, const void *Y, void *Z, void *ws,
             void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_dims(ctx, d, false, kNrAny));
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, Q, 8, "Q", false));
    MPNL_TRY(check_ptr(ctx, Y, 8, "Y", false));
    MPNL_TRY(check_ptr(ctx, Z, 8, "Z", false));
    cudaError_t e = mpnl::launch_qhy(d->n_sc, d->n_sym, d->nr, d->nt, (const float2 *)Q,
                                     (const float2 *)Y, (float2 *)Z, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "qhy launch", e);
    return MPNL_OK;
}

int mpnl_qhy_mixed(mpnl_ctx *ctx, const mpnl_dims *d, const void *Q, const void *Y, void *Z,
                   void *ws, void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_dims(ctx, d, false, kNrAny));
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, Q, 8, "Q", false));
    MPNL_TRY(check_ptr(ctx, Y, 8, "Y", false));
    MPNL_TRY(check_ptr(ctx, Z, 8, "Z", false));
    cudaError_t e = mpnl::launch_qhy_mma(d->n_sc, d->n_sym, d->nr, d->nt, (const float2 *)Q,
                                         (const float2 *)Y, (float2 *)Z, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "qhy_mixed launch", e);
    return MPNL_OK;
}

int mpnl_select_paths(mpnl_ctx *ctx, const mpnl_dims *d, const void *R, float sigma2,
                      uint8_t *paths, void *ws, void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_dims(ctx, d, true));
    MPNL_TRY(check_sigma2(ctx, sigma2));
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, R, 8, "R", false));
    MPNL_TRY(check_ptr(ctx, paths, 1, "paths", false));
    cudaError_t e = mpnl::launch_select_paths(d->n_sc, d->nt, d->qam, d->n_pe, sigma2,
                                              (const float2 *)R, paths, tuned_select_warps(ctx, d),
                                              (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "select_paths launch", e);
    return MPNL_OK;
}

int mpnl_select_paths_lut(mpnl_ctx *ctx, const mpnl_dims *d, const void *R, float sigma2,
                          const mpnl_rank_lut *lut, uint8_t *paths, void *ws, void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_dims(ctx, d, true));
    MPNL_TRY(check_sigma2(ctx, sigma2));
    if (!lut) return fail(ctx, MPNL_ERR_INVALID_ARG, "lut is NULL");
    if (lut->qam != d->qam)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "table qam=%d differs from dims qam=%d", lut->qam,
                    d->qam);
    if (lut->n_bins < 1 || lut->n_bins > 65535)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "n_bins=%d outside 1..65535", lut->n_bins);
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, R, 8, "R", false));
    MPNL_TRY(check_ptr(ctx, paths, 1, "paths", false));
    MPNL_TRY(check_ptr(ctx, lut->cost, 4, "cost", false));
    MPNL_TRY(check_ptr(ctx, lut->edges, 4, "edges", lut->n_bins == 1));
    cudaError_t e = mpnl::launch_select_paths_lut(d->n_sc, d->nt, d->qam, d->n_pe, sigma2,
                                                  (const float2 *)R, lut->edges, lut->cost,
                                                  lut->n_bins, paths, tuned_select_warps(ctx, d),
                                                  (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "select_paths_lut launch", e);
    return MPNL_OK;
}

// The real-valued decomposition: dims describe the complex problem; its 2 nt
// real levels must fit the walks (2 nt <= MPNL_MAX_NT) and n_pe is bounded
// by L^(2 nt) instead of M^nt.
static int check_rvd_dims(mpnl_ctx *ctx, const mpnl_dims *d, bool need_pe)
{
    MPNL_TRY(check_dims(ctx, d, false));
    if (2 * d->nt > MPNL_MAX_NT)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "nt=%d: 2 nt real levels exceed %d", d->nt,
                    MPNL_MAX_NT);
    if (need_pe) {
        const double L = (double)(1 << (bits_of(d->qam) / 2));
        const double cap = pow(L, 2.0 * d->nt);
        if (d->n_pe < 1 || d->n_pe > MPNL_MAX_NPE || (double)d->n_pe > cap)
            return fail(ctx, MPNL_ERR_INVALID_ARG, "n_pe=%d outside 1..min(%d, L^(2 nt))",
                        d->n_pe, MPNL_MAX_NPE);
    }
    return MPNL_OK;
}

int mpnl_rvd_embed(mpnl_ctx *ctx, const mpnl_dims *d, const void *H, const void *Y, void *Hr,
                   void *Yr, void *stream)
{
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_rvd_dims(ctx, d, false));
    if (2 * d->nr > MPNL_MAX_NR)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "nr=%d: 2 nr real rows exceed %d", d->nr,
                    MPNL_MAX_NR);
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, H, 8, "H", false));
    MPNL_TRY(check_ptr(ctx, Y, 8, "Y", false));
    MPNL_TRY(check_ptr(ctx, Hr, 8, "Hr", false));
    MPNL_TRY(check_ptr(ctx, Yr, 8, "Yr", false));
    cudaError_t e = mpnl::launch_rvd_embed(d->n_sc, d->n_sym, d->nr, d->nt, (const float2 *)H,
                                           (const float2 *)Y, (float2 *)Hr, (float2 *)Yr,
                                           (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "rvd_embed launch", e);
    return MPNL_OK;
}

int mpnl_select_paths_pam(mpnl_ctx *ctx, const mpnl_dims *d, const void *R, float sigma2,
                          uint8_t *paths, void *ws, void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_rvd_dims(ctx, d, true));
    MPNL_TRY(check_sigma2(ctx, sigma2));
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, R, 8, "R", false));
    MPNL_TRY(check_ptr(ctx, paths, 1, "paths", false));
    cudaError_t e = mpnl::launch_select_paths_pam(d->n_sc, 2 * d->nt, d->qam, d->n_pe, sigma2,
                                                  (const float2 *)R, paths,
                                                  d->n_pe >= 256 ? 2 : 1, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "select_paths_pam launch", e);
    return MPNL_OK;
}

int mpnl_detect_rvd(mpnl_ctx *ctx, const mpnl_dims *d, const void *R, const float *inv_diag,
                    const uint8_t *perm, const uint8_t *paths, const void *Z, float sigma2,
                    uint8_t *hard, float *llr, float *ped2, void *ws, void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_rvd_dims(ctx, d, true));
    MPNL_TRY(check_sigma2(ctx, sigma2));
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, R, 8, "R", false));
    MPNL_TRY(check_ptr(ctx, inv_diag, 4, "inv_diag", false));
    MPNL_TRY(check_ptr(ctx, perm, 1, "perm", false));
    MPNL_TRY(check_ptr(ctx, paths, 1, "paths", false));
    MPNL_TRY(check_ptr(ctx, Z, 8, "Z", false));
    MPNL_TRY(check_ptr(ctx, hard, 1, "hard", false));
    MPNL_TRY(check_ptr(ctx, llr, 4, "llr", true));
    MPNL_TRY(check_ptr(ctx, ped2, 4, "ped2", true));
    cudaError_t e = mpnl::launch_detect_rvd(d->n_sc, d->n_sym, d->nt, d->qam, d->n_pe, sigma2,
                                            (const float2 *)R, inv_diag, perm, paths,
                                            (const float2 *)Z, hard, llr, ped2, ctx->status,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "detect_rvd launch", e);
    return MPNL_OK;
}

static int check_lut_args(mpnl_ctx *ctx, int qam, int n_bins, long long n_trials)
{
    if (!bits_of(qam)) return fail(ctx, MPNL_ERR_INVALID_ARG, "qam=%d not in {4,16,64}", qam);
    if (n_bins < 1 || n_bins > 65535)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "n_bins=%d outside 1..65535", n_bins);
    if (n_trials < 1 || n_trials >= (1ll << 38))
        return fail(ctx, MPNL_ERR_INVALID_ARG, "n_trials=%lld outside 1..2^38-1", n_trials);
    return MPNL_OK;
}

int mpnl_rank_counts(mpnl_ctx *ctx, int qam, int n_bins, const double *gamma, long long n_trials,
                     unsigned long long seed, unsigned long long *counts, void *stream)
{
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_lut_args(ctx, qam, n_bins, n_trials));
    MPNL_TRY(check_ptr(ctx, gamma, 8, "gamma", false));
    MPNL_TRY(check_ptr(ctx, counts, 8, "counts", false));
    cudaError_t e = mpnl::launch_rank_counts(qam, n_bins, gamma, n_trials, seed, counts,
                                             (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "rank_counts launch", e);
    return MPNL_OK;
}

int mpnl_rank_costs(mpnl_ctx *ctx, int qam, int n_bins, const unsigned long long *counts,
                    long long n_trials, float *cost, void *stream)
{
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_lut_args(ctx, qam, n_bins, n_trials));
    MPNL_TRY(check_ptr(ctx, counts, 8, "counts", false));
    MPNL_TRY(check_ptr(ctx, cost, 4, "cost", false));
    cudaError_t e = mpnl::launch_rank_costs(qam, n_bins, counts, n_trials, cost,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "rank_costs launch", e);
    return MPNL_OK;
}

static int detect_impl(mpnl_ctx *ctx, const mpnl_dims *d, const void *R, const float *inv_diag,
                       const uint8_t *perm, const uint8_t *paths, const void *Z, float sigma2,
                       uint8_t *hard, float *llr, float *ped2, void *stream, bool f16)
{
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_dims(ctx, d, true));
    MPNL_TRY(check_sigma2(ctx, sigma2));
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, R, 8, "R", false));
    MPNL_TRY(check_ptr(ctx, inv_diag, 4, "inv_diag", false));
    MPNL_TRY(check_ptr(ctx, perm, 1, "perm", false));
    MPNL_TRY(check_ptr(ctx, paths, 1, "paths", false));
    MPNL_TRY(check_ptr(ctx, Z, 8, "Z", false));
    MPNL_TRY(check_ptr(ctx, hard, 1, "hard", false));
    MPNL_TRY(check_ptr(ctx, llr, 4, "llr", true));
    MPNL_TRY(check_ptr(ctx, ped2, 4, "ped2", true));
    cudaError_t e = mpnl::launch_detect(d->n_sc, d->n_sym, d->nt, d->qam, d->n_pe, sigma2,
                                        (const float2 *)R, inv_diag, perm, paths, (const float2 *)Z,
                                        hard, llr, ped2, ctx->status, f16, tuned_sym(ctx, d),
                                        (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "detect launch", e);
    return MPNL_OK;
}

int mpnl_detect(mpnl_ctx *ctx, const mpnl_dims *d, const void *R, const float *inv_diag,
                const uint8_t *perm, const uint8_t *paths, const void *Z, float sigma2,
                uint8_t *hard, float *llr, float *ped2, void *ws, void *stream)
{
    (void)ws;
    return detect_impl(ctx, d, R, inv_diag, perm, paths, Z, sigma2, hard, llr, ped2, stream, false);
}

int mpnl_detect_mixed(mpnl_ctx *ctx, const mpnl_dims *d, const void *R, const float *inv_diag,
                      const uint8_t *perm, const uint8_t *paths, const void *Z, float sigma2,
                      uint8_t *hard, float *llr, float *ped2, void *ws, void *stream)
{
    (void)ws;
    return detect_impl(ctx, d, R, inv_diag, perm, paths, Z, sigma2, hard, llr, ped2, stream, true);
}

int mpnl_linear_mmse(mpnl_ctx *ctx, const mpnl_dims *d, const void *H, const void *Y,
                     float sigma2, uint8_t *hard, float *llr, void *ws, void *stream)
{
    (void)ws;
    MPNL_TRY(begin(ctx));
    MPNL_TRY(check_dims(ctx, d, false));
    MPNL_TRY(check_sigma2(ctx, sigma2));
    if (d->n_sc == 0) return MPNL_OK;
    MPNL_TRY(check_ptr(ctx, H, 8, "H", false));
    MPNL_TRY(check_ptr(ctx, Y, 8, "Y", false));
    MPNL_TRY(check_ptr(ctx, hard, 1, "hard", false));
    MPNL_TRY(check_ptr(ctx, llr, 4, "llr", true));
    cudaError_t e = mpnl::launch_mmse(d->n_sc, d->n_sym, d->nr, d->nt, d->qam, sigma2,
                                      (const float2 *)H, (const float2 *)Y, hard, llr,
                                      (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "mmse launch", e);
    return MPNL_OK;
}

int mpnl_check_status(mpnl_ctx *ctx, void *stream)
{
    MPNL_TRY(begin(ctx));
    unsigned h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->status, sizeof h, cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status, 0, sizeof(unsigned), (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "check_status", e);
    if (h & mpnl::kStatusBadPathEntry)
        return fail(ctx, MPNL_ERR_INVALID_ARG,
                    "detect: a position-vector entry was outside 1..qam (clamped)");
    return MPNL_OK;
}

int mpnl_set_tuning(mpnl_ctx *ctx, const mpnl_tuning *t)
{
    if (!ctx) return MPNL_ERR_INVALID_ARG;
    ctx->err[0] = '\0';
    if (!t) {
        memset(&ctx->tuning, 0, sizeof ctx->tuning);
        return MPNL_OK;
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 2; ++c) {
                const int s = t->detect_sym[a][b][c], w = t->select_warps[a][b][c];
                if (s > 2) return fail(ctx, MPNL_ERR_INVALID_ARG, "detect_sym=%d not in {0,1,2}", s);
                if (w != 0 && w != 1 && w != 2 && w != 4)
                    return fail(ctx, MPNL_ERR_INVALID_ARG, "select_warps=%d not in {0,1,2,4}", w);
            }
    if (t->persistent_ctas_per_sm > 3)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "persistent_ctas_per_sm=%d not in {0,1,2,3}",
                    t->persistent_ctas_per_sm);
    {
        const int w = t->persistent_select_warps;
        if (w != 0 && w != 1 && w != 2 && w != 4)
            return fail(ctx, MPNL_ERR_INVALID_ARG, "persistent_select_warps=%d not in {0,1,2,4}", w);
    }
    ctx->tuning = *t;
    return MPNL_OK;
}

int mpnl_get_tuning(mpnl_ctx *ctx, mpnl_tuning *t)
{
    if (!ctx) return MPNL_ERR_INVALID_ARG;
    ctx->err[0] = '\0';
    if (!t) return fail(ctx, MPNL_ERR_INVALID_ARG, "tuning is NULL");
    *t = ctx->tuning;
    return MPNL_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// End-to-end slot call on caller buffers (host or device) with a workspace
// ---------------------------------------------------------------------------
namespace {

struct SlotLayout {
    size_t H, Y, R, invd, perm, Z, paths, hard, llr, ped2, mhard, mllr, bytes;
};

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

SlotLayout slot_layout(const mpnl_dims *d, int flags)
{
    const size_t sc = (size_t)d->n_sc, ns = (size_t)d->n_sym, nr = (size_t)d->nr,
                 nt = (size_t)d->nt, B = (size_t)bits_of(d->qam);
    SlotLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    L.H = take(sc * nr * nt * 8);
    L.Y = take(sc * ns * nr * 8);
    L.R = take(sc * (nt * (nt + 1) / 2) * 8);
    L.invd = take(sc * nt * 4);
    L.perm = take(sc * nt);
    L.Z = take(sc * ns * nt * 8);
    L.paths = take(sc * (size_t)d->n_pe * nt);
    L.hard = take(sc * ns * nt);
    L.llr = take(sc * ns * nt * B * 4);
    L.ped2 = take(sc * ns * 2 * 4);
    const bool mm = flags & MPNL_SLOT_MMSE;
    L.mhard = take(mm ? sc * ns * nt : 0);
    L.mllr = take(mm ? sc * ns * nt * B * 4 : 0);
    L.bytes = o;
    return L;
}

// non-NULL and aligned; host memory of any kind is fine for a copy
int check_buf(mpnl_ctx *ctx, const void *p, size_t align, const char *name, bool nullable)
{
    if (!p) return nullable ? MPNL_OK : fail(ctx, MPNL_ERR_INVALID_ARG, "%s is NULL", name);
    if ((uintptr_t)p % align)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "%s is not %zu-byte aligned", name, align);
    return MPNL_OK;
}

}  // namespace

extern "C" {

size_t mpnl_slot_workspace_bytes(const mpnl_dims *dims, int flags)
{
    if (!dims || dims->n_sc < 0 || dims->n_sym < 0 || dims->nr < 0 || dims->nt < 0 ||
        dims->n_pe < 0 || !bits_of(dims->qam))
        return 0;
    return slot_layout(dims, flags).bytes;
}

// The context's side stream and fork/join events, made on first use (called
// with side_mu held); false if CUDA cannot make them (the caller then runs
// the baseline on its own stream).
static bool side_ready(mpnl_ctx *ctx)
{
    if (ctx->side) return true;
    cudaStream_t s = nullptr;
    cudaEvent_t f = nullptr, j = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreateWithFlags(&f, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess) {
        ctx->side = s;
        ctx->fork = f;
        ctx->join = j;
        return true;
    }
    cudaGetLastError();
    if (s) cudaStreamDestroy(s);
    if (f) cudaEventDestroy(f);
    if (j) cudaEventDestroy(j);
    return false;
}

int mpnl_detect_slot(mpnl_ctx *ctx, const mpnl_dims *d, float sigma2, const void *H,
                     const void *Y, uint8_t *hard, float *llr, float *ped2, uint8_t *mmse_hard,
                     float *mmse_llr, int flags, void *ws, size_t ws_bytes, void *stream)
{
    MPNL_TRY(begin(ctx));
    if (flags & ~(MPNL_SLOT_MMSE | MPNL_SLOT_FP16 | MPNL_SLOT_MMSE_QR))
        return fail(ctx, MPNL_ERR_INVALID_ARG, "unknown slot flags 0x%x", flags);
    const bool mqr = flags & MPNL_SLOT_MMSE_QR;
    MPNL_TRY(check_dims(ctx, d, true, mqr ? kNrAugmented : kNrTall));
    MPNL_TRY(check_sigma2(ctx, sigma2));
    if (d->n_sc == 0) return MPNL_OK;
    const SlotLayout L = slot_layout(d, flags);
    if (ws_bytes < L.bytes)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "workspace of %zu bytes, need %zu", ws_bytes,
                    L.bytes);
    MPNL_TRY(check_ptr(ctx, ws, 256, "ws", false));
    MPNL_TRY(check_buf(ctx, H, 8, "H", false));
    MPNL_TRY(check_buf(ctx, Y, 8, "Y", false));
    MPNL_TRY(check_buf(ctx, hard, 1, "hard", false));
    MPNL_TRY(check_buf(ctx, llr, 4, "llr", true));
    MPNL_TRY(check_buf(ctx, ped2, 4, "ped2", true));
    const bool mm = flags & MPNL_SLOT_MMSE;
    MPNL_TRY(check_buf(ctx, mmse_hard, 1, "mmse_hard", !mm));
    MPNL_TRY(check_buf(ctx, mmse_llr, 4, "mmse_llr", true));
    unsigned char *w = (unsigned char *)ws;
    float2 *dH = (float2 *)(w + L.H), *dY = (float2 *)(w + L.Y), *dR = (float2 *)(w + L.R);
    float2 *dZ = (float2 *)(w + L.Z);
    float *dInv = (float *)(w + L.invd), *dLlr = (float *)(w + L.llr);
    float *dPed = (float *)(w + L.ped2), *dMllr = (float *)(w + L.mllr);
    uint8_t *dPerm = w + L.perm, *dPaths = w + L.paths, *dHard = w + L.hard, *dMhard = w + L.mhard;
    const size_t sc = (size_t)d->n_sc, ns = (size_t)d->n_sym, nt = (size_t)d->nt;
    const size_t B = (size_t)bits_of(d->qam);
    cudaStream_t st = (cudaStream_t)stream;
    const char *what = "slot input copy";
    cudaError_t e = cudaMemcpyAsync(dH, H, sc * d->nr * nt * 8, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dY, Y, sc * ns * d->nr * 8, cudaMemcpyDefault, st);
    // the MMSE baseline needs only H and Y: on the context's side stream,
    // beside the path, joined back before its outputs are copied
    std::unique_lock<std::mutex> side_lock(ctx->side_mu, std::defer_lock);
    bool forked = false;
    if (e == cudaSuccess && mm) {
        what = "mmse launch";
        side_lock.lock();
        if (side_ready(ctx)) {
            e = cudaEventRecord(ctx->fork, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->fork, 0);
            if (e == cudaSuccess)
                e = mpnl::launch_mmse(d->n_sc, d->n_sym, d->nr, d->nt, d->qam, sigma2, dH, dY,
                                      dMhard, mmse_llr ? dMllr : nullptr, ctx->side);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->join, ctx->side);
            forked = e == cudaSuccess;
        } else {
            side_lock.unlock();
            e = mpnl::launch_mmse(d->n_sc, d->n_sym, d->nr, d->nt, d->qam, sigma2, dH, dY, dMhard,
                                  mmse_llr ? dMllr : nullptr, st);
        }
    }
    if (e == cudaSuccess) {
        what = "preprocess launch";
        e = mpnl::launch_preprocess(d->n_sc, d->n_sym, d->nr, d->nt, mqr ? sqrtf(sigma2) : 0.f, dH,
                                    dY, dR, dInv, dPerm, dZ, nullptr, st);
    }
    if (e == cudaSuccess) {
        what = "select_paths launch";
        e = mpnl::launch_select_paths(d->n_sc, d->nt, d->qam, d->n_pe, sigma2, dR, dPaths,
                                      tuned_select_warps(ctx, d), st);
    }
    if (e == cudaSuccess) {
        what = "detect launch";
        e = mpnl::launch_detect(d->n_sc, d->n_sym, d->nt, d->qam, d->n_pe, sigma2, dR, dInv, dPerm,
                                dPaths, dZ, dHard, llr ? dLlr : nullptr, ped2 ? dPed : nullptr,
                                ctx->status, (flags & MPNL_SLOT_FP16) != 0, tuned_sym(ctx, d), st);
    }
    if (e == cudaSuccess) {
        what = "slot output copy";
        e = cudaMemcpyAsync(hard, dHard, sc * ns * nt, cudaMemcpyDefault, st);
    }
    if (e == cudaSuccess && llr)
        e = cudaMemcpyAsync(llr, dLlr, sc * ns * nt * B * 4, cudaMemcpyDefault, st);
    if (e == cudaSuccess && ped2) e = cudaMemcpyAsync(ped2, dPed, sc * ns * 8, cudaMemcpyDefault, st);
    if (forked) {
        // join even after an error, so that the workspace is not reused
        // while the baseline still reads it
        const cudaError_t j = cudaStreamWaitEvent(st, ctx->join, 0);
        if (e == cudaSuccess) e = j;
        side_lock.unlock();
    }
    if (e == cudaSuccess && mm) e = cudaMemcpyAsync(mmse_hard, dMhard, sc * ns * nt, cudaMemcpyDefault, st);
    if (e == cudaSuccess && mm && mmse_llr)
        e = cudaMemcpyAsync(mmse_llr, dMllr, sc * ns * nt * B * 4, cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(ctx, what, e);
    return MPNL_OK;
}

}  // extern "C"
