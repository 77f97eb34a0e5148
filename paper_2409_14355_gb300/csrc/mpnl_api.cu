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

#include "mpnl.h"
#include "mpnl_internal.h"

struct mpnl_ctx {
    int device;
    unsigned *status;  // device word of kStatus* bits, cleared by mpnl_check_status
    char err[512];
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

extern "C" {

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
    mpnl_ctx *ctx = (mpnl_ctx *)calloc(1, sizeof(mpnl_ctx));
    if (!ctx) return MPNL_ERR_CUDA;
    ctx->device = device;
    if (cudaMalloc(&ctx->status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(ctx->status, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->status) cudaFree(ctx->status);
        free(ctx);
        return MPNL_ERR_CUDA;
    }
    *out = ctx;
    return MPNL_OK;
}

void mpnl_destroy(mpnl_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaFree(ctx->status);
    free(ctx);
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
                                            inv_diag, perm, (float2 *)Z, (cudaStream_t)stream);
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
                                              (const float2 *)R, paths, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "select_paths launch", e);
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
                                        hard, llr, ped2, ctx->status, f16, (cudaStream_t)stream);
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

int mpnl_probe_ffma(mpnl_ctx *ctx, int n_blocks, int iters, float *out, double *flops,
                    void *stream)
{
    MPNL_TRY(begin(ctx));
    if (!flops) return fail(ctx, MPNL_ERR_INVALID_ARG, "flops is NULL");
    if (n_blocks < 1 || iters < 1)
        return fail(ctx, MPNL_ERR_INVALID_ARG, "n_blocks=%d, iters=%d must be >= 1", n_blocks, iters);
    // at most ~1e13 flop (about a tenth of a second): the probe never runs long
    const double f = mpnl::ffma_probe_flops(n_blocks, iters);
    if (f > 1e13) return fail(ctx, MPNL_ERR_INVALID_ARG, "probe of %.3g flop exceeds 1e13", f);
    MPNL_TRY(check_ptr(ctx, out, 4, "out", false));
    cudaError_t e = mpnl::launch_ffma_probe(n_blocks, iters, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "ffma probe launch", e);
    *flops = f;
    return MPNL_OK;
}

}  // extern "C"
