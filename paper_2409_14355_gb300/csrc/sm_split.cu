// SM partition for the serving loop (mpnl_sm_split_*): the device's SMs split
// into two disjoint groups with CUDA green contexts, and streams created in
// each group.  A green context is the device's primary context restricted to
// a set of SMs, so device memory, this library's kernels and every other
// call work on its streams as on any stream of the device; only the SMs its
// kernels may occupy differ.  The serving loop gives the small radio units'
// rounds a group of their own, so their CTAs never wait behind the walk CTAs
// of a large unit's round for an SM to free up.
//
// The driver entry points are fetched through the runtime
// (cudaGetDriverEntryPointByVersion): the library links no driver library of
// its own, and a driver without green contexts makes the calls return
// MPNL_ERR_UNSUPPORTED.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>
#include <new>
#include <vector>

#include "mpnl.h"
#include "mpnl_internal.h"

struct mpnl_sm_split {
    CUgreenCtx green[2] = {nullptr, nullptr};
    int sms[2] = {0, 0};
    std::vector<CUstream> streams;
};

namespace {

struct Driver {
    PFN_cuDeviceGet_v2000 device_get = nullptr;
    PFN_cuDeviceGetDevResource_v12040 get_resource = nullptr;
    PFN_cuDevSmResourceSplitByCount_v12040 split = nullptr;
    PFN_cuDevResourceGenerateDesc_v12040 gen_desc = nullptr;
    PFN_cuGreenCtxCreate_v12040 green_create = nullptr;
    PFN_cuGreenCtxDestroy_v12040 green_destroy = nullptr;
    PFN_cuGreenCtxStreamCreate_v12050 stream_create = nullptr;
    PFN_cuStreamSynchronize_v2000 stream_sync = nullptr;
    PFN_cuStreamDestroy_v4000 stream_destroy = nullptr;
    PFN_cuGetErrorName_v6000 error_name = nullptr;
    bool ok = false;
};

template <typename F>
bool entry(const char *name, unsigned version, F &fn)
{
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    fn = reinterpret_cast<F>(p);
    return true;
}

const Driver &driver()
{
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        d.ok = entry("cuDeviceGet", 2000, d.device_get) &&
               entry("cuDeviceGetDevResource", 12040, d.get_resource) &&
               entry("cuDevSmResourceSplitByCount", 12040, d.split) &&
               entry("cuDevResourceGenerateDesc", 12040, d.gen_desc) &&
               entry("cuGreenCtxCreate", 12040, d.green_create) &&
               entry("cuGreenCtxDestroy", 12040, d.green_destroy) &&
               entry("cuGreenCtxStreamCreate", 12050, d.stream_create) &&
               entry("cuStreamSynchronize", 2000, d.stream_sync) &&
               entry("cuStreamDestroy", 4000, d.stream_destroy) &&
               entry("cuGetErrorName", 6000, d.error_name);
    });
    return d;
}

int drv_fail(mpnl_ctx *ctx, const char *what, CUresult r)
{
    const char *name = "?";
    if (driver().error_name) driver().error_name(r, &name);
    return mpnl::api_fail(ctx, MPNL_ERR_CUDA, what, name ? name : "?");
}

}  // namespace

extern "C" int mpnl_sm_split_create(mpnl_ctx *ctx, int sms_first, mpnl_sm_split **split,
                                    int *sms)
{
    int st = mpnl::api_begin(ctx);
    if (st) return st;
    if (!split || !sms) return mpnl::api_fail(ctx, MPNL_ERR_INVALID_ARG, "split or sms is NULL", "");
    *split = nullptr;
    const int device = mpnl::api_device(ctx);
    int n_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return mpnl::api_fail(ctx, MPNL_ERR_CUDA, "cudaDeviceGetAttribute",
                                                cudaGetErrorName(e));
    if (sms_first < 1 || sms_first >= n_sm)
        return mpnl::api_fail(ctx, MPNL_ERR_INVALID_ARG, "sms_first outside 1..SMs-1", "");
    const Driver &d = driver();
    if (!d.ok)
        return mpnl::api_fail(ctx, MPNL_ERR_UNSUPPORTED, "driver has no green contexts", "");
    // the primary context is made current first (the green contexts retain it)
    e = cudaFree(nullptr);
    if (e != cudaSuccess) return mpnl::api_fail(ctx, MPNL_ERR_CUDA, "context init", cudaGetErrorName(e));
    CUdevice dev;
    CUresult r = d.device_get(&dev, device);
    if (r != CUDA_SUCCESS) return drv_fail(ctx, "cuDeviceGet", r);
    CUdevResource all{}, first{}, rest{};
    r = d.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM);
    if (r != CUDA_SUCCESS) return drv_fail(ctx, "cuDeviceGetDevResource", r);
    unsigned n_groups = 1;
    r = d.split(&first, &n_groups, &all, &rest, 0, (unsigned)sms_first);
    if (r != CUDA_SUCCESS) return drv_fail(ctx, "cuDevSmResourceSplitByCount", r);
    if (n_groups != 1 || first.sm.smCount == 0 || rest.type != CU_DEV_RESOURCE_TYPE_SM ||
        rest.sm.smCount == 0)
        return mpnl::api_fail(ctx, MPNL_ERR_INVALID_ARG,
                              "no split with that many SMs in the first group", "");
    mpnl_sm_split *s = new (std::nothrow) mpnl_sm_split;
    if (!s) return mpnl::api_fail(ctx, MPNL_ERR_CUDA, "host allocation", "");
    CUdevResource *parts[2] = {&first, &rest};
    for (int k = 0; k < 2; ++k) {
        CUdevResourceDesc desc;
        r = d.gen_desc(&desc, parts[k], 1);
        if (r == CUDA_SUCCESS) r = d.green_create(&s->green[k], desc, dev, CU_GREEN_CTX_DEFAULT_STREAM);
        if (r != CUDA_SUCCESS) {
            mpnl_sm_split_destroy(ctx, s);
            return drv_fail(ctx, "green context", r);
        }
        s->sms[k] = (int)parts[k]->sm.smCount;
    }
    sms[0] = s->sms[0];
    sms[1] = s->sms[1];
    *split = s;
    return MPNL_OK;
}

extern "C" int mpnl_sm_split_stream(mpnl_ctx *ctx, mpnl_sm_split *split, int part, int priority,
                                    void **stream)
{
    int st = mpnl::api_begin(ctx);
    if (st) return st;
    if (!split || !stream || part < 0 || part > 1)
        return mpnl::api_fail(ctx, MPNL_ERR_INVALID_ARG, "bad split, stream or part", "");
    CUstream s = nullptr;
    const CUresult r = driver().stream_create(&s, split->green[part], CU_STREAM_NON_BLOCKING, priority);
    if (r != CUDA_SUCCESS) return drv_fail(ctx, "cuGreenCtxStreamCreate", r);
    try {
        split->streams.push_back(s);
    } catch (...) {
        driver().stream_destroy(s);
        return mpnl::api_fail(ctx, MPNL_ERR_CUDA, "host allocation", "");
    }
    *stream = s;
    return MPNL_OK;
}

extern "C" int mpnl_sm_split_destroy(mpnl_ctx *ctx, mpnl_sm_split *split)
{
    if (!split) return MPNL_OK;
    int st = ctx ? mpnl::api_begin(ctx) : MPNL_OK;
    const Driver &d = driver();
    CUresult first_err = CUDA_SUCCESS;
    for (CUstream s : split->streams) {
        CUresult r = d.stream_sync(s);
        const CUresult r2 = d.stream_destroy(s);
        if (r == CUDA_SUCCESS) r = r2;
        if (first_err == CUDA_SUCCESS) first_err = r;
    }
    for (int k = 0; k < 2; ++k)
        if (split->green[k]) {
            const CUresult r = d.green_destroy(split->green[k]);
            if (first_err == CUDA_SUCCESS) first_err = r;
        }
    delete split;
    if (st) return st;
    return first_err == CUDA_SUCCESS ? MPNL_OK : drv_fail(ctx, "split teardown", first_err);
}
