// Walks of several radio units for callers that may not allocate device
// memory (mpnl_detect_units_noalloc in include/mpnl.h).
//
// The persistent walk kernel of the batch calls needs scratch in global
// memory beside its inputs and outputs: the units' descriptors, the prefix
// sums of their subcarrier counts, the work counter the CTAs draw items
// from, and the status word for clamped table entries.  mpnl_batch_create
// allocates that scratch with cudaMalloc.  Here it lives in one file-scope
// __device__ array of fixed size instead, which every device that loads the
// library holds from module load until the process exits; the entry point
// itself allocates nothing.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "mpnl.h"
#include "mpnl_internal.h"

namespace {

constexpr int kMaxUnits = MPNL_NOALLOC_MAX_UNITS;
constexpr size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }
// layout of the scratch array
constexpr size_t kItemsOff = 0;
constexpr size_t kStartOff = round256(sizeof(mpnl::BatchItem) * kMaxUnits);
constexpr size_t kCounterOff = kStartOff + round256(sizeof(int) * (kMaxUnits + 1));
constexpr size_t kStatusOff = kCounterOff + 256;
constexpr size_t kScratchBytes = kStatusOff + 256;

}  // namespace

// Shared by every call on a device; it keeps the previous call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// Per device, filled by the first call made with that device current: the
// device address of g_noalloc_scratch (host code cannot use the symbol
// itself, which names a host-side shadow), the SM count and the opt-in
// shared memory per CTA.
constexpr int kMaxDevices = 64;
struct DeviceSetup {
    unsigned char *scratch;
    int sms;
    int smem_optin;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

int setup_device(int dev, DeviceSetup *out)
{
    if (dev < 0 || dev >= kMaxDevices) return MPNL_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.scratch) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return MPNL_ERR_CUDA;
        }
        int sms = 0, smem = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
                cudaSuccess ||
            sms < 1) {
            cudaGetLastError();
            return MPNL_ERR_CUDA;
        }
        s.sms = sms;
        s.smem_optin = smem;
        s.scratch = (unsigned char *)p;
    }
    *out = s;
    return MPNL_OK;
}

// Non-NULL, aligned and reachable from device `dev` (device memory of that
// device, managed or CUDA-registered host memory).
bool ptr_ok(const void *p, size_t align, int dev, bool nullable)
{
    if (!p) return nullable;
    if ((uintptr_t)p % align) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeUnregistered) return false;
    if (a.type == cudaMemoryTypeDevice && a.device != dev) return false;
    return true;
}

int bits_of(int qam) { return qam == 4 ? 2 : qam == 16 ? 4 : qam == 64 ? 6 : 0; }

// One unit's descriptor for the walk stage, or an error code.
int unit_item(const mpnl_batch_item &it, int dev, mpnl::BatchItem *h)
{
    const mpnl_dims &d = it.dims;
    if (d.n_sc < 0 || d.nt < 1 || d.nt > MPNL_MAX_NT || d.nr < 1 || d.nr > MPNL_MAX_NR ||
        d.n_sym < 1 || d.n_sym > MPNL_MAX_NSYM || !bits_of(d.qam))
        return MPNL_ERR_INVALID_ARG;
    if (d.n_pe < 1 || d.n_pe > MPNL_MAX_NPE || (double)d.n_pe > pow((double)d.qam, (double)d.nt))
        return MPNL_ERR_INVALID_ARG;
    if (!(it.sigma2 > 0.0f) || isinf(it.sigma2)) return MPNL_ERR_INVALID_ARG;
    if (it.flags & ~MPNL_ITEM_FP16) return MPNL_ERR_INVALID_ARG;
    if (it.stages != 0 && it.stages != MPNL_STAGE_DETECT) return MPNL_ERR_INVALID_ARG;
    if (d.n_sc > 0) {
        if (!ptr_ok(it.R, 8, dev, false) || !ptr_ok(it.inv_diag, 4, dev, false) ||
            !ptr_ok(it.perm, 1, dev, false) || !ptr_ok(it.paths, 1, dev, false) ||
            !ptr_ok(it.Z, 8, dev, false) || !ptr_ok(it.hard, 1, dev, false) ||
            !ptr_ok(it.llr, 4, dev, true) || !ptr_ok(it.ped2, 4, dev, true))
            return MPNL_ERR_INVALID_ARG;
    }
    *h = mpnl::BatchItem{};
    h->n_sc = d.n_sc;
    h->n_sym = d.n_sym;
    h->nr = d.nr;
    h->nt = d.nt;
    h->qam = d.qam;
    h->n_pe = d.n_pe;
    h->sigma2 = it.sigma2;
    h->sym = d.nt > 8 ? 1 : 2;  // the built-in symbols per lane of the walk kernel
    h->f16 = (it.flags & MPNL_ITEM_FP16) ? 1 : 0;
    h->R = (float2 *)it.R;
    h->inv_diag = it.inv_diag;
    h->perm = it.perm;
    h->Z = (float2 *)it.Z;
    h->paths = it.paths;
    h->hard = it.hard;
    h->llr = it.llr;
    h->ped2 = it.ped2;
    return MPNL_OK;
}

double unit_cost(const mpnl::BatchItem &u) { return (double)u.n_pe * u.nt * (u.nt + 4) * u.n_sym; }

}  // namespace

extern "C" int mpnl_detect_units_noalloc(const mpnl_batch_item *items, int n_items, void *stream)
{
    if (!items || n_items < 1) return MPNL_ERR_INVALID_ARG;
    if (n_items > kMaxUnits) return MPNL_ERR_UNSUPPORTED;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MPNL_ERR_CUDA;
    }
    DeviceSetup s;
    const int rc = setup_device(dev, &s);
    if (rc != MPNL_OK) return rc;

    // descriptors in schedule order (largest units first), on the stack
    mpnl::BatchItem unit[kMaxUnits];
    mpnl::BatchItem h_items[kMaxUnits];
    int order[kMaxUnits];
    int h_start[kMaxUnits + 1];
    size_t smem = 16;
    for (int i = 0; i < n_items; ++i) {
        const int st = unit_item(items[i], dev, &unit[i]);
        if (st != MPNL_OK) return st;
        smem = std::max(smem, mpnl::detect_smem_bytes(unit[i].nt, unit[i].qam, unit[i].n_pe,
                                                      unit[i].n_sym));
        // insertion into the largest-first order (stable)
        int k = i;
        while (k > 0 && unit_cost(unit[order[k - 1]]) < unit_cost(unit[i])) {
            order[k] = order[k - 1];
            --k;
        }
        order[k] = i;
    }
    if (smem > (size_t)s.smem_optin) return MPNL_ERR_UNSUPPORTED;
    int ctas = 3;
    while (ctas > 1 && (size_t)ctas * smem > (size_t)s.smem_optin) --ctas;
    long long total = 0;
    h_start[0] = 0;
    for (int k = 0; k < n_items; ++k) {
        h_items[k] = unit[order[k]];
        total += h_items[k].n_sc;
        if (total > 0x7fffffffLL) return MPNL_ERR_INVALID_ARG;
        h_start[k + 1] = (int)total;
    }
    if (total == 0) return MPNL_OK;

    cudaStream_t st = (cudaStream_t)stream;
    mpnl::BatchItem *d_items = (mpnl::BatchItem *)(s.scratch + kItemsOff);
    int *d_start = (int *)(s.scratch + kStartOff);
    int *d_counter = (int *)(s.scratch + kCounterOff);
    unsigned *d_status = (unsigned *)(s.scratch + kStatusOff);
    // from pageable (stack) memory: each copy has been staged when it returns
    cudaError_t e = cudaMemcpyAsync(d_items, h_items, sizeof(mpnl::BatchItem) * n_items,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_start, h_start, sizeof(int) * (n_items + 1), cudaMemcpyHostToDevice,
                            st);
    // the work counter and the status word start at zero on every call
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = mpnl::launch_detect_batch(d_items, d_start, n_items, d_counter, d_status, smem,
                                      s.sms * ctas, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MPNL_ERR_CUDA;
    }
    return MPNL_OK;
}
