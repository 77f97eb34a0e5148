// Persistent walk kernel of mixed-size batches (mpnl_batch_*), in a
// translation unit of its own: it calls every per-subcarrier instance of
// both precisions as a separate (not inlined) function, so that each keeps
// its own register allocation.  Its arithmetic is that of the per-call
// kernels (no contraction, see the build flags): a unit's results alone and
// in a batch agree bit for bit.
#include "detect_impl.cuh"

namespace mpnl {
namespace {

// Persistent walk kernel over a batch of radio units of mixed sizes: every
// CTA takes (unit, subcarrier) work items from a global counter and runs the
// instance that fits the unit (NT class, QAM, precision, symbols per lane).
template <int NT, int QAM, bool F16>
__device__ __forceinline__ void detect_item_sym(const DetArgs &a, int sym, int sc)
{
    if (sym == 1) detect_sc<NT, QAM, F16, 1>(a, sc);
    else detect_sc<NT, QAM, F16, 2>(a, sc);
}

template <int NT, bool F16>
__device__ __forceinline__ void detect_item_qam(const DetArgs &a, int qam, int sym, int sc)
{
    switch (qam) {
    case 4: detect_item_sym<NT, 4, F16>(a, sym, sc); break;
    case 16: detect_item_sym<NT, 16, F16>(a, sym, sc); break;
    default: detect_item_sym<NT, 64, F16>(a, sym, sc); break;
    }
}

template <bool F16>
__device__ __forceinline__ void detect_item(const DetArgs &a, int nt, int qam, int sym, int sc)
{
    if (nt <= 4) detect_item_qam<4, F16>(a, qam, sym, sc);
    else if (nt <= 8) detect_item_qam<8, F16>(a, qam, sym, sc);
    else detect_item_qam<16, F16>(a, qam, sym, sc);
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
detect_batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ start,
                    int n_items, int *__restrict__ counter, unsigned *__restrict__ status)
{
    __shared__ int s_w;
    const int total = start[n_items];
    for (;;) {
        if (threadIdx.x == 0) s_w = atomicAdd(counter, 1);
        __syncthreads();
        const int w = s_w;
        __syncthreads();  // every thread has read the item before the next fetch
        if (w >= total) break;
        const int i = find_item(start, n_items, w);
        const BatchItem &it = items[i];
        const int sc = w - start[i];
        const DetArgs a{it.n_sym, it.nt,    it.n_pe, it.sigma2, it.R,   it.inv_diag, it.perm,
                        it.paths, it.Z,     it.hard, it.llr,    it.ped2, status};
        if (it.f16) detect_item<true>(a, it.nt, it.qam, it.sym, sc);
        else detect_item<false>(a, it.nt, it.qam, it.sym, sc);
        __syncthreads();  // shared memory is reused by the next item
    }
}

}  // namespace

cudaError_t launch_detect_batch(const BatchItem *items, const int *start, int n_items,
                                int *counter, unsigned *status, size_t smem, int grid,
                                cudaStream_t stream)
{
    cudaError_t e = allow_dynamic_smem(detect_batch_kernel, smem);
    if (e != cudaSuccess) return e;
    detect_batch_kernel<<<grid, kThreads, smem, stream>>>(items, start, n_items, counter, status);
    return cudaGetLastError();
}

}  // namespace mpnl
