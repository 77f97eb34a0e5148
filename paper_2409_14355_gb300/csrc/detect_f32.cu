// Walk kernels of the FP32 path: every (NT, QAM, symbols-per-lane)
// instance, compiled in a translation unit of its own so that the instances
// of the two precisions build in parallel.
#include "detect_impl.cuh"

namespace mpnl {
cudaError_t launch_detect_f32(int n_sc, const DetArgs &a, int qam, int sym, cudaStream_t stream)
{
    return launch_prec<false>(n_sc, a, qam, sym, stream);
}

}  // namespace mpnl
