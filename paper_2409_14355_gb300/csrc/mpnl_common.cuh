// Shared device helpers of the MPNL CUDA path: constellation geometry, limits,
// small complex helpers.  Written for sm_103a (GB300); nothing here is shared
// with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpnl {

constexpr int kMaxNt = 16;
constexpr int kMaxNr = 32;
constexpr int kMaxNsym = 32;
constexpr int kMaxNpe = 1024;
constexpr float kLlrMax = 20.0f;
constexpr float kPeFloor = 1e-12f;
constexpr unsigned kInfBits = 0x7f800000u;  // bit pattern of +inf (float)

// Square M-QAM of TS 38.211 §5.1.3-5.1.5 viewed as two Gray-labelled PAM
// axes.  Along an axis, grid index i = 0..L-1 sits at (2i - (L-1)) * kInvScale
// (most negative first).  The real axis carries bits b0, b2, b4 and the
// imaginary axis b1, b3, b5; the per-axis label is those bits read as an
// integer (first bit most significant).  kAxisLabel[i] is the label at grid
// index i, derived from the standard's mapping formulas:
//   QPSK : x = (1 - 2 b0)                                  -> {1, 0}
//   16QAM: x = (1 - 2 b0)(2 - (1 - 2 b2))                  -> {3, 2, 0, 1}
//   64QAM: x = (1 - 2 b0)(4 - (1 - 2 b2)(2 - (1 - 2 b4)))   -> {7, 6, 4, 5, 1, 0, 2, 3}
template <int QAM>
struct Qam;

template <>
struct Qam<4> {
    static constexpr int L = 2, B = 2;
    static constexpr float kInvScale = 0.70710678118654752f;  // 1/sqrt(2)
    static constexpr float kScale = 1.41421356237309505f;
    __device__ static int axis_label(int i) { return 1 - i; }
};

template <>
struct Qam<16> {
    static constexpr int L = 4, B = 4;
    static constexpr float kInvScale = 0.31622776601683794f;  // 1/sqrt(10)
    static constexpr float kScale = 3.16227766016837933f;
    __device__ static int axis_label(int i) { return (0x1023 >> (4 * i)) & 0xF; }  // {3,2,0,1}
};

template <>
struct Qam<64> {
    static constexpr int L = 8, B = 6;
    static constexpr float kInvScale = 0.15430334996209191f;  // 1/sqrt(42)
    static constexpr float kScale = 6.48074069840786023f;
    __device__ static int axis_label(int i) { return (0x32015467 >> (4 * i)) & 0xF; }  // {7,6,4,5,1,0,2,3}
};

// Coordinate of grid index i along an axis.
template <int QAM>
__device__ __forceinline__ float axis_pos(int i)
{
    return (float)(2 * i - (Qam<QAM>::L - 1)) * Qam<QAM>::kInvScale;
}

// 2-D label from the two axis labels: the real-axis bits go to b0, b2, ...
// and the imaginary-axis bits to b1, b3, ... (b0 is the label's MSB).
template <int QAM>
__device__ __forceinline__ int join_label(int lre, int lim)
{
    constexpr int H = Qam<QAM>::B / 2;
    int lab = 0;
#pragma unroll
    for (int t = 0; t < H; ++t) {
        int rb = (lre >> (H - 1 - t)) & 1;
        int ib = (lim >> (H - 1 - t)) & 1;
        lab = (lab << 2) | (rb << 1) | ib;
    }
    return lab;
}

// Nearest grid index along one axis to coordinate x, exact for the float
// distances: the nearest point is one of the two grid points around x (or
// the clamped end); an exact distance tie goes to the smaller axis label.
template <int QAM>
__device__ __forceinline__ int axis_nearest(float x, float &dist)
{
    constexpr int L = Qam<QAM>::L;
    float f = (x * Qam<QAM>::kScale + (float)(L - 1)) * 0.5f;
    int ia = (int)floorf(f);
    ia = ia < 0 ? 0 : (ia > L - 1 ? L - 1 : ia);
    int ib = ia + 1 < L ? ia + 1 : L - 1;
    float da = x - axis_pos<QAM>(ia);
    float db = x - axis_pos<QAM>(ib);
    da *= da;
    db *= db;
    bool take_b = db < da || (db == da && Qam<QAM>::axis_label(ib) < Qam<QAM>::axis_label(ia));
    dist = take_b ? db : da;
    return take_b ? ib : ia;
}

__device__ __forceinline__ unsigned fbits(float x) { return __float_as_uint(x); }

// Opt a kernel in to `dyn` bytes of dynamic shared memory when its static
// plus dynamic shared memory exceeds the 48 KB available without opt-in.
template <typename Kernel>
inline cudaError_t allow_dynamic_smem(Kernel kernel, size_t dyn)
{
    if (dyn <= 32 * 1024) return cudaSuccess;  // every kernel here has < 16 KB static
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    if (dyn + a.sharedSizeBytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

}  // namespace mpnl
