// z = Q^H y on the tensor cores with FP16 operands and FP32 accumulation
// (mpnl_qhy_mixed): the Q^H y of the mixed-precision path, from a stored Q.
//
// Per subcarrier the 14 symbols share one Q, so z = Q^H y for all of them is
// one small real GEMM: with A = [Re y | Im y] (n_sym x 2nr) and
//   W = [[Re Q, -Im Q], [Im Q, Re Q]]  (2nr x 2nt),
// A W = [Re z | Im z], since Re z_j = sum_i Re y_i Re Q_ij + Im y_i Im Q_ij and
// Im z_j = sum_i Im y_i Re Q_ij - Re y_i Im Q_ij.  A warp stages A and W in
// shared memory as FP16 (zero padding to the 16 x 8 x 16 tile), runs
// mma.sync m16n8k16 (f16 inputs, f32 accumulators) over the tiles, and
// writes z in FP32.  The operation is bandwidth-bound (Q and y are read
// once); the tensor-core form keeps the arithmetic off the FP32 pipe that
// the walks use when both run at once.
#pragma once
#include <cuda_fp16.h>

#include "mpnl_common.cuh"

namespace mpnl {
namespace {

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct QmLayout {
    int MP, KP, NP, off_b, off_c, bytes;
};

// Per-warp shared memory: A [MP][KP] and W^T [NP][KP] in FP16, the result
// [MP][NP] in FP32.
__host__ __device__ inline QmLayout qm_layout(int n_sym, int nr, int nt)
{
    QmLayout L;
    L.MP = round_up(n_sym, 16);
    L.KP = round_up(2 * nr, 16);
    L.NP = round_up(2 * nt, 8);
    L.off_b = round_up(L.MP * L.KP * 2, 16);
    L.off_c = L.off_b + round_up(L.NP * L.KP * 2, 16);
    L.bytes = L.off_c + round_up(L.MP * L.NP * 4, 16);
    return L;
}

__device__ __forceinline__ void mma_16816(float (&c)[4], const unsigned (&a)[4],
                                          const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned ld_pair(const __half *p)
{
    return *reinterpret_cast<const unsigned *>(p);
}

// One subcarrier by one warp, in its shared-memory region at byte offset
// base_off (at least qm_layout(...).bytes).
__device__ __forceinline__ void qhy_mma_warp(int sc, int n_sym, int nr, int nt,
                                             const float2 *__restrict__ Q,
                                             const float2 *__restrict__ Y,
                                             float2 *__restrict__ Z, int base_off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const QmLayout S = qm_layout(n_sym, nr, nt);
    unsigned char *base = smem_raw + base_off;
    __half *As = reinterpret_cast<__half *>(base);
    __half *Bt = reinterpret_cast<__half *>(base + S.off_b);
    float *Cs = reinterpret_cast<float *>(base + S.off_c);
    const int MP = S.MP, KP = S.KP, NP = S.NP;

    // y is scaled by the power of two 2^-x that brings its largest component
    // into [0.5, 1) (exact; FP16's range is +-65504 with subnormals below
    // 2^-14, a caller's y may sit at any scale) and z by 2^x at the end.
    // Q needs none: its columns are orthonormal, every entry within 1.
    const float2 *y = Y + (size_t)sc * n_sym * nr;
    unsigned mx = 0u;
    for (int e = lane; e < n_sym * nr; e += 32) {
        const float2 t = y[e];
        mx = max(mx, max(__float_as_uint(fabsf(t.x)), __float_as_uint(fabsf(t.y))));
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    float ys = 1.f, yu = 1.f;
    {
        const float m = __uint_as_float(mx);
        if (m > 0.f && m < INFINITY) {  // finite and nonzero (NaN bits compare above inf)
            int x;
            frexpf(m, &x);
            x = min(max(x, -100), 100);
            ys = ldexpf(1.f, -x);
            yu = ldexpf(1.f, x);
        }
    }
    // A[m][k]: k < nr the real part of y_k, nr <= k < 2nr the imaginary part
    for (int e = lane; e < MP * KP; e += 32) {
        const int m = e / KP, k = e - m * KP;
        float v = 0.f;
        if (m < n_sym && k < 2 * nr) {
            const float2 t = y[(size_t)m * nr + (k < nr ? k : k - nr)];
            v = (k < nr ? t.x : t.y) * ys;
        }
        As[e] = __float2half_rn(v);
    }
    // W^T[n][k] = W[k][n]: rows k < nr carry (Re Q, -Im Q), rows nr + i
    // carry (Im Q, Re Q)
    const float2 *q = Q + (size_t)sc * nr * nt;
    for (int e = lane; e < NP * KP; e += 32) {
        const int n = e / KP, k = e - n * KP;
        float v = 0.f;
        if (n < 2 * nt && k < 2 * nr) {
            const int i = k < nr ? k : k - nr, j = n < nt ? n : n - nt;
            const float2 t = q[(size_t)i * nt + j];
            if (k < nr) v = n < nt ? t.x : -t.y;
            else v = n < nt ? t.y : t.x;
        }
        Bt[e] = __float2half_rn(v);
    }
    __syncwarp();

    const int g = lane >> 2, t2 = 2 * (lane & 3);
    for (int m0 = 0; m0 < MP; m0 += 16) {
        for (int n0 = 0; n0 < NP; n0 += 8) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k0 = 0; k0 < KP; k0 += 16) {
                unsigned a[4], b[2];
                a[0] = ld_pair(As + (m0 + g) * KP + k0 + t2);
                a[1] = ld_pair(As + (m0 + g + 8) * KP + k0 + t2);
                a[2] = ld_pair(As + (m0 + g) * KP + k0 + t2 + 8);
                a[3] = ld_pair(As + (m0 + g + 8) * KP + k0 + t2 + 8);
                b[0] = ld_pair(Bt + (n0 + g) * KP + k0 + t2);
                b[1] = ld_pair(Bt + (n0 + g) * KP + k0 + t2 + 8);
                mma_16816(c, a, b);
            }
            Cs[(m0 + g) * NP + n0 + t2] = c[0];
            Cs[(m0 + g) * NP + n0 + t2 + 1] = c[1];
            Cs[(m0 + g + 8) * NP + n0 + t2] = c[2];
            Cs[(m0 + g + 8) * NP + n0 + t2 + 1] = c[3];
        }
    }
    __syncwarp();
    float2 *z = Z + (size_t)sc * n_sym * nt;
    for (int e = lane; e < n_sym * nt; e += 32) {
        const int m = e / nt, j = e - m * nt;
        z[e] = make_float2(Cs[m * NP + j] * yu, Cs[m * NP + nt + j] * yu);
    }
    __syncwarp();  // the region may be reused for the warp's next subcarrier
}

}  // namespace
}  // namespace mpnl
