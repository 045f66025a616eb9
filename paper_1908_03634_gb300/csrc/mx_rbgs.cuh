// Single-pass red-black Gauss-Seidel sweep and the per-cell update it shares
// with the two-pass colour kernels.
#pragma once

#include "mx_internal.cuh"

enum { RB_PLAIN = 0, RB_ZERO = 1, RB_PROLONG = 2 };

// Rounded arithmetic without contraction: every kernel that updates a cell
// (two-pass colour passes, the single-pass sweep, the batched and coarse-end
// kernels) evaluates the update with exactly these operations, so they agree
// bit for bit whatever FMA contractions the compiler would choose in each.
// The FP32 update divides with the reciprocal-based fast division (within 2 ulp
// for denominators below 2^126, far above any face-coefficient sum here): the
// smoother only sets the V-cycle's contraction, the refinement loop the accuracy.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }

// Exact solve of cell c's row: e_c = (sum_f b_f e_nb - h^2 f_c) / sum_f b_f.
template <typename T>
__device__ __forceinline__ T gs_update(const T b[6], const T v[6], T f, T h2) {
    T num = rmul(b[0], v[0]);
    num = rfma(b[1], v[1], num);
    num = rfma(b[2], v[2], num);
    num = rfma(b[3], v[3], num);
    num = rfma(b[4], v[4], num);
    num = rfma(b[5], v[5], num);
    num = rfma(-h2, f, num);
    const T den = radd(radd(radd(b[0], b[1]), radd(b[2], b[3])), radd(b[4], b[5]));
    return rdiv(num, den);
}

// Whether the single-pass sweep supports this level (n_x even, periodic extents >= 2).
bool rbgs_fused_ok(const DGeom &g);

// e_out = one red+black sweep applied to e_in (mode RB_ZERO: e_in = 0;
// RB_PROLONG: e_in + piecewise-constant prolongation of coarse->e).
void k_rbgs_fused(cudaStream_t s, const Level<float> &L, const float *ein, float *eout, int mode,
                  const Level<float> *coarse);
