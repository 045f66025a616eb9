// Single-pass red-black Gauss-Seidel sweep and the per-cell update it shares
// with the two-pass colour kernels.
#pragma once

#include "mx_internal.cuh"

enum { RB_PLAIN = 0, RB_ZERO = 1, RB_PROLONG = 2 };

// Exact solve of cell c's row: e_c = (sum_f b_f e_nb - h^2 f_c) / sum_f b_f.
template <typename T>
__device__ __forceinline__ T gs_update(const T b[6], const T v[6], T f, T h2) {
    T num = b[0] * v[0];
    num += b[1] * v[1];
    num += b[2] * v[2];
    num += b[3] * v[3];
    num += b[4] * v[4];
    num += b[5] * v[5];
    num -= h2 * f;
    const T den = ((b[0] + b[1]) + (b[2] + b[3])) + (b[4] + b[5]);
    return num / den;
}

// Whether the single-pass sweep supports this level (n_x even, periodic extents >= 2).
bool rbgs_fused_ok(const DGeom &g);

// e_out = one red+black sweep applied to e_in (mode RB_ZERO: e_in = 0;
// RB_PROLONG: e_in + piecewise-constant prolongation of coarse->e).
void k_rbgs_fused(cudaStream_t s, const Level<float> &L, const float *ein, float *eout, int mode,
                  const Level<float> *coarse);
