// Flexible conjugate gradients FCG(1) around the FP32 V-cycle (mx_krylov.cu).
#pragma once

#include "mx_internal.cuh"

// beta of this iteration from e . q_prev (two launches: dot product, finalize)
void k_kry_dot(cudaStream_t s, long long n, const float *e, const float *q, SolveState *st, double *partials);
// p = e + beta p_prev into p0 (even V-cycle count) or p1 (odd), q = h^2 L p, and
// the line-search step into SolveState::upd (two launches)
void k_kry_dir(cudaStream_t s, const Level<float> &L0, const float *e, float *p0, float *p1, float *q,
               SolveState *st, double *partials);
// reduction partials the direction kernel writes (one triple per tile)
int kry_dir_blocks(const DGeom &g);
