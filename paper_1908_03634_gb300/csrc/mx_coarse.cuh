// Single-CTA coarse end of the V-cycle (all levels of <= COARSE_MAX_CELLS cells).
#pragma once

#include "mx_internal.cuh"

#define COARSE_MAX_LEVELS 8
#define COARSE_MAX_CELLS 4096
#define COARSE_MAX_SMEM (160 * 1024)

// true if levels [0, nl) of `levs` (the last one the bottom) fit the kernel
template <typename T>
bool coarse_fits(const Level<T> *levs, int nl);

// V-cycle on levs[0..nl): reads levs[0].f, writes levs[0].e (global memory)
template <typename T>
void k_coarse_vcycle(cudaStream_t s, const Level<T> *levs, int nl, int nu1, int nu2, int bot_iters, int singular);

cudaError_t coarse_init();

// batched coarse ends: argument blocks for one box each (host fills, device reads)
size_t coarse_args_bytes();
void coarse_fill_args(void *dst, const Level<float> *levs, int nl, int nu1, int nu2, int bot_iters, int singular);
size_t coarse_smem_bytes_f(const Level<float> *levs, int nl);
void k_coarse_vcycle_batch(cudaStream_t s, const void *dev_args, const SolveState *st, int nbox, size_t smem);
