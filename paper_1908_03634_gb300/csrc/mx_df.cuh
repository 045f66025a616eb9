// Double-float (hi + lo float pairs) storage of the refinement loop's
// high-precision quantities; the hi parts of the coefficients are the FP32
// finest-level coefficients of the V-cycle.
#pragma once

#include "mx_dfmath.cuh"
#include "mx_internal.cuh"

struct DFArrays {
    float *bxl, *byl, *bzl;  // lo parts of the lo-face coefficients
    float *hxl, *hyl, *hzl;  // lo parts of the high-boundary planes
    float *fh, *fl;          // h^2 f
    float *ph, *pl;          // phi, buffer 0
    float *ph2, *pl2;        // phi, buffer 1 (the buffers alternate with the V-cycle count)
    float *b0h, *b0l;        // beta0 at the cell centres, split once by the coefficient pass
};

void k_mac_coeffs_df(cudaStream_t s, const Level<float> &L0, const DFArrays &D, const double *rho, const double *beta0,
                     const FaceQ *q = nullptr);
// f = D(beta0 U) - beta0 Sbar in double-float into (D.fh, D.fl), with per-block
// partials (max |f|, sum f^2, sum f) on the stencil grid
// (beta0 comes split from (D.b0h, D.b0l): k_mac_coeffs_df of the same plan must run first)
void k_mac_rhs_df(cudaStream_t s, const DGeom &g, const double *ux, const double *uy, const double *uz,
                  const double *sbar, const DFArrays &D, double *partials);
// (D.fh, D.fl) <- h^2 (f - mean), partials of f - mean on nb grid-stride blocks
void k_sub_mean_scale(cudaStream_t s, const DGeom &g, const SolveState *st, const DFArrays &D, double *partials,
                      int nb);
// partials (max |D(beta0 U) - beta0 Sbar - mean|, 0, 0) on the stencil grid
void k_mac_divcheck_df(cudaStream_t s, const DGeom &g, const double *ux, const double *uy, const double *uz,
                       const double *sbar, const DFArrays &D, const SolveState *st, double *partials);
void k_df_from_double(cudaStream_t s, long long n, const double *x, const DFArrays &D);
void k_df_to_double(cudaStream_t s, long long n, const DFArrays &D, double *x);
void k_df_update(cudaStream_t s, const DGeom &g, const DFArrays &D, const float *e, const SolveState *st);
// r = f - L phi (e == nullptr: phi in buffer iter&1) or, with e, phi_new = phi +
// step e (step = SolveState::upd; phi read from buffer (iter-1)&1, written to
// buffer iter&1) and its residual.  e_odd (optional): the direction to use
// instead of e when iter is odd.
// Returns the number of partial triples written (one per block).
int k_df_resid(cudaStream_t s, const Level<float> &L0, const DFArrays &D, const float *e, const SolveState *st,
               double *partials, const float *e_odd = nullptr);
// the number of partial triples k_df_resid writes for geometry g
int df_resid_parts(const DGeom &g);
int df_resid_blocks(const DGeom &g);
// the residual of phi = 0 (r = f), bit-identical to k_df_resid's there, without the stencil
void k_df_resid_zero(cudaStream_t s, const Level<float> &L0, const DFArrays &D, const SolveState *st, double *partials);
dim3 df_resid_grid(const DGeom &g);

// one box of the batched refinement loop
struct DFBox {
    Level<float> L0;  // finest FP32 level (L0.e: the V-cycle correction, L0.f: rhat)
    DFArrays D;
    int part_off;     // first reduction partial of the box
    int zc;           // z-chunk of the box's march grid (march work lists)
};
// the first residual of every box from phi = 0 over the batched residual's work list
// (cnt: entries per box), bit for bit the stencil kernels' rhat, norms in their slots
void k_df_resid_zero_batch(cudaStream_t s, const DFBox *boxes, const int4 *work, int nwork, const int *cnt,
                           const SolveState *st, double *partials);
// the batched residual over a work list of df_resid_batch_grid entries: the
// z-march (march = 1: element staging, 2: 16-byte row chunks; the smallest
// df_march_usable over the boxes) or the 3D-tile kernel (march = 0)
void k_df_resid_batch(cudaStream_t s, const DFBox *boxes, const int4 *work, int nwork, const SolveState *st,
                      double *partials, int update, int march);
dim3 df_resid_batch_grid(const DGeom &g, int march, int *zc);
int df_march_usable(const DGeom &g);
// phi (double) from the current double-float buffer; partials (may be null):
// per-block (0, sum phi, 0) on red_blocks(n) blocks
void k_df_final(cudaStream_t s, long long n, const DFArrays &D, const SolveState *st, double *x,
                double *partials = nullptr);
