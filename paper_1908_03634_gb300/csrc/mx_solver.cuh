// Solver plans: device workspace for one geometry and precision, holding the
// FP64 finest-level operator and the multigrid hierarchy of the correction solve.
#pragma once

#include <functional>

#include "mx_df.cuh"
#include "mx_internal.cuh"

template <typename T>
struct Hier {
    int nlev = 0;
    Level<T> lev[MX_MAXLEV];
    T *bot_scratch = nullptr;  // 7 vectors of the coarsest level (BiCGStab)
};

struct MacPlan {
    DGeom g;
    int prec = MX_PREC_MIXED;
    void *mem = nullptr;
    size_t bytes = 0;
    Level<double> L64;  // FP64 path: finest-level coefficients; L64.f = FP64 right-hand side
    Hier<float> H32;    // mixed: the FP32 correction hierarchy
    DFArrays D;         // mixed: double-float phi, h^2 f and coefficient lo parts
    Hier<double> H64;   // FP64: the FP64 correction hierarchy (level 0 shares L64's coefficients)
    FaceQ Q;            // correction factors 2/(h (rho_L + rho_R)) of the finest faces
    float *tmp32 = nullptr;
    // FCG (mx_opts::krylov): two direction buffers and q = h^2 L p, allocated on first use
    float *kry_mem = nullptr;
    float *kp0 = nullptr, *kp1 = nullptr, *kq = nullptr;
    // CUDA graph of the refinement loop, keyed by the pointers it was captured with
    cudaGraphExec_t graph = nullptr;
    const void *graph_phi = nullptr;
    int graph_nu1 = -1, graph_nu2 = -1, graph_bot = -1, graph_fused = -1, graph_tilez = -1, graph_krylov = -1;
    long long last_use = 0;
};

MacPlan *get_mac_plan(mx_ctx *c, const DGeom &g, int prec, mx_status *st);
MacPlan *create_mac_plan(mx_ctx *c, const DGeom &g, int prec, mx_status *st);
void free_mac_plan(MacPlan *p);
void setup_coefficients(mx_ctx *c, MacPlan &P, const double *rho, const double *beta0);
void setup_coefficients_on(cudaStream_t s, MacPlan &P, const double *rho, const double *beta0);
mx_status check_opts(mx_ctx *c, const mx_opts *in, mx_opts &o);
template <typename T>
int coarse_start(const Hier<T> &H);
void destroy_plans(mx_ctx *c);
mx_status ensure_partials(mx_ctx *c, long long nblocks);

// Capture body(stream) as the body of a conditional-while graph node and
// instantiate it: one launch then runs body while SolveState::done is 0 (the
// last kernel of each iteration sets the loop condition from it).
mx_status capture_while_graph(mx_ctx *c, cudaGraphExec_t *exec, const std::function<void(cudaStream_t)> &body);

template <typename T>
void vcycle(cudaStream_t s, Hier<T> &H, int nu1, int nu2, int bot_iters, int singular, mx_ctx *prof = nullptr,
            int fused = 0, int zcap = 8);
