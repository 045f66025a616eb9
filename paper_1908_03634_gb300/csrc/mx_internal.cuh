// Internal declarations of the mx projection library (GB300, sm_103a).
//
// Data layout on the device (all levels, both precisions):
//   cell arrays: x fastest, c = i + nx*(j + ny*k);
//   face coefficients in "lo-face" form: bx[c] is the coefficient of the face
//   on the low-x side of cell c (so face i of the API layout), by, bz alike;
//   the faces on the high side of the box are either periodic images (face 0),
//   walls (coefficient 0) or Dirichlet faces, whose coefficients live in the
//   boundary planes hx (ny*nz), hy (nx*nz), hz (nx*ny).
//   Stored coefficients are "effective": a wall face holds 0 and a Dirichlet
//   face holds 2 beta0/rho of its interior cell, so that every face enters the
//   operator as b_f (phi_nb - phi_c) with phi_nb = 0 outside the box.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "mx.h"

#define MX_MAXLEV 24

struct DGeom {
    int n[3];
    long long nxy, N;
    double h;
    int lo[3], hi[3];
};

__host__ __device__ inline bool gper(const DGeom &g, int d) { return g.lo[d] == MX_BC_PERIODIC; }

template <typename T>
struct Level {
    DGeom g;
    T *bx, *by, *bz;  // lo-face coefficients, one per cell
    T *hx, *hy, *hz;  // high-boundary face coefficients (non-periodic axes)
    T *f, *e;         // right-hand side and correction
    T *e2;            // second correction buffer (single-pass sweeps write e2 <-> e)
};

// Device-resident state of one solve (norms, control flags).
struct SolveState {
    double fnorm, fnorm2, fsum;  // ||f||_inf, ||f||_2, sum f (after mean removal)
    double mean;                 // removed RHS mean
    double rnorm, rnorm2, rsum;  // last residual norms
    double scale, inv_scale;     // r is handed to the correction solve as r / scale
    float scale_h, scale_l;      // scale as a double-float pair, and 1/scale as a float,
    float inv_scale_f;           // for kernels that do no FP64 arithmetic
    float upd_h, upd_l;          // step of the double-float update phi += step e: the scale
                                 // (refinement) or the line-search step (FCG)
    double kry_beta;             // FCG: conjugation coefficient of this iteration
    double kry_pq;               // FCG: p . (h^2 L p) of the previous direction
    int kry_restart;             // FCG: 1 = no previous direction (p = e)
    double best;                 // smallest residual seen
    double tol;                  // relative tolerance
    double div_err;              // divergence check of the projected velocity
    double aux;                  // scratch scalar (mean of phi, ...)
    int iter;                    // V-cycles done
    int maxit;                   // V-cycle cap
    int done;                    // 1: leave the refinement loop
    int status;                  // mx_status
};

// set the refinement scale (and its float forms)
__device__ __forceinline__ void set_scale(SolveState *st, double sc) {
    st->scale = sc;
    st->inv_scale = 1.0 / sc;
    st->scale_h = __double2float_rn(sc);
    st->scale_l = __double2float_rn(sc - double(st->scale_h));
    st->inv_scale_f = __double2float_rn(st->inv_scale);
    st->upd_h = st->scale_h;
    st->upd_l = st->scale_l;
}

// Maxima that propagate NaN.  fmax/fmaxf return the other operand when one is
// NaN, so a norm built from them would report a finite value for a residual
// holding NaN; every norm and its block and grid reductions use these instead.
__device__ __forceinline__ double nmax(double a, double b) { return (a > b || a != a) ? a : b; }
__device__ __forceinline__ float nmaxf(float a, float b) {
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// Programmatic dependent launch.  The V-cycle's kernels are launched with
// launch_pdl: the next kernel of the stream may be scheduled while the current
// one drains (its blocks become resident once every block of the current one
// has called pdl_trigger), and waits in pdl_wait -- its first statement -- until
// the current kernel has finished and its writes are visible.  Results are
// those of plain stream order; the launch gaps between the short kernels of the
// coarse levels shrink.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

struct MacPlan;
struct NodalPlan;
struct BatchPlan;
struct RadialPlan;

struct mx_ctx {
    int device;
    cudaStream_t stream;
    std::string err;
    SolveState *state = nullptr;  // device
    SolveState *hstate = nullptr; // pinned host mirror
    double *partials = nullptr;   // device reduction scratch (3 doubles per block)
    int max_partials = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // tune cache (mx_autotune): the fastest setting per operator, precision and geometry
    struct Tune { int op, prec, n[3], lo[3], hi[3], nu1, nu2, fused, tile_z, smoother; double ms; };
    std::vector<Tune> tune;
    std::vector<MacPlan *> plans;        // cached workspaces, one per geometry/precision
    std::vector<NodalPlan *> nplans;
    BatchPlan *batch = nullptr;
    std::vector<RadialPlan *> rplans;    // lateral average / fill plans, one per (n, corner)
    void *base_tmp = nullptr;            // planar-average partial sums
    void *base_flag = nullptr;           // averages: a value outside the fast passes' window
    size_t base_tmp_bytes = 0;
    void *split_tab = nullptr;           // velocity split: per-radius face factors
    size_t split_tab_bytes = 0;
    void *split_cells = nullptr;         // velocity split: the S - Sbar bracket
    size_t split_cells_bytes = 0;
    void *comp = nullptr;                // composite projection: the last geometry's plans and graph
    long long use_counter = 0;
    // tracing (mx_profile_enable)
    bool prof = false;
    double prof_ms[MX_PH_COUNT] = {};
    long long prof_n[MX_PH_COUNT] = {};
    struct Mark { int phase; cudaEvent_t a, b; int n; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> ev_pool;
};

// nu1 = nu2 = 0 in o: replace nu1, nu2, fused, tile_z by the tune cache's
// entry for (op, o.prec, geometry), or nu1 = nu2 = 2 when there is none.
void tune_apply(const mx_ctx *c, int op, const mx_geom *g, mx_opts &o);
// the same for a batch (nu1, nu2 only), keyed by its boxes' geometries
void tune_apply_batch(const mx_ctx *c, int nbox, const mx_geom *geoms, mx_opts &o);

// out = S - Sbar (the velocity split's bracket; mx_base.cu)
mx_status base_subtract_average(mx_ctx *c, const mx_geom *geom, int spherical, const int corner[3], const double *S,
                                double *out);

// phase markers: no-ops unless tracing is on and the stream is not capturing
void prof_begin(mx_ctx *c, cudaStream_t s, int phase);
void prof_end(mx_ctx *c, cudaStream_t s, int phase, int nlaunch);
void prof_flush(mx_ctx *c);

// ---- error helpers --------------------------------------------------------------
mx_status set_err(mx_ctx *ctx, mx_status s, const std::string &msg);
#define MX_CUDA(ctx, call)                                                                     \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return set_err(ctx, MX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ---- workspace: bump allocator over one cudaMalloc (dry run with base = nullptr) -------
struct Bump {
    char *base;
    size_t off;
    template <typename T>
    T *take(size_t n) {
        size_t a = (off + 255) & ~size_t(255);
        off = a + n * sizeof(T);
        return base ? reinterpret_cast<T *>(base + a) : nullptr;
    }
};

// ---- geometry --------------------------------------------------------------------
DGeom make_dgeom(const mx_geom *g);
mx_status check_geom(mx_ctx *ctx, const mx_geom *g, bool nodal);
bool geom_singular(const DGeom &g);

// number of levels and the level geometries of the cell-centred hierarchy
int mac_levels(const DGeom &g0, DGeom *out);

// ---- reductions -------------------------------------------------------------------
constexpr int RED_THREADS = 256;
int red_blocks(long long n);

// ---- kernels, launched from host helpers ------------------------------------------
// MAC (FP64) pieces
void k_fill(cudaStream_t s, const DGeom &g, int spherical, const double *prof, int nr, double dr,
            double cx, double cy, double cz, double *out);
// Correction factors q_f = 2/(h (rho_L + rho_R)) of the MAC faces (a Dirichlet
// face: 2/(h rho) of the interior cell), in the coefficients' lo-face layout
// with the high-boundary planes; written by the coefficient kernels.
struct FaceQ {
    double *x = nullptr, *y = nullptr, *z = nullptr, *hx = nullptr, *hy = nullptr, *hz = nullptr;
};
void k_mac_coeffs64(cudaStream_t s, const Level<double> &L, const double *rho, const double *beta0,
                    const FaceQ *q = nullptr);
void k_mac_rhs(cudaStream_t s, const DGeom &g, const double *ux, const double *uy, const double *uz,
               const double *beta0, const double *sbar, double *f, double *partials, int nb);
void k_sub_mean_norm(cudaStream_t s, const DGeom &g, double *f, const SolveState *st, double *partials, int nb);
void k_finalize_rhs(cudaStream_t s, const double *partials, int nb, SolveState *st, long long N, int remove_mean,
                    int stage);
void k_mac_correct(cudaStream_t s, const DGeom &g, const FaceQ &q, const double *phi, double *ux, double *uy,
                   double *uz);
void k_mac_divcheck(cudaStream_t s, const DGeom &g, const double *ux, const double *uy, const double *uz,
                    const double *beta0, const double *sbar, const SolveState *st, double *partials, int nb);
void k_finalize_max(cudaStream_t s, const double *partials, int nb, double *dst);

// generic multigrid pieces (templated on the V-cycle precision)
template <typename T>
void k_coarsen_coeffs(cudaStream_t s, const Level<T> &fine, const Level<T> &coarse);
void k_round_coeffs(cudaStream_t s, const Level<double> &src, const Level<float> &dst);
template <typename T>
void k_residual64(cudaStream_t s, const Level<double> &L64, const double *phi, const double *f, T *rhat,
                  const SolveState *st, double *partials, int nb);
void k_finalize_residual(cudaStream_t s, const double *partials, int nb, SolveState *st, int scaled = 0);
template <typename T>
void k_update(cudaStream_t s, const DGeom &g, double *phi, const T *e, const SolveState *st);
template <typename T>
void k_rbgs(cudaStream_t s, const Level<T> &L, int colour, int zero = 0, int zcap = 8);
dim3 rbgs_grid(const DGeom &g, int zc);
// batched multigrid phases over a work list of (box, bx, by, bz)
void k_rbgs_batch(cudaStream_t s, const Level<float> *levs, const int4 *work, int nwork, const SolveState *st,
                  int level, int colour, int zero);
// zcf > 0: the fine-cell form, work entries are tiles of resid_restrict_fine_grid(level's
// geometry, zcf) (every box's level has even extents); 0: tiles of the coarse level
void k_resid_restrict_batch(cudaStream_t s, const Level<float> *levs, const int4 *work, int nwork,
                            const SolveState *st, int level, int zcf);
dim3 resid_restrict_fine_grid(const DGeom &fine, int zcf);
void k_prolong_batch(cudaStream_t s, const Level<float> *levs, const int4 *work, int nwork, const SolveState *st,
                     int level);
void k_finalize_residual_batch(cudaStream_t s, const double *partials, const int *off, const int *cnt, SolveState *st,
                               int nbox);
template <typename T>
void k_resid_restrict(cudaStream_t s, const Level<T> &fine, const Level<T> &coarse, int zcap = 8);
template <typename T>
void k_prolong(cudaStream_t s, const Level<T> &coarse, const Level<T> &fine, int zcap = 8);
template <typename T>
void k_bottom(cudaStream_t s, const Level<T> &L, T *scratch, int iters, int singular);
template <typename T>
void k_apply(cudaStream_t s, const Level<T> &L, const T *phi, T *out);
template <typename T>
void k_cast(cudaStream_t s, long long n, const double *src, T *dst);
template <typename T>
void k_uncast(cudaStream_t s, long long n, const T *src, double *dst);
void k_sum_partials(cudaStream_t s, const DGeom &g, const double *x, double *partials, int nb);
void k_finalize_sum(cudaStream_t s, const double *partials, int nb, double *dst, double scale);
void k_sub_scalar(cudaStream_t s, long long n, double *x, const double *val);
void k_residual_plain(cudaStream_t s, const Level<double> &L, const double *phi, const double *f, double *r,
                      double *partials, int nb);
