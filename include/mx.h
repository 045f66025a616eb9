/*
 * mx.h -- C ABI of the GB300 (sm_103a) projection solver for the MAESTROeX low
 * Mach number time step (Fan et al. 2019, "MAESTROeX: A Massively Parallel Low
 * Mach Number Astrophysical Solver").
 *
 * The library enforces the velocity divergence constraint
 *     div(beta0 U) = beta0 Sbar                                  (Eq. div1/div2/div3)
 * by a projection (Appendix A): it solves the variable-coefficient elliptic
 * equation div((beta0/rho) grad phi) = div(beta0 U) - beta0 Sbar with geometric
 * multigrid and subtracts (1/rho) grad phi from U.  Two discretisations:
 *   MAC   (Steps 3 and 7): U on cell faces, phi at cell centres, 7-point operator;
 *   nodal (Step 11):       U at cell centres, phi on nodes, 27-point trilinear
 *                          finite-element operator (an approximate projection).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Domain: n[0] x n[1] x n[2] cubic cells of width dx.  Arrays are contiguous,
 * x fastest: cell (i,j,k) is element i + n0*(j + n1*k).
 * MAC face arrays hold n_d + 1 faces along their own direction d: the x-face
 * array is (n0+1) x n1 x n2, face i sitting at x = i*dx.  On a periodic axis
 * face n_d is the image of face 0; callers pass equal values and the library
 * writes equal values.
 * Nodal arrays hold n_d nodes on a periodic axis and n_d + 1 on a wall axis.
 *
 * Boundaries (per face of the box, lo/hi per axis): periodic (both sides of an
 * axis must then be periodic), Neumann wall (no flux; the normal velocity on the
 * wall is taken as 0 and the projected velocity is 0 there), homogeneous
 * Dirichlet phi = 0 (MAC only).  Periodic axes need an even cell count.
 *
 * Pointers: every array argument is a DEVICE pointer (cudaMalloc / torch CUDA
 * memory) on the context's device, owned by the caller; the library neither
 * frees nor keeps them past the call.  Scalars and structs are host memory.
 * Work is enqueued on the context's stream; calls that report norms return
 * after that stream has synchronised.
 *
 * Errors: every function returns an mx_status; mx_last_error() gives a one-line
 * description of the last failure on that context.  On MX_ERR_NOCONV the best
 * phi and the corrected U are still written and info reports the residual.
 * MX_ERR_CUDA leaves the outputs unspecified.
 */
#ifndef MX_H
#define MX_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mx_ctx mx_ctx;

typedef enum {
    MX_OK = 0,
    MX_ERR_ARG = 1,       /* invalid argument: sizes, boundaries, null pointers */
    MX_ERR_CUDA = 2,      /* a CUDA call failed */
    MX_ERR_OOM = 3,       /* device workspace allocation failed */
    MX_ERR_NOCONV = 4,    /* tolerance not reached within the iteration caps, or divergence */
    MX_ERR_INCOMPAT = 5,  /* singular problem with a right-hand side of non-zero mean */
    MX_ERR_TIMEOUT = 6    /* a device-side loop hit its hard iteration cap */
} mx_status;

typedef enum { MX_BC_PERIODIC = 0, MX_BC_NEUMANN = 1, MX_BC_DIRICHLET = 2 } mx_bc;
typedef enum { MX_PREC_FP64 = 0, MX_PREC_MIXED = 1 } mx_prec;
typedef enum { MX_OP_MAC = 0, MX_OP_NODAL = 1 } mx_op;

/* n = cell counts, dx = cell width, lo/hi = mx_bc per axis */
typedef struct {
    int n[3];
    double dx;
    int lo[3];
    int hi[3];
} mx_geom;

/* Solver options.  mx_default_opts() fills: rel_tol 1e-10, max_outer 100,
 * max_vcycles 100, prec MX_PREC_MIXED, remove_mean 1, use_initial_guess 0,
 * use_graph 1, nu1 = nu2 = 2, bottom_iters 200, fused 0, tile_z 0, krylov 0, smoother 0.
 * nu1 = nu2 = 0 selects the setting mx_autotune() stored in the context for
 * this operator, precision and geometry (nu1, nu2, fused, tile_z; nodal: also
 * smoother), or
 * 2, 2, fused, tile_z as given when nothing is stored. */
typedef struct {
    double rel_tol;        /* stop when ||f - L phi||_inf <= rel_tol ||f||_inf */
    int max_outer;         /* iterative-refinement iterations (one V-cycle each) */
    int max_vcycles;       /* total V-cycle cap */
    int prec;              /* mx_prec: FP32 V-cycles in FP64 refinement, or all FP64 */
    int remove_mean;       /* singular problems: subtract the RHS mean first */
    int use_initial_guess; /* 1: phi holds the initial guess on entry; 0: start from 0 */
    int use_graph;         /* 1: run the refinement loop as one CUDA graph */
    int nu1, nu2;          /* pre/post smoothing sweeps (red+black each) */
    int bottom_iters;      /* BiCGStab iteration cap on the coarsest grid */
    int fused;             /* 1: single-pass tile sweeps with the prolongation fused on load;
                              0: two-pass colour kernels (default; bit-identical results) */
    int tile_z;            /* cells per thread along z in the stencil kernels' tiles (the
                              largest z-chunk; smaller levels use fewer): 0 = default
                              (8 MAC, 16 nodal), else 1, 2, 4, 8 or 16; results do not
                              depend on it */
    int krylov;            /* MAC, MX_PREC_MIXED only: 0 = iterative refinement (phi +=
                              scale e after each V-cycle); 1 = flexible conjugate
                              gradients FCG(1) with the FP32 V-cycle as preconditioner:
                              the direction p = e + beta p_prev is made L-conjugate to
                              the previous one and phi += t p with the exact line-search
                              step t, while the residual is still recomputed from phi in
                              double-float after every step, so the attainable accuracy is
                              that of refinement.  Other solves reject krylov = 1
                              (MX_ERR_ARG). */
    int smoother;          /* nodal solves: 0 = four-colour Gauss-Seidel (default; nu1, nu2
                              sweeps of four colour passes); 1 = Chebyshev smoothing:
                              nu1 / nu2 steps e <- e + w_k D^-1 (f - L e) of one pass each,
                              the weights w_k the inverse roots of one Chebyshev polynomial
                              of degree nu1 + nu2 on [0.4, 1.5] (post-smoothing the nu2
                              largest roots, pre-smoothing the others); 1.5 bounds the
                              spectrum of D^-1 L for every positive coefficient field.
                              MAC, batched and composite solves reject 1 (MX_ERR_ARG). */
} mx_opts;

typedef struct {
    int outer_iters;          /* refinement iterations performed */
    int vcycles;              /* V-cycles performed */
    double rel_resid;         /* final ||f - L phi||_inf / ||f||_inf (FP64) */
    double rel_resid_l2;      /* final ||f - L phi||_2 / ||f||_2 */
    double div_err_linf;      /* MAC: max |D(beta0 U) - beta0 Sbar - c|; nodal: same at nodes */
    double rhs_mean_removed;  /* c, the mean subtracted from the RHS */
    double rhs_linf;          /* ||f||_inf after mean removal */
    double ms;                /* wall time of the call on the stream (CUDA events) */
    int status;               /* mx_status of the solve */
} mx_info;

/* Context calls (no counterpart in the paper: they hold the GPU state that the
 * projections of Appendix A run on).
 * mx_create: a context on CUDA device `device`, enqueuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream); *ctx receives it.  The
 * context owns its device workspace (multigrid hierarchy, reduction scratch,
 * graphs), allocated on first use per geometry and precision.  MX_ERR_ARG for a
 * NULL ctx; MX_ERR_CUDA for a device that does not exist or cannot be used, or
 * when the context's small fixed allocations fail.
 * mx_destroy: synchronises the context's stream and frees everything it owns
 * (never the caller's arrays); NULL is accepted.
 * mx_set_stream: later calls enqueue on cuda_stream; cached CUDA graphs stay
 * valid (graphs are launched on whatever stream is current).
 * mx_last_error: one-line description of the last failure ("" if none). */
mx_status mx_create(mx_ctx **ctx, int device, void *cuda_stream);
mx_status mx_destroy(mx_ctx *ctx);
mx_status mx_set_stream(mx_ctx *ctx, void *cuda_stream);
const char *mx_last_error(const mx_ctx *ctx);
void mx_default_opts(mx_opts *opts);
/* 1 if the library was built for this device (sm_103), else 0 */
int mx_device_supported(int device);

/* Fill (Sec. 3.1): map a 1D base-state profile onto the Cartesian cells.
 * planar (spherical = 0): direct injection, cell (i,j,k) takes prof[k];
 *   requires nr >= n[2].
 * spherical (spherical = 1): prof[m] is the value at radius (m + 1/2) dr from
 *   center (host array of 3 coordinates); each cell centre takes the linear
 *   interpolation in r between the two bracketing radial cell centres (the
 *   first/last interval is extended linearly); requires nr >= 2.
 * prof: device, nr doubles; out_cells: device, n0 n1 n2 doubles. */
mx_status mx_fill_base_state(mx_ctx *ctx, const mx_geom *geom, int spherical, const double *prof,
                             int nr, double dr, const double center[3], double *out_cells);

/* ---- Lateral average and fill of the base state (Sec. 3.1, Eq. radii) --------------
 * Cell arrays are device doubles of n0 n1 n2 entries, x fastest; the boundary
 * types in geom are not used.  The calls queue work on the context's stream and
 * return without synchronising; sums run in double-float arithmetic in a fixed
 * order, so repeated calls give identical bits.  Fields with magnitudes outside
 * 2^-73..2^97 are summed exactly as well, by full-range passes that run only
 * when such a value is present (slower: FP64 for the outliers).
 *
 * Spherical geometry puts the centre of the star on the cell corner corner[3]
 * (host array of three integer corner indices, each within +-2^20; the corner
 * may lie outside the box).  The centre of cell (i,j,k) is then at distance
 * dx sqrt(0.75 + 2m) from it, m = T(i-c0) + T(j-c1) + T(k-c2), T(a) = a(a+1)/2:
 * bin m of the irregularly spaced base state.  The first call for a given
 * (n, corner) builds and caches a plan on the context (host work proportional to
 * n1 n2 plus a device allocation of about 8 bytes per cell at most). */

/* number of radial bins (largest m + 1) for the box and corner; -1 if the corner
 * is out of range or the count reaches 2^31.  Host only. */
long long mx_radial_nbins(const mx_geom *geom, const int corner[3]);

/* Planar Average: prof[k] = mean of field over plane k (n2 doubles out). */
mx_status mx_average_planar(mx_ctx *ctx, const mx_geom *geom, const double *field, double *prof);

/* Spherical Average onto the irregular base state: avg[m] = mean of field over
 * the cells of bin m (0 for bins without cells), count[m] = their number
 * (int64; count may be NULL).  nbins must equal mx_radial_nbins (else
 * MX_ERR_ARG).  MX_ERR_ARG also for n0 above 12000 or a corner whose row radii
 * span more than 2^26 bins; MX_ERR_OOM if the plan cannot be allocated. */
mx_status mx_average_radial(mx_ctx *ctx, const mx_geom *geom, const int corner[3], const double *field,
                            long long nbins, double *avg, long long *count);

/* Fill from the irregular base state, without interpolation: out(i,j,k) =
 * base[m(i,j,k)] (base: nbins device doubles). */
mx_status mx_fill_radial(mx_ctx *ctx, const mx_geom *geom, const int corner[3], const double *base,
                         long long nbins, double *out);

/* Average onto a uniform base state prof[j] at radii (j + 1/2) dr (nr >= 1
 * doubles out) from the bin means avg (nbins doubles, as mx_average_radial
 * writes them): the quadratic (3-point Lagrange) interpolant through the
 * non-empty bin whose radius is nearest to (j + 1/2) dr (the smaller one on a
 * tie) and the non-empty bins on either side, the triple kept one bin inside at
 * either end.  MX_ERR_ARG with fewer than 3 non-empty bins. */
mx_status mx_radial_to_uniform(mx_ctx *ctx, const mx_geom *geom, const int corner[3], const double *avg, int nr,
                               double dr, double *prof);

/* Fill from a uniform base state prof (nr >= 3 device doubles at radii
 * (j + 1/2) dr) by quadratic interpolation: each cell takes the 3-point Lagrange
 * interpolant at its radius through the radial cell centres jc - 1, jc, jc + 1,
 * jc = floor(r / dr) kept within [1, nr - 2].  All cells of a bin share their
 * radius, so the value is computed once per bin (in the context's plan) and
 * gathered. */
mx_status mx_fill_uniform(mx_ctx *ctx, const mx_geom *geom, const int corner[3], const double *prof, int nr,
                          double dr, double *out);

/* ---- Velocity split (Appendix A): U = U~ + w0 e_r --------------------------------------
 * U~ is projected with div(beta0 U~) = beta0 (S - Sbar), Sbar the lateral average of S;
 * w0 solves div(beta0 w0 e_r) = beta0 (Sbar - psi), psi = dp0/dt / (Gamma1bar p0),
 * in one dimension.  Base-state arrays: nr cells between nr + 1 edges r_edge
 * (device, strictly increasing; spherical: r_edge[0] = 0, the star's centre). */

/* w0 on the nr + 1 edges (device out) from beta0 and src = Sbar - psi on the nr
 * cells (device):  Q_0 = 0, Q_{j+1} = Q_j + V_j beta0_j src_j, w0_e = Q_e / (A_e
 * beta0_e); planar A = 1 and V_j = r_{j+1} - r_j, spherical A = r^2 and V_j =
 * (r_{j+1}^3 - r_j^3)/3; beta0 on an interior edge is the mean of its two cells, on
 * the last edge the last cell's.  cutoff >= 0: beyond that edge A w0 keeps its
 * cutoff value (the outer boundary condition at the edge of the star); -1: none.
 * One CTA, FP64; MX_ERR_ARG for nr < 1 or cutoff outside [-1, nr]. */
mx_status mx_w0_integrate(mx_ctx *ctx, int spherical, int nr, const double *r_edge, const double *beta0,
                          const double *src, int cutoff, double *w0);

/* U_f += w0(r_f) (e_r . n_f) on the MAC faces (ux, uy, uz: API face arrays, in/out).
 * planar (spherical = 0): the base-state cells are the cell layers, z-face k takes
 *   w0[k] (needs nr >= n2; r_edge, corner, ux, uy may be NULL).
 * spherical: the star's centre on the cell corner corner[3] (host); w0 linear in r
 *   between the edges, A w0 held beyond the last edge.  The factor dx w0(r)/r is
 *   tabulated once per face radius (4 r^2/dx^2 is an integer K, 2 mod 4) in context
 *   scratch of 2 K_max + 8 bytes; MX_ERR_ARG when K_max / 4 reaches 2^26. */
mx_status mx_add_w0_faces(mx_ctx *ctx, const mx_geom *geom, int spherical, const int corner[3], int nr,
                          const double *r_edge, const double *w0, double *ux, double *uy, double *uz);

/* out = S - Sbar on the cells (device), Sbar the lateral average of S filled back:
 * plane means (spherical = 0) or the irregular radial means of the star centred on
 * corner (spherical = 1). */
mx_status mx_subtract_lateral_average(mx_ctx *ctx, const mx_geom *geom, int spherical, const int corner[3],
                                      const double *S, double *out);

/* The split MAC projection: the bracket S - Sbar (in context scratch of one cell
 * array), mx_mac_project of U~ (ux, uy, uz in: U~ predicted; phi, opts, info as
 * mx_mac_project), then mx_add_w0_faces with the caller's w0 (from
 * mx_w0_integrate).  Returns the solve's status (MX_ERR_NOCONV still adds w0);
 * synchronises the stream before returning. */
mx_status mx_mac_project_split(mx_ctx *ctx, const mx_geom *geom, int spherical, const int corner[3], double *ux,
                               double *uy, double *uz, const double *rho, const double *beta0, const double *S,
                               int nr, const double *r_edge, const double *w0, double *phi, const mx_opts *opts,
                               mx_info *info);

/* MAC projection (Steps 3 and 7; Eq. div1, div2; Appendix A).
 * ux, uy, uz: face velocities U^ADV,dagger (in) -> projected U^ADV (out).
 * rho, beta0, sbar: cell fields; sbar is the whole bracket of the constraint's
 *   right-hand side (S - dp0/dt / (Gamma1 p0)), multiplied by beta0 inside.
 * phi: cell field (out; in as initial guess if opts->use_initial_guess).
 * Face coefficient b = beta0_f / rho_f with arithmetic face averages (the
 * interior cell on a Dirichlet face).  On singular problems (no Dirichlet face)
 * the RHS mean c is removed (remove_mean = 1) and phi has zero mean; with
 * remove_mean = 0 a RHS of mean above 1e-12 ||f||_inf returns MX_ERR_INCOMPAT.
 * opts may be NULL (defaults); info may be NULL. */
mx_status mx_mac_project(mx_ctx *ctx, const mx_geom *geom, double *ux, double *uy, double *uz,
                         const double *rho, const double *beta0, const double *sbar, double *phi,
                         const mx_opts *opts, mx_info *info);

/* Nodal projection (Step 11; Eq. div3; Appendix A).  ux, uy, uz: cell-centred
 * velocity (in/out); phi_nodes: nodal field (out).  Only periodic and Neumann
 * boundaries.  sigma = beta0/rho per cell; the weighted RHS mean is removed. */
mx_status mx_nodal_project(mx_ctx *ctx, const mx_geom *geom, double *ux, double *uy, double *uz,
                           const double *rho, const double *beta0, const double *sbar,
                           double *phi_nodes, const mx_opts *opts, mx_info *info);

/* Apply the operator L = div((beta0/rho) grad .) of the projection's elliptic
 * equation (Appendix A; the MAC form of Steps 3 and 7, Eq. div1/div2, and the
 * nodal form of Step 11, Eq. div3) to phi (MAC: cells -> cells; nodal: nodes ->
 * nodes), with the face coefficients and boundary closures of mx_mac_project /
 * mx_nodal_project.  rho, beta0: cell arrays; phi, Lphi: device arrays in the
 * layout of phi (Lphi written, never read).  prec = MX_PREC_FP64 computes in
 * FP64; MX_PREC_MIXED rounds the coefficients and phi to FP32 and computes in
 * FP32 (the arithmetic of the V-cycle), still writing doubles.  Work is queued
 * on the context's stream (no synchronisation).  MX_ERR_ARG for an unknown op
 * or prec, invalid geometry or a NULL array. */
mx_status mx_apply_op(mx_ctx *ctx, const mx_geom *geom, int op, int prec, const double *rho,
                      const double *beta0, const double *phi, double *Lphi);

/* Residual of the projection's elliptic equation L phi = f (Appendix A; the
 * convergence measure of the solves): r = f - L phi (device, same layout as
 * phi; L as for mx_apply_op) and, if rnorm_linf is not NULL, its max norm to
 * the host after the stream synchronises (NaN if r holds a NaN).  Errors as for
 * mx_apply_op. */
mx_status mx_residual(mx_ctx *ctx, const mx_geom *geom, int op, int prec, const double *rho,
                      const double *beta0, const double *phi, const double *f, double *r,
                      double *rnorm_linf);

/* Batched MAC projections of nbox independent boxes (AMR-style patches, the
 * analogue of the paper's 64^3 grids per MPI task, Sec. 4.1).  Each box has its
 * own geometry and arrays (host arrays of device pointers, length nbox); every
 * smoothing / restriction / prolongation phase runs as one launch over a work
 * list of tiles of all boxes.  infos: host array of nbox (may be NULL). */
mx_status mx_mac_project_batched(mx_ctx *ctx, int nbox, const mx_geom *geoms, double *const *ux,
                                 double *const *uy, double *const *uz, const double *const *rho,
                                 const double *const *beta0, const double *const *sbar,
                                 double *const *phi, const mx_opts *opts, mx_info *infos);

/* FP64 MAC residual r = f - L phi and its max norm, allocating nothing.  This
 * entry point has no counterpart in the paper; it serves callers that may not
 * allocate device memory at all -- code that runs inside a caller-managed pool
 * or arena, or under a policy that forbids cudaMalloc on a hot path -- and so
 * cannot create an mx_ctx (whose workspace is allocated).  It computes the face
 * coefficients on the fly from rho and beta0 and keeps its per-tile partial
 * maxima in a fixed device array built into the library (about 512 KB, held by
 * every GPU that loads the library until the process exits).
 * Arguments as for mx_residual (device arrays, MAC operator, FP64); work runs on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream) of the current
 * device; rnorm_linf (host, may be NULL) is written after the stream syncs.
 * Limit: at most 65536 tiles of 32 x 8 x 8 cells, i.e. ceil(n0/32) *
 * ceil(n1/8) * ceil(n2/8) <= 65536 (512^3 fits), and ceil(n1/8), ceil(n2/8)
 * <= 65535; larger grids return MX_ERR_ARG before any work.  The first call on a device looks up the array's device
 * address; make that first call before capturing a stream into a graph.  All
 * calls share the one array: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  The first-call
 * lookup itself is safe from several host threads.  The looked-up address
 * belongs to the device's primary context: after cudaDeviceReset the library
 * must be unloaded and loaded again.  The norm is NaN if r holds a NaN. */
mx_status mx_residual_noalloc(const mx_geom *geom, const double *rho, const double *beta0, const double *phi,
                              const double *f, double *r, double *rnorm_linf, void *cuda_stream);

/* Tracing: per-phase device time of mx_mac_project.  While enabled, the
 * refinement loop runs from the host (no graph) and every phase is bracketed by
 * CUDA events on the context's stream.  mx_profile_read copies, per phase, the
 * accumulated milliseconds and kernel launches since the last read (host arrays
 * of MX_PH_COUNT entries) and resets the counters. */
enum {
    MX_PH_SETUP = 0,          /* coefficients, hierarchy, right-hand side */
    MX_PH_RESID64 = 1,        /* FP64 residual + norms of the refinement loop */
    MX_PH_SMOOTH_FINE = 2,    /* red-black sweeps on the finest level */
    MX_PH_RESTRICT_FINE = 3,  /* residual + restriction from the finest level */
    MX_PH_PROLONG_FINE = 4,   /* prolongation onto the finest level */
    MX_PH_COARSE = 5,         /* all coarser levels and the bottom solve */
    MX_PH_UPDATE = 6,         /* zeroing of the correction and phi += scale e; with
                                 krylov = 1 the conjugation and line search */
    MX_PH_FINISH = 7,         /* mean normalisation, velocity correction, divergence check */
    MX_PH_COUNT = 8
};
mx_status mx_profile_enable(mx_ctx *ctx, int enable);
mx_status mx_profile_read(mx_ctx *ctx, double *ms, long long *launches);

/* Autotuner (a GPU tuning step; the paper has no counterpart).  Times the
 * projection of the given inputs (op MX_OP_MAC: mx_mac_project, MX_OP_NODAL:
 * mx_nodal_project, same argument layouts) under candidate smoother and tile
 * settings -- sweep counts (nu1, nu2) in {1..4}, then tile_z in {4, 8, 16}
 * (nodal {4, 8, 16, default}), then (MAC, mixed precision) the single-pass
 * sweep or (nodal, base smoother 0) the Chebyshev smoother at degrees (nu1,
 * nu2) in {1..3} -- one at a time from base (NULL = defaults), keeping a change only if
 * the solve converges and is faster (CUDA-event time of a whole call, after
 * one untimed call that builds the graph).  Candidates needing more than
 * 3 x (the best's V-cycles) + 4 V-cycles are cut off.  The winner is stored in
 * the context's tune cache for (op, prec, geometry) and used by later calls
 * with nu1 = nu2 = 0.  The inputs are not modified: the tuner copies U and
 * phi into scratch it allocates and frees (about 4 fields of device memory).
 * best (may be NULL): the chosen options (base with nu1, nu2, fused, tile_z,
 * smoother replaced); ms_best (may be NULL): the tuned solve's time in ms.  Returns
 * MX_ERR_NOCONV if no candidate converges, MX_ERR_OOM if the scratch cannot
 * be allocated, or the error of the first failing solve. */
mx_status mx_autotune(mx_ctx *ctx, int op, const mx_geom *geom, const double *ux, const double *uy,
                      const double *uz, const double *rho, const double *beta0, const double *sbar,
                      const mx_opts *base, mx_opts *best, double *ms_best);

/* Autotuner for a batch (mx_mac_project_batched arguments; mixed precision):
 * times the whole batch under each candidate (nu1, nu2) of mx_autotune, one
 * setting for every box, and stores the fastest converging one in the tune
 * cache under the batch's box count and geometries; mx_mac_project_batched
 * with nu1 = nu2 = 0 uses it.  The inputs are not modified (scratch copies of
 * every box's U and phi are allocated and freed).  Same outputs and errors as
 * mx_autotune. */
mx_status mx_autotune_batched(mx_ctx *ctx, int nbox, const mx_geom *geoms, const double *const *ux,
                              const double *const *uy, const double *const *uz, const double *const *rho,
                              const double *const *beta0, const double *const *sbar, const mx_opts *base,
                              mx_opts *best, double *ms_best);

/* ---- Two-level composite (AMR) operator, refinement ratio 2 (end of Sec. 3.2:
 * AMR as in the paper's Paper V, ratio 2 between levels) -------------------------
 * geom: the coarse level (cells, dx = H, domain boundary types).  plo, phi (host):
 * the fine patch as the coarse-index box [plo, phi), at least one coarse cell from
 * every domain face and at least one coarse cell thick (else MX_ERR_ARG); the fine
 * level has 2 (phi - plo) cells per axis of width H/2.  Coarse arrays cover the
 * whole coarse grid (values on covered cells are not read); fine arrays cover the
 * patch; face arrays carry n_d + 1 entries along their own direction.  All arrays
 * are device pointers, x fastest.  Discretisation: fine ghost values across the
 * patch boundary by linear tangential interpolation of the coarse value across
 * and the normal quadratic 8/15 C~ + 2/3 F1 - 1/5 F2; coarse fluxes through
 * coarse-fine faces are the means of the four fine fluxes (flux matching); face
 * coefficients beta0_f / rho_f by arithmetic face means (of the fine cell and
 * the coarse cell across on a coarse-fine face).  FP64; both calls queue their
 * work on the context's stream and return without synchronising (the outputs
 * are ready in stream order, as for mx_apply_op). */

/* out = L phi on the uncovered coarse cells (0 on covered ones) and the fine cells */
mx_status mx_composite_apply(mx_ctx *ctx, const mx_geom *geom, const int plo[3], const int phi[3],
                             const double *rho_c, const double *beta0_c, const double *rho_f, const double *beta0_f,
                             const double *phi_c, const double *phi_f, double *out_c, double *out_f);

/* out = D(beta0 U) on the uncovered coarse cells (0 on covered ones) and the fine
 * cells; U on a wall face is taken as 0, beta0 of the interior cell on a Dirichlet
 * face, and a coarse cell's coarse-fine flux is the mean of the four fine
 * beta0_f U_f on its face. */
mx_status mx_composite_divergence(mx_ctx *ctx, const mx_geom *geom, const int plo[3], const int phi[3],
                                  const double *ux_c, const double *uy_c, const double *uz_c, const double *ux_f,
                                  const double *uy_f, const double *uz_f, const double *beta0_c,
                                  const double *beta0_f, double *out_c, double *out_f);

/* Measurement helper (no counterpart in the paper): the FMA rate of the
 * device's FP64 (fp64 = 1) or FP32 (fp64 = 0) pipe in TFLOP/s (2 flops per
 * FMA), the best of three CUDA-event-timed launches of independent FMA chains
 * on every SM (after one warm-up launch).  It is the arithmetic bound beside the
 * HBM bound for the plain FP64 solve.  Runs on the legacy default stream of
 * `device` (made current), allocates and frees a small device buffer and
 * synchronises; *tflops is written on MX_OK.  MX_ERR_ARG for a NULL tflops,
 * MX_ERR_CUDA if the device cannot run it. */
mx_status mx_probe_fma_peak(int device, int fp64, double *tflops);

/* Composite (two-level, ratio 2) MAC projection (Steps 3 and 7, Eq. div1/div2,
 * Appendix A, on the AMR levels of the end of Sec. 3.2): the projection of the
 * coarse level and one fine patch together, with the composite operator and
 * divergence of mx_composite_apply / mx_composite_divergence (ghost values,
 * flux matching at the coarse-fine faces).  Solves L phi = f, f = D(beta0 U) -
 * beta0 Sbar on the uncovered coarse cells and the fine cells, the
 * volume-weighted mean removed when no face is Dirichlet, to ||f - L phi||_inf
 * <= rel_tol ||f||_inf (FP64 composite residual); then U -= grad(phi)/rho_f on
 * both levels (the fine coarse-fine faces with the ghost value), the coarse
 * faces on and inside the patch take the mean of the four fine faces on them,
 * and the covered coarse phi the mean of its eight fine cells.  phi has zero
 * volume-weighted mean over the uncovered coarse and the fine cells on singular
 * problems.
 * Arguments: geom, plo, phi as for mx_composite_apply (phi[3] is the patch's
 * high corner, phi_c / phi_f the potentials); coarse arrays cover the whole
 * coarse grid (U faces in/out, rho, beta0, sbar in; rho and beta0 on covered
 * cells are not read), fine arrays cover the patch; all device pointers.
 * opts: prec must be MX_PREC_MIXED (FP32 V-cycles as the corrections inside the
 * FP64 refinement) and krylov 0 (else MX_ERR_ARG); nu1 = nu2 = 0 means 2, 2;
 * max_outer / max_vcycles cap the refinement iterations (each runs one V-cycle
 * of the coarse grid and one of the patch; info->vcycles counts both).
 * The context keeps the workspace of the last composite geometry (two multigrid
 * plans, six FP64 cell fields and the FP64 face coefficients of both levels) and
 * the CUDA graph of its refinement loop (use_graph = 1; keyed by phi_c, phi_f and
 * the smoother options); a new geometry replaces them.  Synchronises the stream. */
mx_status mx_mac_project_composite(mx_ctx *ctx, const mx_geom *geom, const int plo[3], const int phi[3],
                                   double *ux_c, double *uy_c, double *uz_c, const double *rho_c,
                                   const double *beta0_c, const double *sbar_c, double *phi_c, double *ux_f,
                                   double *uy_f, double *uz_f, const double *rho_f, const double *beta0_f,
                                   const double *sbar_f, double *phi_f, const mx_opts *opts, mx_info *info);

/* Look up the tune cache: 1 and *out = the stored setting (base fields from
 * *out as passed) if mx_autotune stored one for (op, prec, geometry), else 0. */
int mx_tune_lookup(const mx_ctx *ctx, int op, int prec, const mx_geom *geom, mx_opts *out);

#ifdef __cplusplus
}
#endif
#endif /* MX_H */
