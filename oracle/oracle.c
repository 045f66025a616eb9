/*
 * FP64 CPU oracle for the MAESTROeX projections (Fan et al., "MAESTROeX: A
 * Massively Parallel Low Mach Number Astrophysical Solver", Appendix A and
 * Steps 3, 7, 11 of Sec. 3.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this code.  It shares nothing with the CUDA library:
 * separate source, separate data layout (API face arrays throughout), separate
 * solver (multigrid-preconditioned conjugate gradients with lexicographic
 * symmetric Gauss-Seidel, plus a dense Gaussian-elimination solve).
 *
 * Everything is plain, slow, double precision and single threaded.
 *
 * Discretisation readings (the paper defers the stencils to its Paper III):
 *   - face coefficient b_f = beta0_f / rho_f with arithmetic face averages of
 *     the two adjacent cells; on a Dirichlet face the single interior cell;
 *   - (L phi)_c = sum_d (F_hi - F_lo)/h with the face flux F = b_f dphi/dn;
 *     periodic faces wrap, wall (Neumann) faces carry no flux, Dirichlet
 *     phi = 0 faces use the one-sided difference (0 - phi_c)/(h/2);
 *   - RHS f = D(beta0_f U_f) - beta0 Sbar (Eq. div1/div2), U_f treated as 0 on
 *     wall faces, mean removed when no face is Dirichlet;
 *   - correction U_f <- U_f - dphi/dn / rho_f, wall faces set to 0.
 *
 * Nodal projection (Step 11, Eq. div3): trilinear finite-element operator on
 * nodes with cell-centred sigma = beta0/rho, lumped node weights, the weak
 * divergence of cell-centred velocities and the cell-averaged nodal gradient.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_PERIODIC 0
#define OR_NEUMANN 1
#define OR_DIRICHLET 2

typedef struct {
    int n[3];
    double h;
    int lo[3], hi[3];
} or_geom;

/* ------------------------------------------------------------------------ */
/* indexing                                                                   */

static long cidx(const or_geom *g, int i, int j, int k) {
    return (long)i + (long)g->n[0] * ((long)j + (long)g->n[1] * k);
}

/* face p (0..n_d) along d, transverse indices taken from (i,j,k) */
static long fidx(const or_geom *g, int d, int i, int j, int k) {
    long nx = g->n[0], ny = g->n[1];
    if (d == 0) return (long)i + (nx + 1) * ((long)j + ny * k);
    if (d == 1) return (long)i + nx * ((long)j + (ny + 1) * k);
    return (long)i + nx * ((long)j + ny * k);
}

long or_ncell(const or_geom *g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

long or_nface(const or_geom *g, int d) {
    long m = 1;
    for (int a = 0; a < 3; a++) m *= g->n[a] + (a == d ? 1 : 0);
    return m;
}

int or_singular(const or_geom *g) {
    for (int d = 0; d < 3; d++)
        if (g->lo[d] == OR_DIRICHLET || g->hi[d] == OR_DIRICHLET) return 0;
    return 1;
}

/* The two cells beside face p along d: returns 1 if the left (or right) cell is
 * a real cell (with periodic wrap), 0 if it lies outside a non-periodic wall. */
static int face_cells(const or_geom *g, int d, int p, int *left, int *right) {
    int n = g->n[d];
    *left = p - 1;
    *right = p;
    int has_l = 1, has_r = 1;
    if (p == 0) {
        if (g->lo[d] == OR_PERIODIC) *left = n - 1; else has_l = 0;
    }
    if (p == n) {
        if (g->hi[d] == OR_PERIODIC) *right = 0; else has_r = 0;
    }
    return has_l | (has_r << 1);
}

static int face_bc(const or_geom *g, int d, int p) {
    if (p == 0) return g->lo[d];
    if (p == g->n[d]) return g->hi[d];
    return -1; /* interior */
}

/* cell index with coordinate along d replaced */
static long cell_along(const or_geom *g, int d, int i, int j, int k, int m) {
    if (d == 0) return cidx(g, m, j, k);
    if (d == 1) return cidx(g, i, m, k);
    return cidx(g, i, j, m);
}

/* ------------------------------------------------------------------------ */
/* Fill (Sec. 3.1): base state -> Cartesian cells                             */

/* planar: direct injection, cell (i,j,k) takes prof[k] */
int or_fill_planar(const or_geom *g, const double *prof, int nr, double *out) {
    if (nr < g->n[2]) return -1;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) out[cidx(g, i, j, k)] = prof[k];
    return 0;
}

/* spherical: prof[m] is the value at radius (m + 1/2) dr; linear interpolation
 * in r between the two bracketing radial cell centres (end intervals extended
 * linearly). */
int or_fill_spherical(const or_geom *g, const double *prof, int nr, double dr,
                      const double *center, double *out) {
    if (nr < 2) return -1;
    double h = g->h;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                double x = (i + 0.5) * h - center[0];
                double y = (j + 0.5) * h - center[1];
                double z = (k + 0.5) * h - center[2];
                double r = sqrt(x * x + y * y + z * z);
                double s = r / dr - 0.5;      /* fractional radial cell-centre index */
                int m = (int)floor(s);
                if (m < 0) m = 0;
                if (m > nr - 2) m = nr - 2;
                double t = s - m;
                out[cidx(g, i, j, k)] = prof[m] + t * (prof[m + 1] - prof[m]);
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* MAC projection: coefficients, operator, RHS, correction, divergence        */

/* b_f = beta0_f / rho_f on all faces of direction d (API face layout). */
void or_mac_coeffs(const or_geom *g, const double *rho, const double *beta0,
                   double *bx, double *by, double *bz) {
    double *b[3] = {bx, by, bz};
    for (int d = 0; d < 3; d++) {
        int m[3] = {g->n[0], g->n[1], g->n[2]};
        m[d] += 1;
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    int p = d == 0 ? i : d == 1 ? j : k;
                    int L, R;
                    int has = face_cells(g, d, p, &L, &R);
                    double v;
                    if (has == 3) {
                        long cl = cell_along(g, d, i, j, k, L), cr = cell_along(g, d, i, j, k, R);
                        double beta_f = 0.5 * (beta0[cl] + beta0[cr]);
                        double rho_f = 0.5 * (rho[cl] + rho[cr]);
                        v = beta_f / rho_f;
                    } else if (face_bc(g, d, p) == OR_DIRICHLET) {
                        long c = cell_along(g, d, i, j, k, has == 2 ? R : L);
                        v = beta0[c] / rho[c];
                    } else {
                        v = 0.0; /* wall: no flux, coefficient unused */
                    }
                    b[d][fidx(g, d, i, j, k)] = v;
                }
    }
}

/* normal derivative of phi on face p along d (cell (i,j,k) supplies the
 * transverse indices); phi = 0 beyond a Dirichlet face, 0 on a wall. */
static double face_grad(const or_geom *g, const double *phi, int d, int i, int j, int k, int p) {
    int L, R;
    int has = face_cells(g, d, p, &L, &R);
    double h = g->h;
    if (has == 3)
        return (phi[cell_along(g, d, i, j, k, R)] - phi[cell_along(g, d, i, j, k, L)]) / h;
    if (face_bc(g, d, p) == OR_DIRICHLET) {
        if (has == 2) return (phi[cell_along(g, d, i, j, k, R)] - 0.0) / (0.5 * h);
        return (0.0 - phi[cell_along(g, d, i, j, k, L)]) / (0.5 * h);
    }
    return 0.0;
}

static long face_of_cell(const or_geom *g, int d, int i, int j, int k, int p) {
    if (d == 0) return fidx(g, 0, p, j, k);
    if (d == 1) return fidx(g, 1, i, p, k);
    return fidx(g, 2, i, j, p);
}

/* Lphi = sum_d (b dphi/dn |hi - b dphi/dn |lo) / h */
void or_mac_apply(const or_geom *g, const double *bx, const double *by, const double *bz,
                  const double *phi, double *out) {
    const double *b[3] = {bx, by, bz};
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                int c3[3] = {i, j, k};
                double s = 0.0;
                for (int d = 0; d < 3; d++) {
                    int plo = c3[d], phi_ = c3[d] + 1;
                    double flo = b[d][face_of_cell(g, d, i, j, k, plo)] * face_grad(g, phi, d, i, j, k, plo);
                    double fhi = b[d][face_of_cell(g, d, i, j, k, phi_)] * face_grad(g, phi, d, i, j, k, phi_);
                    s += (fhi - flo) / g->h;
                }
                out[cidx(g, i, j, k)] = s;
            }
}

/* beta0 on face p: average of the two cells, the interior cell on a Dirichlet
 * face; 0 on a wall (U_f is taken as 0 there). */
static double face_beta(const or_geom *g, const double *beta0, int d, int i, int j, int k, int p) {
    int L, R;
    int has = face_cells(g, d, p, &L, &R);
    if (has == 3)
        return 0.5 * (beta0[cell_along(g, d, i, j, k, L)] + beta0[cell_along(g, d, i, j, k, R)]);
    if (face_bc(g, d, p) == OR_DIRICHLET) return beta0[cell_along(g, d, i, j, k, has == 2 ? R : L)];
    return 0.0;
}

/* D(beta0 U) on cells from face velocities */
void or_mac_divergence(const or_geom *g, const double *ux, const double *uy, const double *uz,
                       const double *beta0, double *out) {
    const double *u[3] = {ux, uy, uz};
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                int c3[3] = {i, j, k};
                double s = 0.0;
                for (int d = 0; d < 3; d++) {
                    int plo = c3[d], phi_ = c3[d] + 1;
                    double flo = face_beta(g, beta0, d, i, j, k, plo) * u[d][face_of_cell(g, d, i, j, k, plo)];
                    double fhi = face_beta(g, beta0, d, i, j, k, phi_) * u[d][face_of_cell(g, d, i, j, k, phi_)];
                    s += (fhi - flo) / g->h;
                }
                out[cidx(g, i, j, k)] = s;
            }
}

/* f = D(beta0 U) - beta0 Sbar; mean removed when the problem is singular and
 * remove_mean != 0.  Returns the removed mean in *mean. */
void or_mac_rhs(const or_geom *g, const double *ux, const double *uy, const double *uz,
                const double *beta0, const double *sbar, int remove_mean, double *f, double *mean) {
    or_mac_divergence(g, ux, uy, uz, beta0, f);
    long N = or_ncell(g);
    for (long c = 0; c < N; c++) f[c] -= beta0[c] * sbar[c];
    double m = 0.0;
    if (remove_mean && or_singular(g)) {
        double s = 0.0;
        for (long c = 0; c < N; c++) s += f[c];
        m = s / (double)N;
        for (long c = 0; c < N; c++) f[c] -= m;
    }
    if (mean) *mean = m;
}

/* U_f <- U_f - (dphi/dn)/rho_f on every face; wall faces get U = 0 */
void or_mac_correct(const or_geom *g, const double *rho, const double *phi,
                    double *ux, double *uy, double *uz) {
    double *u[3] = {ux, uy, uz};
    for (int d = 0; d < 3; d++) {
        int m[3] = {g->n[0], g->n[1], g->n[2]};
        m[d] += 1;
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    int p = d == 0 ? i : d == 1 ? j : k;
                    int L, R;
                    int has = face_cells(g, d, p, &L, &R);
                    long f = fidx(g, d, i, j, k);
                    /* the transverse indices of (i,j,k) are valid cell indices;
                       face_grad only reads cells along d */
                    if (has == 3) {
                        double rho_f = 0.5 * (rho[cell_along(g, d, i, j, k, L)] + rho[cell_along(g, d, i, j, k, R)]);
                        u[d][f] -= face_grad(g, phi, d, i, j, k, p) / rho_f;
                    } else if (face_bc(g, d, p) == OR_DIRICHLET) {
                        double rho_f = rho[cell_along(g, d, i, j, k, has == 2 ? R : L)];
                        u[d][f] -= face_grad(g, phi, d, i, j, k, p) / rho_f;
                    } else {
                        u[d][f] = 0.0;
                    }
                }
    }
}

/* ------------------------------------------------------------------------ */
/* norms and small helpers                                                    */

double or_norm_inf(long n, const double *a) {
    double m = 0.0;
    for (long i = 0; i < n; i++) m = fmax(m, fabs(a[i]));
    return m;
}

static double dot(long n, const double *a, const double *b) {
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static void remove_mean(long n, double *a) {
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i];
    s /= (double)n;
    for (long i = 0; i < n; i++) a[i] -= s;
}

/* ------------------------------------------------------------------------ */
/* Dense direct solve (Gaussian elimination with partial pivoting).  Used as
 * an independent check of the iterative solve on small grids.                */

typedef void (*or_apply_fn)(const void *ctx, const double *x, double *y);

/* Solve A x = f, A given as an operator on n unknowns.  If pin_row is >= 0,
 * equation pin_row is replaced by sum_i w_i x_i = 0 (w = NULL: all ones),
 * which selects the normalised solution of a singular, consistent system. */
int or_dense_solve(long n, or_apply_fn apply, const void *ctx, const double *f, double *x,
                   long pin_row, const double *w) {
    double *A = (double *)malloc(sizeof(double) * n * n);
    double *e = (double *)calloc(n, sizeof(double));
    double *col = (double *)malloc(sizeof(double) * n);
    double *rhs = (double *)malloc(sizeof(double) * n);
    if (!A || !e || !col || !rhs) { free(A); free(e); free(col); free(rhs); return -1; }
    for (long j = 0; j < n; j++) {
        e[j] = 1.0;
        apply(ctx, e, col);
        e[j] = 0.0;
        for (long i = 0; i < n; i++) A[i * n + j] = col[i];
    }
    for (long i = 0; i < n; i++) rhs[i] = f[i];
    if (pin_row >= 0) {
        for (long j = 0; j < n; j++) A[pin_row * n + j] = w ? w[j] : 1.0;
        rhs[pin_row] = 0.0;
    }
    for (long c = 0; c < n; c++) {
        long p = c;
        for (long r = c + 1; r < n; r++)
            if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
        if (A[p * n + c] == 0.0) { free(A); free(e); free(col); free(rhs); return -2; }
        if (p != c) {
            for (long j = 0; j < n; j++) { double t = A[c * n + j]; A[c * n + j] = A[p * n + j]; A[p * n + j] = t; }
            double t = rhs[c]; rhs[c] = rhs[p]; rhs[p] = t;
        }
        for (long r = c + 1; r < n; r++) {
            double m = A[r * n + c] / A[c * n + c];
            if (m == 0.0) continue;
            for (long j = c; j < n; j++) A[r * n + j] -= m * A[c * n + j];
            rhs[r] -= m * rhs[c];
        }
    }
    for (long r = n - 1; r >= 0; r--) {
        double s = rhs[r];
        for (long j = r + 1; j < n; j++) s -= A[r * n + j] * x[j];
        x[r] = s / A[r * n + r];
    }
    free(A); free(e); free(col); free(rhs);
    return 0;
}

typedef struct { const or_geom *g; const double *b[3]; } mac_op_ctx;

static void mac_apply_cb(const void *vctx, const double *x, double *y) {
    const mac_op_ctx *c = (const mac_op_ctx *)vctx;
    or_mac_apply(c->g, c->b[0], c->b[1], c->b[2], x, y);
}

int or_mac_dense_solve(const or_geom *g, const double *bx, const double *by, const double *bz,
                       const double *f, double *phi) {
    mac_op_ctx c = {g, {bx, by, bz}};
    return or_dense_solve(or_ncell(g), mac_apply_cb, &c, f, phi, or_singular(g) ? 0 : -1, NULL);
}

/* ------------------------------------------------------------------------ */
/* Multigrid-preconditioned conjugate gradients for the MAC system.
 * A = -L is symmetric positive (semi)definite.  The preconditioner is one
 * V-cycle: lexicographic Gauss-Seidel forward before and backward after the
 * coarse correction, 8-cell average restriction, piecewise-constant
 * prolongation, coarse faces = mean of the 4 fine faces they cover, exact
 * dense coarsest solve.  Forward/backward smoothing and R = P^T/8 make the
 * preconditioner symmetric, as CG requires.                                   */

#define OR_MAXLEV 24

typedef struct {
    or_geom g;
    double *b[3];
    double *x, *r, *t;
    double *diag;
    double *chol; /* coarsest level: Cholesky factor of -L (+ mean shift) */
    long n;
} mac_level;

typedef struct {
    int nlev;
    mac_level lev[OR_MAXLEV];
    int singular;
} mac_mg;

/* row of L at cell (i,j,k): neighbour cells and coefficients, diagonal */
static int mac_row(const or_geom *g, double *const *b, int i, int j, int k, long *nb, double *a, double *diag) {
    int c3[3] = {i, j, k};
    int cnt = 0;
    double dg = 0.0;
    double ih2 = 1.0 / (g->h * g->h);
    for (int d = 0; d < 3; d++) {
        for (int side = 0; side < 2; side++) {
            int p = c3[d] + side;
            int L, R;
            int has = face_cells(g, d, p, &L, &R);
            double bf = b[d][face_of_cell(g, d, i, j, k, p)];
            if (has == 3) {
                nb[cnt] = cell_along(g, d, i, j, k, side ? R : L);
                a[cnt] = bf * ih2;
                dg -= bf * ih2;
                cnt++;
            } else if (face_bc(g, d, p) == OR_DIRICHLET) {
                dg -= 2.0 * bf * ih2;
            }
        }
    }
    *diag = dg;
    return cnt;
}

/* Gauss-Seidel on L x = r, lexicographic, forward (dir=+1) or backward */
static void mac_gs(mac_level *lv, int dir) {
    const or_geom *g = &lv->g;
    long nb[6];
    double a[6], dg;
    long N = lv->n;
    for (long s = 0; s < N; s++) {
        long c = dir > 0 ? s : N - 1 - s;
        int i = (int)(c % g->n[0]);
        int j = (int)((c / g->n[0]) % g->n[1]);
        int k = (int)(c / ((long)g->n[0] * g->n[1]));
        int m = mac_row(g, lv->b, i, j, k, nb, a, &dg);
        double acc = lv->r[c];
        for (int q = 0; q < m; q++) acc -= a[q] * lv->x[nb[q]];
        lv->x[c] = acc / dg;
    }
}

static void mac_coarsen_faces(const or_geom *gf, double *const *bf, const or_geom *gc, double **bc) {
    for (int d = 0; d < 3; d++) {
        int m[3] = {gc->n[0], gc->n[1], gc->n[2]};
        m[d] += 1;
        for (int K = 0; K < m[2]; K++)
            for (int J = 0; J < m[1]; J++)
                for (int I = 0; I < m[0]; I++) {
                    int C[3] = {I, J, K};
                    double s = 0.0;
                    for (int u = 0; u < 2; u++)
                        for (int v = 0; v < 2; v++) {
                            int f3[3];
                            int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
                            f3[d] = 2 * C[d];
                            f3[t1] = 2 * C[t1] + u;
                            f3[t2] = 2 * C[t2] + v;
                            s += bf[d][fidx(gf, d, f3[0], f3[1], f3[2])];
                        }
                    bc[d][fidx(gc, d, I, J, K)] = 0.25 * s;
                }
    }
}

static int cholesky(long n, double *A) {
    for (long j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (long k = 0; k < j; k++) s -= A[j * n + k] * A[j * n + k];
        if (s <= 0.0) return -1;
        A[j * n + j] = sqrt(s);
        for (long i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (long k = 0; k < j; k++) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / A[j * n + j];
        }
    }
    return 0;
}

static void chol_solve(long n, const double *Lf, double *x) {
    for (long i = 0; i < n; i++) {
        double s = x[i];
        for (long k = 0; k < i; k++) s -= Lf[i * n + k] * x[k];
        x[i] = s / Lf[i * n + i];
    }
    for (long i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (long k = i + 1; k < n; k++) s -= Lf[k * n + i] * x[k];
        x[i] = s / Lf[i * n + i];
    }
}

#define OR_DENSE_MAX 1024

static void mac_mg_free(mac_mg *mg) {
    for (int l = 0; l < mg->nlev; l++) {
        mac_level *lv = &mg->lev[l];
        if (l > 0) for (int d = 0; d < 3; d++) free(lv->b[d]);
        free(lv->x); free(lv->r); free(lv->t); free(lv->chol);
    }
}

static int mac_mg_build(mac_mg *mg, const or_geom *g, const double *bx, const double *by, const double *bz) {
    memset(mg, 0, sizeof(*mg));
    mg->singular = or_singular(g);
    mac_level *lv = &mg->lev[0];
    lv->g = *g;
    lv->b[0] = (double *)bx; lv->b[1] = (double *)by; lv->b[2] = (double *)bz;
    int l = 0;
    for (;;) {
        lv = &mg->lev[l];
        lv->n = or_ncell(&lv->g);
        lv->x = (double *)calloc(lv->n, sizeof(double));
        lv->r = (double *)calloc(lv->n, sizeof(double));
        lv->t = (double *)calloc(lv->n, sizeof(double));
        mg->nlev = l + 1;
        int even = 1;
        for (int d = 0; d < 3; d++) even &= (lv->g.n[d] % 2 == 0) && lv->g.n[d] >= 2;
        if (!even || lv->n <= 64 || l + 1 >= OR_MAXLEV) break;
        mac_level *cv = &mg->lev[l + 1];
        cv->g = lv->g;
        for (int d = 0; d < 3; d++) cv->g.n[d] = lv->g.n[d] / 2;
        cv->g.h = 2.0 * lv->g.h;
        for (int d = 0; d < 3; d++) cv->b[d] = (double *)malloc(sizeof(double) * or_nface(&cv->g, d));
        mac_coarsen_faces(&lv->g, lv->b, &cv->g, cv->b);
        l++;
    }
    lv = &mg->lev[mg->nlev - 1];
    if (lv->n <= OR_DENSE_MAX) {
        long n = lv->n;
        lv->chol = (double *)malloc(sizeof(double) * n * n);
        double *e = (double *)calloc(n, sizeof(double));
        double *col = (double *)malloc(sizeof(double) * n);
        double shift = 0.0;
        for (long j = 0; j < n; j++) {
            e[j] = 1.0;
            or_mac_apply(&lv->g, lv->b[0], lv->b[1], lv->b[2], e, col);
            e[j] = 0.0;
            for (long i = 0; i < n; i++) lv->chol[i * n + j] = -col[i];
            shift = fmax(shift, -col[j]);
        }
        /* singular: A + shift * 11^T/n is SPD and agrees with A on mean-free vectors */
        if (mg->singular)
            for (long i = 0; i < n * n; i++) lv->chol[i] += shift / (double)n;
        free(e); free(col);
        if (cholesky(n, lv->chol)) { mac_mg_free(mg); return -1; }
    }
    return 0;
}

static void mac_vcycle(mac_mg *mg, int l) {
    mac_level *lv = &mg->lev[l];
    if (l == mg->nlev - 1) {
        if (lv->chol) {
            memcpy(lv->x, lv->r, sizeof(double) * lv->n);
            if (mg->singular) remove_mean(lv->n, lv->x);
            /* x holds -r: we factored -L */
            for (long c = 0; c < lv->n; c++) lv->x[c] = -lv->x[c];
            chol_solve(lv->n, lv->chol, lv->x);
            if (mg->singular) remove_mean(lv->n, lv->x);
        } else {
            memset(lv->x, 0, sizeof(double) * lv->n);
            for (int s = 0; s < 20; s++) { mac_gs(lv, +1); mac_gs(lv, -1); }
        }
        return;
    }
    memset(lv->x, 0, sizeof(double) * lv->n);
    mac_gs(lv, +1);
    mac_gs(lv, +1);
    or_mac_apply(&lv->g, lv->b[0], lv->b[1], lv->b[2], lv->x, lv->t);
    for (long c = 0; c < lv->n; c++) lv->t[c] = lv->r[c] - lv->t[c];
    mac_level *cv = &mg->lev[l + 1];
    const or_geom *gc = &cv->g;
    for (int K = 0; K < gc->n[2]; K++)
        for (int J = 0; J < gc->n[1]; J++)
            for (int I = 0; I < gc->n[0]; I++) {
                double s = 0.0;
                for (int dk = 0; dk < 2; dk++)
                    for (int dj = 0; dj < 2; dj++)
                        for (int di = 0; di < 2; di++)
                            s += lv->t[cidx(&lv->g, 2 * I + di, 2 * J + dj, 2 * K + dk)];
                cv->r[cidx(gc, I, J, K)] = s / 8.0;
            }
    mac_vcycle(mg, l + 1);
    for (int k = 0; k < lv->g.n[2]; k++)
        for (int j = 0; j < lv->g.n[1]; j++)
            for (int i = 0; i < lv->g.n[0]; i++)
                lv->x[cidx(&lv->g, i, j, k)] += cv->x[cidx(gc, i / 2, j / 2, k / 2)];
    mac_gs(lv, -1);
    mac_gs(lv, -1);
}

/* Solve L phi = f to ||f - L phi||_inf <= tol ||f||_inf.  phi holds the initial
 * guess on entry.  For singular problems the returned phi has zero mean.
 * Returns the iteration count, or -1 if maxit was reached. */
int or_mac_solve(const or_geom *g, const double *bx, const double *by, const double *bz,
                 const double *f, double *phi, double tol, int maxit, double *relres) {
    mac_mg mg;
    if (mac_mg_build(&mg, g, bx, by, bz)) return -2;
    long N = or_ncell(g);
    double *r = (double *)malloc(sizeof(double) * N);
    double *z = (double *)malloc(sizeof(double) * N);
    double *p = (double *)malloc(sizeof(double) * N);
    double *q = (double *)malloc(sizeof(double) * N);
    double fn = or_norm_inf(N, f);
    int it = 0, ok = 0;
    double rz = 0.0;
    if (mg.singular) remove_mean(N, phi);
    for (it = 0; it <= maxit; it++) {
        /* true residual of the A-system, A = -L, b = -f:  s = b - A phi = L phi - f */
        or_mac_apply(g, bx, by, bz, phi, r);
        for (long c = 0; c < N; c++) r[c] = r[c] - f[c];
        double rn = or_norm_inf(N, r);
        if (relres) *relres = fn > 0 ? rn / fn : rn;
        if (rn <= tol * fn || rn == 0.0) { ok = 1; break; }
        if (it == maxit) break;
        /* preconditioner: one V-cycle on L e = -s, i.e. z = A^-1 s approximately */
        mac_level *lv = &mg.lev[0];
        for (long c = 0; c < N; c++) lv->r[c] = -r[c];
        if (mg.singular) remove_mean(N, lv->r);
        mac_vcycle(&mg, 0);
        memcpy(z, lv->x, sizeof(double) * N);
        if (mg.singular) remove_mean(N, z);
        double rz_new = dot(N, r, z);
        if (it == 0) memcpy(p, z, sizeof(double) * N);
        else {
            double beta = rz_new / rz;
            for (long c = 0; c < N; c++) p[c] = z[c] + beta * p[c];
        }
        rz = rz_new;
        or_mac_apply(g, bx, by, bz, p, q);
        for (long c = 0; c < N; c++) q[c] = -q[c];  /* q = A p */
        double alpha = rz / dot(N, p, q);
        for (long c = 0; c < N; c++) phi[c] += alpha * p[c];
    }
    if (mg.singular) remove_mean(N, phi);
    free(r); free(z); free(p); free(q);
    mac_mg_free(&mg);
    return ok ? it : -1;
}

/* One full MAC projection: coefficients, RHS, solve, correction, divergence
 * check.  u* are overwritten with the projected velocity.  out[0] = removed
 * mean c, out[1] = relative residual, out[2] = max |D(beta0 U) - beta0 Sbar - c|,
 * out[3] = iterations. */
int or_mac_project(const or_geom *g, double *ux, double *uy, double *uz, const double *rho,
                   const double *beta0, const double *sbar, double *phi, double tol, int maxit,
                   int remove_mean_flag, double *out) {
    long N = or_ncell(g);
    double *b[3];
    for (int d = 0; d < 3; d++) b[d] = (double *)malloc(sizeof(double) * or_nface(g, d));
    double *f = (double *)malloc(sizeof(double) * N);
    double *dv = (double *)malloc(sizeof(double) * N);
    or_mac_coeffs(g, rho, beta0, b[0], b[1], b[2]);
    double c = 0.0, rr = 0.0;
    or_mac_rhs(g, ux, uy, uz, beta0, sbar, remove_mean_flag, f, &c);
    int it = or_mac_solve(g, b[0], b[1], b[2], f, phi, tol, maxit, &rr);
    or_mac_correct(g, rho, phi, ux, uy, uz);
    or_mac_divergence(g, ux, uy, uz, beta0, dv);
    double e = 0.0;
    for (long q = 0; q < N; q++) e = fmax(e, fabs(dv[q] - beta0[q] * sbar[q] - c));
    out[0] = c; out[1] = rr; out[2] = e; out[3] = it;
    for (int d = 0; d < 3; d++) free(b[d]);
    free(f); free(dv);
    return it < 0 ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Sampled outputs for large grids: the residual f - L phi and the divergence
 * D(beta0 U) at a list of cells, computed one cell at a time from the inputs
 * with the same definitions as the full-array functions above.              */

static double face_b_direct(const or_geom *g, const double *rho, const double *beta0, int d, int i, int j, int k, int p) {
    int L, R;
    int has = face_cells(g, d, p, &L, &R);
    if (has == 3) {
        long cl = cell_along(g, d, i, j, k, L), cr = cell_along(g, d, i, j, k, R);
        return (0.5 * (beta0[cl] + beta0[cr])) / (0.5 * (rho[cl] + rho[cr]));
    }
    if (face_bc(g, d, p) == OR_DIRICHLET) {
        long c = cell_along(g, d, i, j, k, has == 2 ? R : L);
        return beta0[c] / rho[c];
    }
    return 0.0;
}

/* r[q] = f[c] - (L phi)_c at cells idx[q] */
void or_mac_residual_sample(const or_geom *g, const double *rho, const double *beta0, const double *phi,
                            const double *f, const long *idx, long n, double *r) {
    for (long q = 0; q < n; q++) {
        long c = idx[q];
        int i = (int)(c % g->n[0]), j = (int)((c / g->n[0]) % g->n[1]), k = (int)(c / ((long)g->n[0] * g->n[1]));
        int c3[3] = {i, j, k};
        double s = 0.0;
        for (int d = 0; d < 3; d++) {
            int plo = c3[d], phi_ = c3[d] + 1;
            double flo = face_b_direct(g, rho, beta0, d, i, j, k, plo) * face_grad(g, phi, d, i, j, k, plo);
            double fhi = face_b_direct(g, rho, beta0, d, i, j, k, phi_) * face_grad(g, phi, d, i, j, k, phi_);
            s += (fhi - flo) / g->h;
        }
        r[q] = f[c] - s;
    }
}

/* out[q] = D(beta0 U) at cells idx[q] */
void or_mac_divergence_sample(const or_geom *g, const double *ux, const double *uy, const double *uz,
                              const double *beta0, const long *idx, long n, double *out) {
    const double *u[3] = {ux, uy, uz};
    for (long q = 0; q < n; q++) {
        long c = idx[q];
        int i = (int)(c % g->n[0]), j = (int)((c / g->n[0]) % g->n[1]), k = (int)(c / ((long)g->n[0] * g->n[1]));
        int c3[3] = {i, j, k};
        double s = 0.0;
        for (int d = 0; d < 3; d++) {
            int plo = c3[d], phi_ = c3[d] + 1;
            double flo = face_beta(g, beta0, d, i, j, k, plo) * u[d][face_of_cell(g, d, i, j, k, plo)];
            double fhi = face_beta(g, beta0, d, i, j, k, phi_) * u[d][face_of_cell(g, d, i, j, k, phi_)];
            s += (fhi - flo) / g->h;
        }
        out[q] = s;
    }
}
