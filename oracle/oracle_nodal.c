/*
 * FP64 CPU oracle, nodal projection (Step 11 of Sec. 3.2, Eq. div3; Appendix A).
 * TEST INFRASTRUCTURE ONLY (see oracle.c).
 *
 * Reading of the nodal discretisation (the paper defers it to Paper III):
 *   - phi lives on nodes; a periodic axis with n cells has n nodes, a wall
 *     (Neumann) axis has n+1 nodes including both walls;
 *   - node weight w = (number of cells touching the node)/8;
 *   - (L phi)_n = 1/(w_n h^2) sum_{cells c at n} sigma_c sum_{corners m of c}
 *     a(n,m) phi_m, the trilinear finite-element stiffness on a cube:
 *     a = -1/3 on the diagonal, 0 between corners differing in one index,
 *     +1/12 between corners differing in two or three indices;
 *   - divergence of cell-centred V:
 *     (D V)_n = 1/(4 h w_n) sum_{c at n} sum_d s_d(c,n) V_{d,c}, s = +1 when
 *     the cell lies on the +d side of the node;
 *   - cell gradient (G phi)_{d,c} = 1/(4h) sum over the 4 d-edges of c of
 *     (phi_hi - phi_lo);
 *   - nodal Sbar = mean over the touching cells of beta0 Sbar;
 *   - the weighted mean sum_n w_n f_n is removed; phi normalised to
 *     sum_n w_n phi_n = 0.
 */
#include <math.h>
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

typedef void (*or_apply_fn)(const void *ctx, const double *x, double *y);
int or_dense_solve(long n, or_apply_fn apply, const void *ctx, const double *f, double *x,
                   long pin_row, const double *w);
double or_norm_inf(long n, const double *a);

static int nnodes_axis(const or_geom *g, int d) {
    return g->n[d] + (g->lo[d] == OR_PERIODIC ? 0 : 1);
}

long or_nd_nnode(const or_geom *g) {
    return (long)nnodes_axis(g, 0) * nnodes_axis(g, 1) * nnodes_axis(g, 2);
}

static long nidx(const or_geom *g, int a, int b, int c) {
    return (long)a + (long)nnodes_axis(g, 0) * ((long)b + (long)nnodes_axis(g, 1) * c);
}

static long ccidx(const or_geom *g, int i, int j, int k) {
    return (long)i + (long)g->n[0] * ((long)j + (long)g->n[1] * k);
}

/* node coordinate of corner e (0/1) of cell index i along d, wrapping periodic axes */
static int corner(const or_geom *g, int d, int i, int e) {
    int a = i + e;
    if (g->lo[d] == OR_PERIODIC && a == g->n[d]) a = 0;
    return a;
}

/* corner-pair stiffness of the unit cube Q1 element, with the sign of L */
static double elem_a(int e1, int e2) {
    int diff = e1 ^ e2;
    int cnt = (diff & 1) + ((diff >> 1) & 1) + ((diff >> 2) & 1);
    if (cnt == 0) return -1.0 / 3.0;
    if (cnt == 1) return 0.0;
    return 1.0 / 12.0;
}

static long corner_node(const or_geom *g, int i, int j, int k, int e) {
    return nidx(g, corner(g, 0, i, e & 1), corner(g, 1, j, (e >> 1) & 1), corner(g, 2, k, (e >> 2) & 1));
}

/* number of cells touching each node */
static void node_counts(const or_geom *g, double *cnt) {
    long M = or_nd_nnode(g);
    for (long q = 0; q < M; q++) cnt[q] = 0.0;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++)
                for (int e = 0; e < 8; e++) cnt[corner_node(g, i, j, k, e)] += 1.0;
}

void or_nd_weights(const or_geom *g, double *w) {
    node_counts(g, w);
    long M = or_nd_nnode(g);
    for (long q = 0; q < M; q++) w[q] /= 8.0;
}

void or_nd_apply(const or_geom *g, const double *sigma, const double *phi, double *out) {
    long M = or_nd_nnode(g);
    double *w = (double *)malloc(sizeof(double) * M);
    or_nd_weights(g, w);
    for (long q = 0; q < M; q++) out[q] = 0.0;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                double s = sigma[ccidx(g, i, j, k)];
                for (int e1 = 0; e1 < 8; e1++) {
                    double acc = 0.0;
                    for (int e2 = 0; e2 < 8; e2++) acc += elem_a(e1, e2) * phi[corner_node(g, i, j, k, e2)];
                    out[corner_node(g, i, j, k, e1)] += s * acc;
                }
            }
    for (long q = 0; q < M; q++) out[q] /= w[q] * g->h * g->h;
    free(w);
}

/* nodal divergence of the cell-centred field (vx, vy, vz) */
void or_nd_divergence(const or_geom *g, const double *vx, const double *vy, const double *vz, double *out) {
    long M = or_nd_nnode(g);
    const double *v[3] = {vx, vy, vz};
    double *w = (double *)malloc(sizeof(double) * M);
    or_nd_weights(g, w);
    for (long q = 0; q < M; q++) out[q] = 0.0;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                long c = ccidx(g, i, j, k);
                for (int e = 0; e < 8; e++) {
                    double s = 0.0;
                    for (int d = 0; d < 3; d++) {
                        /* node is the cell's lower corner along d -> cell on the +d side */
                        double sg = ((e >> d) & 1) ? -1.0 : 1.0;
                        s += sg * v[d][c];
                    }
                    out[corner_node(g, i, j, k, e)] += s;
                }
            }
    for (long q = 0; q < M; q++) out[q] /= 4.0 * g->h * w[q];
    free(w);
}

/* cell gradient of nodal phi: G[d][c] */
void or_nd_gradient(const or_geom *g, const double *phi, double *gx, double *gy, double *gz) {
    double *G[3] = {gx, gy, gz};
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                long c = ccidx(g, i, j, k);
                for (int d = 0; d < 3; d++) {
                    double s = 0.0;
                    for (int e = 0; e < 8; e++) {
                        if ((e >> d) & 1) continue;
                        int e_hi = e | (1 << d);
                        s += phi[corner_node(g, i, j, k, e_hi)] - phi[corner_node(g, i, j, k, e)];
                    }
                    G[d][c] = s / (4.0 * g->h);
                }
            }
}

/* f = D(beta0 U) - Sbar_n, Sbar_n = mean of beta0 Sbar over the touching cells;
 * the weighted mean is removed when remove_mean != 0 */
void or_nd_rhs(const or_geom *g, const double *ux, const double *uy, const double *uz,
               const double *beta0, const double *sbar, int remove_mean, double *f, double *mean) {
    long N = (long)g->n[0] * g->n[1] * g->n[2], M = or_nd_nnode(g);
    double *bv[3];
    const double *u[3] = {ux, uy, uz};
    for (int d = 0; d < 3; d++) {
        bv[d] = (double *)malloc(sizeof(double) * N);
        for (long c = 0; c < N; c++) bv[d][c] = beta0[c] * u[d][c];
    }
    or_nd_divergence(g, bv[0], bv[1], bv[2], f);
    double *cnt = (double *)malloc(sizeof(double) * M);
    double *sn = (double *)calloc(M, sizeof(double));
    node_counts(g, cnt);
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                long c = ccidx(g, i, j, k);
                for (int e = 0; e < 8; e++) sn[corner_node(g, i, j, k, e)] += beta0[c] * sbar[c];
            }
    for (long q = 0; q < M; q++) f[q] -= sn[q] / cnt[q];
    double m = 0.0;
    if (remove_mean) {
        double sw = 0.0, sf = 0.0;
        for (long q = 0; q < M; q++) { sw += cnt[q] / 8.0; sf += cnt[q] / 8.0 * f[q]; }
        m = sf / sw;
        for (long q = 0; q < M; q++) f[q] -= m;
    }
    if (mean) *mean = m;
    for (int d = 0; d < 3; d++) free(bv[d]);
    free(cnt); free(sn);
}

void or_nd_correct(const or_geom *g, const double *rho, const double *phi,
                   double *ux, double *uy, double *uz) {
    long N = (long)g->n[0] * g->n[1] * g->n[2];
    double *G[3];
    double *u[3] = {ux, uy, uz};
    for (int d = 0; d < 3; d++) G[d] = (double *)malloc(sizeof(double) * N);
    or_nd_gradient(g, phi, G[0], G[1], G[2]);
    for (int d = 0; d < 3; d++)
        for (long c = 0; c < N; c++) u[d][c] -= G[d][c] / rho[c];
    for (int d = 0; d < 3; d++) free(G[d]);
}

typedef struct { const or_geom *g; const double *sigma; } nd_ctx;

static void nd_apply_cb(const void *v, const double *x, double *y) {
    const nd_ctx *c = (const nd_ctx *)v;
    or_nd_apply(c->g, c->sigma, x, y);
}

int or_nd_dense_solve(const or_geom *g, const double *sigma, const double *f, double *phi) {
    long M = or_nd_nnode(g);
    double *w = (double *)malloc(sizeof(double) * M);
    or_nd_weights(g, w);
    nd_ctx c = {g, sigma};
    int rc = or_dense_solve(M, nd_apply_cb, &c, f, phi, 0, w);
    free(w);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Multigrid-preconditioned CG on A = -W L (symmetric, semidefinite).  V-cycle:
 * lexicographic Gauss-Seidel forward/backward, trilinear prolongation P,
 * restriction P^T/8 (the nested finite-element spaces give
 * P^T A_h P = 8 A_2h for sigma constant on coarse cells), coarse sigma = mean
 * of the 8 fine cells, dense coarsest solve.                                 */

#define ND_MAXLEV 24
#define ND_DENSE_MAX 1200

typedef struct {
    or_geom g;
    double *sigma;
    double *w;
    double *x, *r, *t;
    double *chol;
    long m;
} nd_level;

typedef struct { int nlev; nd_level lev[ND_MAXLEV]; } nd_mg;

/* row of A = -W L at node (a,b,c): 27 offsets, coefficients of phi */
static void nd_row(const or_geom *g, const double *sigma, int a, int b, int c, double *coef, long *nb) {
    int p[3] = {a, b, c};
    for (int q = 0; q < 27; q++) { coef[q] = 0.0; nb[q] = -1; }
    double ih2 = 1.0 / (g->h * g->h);
    for (int dz = -1; dz <= 0; dz++)
        for (int dy = -1; dy <= 0; dy++)
            for (int dx = -1; dx <= 0; dx++) {
                int del[3] = {dx, dy, dz}, cell[3];
                int ok = 1;
                for (int d = 0; d < 3; d++) {
                    cell[d] = p[d] + del[d];
                    if (g->lo[d] == OR_PERIODIC) {
                        if (cell[d] < 0) cell[d] += g->n[d];
                    } else if (cell[d] < 0 || cell[d] >= g->n[d]) ok = 0;
                }
                if (!ok) continue;
                double s = sigma[ccidx(g, cell[0], cell[1], cell[2])];
                int e_n = (-dx) | ((-dy) << 1) | ((-dz) << 2);   /* node's corner in this cell */
                for (int e = 0; e < 8; e++) {
                    int off[3] = {del[0] + (e & 1), del[1] + ((e >> 1) & 1), del[2] + ((e >> 2) & 1)};
                    int q = (off[0] + 1) + 3 * ((off[1] + 1) + 3 * (off[2] + 1));
                    coef[q] += -s * elem_a(e_n, e) * ih2;
                    nb[q] = corner_node(g, cell[0], cell[1], cell[2], e);
                }
            }
}

static void nd_gs(nd_level *lv, int dir) {
    const or_geom *g = &lv->g;
    int mx = nnodes_axis(g, 0), my = nnodes_axis(g, 1);
    double coef[27];
    long nb[27];
    for (long s = 0; s < lv->m; s++) {
        long q = dir > 0 ? s : lv->m - 1 - s;
        int a = (int)(q % mx), b = (int)((q / mx) % my), c = (int)(q / ((long)mx * my));
        nd_row(g, lv->sigma, a, b, c, coef, nb);
        double acc = lv->r[q], dg = coef[13];
        for (int o = 0; o < 27; o++)
            if (o != 13 && nb[o] >= 0) acc -= coef[o] * lv->x[nb[o]];
        lv->x[q] = acc / dg;
    }
}

/* y = A x with A = -W L (the weak-form matrix divided by h^3) */
static void nd_applyA(const nd_level *lv, const double *x, double *y) {
    or_nd_apply(&lv->g, lv->sigma, x, y);
    for (long q = 0; q < lv->m; q++) y[q] = -lv->w[q] * y[q];
}

static int nd_fine_to_coarse(int af, int *ac, double *wt) {
    /* returns the number of coarse parents along one axis */
    if ((af & 1) == 0) { ac[0] = af / 2; wt[0] = 1.0; return 1; }
    ac[0] = (af - 1) / 2; ac[1] = (af + 1) / 2; wt[0] = wt[1] = 0.5;
    return 2;
}

static int cholesky_nd(long n, double *A) {
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

static void chol_solve_nd(long n, const double *Lf, double *x) {
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

static void plain_mean0(long n, double *a) {
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i];
    s /= (double)n;
    for (long i = 0; i < n; i++) a[i] -= s;
}

static void nd_mg_free(nd_mg *mg) {
    for (int l = 0; l < mg->nlev; l++) {
        nd_level *lv = &mg->lev[l];
        if (l > 0) free(lv->sigma);
        free(lv->w); free(lv->x); free(lv->r); free(lv->t); free(lv->chol);
    }
}

static int nd_mg_build(nd_mg *mg, const or_geom *g, const double *sigma) {
    memset(mg, 0, sizeof(*mg));
    mg->lev[0].g = *g;
    mg->lev[0].sigma = (double *)sigma;
    int l = 0;
    for (;;) {
        nd_level *lv = &mg->lev[l];
        lv->m = or_nd_nnode(&lv->g);
        lv->w = (double *)malloc(sizeof(double) * lv->m);
        or_nd_weights(&lv->g, lv->w);
        lv->x = (double *)calloc(lv->m, sizeof(double));
        lv->r = (double *)calloc(lv->m, sizeof(double));
        lv->t = (double *)calloc(lv->m, sizeof(double));
        mg->nlev = l + 1;
        int even = 1;
        for (int d = 0; d < 3; d++) even &= (lv->g.n[d] % 2 == 0) && lv->g.n[d] >= 4;
        if (!even || lv->m <= 64 || l + 1 >= ND_MAXLEV) break;
        nd_level *cv = &mg->lev[l + 1];
        cv->g = lv->g;
        for (int d = 0; d < 3; d++) cv->g.n[d] = lv->g.n[d] / 2;
        cv->g.h = 2.0 * lv->g.h;
        long Nc = (long)cv->g.n[0] * cv->g.n[1] * cv->g.n[2];
        cv->sigma = (double *)malloc(sizeof(double) * Nc);
        for (int K = 0; K < cv->g.n[2]; K++)
            for (int J = 0; J < cv->g.n[1]; J++)
                for (int I = 0; I < cv->g.n[0]; I++) {
                    double s = 0.0;
                    for (int e = 0; e < 8; e++)
                        s += lv->sigma[ccidx(&lv->g, 2 * I + (e & 1), 2 * J + ((e >> 1) & 1), 2 * K + ((e >> 2) & 1))];
                    cv->sigma[ccidx(&cv->g, I, J, K)] = s / 8.0;
                }
        l++;
    }
    nd_level *lv = &mg->lev[mg->nlev - 1];
    if (lv->m <= ND_DENSE_MAX) {
        long n = lv->m;
        lv->chol = (double *)malloc(sizeof(double) * n * n);
        double *e = (double *)calloc(n, sizeof(double));
        double *col = (double *)malloc(sizeof(double) * n);
        double shift = 0.0;
        for (long j = 0; j < n; j++) {
            e[j] = 1.0;
            nd_applyA(lv, e, col);
            e[j] = 0.0;
            for (long i = 0; i < n; i++) lv->chol[i * n + j] = col[i];
            shift = fmax(shift, col[j]);
        }
        for (long i = 0; i < n * n; i++) lv->chol[i] += shift / (double)n;
        free(e); free(col);
        if (cholesky_nd(n, lv->chol)) { nd_mg_free(mg); return -1; }
    }
    return 0;
}

/* V-cycle on A x = r (A = -W L) */
static void nd_vcycle(nd_mg *mg, int l) {
    nd_level *lv = &mg->lev[l];
    if (l == mg->nlev - 1) {
        if (lv->chol) {
            memcpy(lv->x, lv->r, sizeof(double) * lv->m);
            plain_mean0(lv->m, lv->x);
            chol_solve_nd(lv->m, lv->chol, lv->x);
            plain_mean0(lv->m, lv->x);
        } else {
            memset(lv->x, 0, sizeof(double) * lv->m);
            for (int s = 0; s < 20; s++) { nd_gs(lv, +1); nd_gs(lv, -1); }
        }
        return;
    }
    memset(lv->x, 0, sizeof(double) * lv->m);
    nd_gs(lv, +1);
    nd_gs(lv, +1);
    nd_applyA(lv, lv->x, lv->t);
    for (long q = 0; q < lv->m; q++) lv->t[q] = lv->r[q] - lv->t[q];
    nd_level *cv = &mg->lev[l + 1];
    memset(cv->r, 0, sizeof(double) * cv->m);
    int mx = nnodes_axis(&lv->g, 0), my = nnodes_axis(&lv->g, 1), mz = nnodes_axis(&lv->g, 2);
    int cmx = nnodes_axis(&cv->g, 0), cmy = nnodes_axis(&cv->g, 1), cmz = nnodes_axis(&cv->g, 2);
    for (int c = 0; c < mz; c++)
        for (int b = 0; b < my; b++)
            for (int a = 0; a < mx; a++) {
                int ia[2], ib[2], ic[2];
                double wa[2], wb[2], wc[2];
                int na = nd_fine_to_coarse(a, ia, wa), nb_ = nd_fine_to_coarse(b, ib, wb), nc = nd_fine_to_coarse(c, ic, wc);
                double v = lv->t[nidx(&lv->g, a, b, c)];
                for (int u = 0; u < nc; u++)
                    for (int s = 0; s < nb_; s++)
                        for (int t = 0; t < na; t++) {
                            int A_ = ia[t] % cmx, B_ = ib[s] % cmy, C_ = ic[u] % cmz;
                            cv->r[nidx(&cv->g, A_, B_, C_)] += wa[t] * wb[s] * wc[u] * v / 8.0;
                        }
            }
    nd_vcycle(mg, l + 1);
    for (int c = 0; c < mz; c++)
        for (int b = 0; b < my; b++)
            for (int a = 0; a < mx; a++) {
                int ia[2], ib[2], ic[2];
                double wa[2], wb[2], wc[2];
                int na = nd_fine_to_coarse(a, ia, wa), nb_ = nd_fine_to_coarse(b, ib, wb), nc = nd_fine_to_coarse(c, ic, wc);
                double s_ = 0.0;
                for (int u = 0; u < nc; u++)
                    for (int s = 0; s < nb_; s++)
                        for (int t = 0; t < na; t++) {
                            int A_ = ia[t] % cmx, B_ = ib[s] % cmy, C_ = ic[u] % cmz;
                            s_ += wa[t] * wb[s] * wc[u] * cv->x[nidx(&cv->g, A_, B_, C_)];
                        }
                lv->x[nidx(&lv->g, a, b, c)] += s_;
            }
    nd_gs(lv, -1);
    nd_gs(lv, -1);
}

static void weighted_mean0(long n, const double *w, double *a) {
    double sw = 0.0, s = 0.0;
    for (long i = 0; i < n; i++) { sw += w[i]; s += w[i] * a[i]; }
    s /= sw;
    for (long i = 0; i < n; i++) a[i] -= s;
}

/* Solve L phi = f (f weighted-mean-free) to ||f - L phi||_inf <= tol ||f||_inf,
 * phi normalised to zero weighted mean.  Returns iterations or -1. */
int or_nd_solve(const or_geom *g, const double *sigma, const double *f, double *phi,
                double tol, int maxit, double *relres) {
    nd_mg mg;
    if (nd_mg_build(&mg, g, sigma)) return -2;
    nd_level *top = &mg.lev[0];
    long M = top->m;
    double *s = (double *)malloc(sizeof(double) * M);
    double *z = (double *)malloc(sizeof(double) * M);
    double *p = (double *)malloc(sizeof(double) * M);
    double *q = (double *)malloc(sizeof(double) * M);
    double *lf = (double *)malloc(sizeof(double) * M);
    double fn = or_norm_inf(M, f);
    double rz = 0.0;
    int it, ok = 0;
    for (it = 0; it <= maxit; it++) {
        or_nd_apply(g, sigma, phi, lf);
        double rn = 0.0;
        for (long k = 0; k < M; k++) {
            double r = f[k] - lf[k];
            rn = fmax(rn, fabs(r));
            s[k] = -top->w[k] * r;   /* residual of A phi = b, b = -W f */
        }
        if (relres) *relres = fn > 0 ? rn / fn : rn;
        if (rn <= tol * fn || rn == 0.0) { ok = 1; break; }
        if (it == maxit) break;
        memcpy(top->r, s, sizeof(double) * M);
        plain_mean0(M, top->r);
        nd_vcycle(&mg, 0);
        memcpy(z, top->x, sizeof(double) * M);
        plain_mean0(M, z);
        double rz_new = 0.0;
        for (long k = 0; k < M; k++) rz_new += s[k] * z[k];
        if (it == 0) memcpy(p, z, sizeof(double) * M);
        else {
            double beta = rz_new / rz;
            for (long k = 0; k < M; k++) p[k] = z[k] + beta * p[k];
        }
        rz = rz_new;
        nd_applyA(top, p, q);
        double pq = 0.0;
        for (long k = 0; k < M; k++) pq += p[k] * q[k];
        double alpha = rz / pq;
        for (long k = 0; k < M; k++) phi[k] += alpha * p[k];
    }
    weighted_mean0(M, top->w, phi);
    free(s); free(z); free(p); free(q); free(lf);
    nd_mg_free(&mg);
    return ok ? it : -1;
}

/* Full nodal projection.  u* (cell fields) are overwritten.  out[0] = removed
 * weighted mean c, out[1] = relative residual, out[2] = max over nodes of
 * |D(beta0 U) - Sbar_n - c| (an O(h^2) quantity: the projection is
 * approximate), out[3] = iterations. */
int or_nd_project(const or_geom *g, double *ux, double *uy, double *uz, const double *rho,
                  const double *beta0, const double *sbar, double *phi, double tol, int maxit,
                  double *out) {
    long N = (long)g->n[0] * g->n[1] * g->n[2], M = or_nd_nnode(g);
    double *sigma = (double *)malloc(sizeof(double) * N);
    double *f = (double *)malloc(sizeof(double) * M);
    double *d = (double *)malloc(sizeof(double) * M);
    for (long c = 0; c < N; c++) sigma[c] = beta0[c] / rho[c];
    double cm = 0.0, rr = 0.0;
    or_nd_rhs(g, ux, uy, uz, beta0, sbar, 1, f, &cm);
    int it = or_nd_solve(g, sigma, f, phi, tol, maxit, &rr);
    or_nd_correct(g, rho, phi, ux, uy, uz);
    double c2 = 0.0;
    or_nd_rhs(g, ux, uy, uz, beta0, sbar, 0, d, &c2);
    double e = 0.0;
    for (long q = 0; q < M; q++) e = fmax(e, fabs(d[q] - cm));
    out[0] = cm; out[1] = rr; out[2] = e; out[3] = it;
    free(sigma); free(f); free(d);
    return it < 0 ? -1 : 0;
}

/* Sampled nodal residual f - L phi at nodes idx[q] (same definition as
 * or_nd_apply, evaluated node by node). */
void or_nd_residual_sample(const or_geom *g, const double *sigma, const double *phi, const double *f,
                           const long *idx, long n, double *r) {
    int mx = nnodes_axis(g, 0), my = nnodes_axis(g, 1);
    for (long q = 0; q < n; q++) {
        long nd = idx[q];
        int a = (int)(nd % mx), b = (int)((nd / mx) % my), c = (int)(nd / ((long)mx * my));
        double acc = 0.0, cnt = 0.0;
        for (int dz = -1; dz <= 0; dz++)
            for (int dy = -1; dy <= 0; dy++)
                for (int dx = -1; dx <= 0; dx++) {
                    int cell[3] = {a + dx, b + dy, c + dz}, ok = 1;
                    for (int d = 0; d < 3; d++) {
                        if (g->lo[d] == OR_PERIODIC) {
                            if (cell[d] < 0) cell[d] += g->n[d];
                        } else if (cell[d] < 0 || cell[d] >= g->n[d]) ok = 0;
                    }
                    if (!ok) continue;
                    cnt += 1.0;
                    double s = sigma[ccidx(g, cell[0], cell[1], cell[2])];
                    int e_n = (-dx) | ((-dy) << 1) | ((-dz) << 2);
                    double inner = 0.0;
                    for (int e = 0; e < 8; e++)
                        inner += elem_a(e_n, e) * phi[corner_node(g, cell[0], cell[1], cell[2], e)];
                    acc += s * inner;
                }
        r[q] = f[nd] - acc / ((cnt / 8.0) * g->h * g->h);
    }
}
