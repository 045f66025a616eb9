/*
 * FP64 CPU oracle for the base-state mapping modules of MAESTROeX (Sec. 3.1):
 * the lateral average (Cartesian cells -> 1D base state) and the fill
 * (1D base state -> Cartesian cells); and for the velocity split of Appendix A
 * (the w0 integration, w0 e_r on the MAC faces, the S - Sbar bracket).
 *
 * TEST INFRASTRUCTURE ONLY (the tests, the smoke check and the benchmark's CPU
 * legs load it).  Shares nothing with the CUDA library.  Plain loops, double
 * precision, single threaded.
 *
 * Definitions (Sec. 3.1; Eq. radii):
 *   - planar average: the arithmetic mean of the cells at each height k;
 *   - spherical geometry with the star's centre on a cell corner (corner index
 *     c = (c0, c1, c2): the centre sits at x_d = c_d dx): the centre of cell
 *     (i, j, k) lies at offsets (a + 1/2, b + 1/2, e + 1/2) dx with a = i - c0,
 *     b = j - c1, e = k - c2, so its radius is dx sqrt(0.75 + 2m) with
 *         m = (a (a + 1) + b (b + 1) + e (e + 1)) / 2   (an integer);
 *     the irregular base state holds, for each m, the mean of the cells of that
 *     radius (with their count), and its fill gives every cell the value of
 *     its own m (no interpolation);
 *   - the uniform base state (radial cells (j + 1/2) dr): its fill assigns each
 *     cell centre the quadratic (3-point Lagrange) interpolant through three
 *     consecutive radial cell centres, centred on the one nearest to the
 *     cell's radius (the radial cell containing it), shifted inward at the
 *     first and last radial cell; the average onto it interpolates the
 *     irregular means quadratically the same way: through the non-empty radius
 *     nearest to each uniform radius (the smaller one on a tie) and its two
 *     non-empty neighbours.
 */
#include <math.h>
#include <stdlib.h>

typedef struct {
    int n[3];
    double dx;
    int lo[3], hi[3];
} or_geom;

/* ---- planar ----------------------------------------------------------------------- */
void or_average_planar(const or_geom *g, const double *field, double *out) {
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    for (int k = 0; k < nz; k++) {
        double s = 0.0;
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) s += field[i + (long)nx * (j + (long)ny * k)];
        out[k] = s / ((double)nx * ny);
    }
}

/* ---- spherical, irregular base state ------------------------------------------------- */
long or_radial_m(int i, int j, int k, const int *corner) {
    const long a = i - corner[0], b = j - corner[1], e = k - corner[2];
    return (a * (a + 1) + b * (b + 1) + e * (e + 1)) / 2;
}

long or_radial_nbins(const or_geom *g, const int *corner) {
    long mmax = 0;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                const long m = or_radial_m(i, j, k, corner);
                if (m > mmax) mmax = m;
            }
    return mmax + 1;
}

void or_radial_index(const or_geom *g, const int *corner, long *m_out) {
    long c = 0;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) m_out[c++] = or_radial_m(i, j, k, corner);
}

/* mean over the cells of each radius; bins without cells get 0 */
void or_average_radial(const or_geom *g, const int *corner, const double *field, long nbins, double *out,
                       long *count) {
    for (long m = 0; m < nbins; m++) {
        out[m] = 0.0;
        count[m] = 0;
    }
    long c = 0;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++, c++) {
                const long m = or_radial_m(i, j, k, corner);
                out[m] += field[c];
                count[m] += 1;
            }
    for (long m = 0; m < nbins; m++)
        if (count[m] > 0) out[m] /= (double)count[m];
}

void or_fill_irregular(const or_geom *g, const int *corner, const double *base, double *out) {
    long c = 0;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++, c++) out[c] = base[or_radial_m(i, j, k, corner)];
}

/* ---- quadratic interpolation ---------------------------------------------------------- */
/* value at r of the Lagrange quadratic through (x0,y0), (x1,y1), (x2,y2) */
static double lagrange3(double r, double x0, double y0, double x1, double y1, double x2, double y2) {
    return y0 * (r - x1) * (r - x2) / ((x0 - x1) * (x0 - x2)) + y1 * (r - x0) * (r - x2) / ((x1 - x0) * (x1 - x2)) +
           y2 * (r - x0) * (r - x1) / ((x2 - x0) * (x2 - x1));
}

/* uniform base state prof[j] at radii (j + 1/2) dr (nr >= 3) onto the cells,
 * the star's centre at center[3] (physical coordinates) */
int or_fill_quadratic(const or_geom *g, const double *prof, int nr, double dr, const double *center, double *out) {
    if (nr < 3) return -1;
    const double h = g->dx;
    long c = 0;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++, c++) {
                const double x = (i + 0.5) * h - center[0], y = (j + 0.5) * h - center[1];
                const double z = (k + 0.5) * h - center[2];
                const double r = sqrt(x * x + y * y + z * z);
                /* the radial cell centre nearest to r, as the middle of the stencil */
                long jc = (long)floor(r / dr);
                if (jc < 1) jc = 1;
                if (jc > nr - 2) jc = nr - 2;
                out[c] = lagrange3(r, (jc - 0.5) * dr, prof[jc - 1], (jc + 0.5) * dr, prof[jc], (jc + 1.5) * dr,
                                   prof[jc + 1]);
            }
    return 0;
}

/* irregular means avg[m] (count[m] cells at radius dx sqrt(0.75 + 2m)) onto the
 * uniform base state out[j] at radii (j + 1/2) dr, quadratically through the
 * non-empty radius nearest to each uniform radius and its non-empty neighbours
 * (needs >= 3 non-empty bins) */
int or_average_to_uniform(long nbins, const double *avg, const long *count, double dx, int nr, double dr,
                          double *out) {
    long nz = 0;
    for (long m = 0; m < nbins; m++)
        if (count[m] > 0) nz++;
    if (nz < 3) return -1;
    double *rr = (double *)malloc(sizeof(double) * nz), *vv = (double *)malloc(sizeof(double) * nz);
    long q = 0;
    for (long m = 0; m < nbins; m++)
        if (count[m] > 0) {
            rr[q] = dx * sqrt(0.75 + 2.0 * (double)m);
            vv[q] = avg[m];
            q++;
        }
    for (int j = 0; j < nr; j++) {
        const double r = (j + 0.5) * dr;
        /* the non-empty radius nearest to r, the first one on a tie */
        long best = 0;
        double bd = fabs(rr[0] - r);
        for (long t = 1; t < nz; t++) {
            const double d = fabs(rr[t] - r);
            if (d < bd) {
                bd = d;
                best = t;
            }
        }
        if (best < 1) best = 1;
        if (best > nz - 2) best = nz - 2;
        out[j] = lagrange3(r, rr[best - 1], vv[best - 1], rr[best], vv[best], rr[best + 1], vv[best + 1]);
    }
    free(rr);
    free(vv);
    return 0;
}

/* ---- velocity split: w0 and the lateral-average constraint (Appendix A) -------------
 * U = U~ + w0 e_r.  U~ satisfies div(beta0 U~) = beta0 (S - Sbar) (Sbar: the lateral
 * average of S, filled back onto the cells); w0 satisfies
 *     div(beta0 w0 e_r) = beta0 (Sbar - psi),   psi = dp0/dt / (Gamma1bar p0),
 * integrated in one dimension over base-state cells j (edges e = j and j + 1):
 *     Q_0 = 0,  Q_{j+1} = Q_j + V_j beta0_j src_j,  src_j = Sbar_j - psi_j,
 *     w0_e = Q_e / (A_e beta0e_e)      (w0_0 = 0),
 * planar: A = 1, V_j = r_{j+1} - r_j; spherical: A = r^2, V_j = (r_{j+1}^3 - r_j^3)/3
 * (the exact shell integral of r^2).  beta0 on an interior edge is the mean of its two
 * cells, on the last edge that of the last cell.  With a cutoff edge c >= 0 the
 * edges beyond it keep A w0 constant: w0_e = w0_c A_c / A_e. */
int or_w0_integrate(int spherical, int nr, const double *r_edge, const double *beta0, const double *src,
                    int cutoff, double *w0) {
    if (nr < 1) return -1;
    double Q = 0.0;
    w0[0] = 0.0;
    for (int j = 0; j < nr; j++) {
        const double r0 = r_edge[j], r1 = r_edge[j + 1];
        const double V = spherical ? (r1 * r1 * r1 - r0 * r0 * r0) / 3.0 : r1 - r0;
        Q += V * beta0[j] * src[j];
        const double be = j + 1 < nr ? 0.5 * (beta0[j] + beta0[j + 1]) : beta0[j];
        const double A = spherical ? r1 * r1 : 1.0;
        w0[j + 1] = Q / (A * be);
    }
    if (cutoff >= 0 && cutoff < nr) {
        const double rc = r_edge[cutoff];
        for (int e = cutoff + 1; e <= nr; e++) {
            const double re = r_edge[e];
            w0[e] = spherical ? w0[cutoff] * (rc * rc) / (re * re) : w0[cutoff];
        }
    }
    return 0;
}

/* w0 at radius r: linear between the edges around it; beyond the last edge A w0 is
 * held constant (planar: w0 constant) */
static double w0_at(int spherical, int nr, const double *r_edge, const double *w0, double r) {
    if (r >= r_edge[nr]) {
        const double rl = r_edge[nr];
        return spherical ? w0[nr] * (rl * rl) / (r * r) : w0[nr];
    }
    if (r <= r_edge[0]) return w0[0];
    int e = 0;
    while (r_edge[e + 1] < r) e++;
    const double t = (r - r_edge[e]) / (r_edge[e + 1] - r_edge[e]);
    return w0[e] + t * (w0[e + 1] - w0[e]);
}

/* U_f += w0(r_f) (e_r . n_f) on every MAC face (API face layout: n_d + 1 faces along d).
 * planar: e_r = e_z; the base-state cells are the cell layers, so z-face k gets w0_k.
 * spherical: the star's centre on corner c; face centre x_f, r_f = |x_f - c dx|. */
void or_add_w0_faces(const or_geom *g, int spherical, const int *corner, int nr, const double *r_edge,
                     const double *w0, double *ux, double *uy, double *uz) {
    const double h = g->dx;
    double *u[3] = {ux, uy, uz};
    for (int d = 0; d < 3; d++) {
        if (!spherical && d != 2) continue;
        const int m0 = g->n[0] + (d == 0), m1 = g->n[1] + (d == 1), m2 = g->n[2] + (d == 2);
        long c = 0;
        for (int k = 0; k < m2; k++)
            for (int j = 0; j < m1; j++)
                for (int i = 0; i < m0; i++, c++) {
                    if (!spherical) {  /* base-state edges are the z faces: needs nr >= n2 */
                        u[2][c] += w0[k];
                        continue;
                    }
                    /* face centre: integer position along d, half-integer along the others */
                    const double x = (d == 0 ? i : i + 0.5) * h - corner[0] * h;
                    const double y = (d == 1 ? j : j + 0.5) * h - corner[1] * h;
                    const double z = (d == 2 ? k : k + 0.5) * h - corner[2] * h;
                    const double r = sqrt(x * x + y * y + z * z);
                    const double comp = d == 0 ? x : (d == 1 ? y : z);
                    u[d][c] += w0_at(1, nr, r_edge, w0, r) * comp / r;
                }
    }
}

/* the right-hand-side bracket of the U~ constraint: out = S - Sbar on every cell, Sbar
 * the lateral average of S (planar: plane means; spherical: the irregular radial
 * means of the corner-centred star) filled back without interpolation */
void or_subtract_lateral_average(const or_geom *g, int spherical, const int *corner, const double *S,
                                 double *out) {
    const long n = (long)g->n[0] * g->n[1] * g->n[2];
    double *fillv = (double *)malloc(sizeof(double) * n);
    if (!spherical) {
        double *prof = (double *)malloc(sizeof(double) * g->n[2]);
        or_average_planar(g, S, prof);
        long c = 0;
        for (int k = 0; k < g->n[2]; k++)
            for (long q = 0; q < (long)g->n[0] * g->n[1]; q++, c++) fillv[c] = prof[k];
        free(prof);
    } else {
        const long nb = or_radial_nbins(g, corner);
        double *avg = (double *)malloc(sizeof(double) * nb);
        long *cnt = (long *)malloc(sizeof(long) * nb);
        or_average_radial(g, corner, S, nb, avg, cnt);
        or_fill_irregular(g, corner, avg, fillv);
        free(avg);
        free(cnt);
    }
    for (long c = 0; c < n; c++) out[c] = S[c] - fillv[c];
    free(fillv);
}
