/*
 * FP64 CPU oracle for the base-state mapping modules of MAESTROeX (Sec. 3.1):
 * the lateral average (Cartesian cells -> 1D base state) and the fill
 * (1D base state -> Cartesian cells).
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
