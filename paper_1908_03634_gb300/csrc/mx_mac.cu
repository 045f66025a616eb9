// MAC projection kernels in FP64 (Steps 3 and 7; Eq. div1, div2; Appendix A):
// base-state Fill (Sec. 3.1), face coefficients beta0_f/rho_f, the right-hand
// side D(beta0 U) - beta0 Sbar with mean removal, the velocity correction
// U -= grad(phi)/rho_f and the divergence check of the projected velocity.
#include "mx_stencil.cuh"

int red_blocks(long long n) {
    long long b = (n + RED_THREADS - 1) / RED_THREADS;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    return int(b);
}

// ------------------------------------------------------------------------------
// Fill: planar injection by z index, or linear interpolation in radius.
__global__ void fill_kernel(DGeom g, int spherical, const double *__restrict__ prof, int nr, double dr, double cx,
                            double cy, double cz, double *__restrict__ out) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.N; c += (long long)gridDim.x * blockDim.x) {
        const int i = int(c % g.n[0]);
        const int j = int((c / g.n[0]) % g.n[1]);
        const int k = int(c / g.nxy);
        if (!spherical) {
            out[c] = prof[k];
        } else {
            const double x = (i + 0.5) * g.h - cx, y = (j + 0.5) * g.h - cy, z = (k + 0.5) * g.h - cz;
            const double r = sqrt(x * x + y * y + z * z);
            const double s = r / dr - 0.5;  // fractional index of the radial cell centres
            int m = int(floor(s));
            m = m < 0 ? 0 : (m > nr - 2 ? nr - 2 : m);
            const double t = s - m;
            out[c] = prof[m] + t * (prof[m + 1] - prof[m]);
        }
    }
}

void k_fill(cudaStream_t s, const DGeom &g, int spherical, const double *prof, int nr, double dr, double cx, double cy,
            double cz, double *out) {
    fill_kernel<<<red_blocks(g.N), RED_THREADS, 0, s>>>(g, spherical, prof, nr, dr, cx, cy, cz, out);
}

// ------------------------------------------------------------------------------
// Face coefficients b_f = beta0_f / rho_f (arithmetic face averages), stored in
// lo-face form; wall faces 0, Dirichlet faces 2 beta0/rho of the interior cell.
__global__ void mac_coeffs_kernel(Level<double> L, const double *__restrict__ rho, const double *__restrict__ beta0) {
    const DGeom &g = L.g;
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int k1 = min(k0 + ZC, nz);
    for (int k = k0; k < k1; k++) {
        const long long c = i + (long long)nx * (j + (long long)ny * k);
        const double bc = beta0[c], rc = rho[c];
        auto own = [&]() { return 2.0 * (bc * rcp64(rc)); };  // a Dirichlet face's coefficient
        // x
        if (i > 0) L.bx[c] = (beta0[c - 1] + bc) * rcp64(rho[c - 1] + rc);
        else if (gper(g, 0)) L.bx[c] = (beta0[c + nx - 1] + bc) * rcp64(rho[c + nx - 1] + rc);
        else L.bx[c] = g.lo[0] == MX_BC_DIRICHLET ? own() : 0.0;
        // y
        if (j > 0) L.by[c] = (beta0[c - nx] + bc) * rcp64(rho[c - nx] + rc);
        else if (gper(g, 1)) {
            const long long o = c + (long long)(ny - 1) * nx;
            L.by[c] = (beta0[o] + bc) * rcp64(rho[o] + rc);
        } else L.by[c] = g.lo[1] == MX_BC_DIRICHLET ? own() : 0.0;
        // z
        if (k > 0) L.bz[c] = (beta0[c - g.nxy] + bc) * rcp64(rho[c - g.nxy] + rc);
        else if (gper(g, 2)) {
            const long long o = c + (long long)(nz - 1) * g.nxy;
            L.bz[c] = (beta0[o] + bc) * rcp64(rho[o] + rc);
        } else L.bz[c] = g.lo[2] == MX_BC_DIRICHLET ? own() : 0.0;
        // high boundary planes
        if (i == nx - 1 && L.hx) L.hx[j + (long long)ny * k] = g.hi[0] == MX_BC_DIRICHLET ? own() : 0.0;
        if (j == ny - 1 && L.hy) L.hy[i + (long long)nx * k] = g.hi[1] == MX_BC_DIRICHLET ? own() : 0.0;
        if (k == nz - 1 && L.hz) L.hz[i + (long long)nx * j] = g.hi[2] == MX_BC_DIRICHLET ? own() : 0.0;
    }
}

void k_mac_coeffs64(cudaStream_t s, const Level<double> &L, const double *rho, const double *beta0) {
    mac_coeffs_kernel<<<stencil_grid(L.g), dim3(SX, SY), 0, s>>>(L, rho, beta0);
}

// ------------------------------------------------------------------------------
// D(beta0 U) at cell (i,j,k) from API-layout face velocities.

__device__ __forceinline__ double face_beta_u(const DGeom &g, const double *__restrict__ beta0, int d, int p,
                                              long long c_lo, long long c_hi, double u) {
    // face p along d joins cells c_lo (p-1, possibly wrapped) and c_hi (p)
    const int n = g.n[d];
    if (p > 0 && p < n) return 0.5 * (beta0[c_lo] + beta0[c_hi]) * u;
    const int bc = p == 0 ? g.lo[d] : g.hi[d];
    if (bc == MX_BC_PERIODIC) return 0.5 * (beta0[c_lo] + beta0[c_hi]) * u;
    if (bc == MX_BC_DIRICHLET) return beta0[p == 0 ? c_hi : c_lo] * u;
    return 0.0;  // wall: U_n taken as 0
}

__device__ __forceinline__ double div_beta_u(const DGeom &g, const double *__restrict__ beta0,
                                             const double *__restrict__ ux, const double *__restrict__ uy,
                                             const double *__restrict__ uz, int i, int j, int k, long long c,
                                             double ih) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    // x faces i and i+1 in the (nx+1)-wide layout
    const long long fx = i + (long long)(nx + 1) * (j + (long long)ny * k);
    const long long cw = i > 0 ? c - 1 : c + nx - 1;   // wrapped neighbour (used only if periodic)
    const long long ce = i + 1 < nx ? c + 1 : c - (nx - 1);
    const double fxl = face_beta_u(g, beta0, 0, i, cw, c, ux[fx]);
    const double fxh = face_beta_u(g, beta0, 0, i + 1, c, ce, ux[fx + 1]);
    const long long fy = i + (long long)nx * (j + (long long)(ny + 1) * k);
    const long long cs = j > 0 ? c - nx : c + (long long)(ny - 1) * nx;
    const long long cn = j + 1 < ny ? c + nx : c - (long long)(ny - 1) * nx;
    const double fyl = face_beta_u(g, beta0, 1, j, cs, c, uy[fy]);
    const double fyh = face_beta_u(g, beta0, 1, j + 1, c, cn, uy[fy + nx]);
    const long long fz = c;  // z faces: i + nx*(j + ny*k), k in [0, nz]
    const long long cb = k > 0 ? c - g.nxy : c + (long long)(nz - 1) * g.nxy;
    const long long ct = k + 1 < nz ? c + g.nxy : c - (long long)(nz - 1) * g.nxy;
    const double fzl = face_beta_u(g, beta0, 2, k, cb, c, uz[fz]);
    const double fzh = face_beta_u(g, beta0, 2, k + 1, c, ct, uz[fz + g.nxy]);
    return (fxh - fxl) * ih + (fyh - fyl) * ih + (fzh - fzl) * ih;
}

__global__ void mac_rhs_kernel(DGeom g, const double *__restrict__ ux, const double *__restrict__ uy,
                               const double *__restrict__ uz, const double *__restrict__ beta0,
                               const double *__restrict__ sbar, double *__restrict__ f, double *part, double ih) {
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + ZC, g.n[2]);
        for (int k = k0; k < k1; k++) {
            const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
            const double v = div_beta_u(g, beta0, ux, uy, uz, i, j, k, c, ih) - beta0[c] * sbar[c];
            f[c] = v;
            mx = fmax(mx, fabs(v));
            s2 += v * v;
            s1 += v;
        }
    }
    block_red3(mx, s2, s1);
    if (flat_tid() == 0) {
        double *p = part + 3 * flat_bid();
        p[0] = mx;
        p[1] = s2;
        p[2] = s1;
    }
}

void k_mac_rhs(cudaStream_t s, const DGeom &g, const double *ux, const double *uy, const double *uz,
               const double *beta0, const double *sbar, double *f, double *partials, int nb) {
    (void)nb;
    mac_rhs_kernel<<<stencil_grid(g), dim3(SX, SY), 0, s>>>(g, ux, uy, uz, beta0, sbar, f, partials, 1.0 / g.h);
}

// stage 0: the RHS mean (if removed); stage 1: norms of the final RHS and the
// initial solve state (scale = ||f||_inf).
__global__ void finalize_rhs_kernel(const double *part, int nb, SolveState *st, long long N, int remove_mean,
                                    int stage) {
    double a, b, c;
    reduce_partials3(part, nb, a, b, c);
    if (flat_tid() == 0) {
        if (stage == 0) {
            st->mean = remove_mean ? c / double(N) : 0.0;
            st->aux = c / double(N);  // the raw mean, for the compatibility check
            st->fnorm = a;
        } else {
            st->fnorm = a;
            st->fnorm2 = sqrt(b);
            st->fsum = c;
            st->scale = a > 0.0 ? a : 1.0;
            st->inv_scale = 1.0 / st->scale;
            st->best = INFINITY;
            st->iter = 0;
            st->done = 0;
            st->status = MX_OK;
        }
    }
}

void k_finalize_rhs(cudaStream_t s, const double *partials, int nb, SolveState *st, long long N, int remove_mean,
                    int stage) {
    finalize_rhs_kernel<<<1, 1024, 0, s>>>(partials, nb, st, N, remove_mean, stage);
}

__global__ void sub_mean_norm_kernel(double *f, long long n, const SolveState *st, double *part) {
    const double m = st->mean;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const double v = f[q] - m;
        f[q] = v;
        mx = fmax(mx, fabs(v));
        s2 += v * v;
        s1 += v;
    }
    block_red3(mx, s2, s1);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = mx;
        part[3 * blockIdx.x + 1] = s2;
        part[3 * blockIdx.x + 2] = s1;
    }
}

void k_sub_mean_norm(cudaStream_t s, const DGeom &g, double *f, const SolveState *st, double *partials, int nb) {
    sub_mean_norm_kernel<<<nb, RED_THREADS, 0, s>>>(f, g.N, st, partials);
}

// ------------------------------------------------------------------------------
// Correction U_f -= (dphi/dn)_f / rho_f on the API face layout.  One thread per
// cell updates the cell's three low faces and, on the last cell of a row, the
// high boundary face.  The face gradient is (phi_R - phi_L)/h inside and across
// periodic faces (faces 0 and n then both get the same value), one-sided with
// phi = 0 across a Dirichlet face; wall faces are set to 0.
__device__ __forceinline__ void correct_face(const DGeom &g, int d, int p, long long cl, long long cr, long long ci,
                                             const double *__restrict__ rho, const double *__restrict__ phi,
                                             double *__restrict__ u, long long f, double ih) {
    const int n = g.n[d];
    if ((p > 0 && p < n) || gper(g, d)) {
        const double rf = 0.5 * (rho[cl] + rho[cr]);
        u[f] -= ((phi[cr] - phi[cl]) * ih) * rcp64(rf);
    } else {
        const int bc = p == 0 ? g.lo[d] : g.hi[d];
        if (bc == MX_BC_DIRICHLET) {
            const double grad = p == 0 ? (phi[ci] - 0.0) * (2.0 * ih) : (0.0 - phi[ci]) * (2.0 * ih);
            u[f] -= grad * rcp64(rho[ci]);
        } else {
            u[f] = 0.0;
        }
    }
}

__global__ void mac_correct_kernel(DGeom g, const double *__restrict__ rho, const double *__restrict__ phi,
                                   double *__restrict__ ux, double *__restrict__ uy, double *__restrict__ uz, double ih) {
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int k1 = min(k0 + ZC, nz);
    for (int k = k0; k < k1; k++) {
        const long long c = i + (long long)nx * (j + (long long)ny * k);
        // x faces i (and nx on the last cell)
        const long long fx = i + (long long)(nx + 1) * (j + (long long)ny * k);
        correct_face(g, 0, i, i > 0 ? c - 1 : c + nx - 1, c, c, rho, phi, ux, fx, ih);
        if (i == nx - 1) correct_face(g, 0, nx, c, c - (nx - 1), c, rho, phi, ux, fx + 1, ih);
        const long long fy = i + (long long)nx * (j + (long long)(ny + 1) * k);
        correct_face(g, 1, j, j > 0 ? c - nx : c + (long long)(ny - 1) * nx, c, c, rho, phi, uy, fy, ih);
        if (j == ny - 1) correct_face(g, 1, ny, c, c - (long long)(ny - 1) * nx, c, rho, phi, uy, fy + nx, ih);
        correct_face(g, 2, k, k > 0 ? c - g.nxy : c + (long long)(nz - 1) * g.nxy, c, c, rho, phi, uz, c, ih);
        if (k == nz - 1) correct_face(g, 2, nz, c, c - (long long)(nz - 1) * g.nxy, c, rho, phi, uz, c + g.nxy, ih);
    }
}

void k_mac_correct(cudaStream_t s, const DGeom &g, const double *rho, const double *phi, double *ux, double *uy,
                   double *uz) {
    mac_correct_kernel<<<stencil_grid(g), dim3(SX, SY), 0, s>>>(g, rho, phi, ux, uy, uz, 1.0 / g.h);
}

// max |D(beta0 U) - beta0 Sbar - c| of the projected velocity
__global__ void mac_divcheck_kernel(DGeom g, const double *__restrict__ ux, const double *__restrict__ uy,
                                    const double *__restrict__ uz, const double *__restrict__ beta0,
                                    const double *__restrict__ sbar, const SolveState *st, double *part, double ih) {
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    const double cm = st->mean;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + ZC, g.n[2]);
        for (int k = k0; k < k1; k++) {
            const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
            const double v = div_beta_u(g, beta0, ux, uy, uz, i, j, k, c, ih) - beta0[c] * sbar[c] - cm;
            mx = fmax(mx, fabs(v));
            s2 += v * v;
        }
    }
    block_red3(mx, s2, s1);
    if (flat_tid() == 0) {
        double *p = part + 3 * flat_bid();
        p[0] = mx;
        p[1] = s2;
        p[2] = s1;
    }
}

void k_mac_divcheck(cudaStream_t s, const DGeom &g, const double *ux, const double *uy, const double *uz,
                    const double *beta0, const double *sbar, const SolveState *st, double *partials, int nb) {
    (void)nb;
    mac_divcheck_kernel<<<stencil_grid(g), dim3(SX, SY), 0, s>>>(g, ux, uy, uz, beta0, sbar, st, partials, 1.0 / g.h);
}

__global__ void finalize_max_kernel(const double *part, int nb, double *dst) {
    double a, b, c;
    reduce_partials3(part, nb, a, b, c);
    if (flat_tid() == 0) *dst = a;
}

void k_finalize_max(cudaStream_t s, const double *partials, int nb, double *dst) {
    finalize_max_kernel<<<1, 1024, 0, s>>>(partials, nb, dst);
}
