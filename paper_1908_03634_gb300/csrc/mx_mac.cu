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
// With Q: the correction factors q_f = 2/(h (rho_L + rho_R)) (Dirichlet 2/(h rho)).
__global__ void mac_coeffs_kernel(Level<double> L, FaceQ Q, const double *__restrict__ rho,
                                  const double *__restrict__ beta0, double ih2x) {
    const DGeom &g = L.g;
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int k1 = min(k0 + ZC, nz);
    const bool wq = Q.x != nullptr;
    for (int k = k0; k < k1; k++) {
        const long long c = i + (long long)nx * (j + (long long)ny * k);
        const double bc = beta0[c], rc = rho[c];
        auto face = [&](long long cl, double *b, double *q) {
            const double r = rcp64(rho[cl] + rc);
            *b = (beta0[cl] + bc) * r;
            if (wq) *q = ih2x * r;
        };
        auto own = [&](int bcnd, double *b, double *q) {
            if (bcnd == MX_BC_DIRICHLET) {
                const double r = rcp64(rc);
                *b = 2.0 * (bc * r);
                if (wq) *q = ih2x * r;
            } else {
                *b = 0.0;
                if (wq) *q = 0.0;
            }
        };
        // x
        if (i > 0) face(c - 1, L.bx + c, Q.x + c);
        else if (gper(g, 0)) face(c + nx - 1, L.bx + c, Q.x + c);
        else own(g.lo[0], L.bx + c, Q.x + c);
        // y
        if (j > 0) face(c - nx, L.by + c, Q.y + c);
        else if (gper(g, 1)) face(c + (long long)(ny - 1) * nx, L.by + c, Q.y + c);
        else own(g.lo[1], L.by + c, Q.y + c);
        // z
        if (k > 0) face(c - g.nxy, L.bz + c, Q.z + c);
        else if (gper(g, 2)) face(c + (long long)(nz - 1) * g.nxy, L.bz + c, Q.z + c);
        else own(g.lo[2], L.bz + c, Q.z + c);
        // high boundary planes
        if (i == nx - 1 && L.hx) {
            const long long q = j + (long long)ny * k;
            own(g.hi[0], L.hx + q, Q.hx + q);
        }
        if (j == ny - 1 && L.hy) {
            const long long q = i + (long long)nx * k;
            own(g.hi[1], L.hy + q, Q.hy + q);
        }
        if (k == nz - 1 && L.hz) {
            const long long q = i + (long long)nx * j;
            own(g.hi[2], L.hz + q, Q.hz + q);
        }
    }
}

void k_mac_coeffs64(cudaStream_t s, const Level<double> &L, const double *rho, const double *beta0, const FaceQ *q) {
    mac_coeffs_kernel<<<stencil_grid(L.g), dim3(SX, SY), 0, s>>>(L, q ? *q : FaceQ{}, rho, beta0, 2.0 / L.g.h);
}

// ------------------------------------------------------------------------------
// D(beta0 U) - beta0 Sbar along a cell column, from API-layout face velocities.
// Face flux times 2: (beta0_L + beta0_R) U_f inside and across periodic faces,
// 2 beta0 U_f of the interior cell on a Dirichlet face, 0 on a wall; the factor
// 1/2 and 1/h are applied once per cell.  The column walks up k and carries each
// cell's high z-face flux over as the next cell's low one.
__device__ __forceinline__ double face_flux2(const DGeom &g, const double *__restrict__ beta0, int d, int p,
                                             long long c_lo, long long c_hi, double u) {
    // one FP64 expression for every face kind (branches with FP64 arithmetic
    // are predicated by the compiler and would all occupy the FP64 pipe):
    // inside / periodic (beta0_lo + beta0_hi) u; Dirichlet (beta0_in + beta0_in) u;
    // wall 0 u
    const int n = g.n[d];
    const bool inner = (p > 0 && p < n) || gper(g, d);
    const int bc = p == 0 ? g.lo[d] : g.hi[d];
    const long long cin = p == 0 ? c_hi : c_lo;
    const bool wall = !inner && bc != MX_BC_DIRICHLET;
    const double a = wall ? 0.0 : beta0[inner ? c_lo : cin];
    const double b = wall ? 0.0 : beta0[inner ? c_hi : cin];
    return (a + b) * u;
}

template <typename F>
__device__ __forceinline__ void div_column(const DGeom &g, const double *__restrict__ ux,
                                           const double *__restrict__ uy, const double *__restrict__ uz,
                                           const double *__restrict__ beta0, const double *__restrict__ sbar, int i,
                                           int j, int k0, int k1, double hih, F fn) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long nxy = g.nxy;
    long long c = i + (long long)nx * (j + (long long)ny * k0);
    double fzl = face_flux2(g, beta0, 2, k0, k0 > 0 ? c - nxy : c + (long long)(nz - 1) * nxy, c, uz[c]);
    for (int k = k0; k < k1; k++, c += nxy) {
        // x faces i and i+1 in the (nx+1)-wide layout
        const long long fx = i + (long long)(nx + 1) * (j + (long long)ny * k);
        const long long cw = i > 0 ? c - 1 : c + nx - 1;  // wrapped neighbours (used only if periodic)
        const long long ce = i + 1 < nx ? c + 1 : c - (nx - 1);
        const double fxl = face_flux2(g, beta0, 0, i, cw, c, ux[fx]);
        const double fxh = face_flux2(g, beta0, 0, i + 1, c, ce, ux[fx + 1]);
        const long long fy = i + (long long)nx * (j + (long long)(ny + 1) * k);
        const long long cs = j > 0 ? c - nx : c + (long long)(ny - 1) * nx;
        const long long cn = j + 1 < ny ? c + nx : c - (long long)(ny - 1) * nx;
        const double fyl = face_flux2(g, beta0, 1, j, cs, c, uy[fy]);
        const double fyh = face_flux2(g, beta0, 1, j + 1, c, cn, uy[fy + nx]);
        const long long ct = k + 1 < nz ? c + nxy : c - (long long)(nz - 1) * nxy;
        const double fzh = face_flux2(g, beta0, 2, k + 1, c, ct, uz[c + nxy]);  // z faces: c + nxy*k', k' <= nz
        fn(c, fma(((fxh - fxl) + (fyh - fyl)) + (fzh - fzl), hih, -beta0[c] * sbar[c]));
        fzl = fzh;
    }
}

__global__ void mac_rhs_kernel(DGeom g, const double *__restrict__ ux, const double *__restrict__ uy,
                               const double *__restrict__ uz, const double *__restrict__ beta0,
                               const double *__restrict__ sbar, double *__restrict__ f, double *part, double hih) {
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    if (i < g.n[0] && j < g.n[1])
        div_column(g, ux, uy, uz, beta0, sbar, i, j, k0, min(k0 + ZC, g.n[2]), hih, [&](long long c, double v) {
            f[c] = v;
            mx = nmax(mx, fabs(v));
            s2 = fma(v, v, s2);
            s1 += v;
        });
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
    mac_rhs_kernel<<<stencil_grid(g), dim3(SX, SY), 0, s>>>(g, ux, uy, uz, beta0, sbar, f, partials, 0.5 / g.h);
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
            set_scale(st, a > 0.0 ? a : 1.0);
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
        mx = nmax(mx, fabs(v));
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
// Correction U_f -= (dphi/dn)_f / rho_f on the API face layout, with the face
// factors q_f = 2/(h (rho_L + rho_R)) of the coefficient setup: inside and
// across periodic faces U_f -= q_f (phi_R - phi_L) (faces 0 and n of a periodic
// axis get the same value); across a Dirichlet face (phi = 0 outside, distance
// h/2) U_f -= +-q_f phi_c; wall faces are set to 0.  One thread per cell
// updates the cell's three low faces and, on the last cell of a row, the high
// boundary face.
__device__ __forceinline__ void correct_face(const DGeom &g, int d, int p, long long cl, long long cr, long long ci,
                                             const double *__restrict__ phi, double q, double *__restrict__ u,
                                             long long f) {
    u[f] = corr_face_value(g, d, p, cl, cr, ci, phi, q, u[f]);
}

__global__ void mac_correct_kernel(DGeom g, FaceQ Q, const double *__restrict__ phi, double *__restrict__ ux,
                                   double *__restrict__ uy, double *__restrict__ uz) {
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int k1 = min(k0 + ZC, nz);
    for (int k = k0; k < k1; k++) {
        const long long c = i + (long long)nx * (j + (long long)ny * k);
        // x faces i (and nx on the last cell)
        const long long fx = i + (long long)(nx + 1) * (j + (long long)ny * k);
        correct_face(g, 0, i, i > 0 ? c - 1 : c + nx - 1, c, c, phi, Q.x[c], ux, fx);
        if (i == nx - 1)
            correct_face(g, 0, nx, c, c - (nx - 1), c, phi, gper(g, 0) ? Q.x[c - (nx - 1)] : Q.hx[j + (long long)ny * k],
                         ux, fx + 1);
        const long long fy = i + (long long)nx * (j + (long long)(ny + 1) * k);
        correct_face(g, 1, j, j > 0 ? c - nx : c + (long long)(ny - 1) * nx, c, c, phi, Q.y[c], uy, fy);
        if (j == ny - 1)
            correct_face(g, 1, ny, c, c - (long long)(ny - 1) * nx, c, phi,
                         gper(g, 1) ? Q.y[c - (long long)(ny - 1) * nx] : Q.hy[i + (long long)nx * k], uy, fy + nx);
        correct_face(g, 2, k, k > 0 ? c - g.nxy : c + (long long)(nz - 1) * g.nxy, c, c, phi, Q.z[c], uz, c);
        if (k == nz - 1)
            correct_face(g, 2, nz, c, c - (long long)(nz - 1) * g.nxy, c, phi,
                         gper(g, 2) ? Q.z[c - (long long)(nz - 1) * g.nxy] : Q.hz[i + (long long)nx * j], uz,
                         c + g.nxy);
    }
}

void k_mac_correct(cudaStream_t s, const DGeom &g, const FaceQ &q, const double *phi, double *ux, double *uy,
                   double *uz) {
    mac_correct_kernel<<<stencil_grid(g), dim3(SX, SY), 0, s>>>(g, q, phi, ux, uy, uz);
}

// max |D(beta0 U) - beta0 Sbar - c| of the projected velocity
__global__ void mac_divcheck_kernel(DGeom g, const double *__restrict__ ux, const double *__restrict__ uy,
                                    const double *__restrict__ uz, const double *__restrict__ beta0,
                                    const double *__restrict__ sbar, const SolveState *st, double *part, double hih) {
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    const double cm = st->mean;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    if (i < g.n[0] && j < g.n[1])
        div_column(g, ux, uy, uz, beta0, sbar, i, j, k0, min(k0 + ZC, g.n[2]), hih,
                   [&](long long, double v) { mx = nmax(mx, fabs(v - cm)); });
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
    mac_divcheck_kernel<<<stencil_grid(g), dim3(SX, SY), 0, s>>>(g, ux, uy, uz, beta0, sbar, st, partials, 0.5 / g.h);
}

__global__ void finalize_max_kernel(const double *part, int nb, double *dst) {
    double a, b, c;
    reduce_partials3(part, nb, a, b, c);
    if (flat_tid() == 0) *dst = a;
}

void k_finalize_max(cudaStream_t s, const double *partials, int nb, double *dst) {
    finalize_max_kernel<<<1, 1024, 0, s>>>(partials, nb, dst);
}
