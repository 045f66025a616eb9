// Two-level composite MAC operator and divergence, refinement ratio 2 (the
// paper keeps its AMR as in its Paper V, ratio 2, end of Sec. 3.2): a coarse
// level with one fine patch over the coarse box [plo, phi), at least one coarse
// cell from every domain face and at least one coarse cell thick.
//
//   * a fine cell's neighbour across the patch boundary is a ghost value: the
//     coarse value C across, interpolated linearly to the ghost's tangential
//     position with the central differences of C's tangential neighbours
//     (offsets -H/4 or +H/4, i.e. a coefficient of -1/8 or +1/8 on each
//     difference), then the quadratic in the normal direction through C~, the
//     boundary fine cell F1 and the next one F2: 8/15 C~ + 2/3 F1 - 1/5 F2;
//   * a coarse cell's flux through a coarse-fine face is the mean of the four
//     fine fluxes b_f (phi_F1 - phi_g)/h on it (flux matching), so the volume
//     sum of L phi telescopes;
//   * face coefficients b = beta0_f/rho_f with arithmetic face means, of the
//     fine cell and the coarse cell across on a coarse-fine face; the domain
//     faces as on one level (wall: no flux; Dirichlet phi = 0: (0 - phi)/(H/2)).
//
// FP64, one thread per cell: the operator and divergence, and on them the
// composite projection (mx_mac_project_composite): refinement on the composite
// residual with a two-level correction per iteration (a V-cycle of the whole
// coarse grid, then a V-cycle of the patch).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mx_internal.cuh"
#include "mx_solver.cuh"
#include "mx_stencil.cuh"

namespace {

struct CompGeom {
    int n[3];       // coarse cells
    int lo[3], hi[3];
    int plo[3], phi[3];
    int nf[3];      // fine cells of the patch
    double H, h;
};

__device__ __forceinline__ long long cix(const CompGeom &G, int i, int j, int k) {
    return i + (long long)G.n[0] * (j + (long long)G.n[1] * k);
}
__device__ __forceinline__ long long fix_(const CompGeom &G, int i, int j, int k) {
    return i + (long long)G.nf[0] * (j + (long long)G.nf[1] * k);
}
__device__ __forceinline__ bool in_patch(const CompGeom &G, const int c[3]) {
    return c[0] >= G.plo[0] && c[0] < G.phi[0] && c[1] >= G.plo[1] && c[1] < G.phi[1] && c[2] >= G.plo[2] &&
           c[2] < G.phi[2];
}
__device__ __forceinline__ double bmean(double ba, double ra, double bb, double rb) {
    return (0.5 * (ba + bb)) / (0.5 * (ra + rb));
}

// ghost value of fine cell F (patch-local) across its patch face along d on
// side s (-1 / +1), and the coarse cell C across
__device__ double ghost(const CompGeom &G, const double *__restrict__ pc, const double *__restrict__ pf,
                        const int F[3], int d, int s, int C[3]) {
    for (int a = 0; a < 3; a++) C[a] = G.plo[a] + F[a] / 2;
    C[d] += s;
    const double vc = pc[cix(G, C[0], C[1], C[2])];
    double ct = vc;
    for (int t = 0; t < 3; t++) {
        if (t == d) continue;
        int cp[3] = {C[0], C[1], C[2]}, cm[3] = {C[0], C[1], C[2]};
        cp[t] += 1;
        cm[t] -= 1;
        const double sig = (F[t] & 1) ? 0.125 : -0.125;
        ct += sig * (pc[cix(G, cp[0], cp[1], cp[2])] - pc[cix(G, cm[0], cm[1], cm[2])]);
    }
    int F2[3] = {F[0], F[1], F[2]};
    F2[d] -= s;
    return (8.0 / 15.0) * ct + (2.0 / 3.0) * pf[fix_(G, F[0], F[1], F[2])] - 0.2 * pf[fix_(G, F2[0], F2[1], F2[2])];
}

// out = L phi on the uncovered coarse cells (0 on covered ones), or with f
// non-null the residual f - L phi and per-block maxima of its magnitude in part
__global__ void comp_apply_coarse_kernel(CompGeom G, const double *__restrict__ rc, const double *__restrict__ bc,
                                         const double *__restrict__ rf, const double *__restrict__ bf,
                                         const double *__restrict__ pc, const double *__restrict__ pf,
                                         double *__restrict__ out, const double *__restrict__ f = nullptr,
                                         double *part = nullptr) {
    double rmax = 0.0;
    const long long N = (long long)G.n[0] * G.n[1] * G.n[2];
    const double iH2 = 1.0 / (G.H * G.H), ihH = 1.0 / (G.h * G.H);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int c[3] = {int(q % G.n[0]), int((q / G.n[0]) % G.n[1]), int(q / ((long long)G.n[0] * G.n[1]))};
        if (in_patch(G, c)) {
            out[q] = 0.0;
            continue;
        }
        const double r0 = rc[q], b0 = bc[q], p0 = pc[q];
        double acc = 0.0;
        for (int d = 0; d < 3; d++) {
            for (int s = -1; s <= 1; s += 2) {
                int nb[3] = {c[0], c[1], c[2]};
                nb[d] += s;
                if (nb[d] < 0 || nb[d] >= G.n[d]) {
                    if (G.lo[d] != MX_BC_PERIODIC) {
                        const int bcd = s < 0 ? G.lo[d] : G.hi[d];
                        if (bcd == MX_BC_DIRICHLET) acc += -2.0 * (b0 / r0) * p0 * iH2;
                        continue;
                    }
                    nb[d] = (nb[d] + G.n[d]) % G.n[d];
                }
                if (!in_patch(G, nb)) {
                    const long long qn = cix(G, nb[0], nb[1], nb[2]);
                    acc += bmean(b0, r0, bc[qn], rc[qn]) * (pc[qn] - p0) * iH2;
                    continue;
                }
                // coarse-fine face: mean of the four fine fluxes
                const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
                const int Fd = 2 * (nb[d] - G.plo[d]) + (s > 0 ? 0 : 1);
                double m = 0.0;
                for (int a = 0; a < 2; a++)
                    for (int e = 0; e < 2; e++) {
                        int F[3];
                        F[d] = Fd;
                        F[t1] = 2 * (c[t1] - G.plo[t1]) + a;
                        F[t2] = 2 * (c[t2] - G.plo[t2]) + e;
                        int C[3];
                        const double g = ghost(G, pc, pf, F, d, -s, C);
                        const long long qf = fix_(G, F[0], F[1], F[2]);
                        m += bmean(bf[qf], rf[qf], b0, r0) * (pf[qf] - g);
                    }
                acc += 0.25 * m * ihH;
            }
        }
        if (f) {
            acc = f[q] - acc;
            rmax = nmax(rmax, fabs(acc));
        }
        out[q] = acc;
    }
    if (part) {
        double z1 = 0.0, z2 = 0.0;
        block_red3(rmax, z1, z2);
        if (threadIdx.x == 0) part[3 * blockIdx.x] = rmax;
    }
}

__global__ void comp_apply_fine_kernel(CompGeom G, const double *__restrict__ rc, const double *__restrict__ bc,
                                       const double *__restrict__ rf, const double *__restrict__ bf,
                                       const double *__restrict__ pc, const double *__restrict__ pf,
                                       double *__restrict__ out, const double *__restrict__ f = nullptr,
                                       double *part = nullptr) {
    double rmax = 0.0;
    const long long N = (long long)G.nf[0] * G.nf[1] * G.nf[2];
    const double ih2 = 1.0 / (G.h * G.h);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int F[3] = {int(q % G.nf[0]), int((q / G.nf[0]) % G.nf[1]), int(q / ((long long)G.nf[0] * G.nf[1]))};
        const double r0 = rf[q], b0 = bf[q], p0 = pf[q];
        double acc = 0.0;
        for (int d = 0; d < 3; d++) {
            for (int s = -1; s <= 1; s += 2) {
                int nb[3] = {F[0], F[1], F[2]};
                nb[d] += s;
                if (nb[d] >= 0 && nb[d] < G.nf[d]) {
                    const long long qn = fix_(G, nb[0], nb[1], nb[2]);
                    acc += bmean(b0, r0, bf[qn], rf[qn]) * (pf[qn] - p0) * ih2;
                } else {
                    int C[3];
                    const double g = ghost(G, pc, pf, F, d, s, C);
                    const long long qc = cix(G, C[0], C[1], C[2]);
                    acc += bmean(b0, r0, bc[qc], rc[qc]) * (g - p0) * ih2;
                }
            }
        }
        if (f) {
            acc = f[q] - acc;
            rmax = nmax(rmax, fabs(acc));
        }
        out[q] = acc;
    }
    if (part) {
        double z1 = 0.0, z2 = 0.0;
        block_red3(rmax, z1, z2);
        if (threadIdx.x == 0) part[3 * blockIdx.x] = rmax;
    }
}

// D(beta0 U): coarse faces with the single-level rules (U taken as 0 on a wall,
// beta0 of the interior cell on a Dirichlet face) except the coarse-fine faces,
// whose flux is the mean of the four fine beta0_f U_f
__global__ void comp_div_coarse_kernel(CompGeom G, const double *__restrict__ ux, const double *__restrict__ uy,
                                       const double *__restrict__ uz, const double *__restrict__ fx,
                                       const double *__restrict__ fy, const double *__restrict__ fz,
                                       const double *__restrict__ bc, const double *__restrict__ bf,
                                       double *__restrict__ out) {
    const long long N = (long long)G.n[0] * G.n[1] * G.n[2];
    const double *uc[3] = {ux, uy, uz};
    const double *uf[3] = {fx, fy, fz};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int c[3] = {int(q % G.n[0]), int((q / G.n[0]) % G.n[1]), int(q / ((long long)G.n[0] * G.n[1]))};
        if (in_patch(G, c)) {
            out[q] = 0.0;
            continue;
        }
        const double b0 = bc[q];
        double acc = 0.0;
        for (int d = 0; d < 3; d++) {
            int m3[3] = {G.n[0], G.n[1], G.n[2]};
            m3[d] += 1;  // the coarse face array along d
            for (int s = -1; s <= 1; s += 2) {
                int face[3] = {c[0], c[1], c[2]};
                if (s > 0) face[d] += 1;
                const long long qfc = face[0] + (long long)m3[0] * (face[1] + (long long)m3[1] * face[2]);
                int nb[3] = {c[0], c[1], c[2]};
                nb[d] += s;
                if (nb[d] < 0 || nb[d] >= G.n[d]) {
                    if (G.lo[d] != MX_BC_PERIODIC) {
                        const int bcd = s < 0 ? G.lo[d] : G.hi[d];
                        if (bcd == MX_BC_DIRICHLET) acc += s * b0 * uc[d][qfc];
                        continue;
                    }
                    nb[d] = (nb[d] + G.n[d]) % G.n[d];
                }
                if (!in_patch(G, nb)) {
                    acc += s * 0.5 * (b0 + bc[cix(G, nb[0], nb[1], nb[2])]) * uc[d][qfc];
                    continue;
                }
                const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
                const int Fd = 2 * (nb[d] - G.plo[d]) + (s > 0 ? 0 : 1);
                int mf[3] = {G.nf[0], G.nf[1], G.nf[2]};
                mf[d] += 1;
                double m = 0.0;
                for (int a = 0; a < 2; a++)
                    for (int e = 0; e < 2; e++) {
                        int F[3];
                        F[d] = Fd;
                        F[t1] = 2 * (c[t1] - G.plo[t1]) + a;
                        F[t2] = 2 * (c[t2] - G.plo[t2]) + e;
                        int ff[3] = {F[0], F[1], F[2]};
                        if (s < 0) ff[d] += 1;  // the fine cell's high face
                        const long long qff = ff[0] + (long long)mf[0] * (ff[1] + (long long)mf[1] * ff[2]);
                        m += 0.25 * 0.5 * (bf[fix_(G, F[0], F[1], F[2])] + b0) * uf[d][qff];
                    }
                acc += s * m;
            }
        }
        out[q] = acc / G.H;
    }
}

__global__ void comp_div_fine_kernel(CompGeom G, const double *__restrict__ fx, const double *__restrict__ fy,
                                     const double *__restrict__ fz, const double *__restrict__ bc,
                                     const double *__restrict__ bf, double *__restrict__ out) {
    const long long N = (long long)G.nf[0] * G.nf[1] * G.nf[2];
    const double *uf[3] = {fx, fy, fz};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int F[3] = {int(q % G.nf[0]), int((q / G.nf[0]) % G.nf[1]), int(q / ((long long)G.nf[0] * G.nf[1]))};
        const double b0 = bf[q];
        double acc = 0.0;
        for (int d = 0; d < 3; d++) {
            int mf[3] = {G.nf[0], G.nf[1], G.nf[2]};
            mf[d] += 1;
            for (int s = -1; s <= 1; s += 2) {
                int nb[3] = {F[0], F[1], F[2]};
                nb[d] += s;
                int ff[3] = {F[0], F[1], F[2]};
                if (s > 0) ff[d] += 1;
                const long long qff = ff[0] + (long long)mf[0] * (ff[1] + (long long)mf[1] * ff[2]);
                double bn;
                if (nb[d] >= 0 && nb[d] < G.nf[d]) {
                    bn = bf[fix_(G, nb[0], nb[1], nb[2])];
                } else {
                    int C[3];
                    for (int a = 0; a < 3; a++) C[a] = G.plo[a] + F[a] / 2;
                    C[d] += s;
                    bn = bc[cix(G, C[0], C[1], C[2])];
                }
                acc += s * 0.5 * (b0 + bn) * uf[d][qff];
            }
        }
        out[q] = acc / G.h;
    }
}

// grid-stride launch shape of the per-cell kernels below
inline int gs_blocks(long long n) { return red_blocks(n); }

__device__ __forceinline__ void coarse_ijk(const CompGeom &G, long long q, int c[3]) {
    c[0] = int(q % G.n[0]);
    c[1] = int((q / G.n[0]) % G.n[1]);
    c[2] = int(q / ((long long)G.n[0] * G.n[1]));
}
__device__ __forceinline__ void fine_ijk(const CompGeom &G, long long q, int F[3]) {
    F[0] = int(q % G.nf[0]);
    F[1] = int((q / G.nf[0]) % G.nf[1]);
    F[2] = int(q / ((long long)G.nf[0] * G.nf[1]));
}
// the fine cell (patch-local) of child (a, b, e) of covered coarse cell c
__device__ __forceinline__ long long child(const CompGeom &G, const int c[3], int a, int b, int e) {
    return fix_(G, 2 * (c[0] - G.plo[0]) + a, 2 * (c[1] - G.plo[1]) + b, 2 * (c[2] - G.plo[2]) + e);
}
__device__ __forceinline__ double mean8(const CompGeom &G, const double *__restrict__ xf, const int c[3]) {
    double s = 0.0;
    for (int e = 0; e < 2; e++)
        for (int b = 0; b < 2; b++)
            for (int a = 0; a < 2; a++) s += xf[child(G, c, a, b, e)];
    return 0.125 * s;
}

// ---- composite projection ---------------------------------------------------------------
// Face coefficients of both levels, computed once per solve (the iteration then
// does no FP64 division): API face layout, n_d + 1 faces along d.
//   coarse: faces between two uncovered cells (periodic images included) the
//   arithmetic face mean, a Dirichlet domain face 2 beta0/rho of its cell, a wall
//   0; faces touching a covered cell 0 (their fluxes come from the fine faces);
//   fine: the face mean inside the patch, on the patch boundary of the fine cell
//   and the coarse cell across.
__device__ __forceinline__ long long face_ix(const int m[3], const int f[3]) {
    return f[0] + (long long)m[0] * (f[1] + (long long)m[1] * f[2]);
}
__global__ void comp_coef_coarse_kernel(CompGeom G, int d, double *__restrict__ B, const double *__restrict__ rc,
                                        const double *__restrict__ bc) {
    int m[3] = {G.n[0], G.n[1], G.n[2]};
    m[d] += 1;
    const long long N = (long long)m[0] * m[1] * m[2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int f[3] = {int(q % m[0]), int((q / m[0]) % m[1]), int(q / ((long long)m[0] * m[1]))};
        const int p = f[d];
        int L[3] = {f[0], f[1], f[2]}, R[3] = {f[0], f[1], f[2]};
        L[d] = p - 1;
        double b = 0.0;
        if (p == 0 || p == G.n[d]) {
            if (G.lo[d] == MX_BC_PERIODIC) {
                L[d] = (L[d] + G.n[d]) % G.n[d];
                R[d] = R[d] % G.n[d];
                const long long ql = cix(G, L[0], L[1], L[2]), qr = cix(G, R[0], R[1], R[2]);
                b = bmean(bc[ql], rc[ql], bc[qr], rc[qr]);
            } else if ((p == 0 ? G.lo[d] : G.hi[d]) == MX_BC_DIRICHLET) {
                const int *in = p == 0 ? R : L;
                const long long qi = cix(G, in[0], in[1], in[2]);
                b = 2.0 * (bc[qi] / rc[qi]);
            }
        } else if (!in_patch(G, L) && !in_patch(G, R)) {
            const long long ql = cix(G, L[0], L[1], L[2]), qr = cix(G, R[0], R[1], R[2]);
            b = bmean(bc[ql], rc[ql], bc[qr], rc[qr]);
        }
        B[q] = b;
    }
}
__global__ void comp_coef_fine_kernel(CompGeom G, int d, double *__restrict__ B, const double *__restrict__ rc,
                                      const double *__restrict__ bc, const double *__restrict__ rf,
                                      const double *__restrict__ bf) {
    int m[3] = {G.nf[0], G.nf[1], G.nf[2]};
    m[d] += 1;
    const long long N = (long long)m[0] * m[1] * m[2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int f[3] = {int(q % m[0]), int((q / m[0]) % m[1]), int(q / ((long long)m[0] * m[1]))};
        const int p = f[d];
        int L[3] = {f[0], f[1], f[2]};
        L[d] = p - 1;
        if (p > 0 && p < G.nf[d]) {
            const long long ql = fix_(G, L[0], L[1], L[2]), qr = fix_(G, f[0], f[1], f[2]);
            B[q] = bmean(bf[ql], rf[ql], bf[qr], rf[qr]);
        } else {
            const int *F = p == 0 ? f : L;
            int C[3];
            for (int a = 0; a < 3; a++) C[a] = G.plo[a] + F[a] / 2;
            C[d] += p == 0 ? -1 : 1;
            const long long qf = fix_(G, F[0], F[1], F[2]), qc = cix(G, C[0], C[1], C[2]);
            B[q] = bmean(bf[qf], rf[qf], bc[qc], rc[qc]);
        }
    }
}
struct CompCoefs {
    const double *c[3], *f[3];
};
// r = f - L phi with the cached face coefficients (the operator of
// comp_apply_*_kernel), and per-block maxima of |r| in part (if non-null)
__global__ void comp_resid_coarse_kernel(CompGeom G, CompCoefs B, const double *__restrict__ pc,
                                         const double *__restrict__ pf, const double *__restrict__ f,
                                         double *__restrict__ out, double *part) {
    const long long N = (long long)G.n[0] * G.n[1] * G.n[2];
    const double iH2 = 1.0 / (G.H * G.H), ihH = 1.0 / (G.h * G.H);
    double rmax = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int c[3];
        coarse_ijk(G, q, c);
        if (in_patch(G, c)) {
            out[q] = 0.0;
            continue;
        }
        const double p0 = pc[q];
        double acc = 0.0;
        for (int d = 0; d < 3; d++) {
            int m[3] = {G.n[0], G.n[1], G.n[2]};
            m[d] += 1;
            for (int s = -1; s <= 1; s += 2) {
                int face[3] = {c[0], c[1], c[2]};
                if (s > 0) face[d] += 1;
                const double b = B.c[d][face_ix(m, face)];
                int nb[3] = {c[0], c[1], c[2]};
                nb[d] += s;
                if (nb[d] < 0 || nb[d] >= G.n[d]) {
                    if (G.lo[d] != MX_BC_PERIODIC) {
                        acc -= b * p0 * iH2;  // Dirichlet (b = 2 beta0/rho) or wall (b = 0)
                        continue;
                    }
                    nb[d] = (nb[d] + G.n[d]) % G.n[d];
                }
                if (!in_patch(G, nb)) {
                    acc += b * (pc[cix(G, nb[0], nb[1], nb[2])] - p0) * iH2;
                    continue;
                }
                // coarse-fine face: the mean of the four fine fluxes
                const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
                const int Fd = 2 * (nb[d] - G.plo[d]) + (s > 0 ? 0 : 1);
                int mf[3] = {G.nf[0], G.nf[1], G.nf[2]};
                mf[d] += 1;
                double mm = 0.0;
                for (int a = 0; a < 2; a++)
                    for (int e = 0; e < 2; e++) {
                        int F[3];
                        F[d] = Fd;
                        F[t1] = 2 * (c[t1] - G.plo[t1]) + a;
                        F[t2] = 2 * (c[t2] - G.plo[t2]) + e;
                        int ff[3] = {F[0], F[1], F[2]};
                        if (s < 0) ff[d] += 1;  // the fine cell's high face
                        int C[3];
                        const double g = ghost(G, pc, pf, F, d, -s, C);
                        mm += B.f[d][face_ix(mf, ff)] * (pf[fix_(G, F[0], F[1], F[2])] - g);
                    }
                acc += 0.25 * mm * ihH;
            }
        }
        acc = f[q] - acc;
        rmax = nmax(rmax, fabs(acc));
        out[q] = acc;
    }
    if (part) {
        double z1 = 0.0, z2 = 0.0;
        block_red3(rmax, z1, z2);
        if (threadIdx.x == 0) part[3 * blockIdx.x] = rmax;
    }
}
__global__ void comp_resid_fine_kernel(CompGeom G, CompCoefs B, const double *__restrict__ pc,
                                       const double *__restrict__ pf, const double *__restrict__ f,
                                       double *__restrict__ out, double *part) {
    const long long N = (long long)G.nf[0] * G.nf[1] * G.nf[2];
    const double ih2 = 1.0 / (G.h * G.h);
    double rmax = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int F[3];
        fine_ijk(G, q, F);
        const double p0 = pf[q];
        double acc = 0.0;
        for (int d = 0; d < 3; d++) {
            int m[3] = {G.nf[0], G.nf[1], G.nf[2]};
            m[d] += 1;
            for (int s = -1; s <= 1; s += 2) {
                int face[3] = {F[0], F[1], F[2]};
                if (s > 0) face[d] += 1;
                const double b = B.f[d][face_ix(m, face)];
                int nb[3] = {F[0], F[1], F[2]};
                nb[d] += s;
                if (nb[d] >= 0 && nb[d] < G.nf[d]) {
                    acc += b * (pf[fix_(G, nb[0], nb[1], nb[2])] - p0) * ih2;
                } else {
                    int C[3];
                    acc += b * (ghost(G, pc, pf, F, d, s, C) - p0) * ih2;
                }
            }
        }
        acc = f[q] - acc;
        rmax = nmax(rmax, fabs(acc));
        out[q] = acc;
    }
    if (part) {
        double z1 = 0.0, z2 = 0.0;
        block_red3(rmax, z1, z2);
        if (threadIdx.x == 0) part[3 * blockIdx.x] = rmax;
    }
}



// f = D(beta0 U) - beta0 Sbar on the uncovered coarse cells (0 on covered ones)
// and the fine cells, in place over the divergence; partials (max |f|,
// volume-weighted sum of f, volume) per block, the coarse level's blocks first
__global__ void comp_rhs_kernel(CompGeom G, double *__restrict__ fc, double *__restrict__ ff,
                                const double *__restrict__ bc, const double *__restrict__ sc,
                                const double *__restrict__ bf, const double *__restrict__ sf, double *part,
                                int nbc) {
    const bool fine = blockIdx.x >= nbc;
    const long long N = fine ? (long long)G.nf[0] * G.nf[1] * G.nf[2] : (long long)G.n[0] * G.n[1] * G.n[2];
    const int b0 = fine ? blockIdx.x - nbc : blockIdx.x, nb = fine ? gridDim.x - nbc : nbc;
    const double vol = fine ? G.h * G.h * G.h : G.H * G.H * G.H;
    double mx = 0.0, sum = 0.0, v = 0.0;
    for (long long q = b0 * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)nb * blockDim.x) {
        if (fine) {
            const double x = ff[q] - bf[q] * sf[q];
            ff[q] = x;
            mx = nmax(mx, fabs(x));
            sum += vol * x;
            v += vol;
        } else {
            int c[3];
            coarse_ijk(G, q, c);
            if (in_patch(G, c)) {
                fc[q] = 0.0;
                continue;
            }
            const double x = fc[q] - bc[q] * sc[q];
            fc[q] = x;
            mx = nmax(mx, fabs(x));
            sum += vol * x;
            v += vol;
        }
    }
    block_red3(mx, sum, v);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = mx;
        part[3 * blockIdx.x + 1] = sum;
        part[3 * blockIdx.x + 2] = v;
    }
}

// one block: st->mean = volume-weighted mean (when singular and asked), st->fnorm = max |f|
__global__ void comp_rhs_final_kernel(const double *part, int nb, SolveState *st, int remove_mean) {
    double a, b, c;
    reduce_partials3(part, nb, a, b, c);
    if (threadIdx.x == 0) {
        st->mean = remove_mean ? b / c : 0.0;
        st->fnorm = a;
        st->aux = b / c;
    }
}

// f -= mean on the uncovered coarse and the fine cells; partials of max |f|
__global__ void comp_sub_mean_kernel(CompGeom G, double *__restrict__ fc, double *__restrict__ ff,
                                     const SolveState *st, double *part, int nbc) {
    const bool fine = blockIdx.x >= nbc;
    const long long N = fine ? (long long)G.nf[0] * G.nf[1] * G.nf[2] : (long long)G.n[0] * G.n[1] * G.n[2];
    const int b0 = fine ? blockIdx.x - nbc : blockIdx.x, nb = fine ? gridDim.x - nbc : nbc;
    const double m = st->mean;
    double mx = 0.0, z1 = 0.0, z2 = 0.0;
    for (long long q = b0 * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)nb * blockDim.x) {
        double *x = fine ? ff : fc;
        if (!fine) {
            int c[3];
            coarse_ijk(G, q, c);
            if (in_patch(G, c)) continue;
        }
        x[q] -= m;
        mx = nmax(mx, fabs(x[q]));
    }
    block_red3(mx, z1, z2);
    if (threadIdx.x == 0) part[3 * blockIdx.x] = mx;
}

// one block: convergence decision from the partial maxima of the residual
__global__ void comp_decide_kernel(const double *part, int nb, SolveState *st) {
    double mx = 0.0, z1 = 0.0, z2 = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) mx = nmax(mx, part[3 * q]);
    block_red3(mx, z1, z2);
    if (threadIdx.x == 0) {
        st->rnorm = mx;
        const bool conv = mx <= st->tol * st->fnorm;
        if (!(mx == mx) || isinf(mx)) {
            st->status = MX_ERR_NOCONV;
            st->done = 1;
        } else if (conv) {
            st->status = MX_OK;
            st->done = 1;
        } else if (st->iter >= st->maxit) {
            st->status = MX_ERR_NOCONV;
            st->done = 1;
        } else if (st->iter > 3 && mx > 1e3 * st->best) {
            st->status = MX_ERR_NOCONV;
            st->done = 1;
        } else {
            st->done = 0;
            st->iter += 1;
        }
        if (mx < st->best) st->best = mx;
    }
}
__global__ void comp_scale_kernel(SolveState *st) { set_scale(st, st->fnorm > 0.0 ? st->fnorm : 1.0); }
__global__ void comp_rmax_kernel(const double *part, int nb, double *dst) {
    double mx = 0.0, z1 = 0.0, z2 = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) mx = nmax(mx, part[3 * q]);
    block_red3(mx, z1, z2);
    if (threadIdx.x == 0) *dst = mx;
}

// right-hand side of the coarse correction: r / scale on the uncovered cells,
// the mean of the eight fine residuals on the covered ones (FP32)
__global__ void comp_coarse_rhs_kernel(CompGeom G, const double *__restrict__ rc, const double *__restrict__ rf,
                                       const SolveState *st, float *__restrict__ out) {
    const long long N = (long long)G.n[0] * G.n[1] * G.n[2];
    const double is = st->inv_scale;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int c[3];
        coarse_ijk(G, q, c);
        out[q] = float((in_patch(G, c) ? mean8(G, rf, c) : rc[q]) * is);
    }
}
__global__ void comp_fine_rhs_kernel(long long n, const double *__restrict__ rf, const SolveState *st,
                                     float *__restrict__ out) {
    const double is = st->inv_scale;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        out[q] = float(rf[q] * is);
}
// phi_c += scale e_c on the uncovered cells, phi_f += scale e_c(parent)
__global__ void comp_coarse_update_kernel(CompGeom G, double *__restrict__ pc, double *__restrict__ pf,
                                          const float *__restrict__ ec, const SolveState *st, int nbc) {
    const double sc = st->scale;
    const bool fine = blockIdx.x >= nbc;
    const int b0 = fine ? blockIdx.x - nbc : blockIdx.x, nb = fine ? gridDim.x - nbc : nbc;
    if (fine) {
        const long long N = (long long)G.nf[0] * G.nf[1] * G.nf[2];
        for (long long q = b0 * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)nb * blockDim.x) {
            int F[3];
            fine_ijk(G, q, F);
            pf[q] += sc * double(ec[cix(G, G.plo[0] + F[0] / 2, G.plo[1] + F[1] / 2, G.plo[2] + F[2] / 2)]);
        }
    } else {
        const long long N = (long long)G.n[0] * G.n[1] * G.n[2];
        for (long long q = b0 * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)nb * blockDim.x) {
            int c[3];
            coarse_ijk(G, q, c);
            if (!in_patch(G, c)) pc[q] += sc * double(ec[q]);
        }
    }
}
__global__ void comp_fine_update_kernel(long long n, double *__restrict__ pf, const float *__restrict__ ef,
                                        const SolveState *st) {
    const double sc = st->scale;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        pf[q] += sc * double(ef[q]);
}

// coefficient inputs of the coarse correction operator: rho, beta0 of the coarse
// level with the covered cells replaced by the means of their fine cells
__global__ void comp_coarse_fields_kernel(CompGeom G, const double *__restrict__ rc, const double *__restrict__ bc,
                                          const double *__restrict__ rf, const double *__restrict__ bf,
                                          double *__restrict__ rm, double *__restrict__ bm) {
    const long long N = (long long)G.n[0] * G.n[1] * G.n[2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int c[3];
        coarse_ijk(G, q, c);
        const bool cov = in_patch(G, c);
        rm[q] = cov ? mean8(G, rf, c) : rc[q];
        bm[q] = cov ? mean8(G, bf, c) : bc[q];
    }
}

// The patch's correction operator: the patch as a box with phi = 0 beyond its
// faces, whose boundary faces (stored as the Dirichlet coefficient 2 b of the
// boundary cell) get the weight the ghost gives the boundary cell when the
// coarse correction is held at 0 and the next cell inward is taken equal to it:
// phi_g - phi_F1 = (2/3 - 1/5 - 1) phi_F1, i.e. 8/15 b instead of 2 b.
__global__ void comp_patch_bnd_kernel(Level<float> L, float w) {
    const DGeom &g = L.g;
    const long long N = g.N;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int i = int(q % g.n[0]), j = int((q / g.n[0]) % g.n[1]), k = int(q / g.nxy);
        if (i == 0) L.bx[q] *= w;
        if (j == 0) L.by[q] *= w;
        if (k == 0) L.bz[q] *= w;
        if (i == g.n[0] - 1) L.hx[j + (long long)g.n[1] * k] *= w;
        if (j == g.n[1] - 1) L.hy[i + (long long)g.n[0] * k] *= w;
        if (k == g.n[2] - 1) L.hz[i + (long long)g.n[0] * j] *= w;
    }
}

// volume-weighted sum of phi over the unknowns (uncovered coarse, fine): partials (0, sum, volume)
__global__ void comp_phi_sum_kernel(CompGeom G, const double *__restrict__ pc, const double *__restrict__ pf,
                                    double *part, int nbc) {
    const bool fine = blockIdx.x >= nbc;
    const long long N = fine ? (long long)G.nf[0] * G.nf[1] * G.nf[2] : (long long)G.n[0] * G.n[1] * G.n[2];
    const int b0 = fine ? blockIdx.x - nbc : blockIdx.x, nb = fine ? gridDim.x - nbc : nbc;
    const double vol = fine ? G.h * G.h * G.h : G.H * G.H * G.H;
    double z = 0.0, sum = 0.0, v = 0.0;
    for (long long q = b0 * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)nb * blockDim.x) {
        if (!fine) {
            int c[3];
            coarse_ijk(G, q, c);
            if (in_patch(G, c)) continue;
        }
        sum += vol * (fine ? pf[q] : pc[q]);
        v += vol;
    }
    block_red3(z, sum, v);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = 0.0;
        part[3 * blockIdx.x + 1] = sum;
        part[3 * blockIdx.x + 2] = v;
    }
}
__global__ void comp_phi_mean_kernel(const double *part, int nb, double *dst) {
    double a, b, c;
    reduce_partials3(part, nb, a, b, c);
    if (threadIdx.x == 0) *dst = b / c;
}
// phi -= mean (singular problems) on both levels, then the covered coarse phi = mean of its fine cells
__global__ void comp_phi_fine_shift_kernel(long long n, double *__restrict__ pf, const double *mean) {
    const double m = mean ? *mean : 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        pf[q] -= m;
}
__global__ void comp_phi_coarse_final_kernel(CompGeom G, double *__restrict__ pc, const double *__restrict__ pf,
                                             const double *mean) {
    const double m = mean ? *mean : 0.0;
    const long long N = (long long)G.n[0] * G.n[1] * G.n[2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int c[3];
        coarse_ijk(G, q, c);
        pc[q] = in_patch(G, c) ? mean8(G, pf, c) : pc[q] - m;
    }
}

// U <- U - (dphi/dn)/rho_f on the coarse faces off the patch (single-level rules:
// periodic faces wrap, a wall face keeps U = 0, a Dirichlet face uses (0 - phi)
// over H/2); faces touching a covered cell are left to comp_face_mean_kernel
__global__ void comp_correct_coarse_kernel(CompGeom G, int d, double *__restrict__ u, const double *__restrict__ pc,
                                           const double *__restrict__ rc) {
    int m[3] = {G.n[0], G.n[1], G.n[2]};
    m[d] += 1;
    const long long N = (long long)m[0] * m[1] * m[2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int f[3] = {int(q % m[0]), int((q / m[0]) % m[1]), int(q / ((long long)m[0] * m[1]))};
        const int p = f[d];
        int L[3] = {f[0], f[1], f[2]}, R[3] = {f[0], f[1], f[2]};
        L[d] = p - 1;
        if (p == 0 || p == G.n[d]) {
            if (G.lo[d] == MX_BC_PERIODIC) {
                L[d] = (L[d] + G.n[d]) % G.n[d];
                R[d] = R[d] % G.n[d];
            } else {
                const int bc = p == 0 ? G.lo[d] : G.hi[d];
                const int *in = p == 0 ? R : L;
                const long long qi = cix(G, in[0], in[1], in[2]);
                if (bc == MX_BC_DIRICHLET) {
                    const double g = p == 0 ? pc[qi] / (0.5 * G.H) : -pc[qi] / (0.5 * G.H);
                    u[q] -= g / rc[qi];
                } else {
                    u[q] = 0.0;
                }
                continue;
            }
        }
        if (in_patch(G, L) || in_patch(G, R)) continue;
        const long long ql = cix(G, L[0], L[1], L[2]), qr = cix(G, R[0], R[1], R[2]);
        u[q] -= ((pc[qr] - pc[ql]) / G.H) / (0.5 * (rc[ql] + rc[qr]));
    }
}
// the fine faces: interior ones by the fine difference, patch-boundary ones with the ghost value
__global__ void comp_correct_fine_kernel(CompGeom G, int d, double *__restrict__ u, const double *__restrict__ pc,
                                         const double *__restrict__ pf, const double *__restrict__ rc,
                                         const double *__restrict__ rf) {
    int m[3] = {G.nf[0], G.nf[1], G.nf[2]};
    m[d] += 1;
    const long long N = (long long)m[0] * m[1] * m[2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int f[3] = {int(q % m[0]), int((q / m[0]) % m[1]), int(q / ((long long)m[0] * m[1]))};
        const int p = f[d];
        int L[3] = {f[0], f[1], f[2]};
        L[d] = p - 1;
        if (p > 0 && p < G.nf[d]) {
            const long long ql = fix_(G, L[0], L[1], L[2]), qr = fix_(G, f[0], f[1], f[2]);
            u[q] -= ((pf[qr] - pf[ql]) / G.h) / (0.5 * (rf[ql] + rf[qr]));
        } else {
            const int *F = p == 0 ? f : L;
            const int s = p == 0 ? -1 : 1;
            int C[3];
            const double pg = ghost(G, pc, pf, F, d, s, C);
            const long long qf = fix_(G, F[0], F[1], F[2]);
            const double g = p == 0 ? (pf[qf] - pg) / G.h : (pg - pf[qf]) / G.h;
            u[q] -= g / (0.5 * (rf[qf] + rc[cix(G, C[0], C[1], C[2])]));
        }
    }
}
// coarse faces on and inside the patch: the mean of the four fine faces on them
__global__ void comp_face_mean_kernel(CompGeom G, int d, double *__restrict__ uc, const double *__restrict__ uf) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int np = G.phi[d] - G.plo[d] + 1, na = G.phi[t1] - G.plo[t1], nb = G.phi[t2] - G.plo[t2];
    int mc[3] = {G.n[0], G.n[1], G.n[2]}, mf[3] = {G.nf[0], G.nf[1], G.nf[2]};
    mc[d] += 1;
    mf[d] += 1;
    const long long N = (long long)np * na * nb;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int p = G.plo[d] + int(q % np), a = G.plo[t1] + int((q / np) % na), b = G.plo[t2] + int(q / ((long long)np * na));
        int face[3];
        face[d] = p;
        face[t1] = a;
        face[t2] = b;
        double m = 0.0;
        for (int e2 = 0; e2 < 2; e2++)
            for (int e1 = 0; e1 < 2; e1++) {
                int ff[3];
                ff[d] = 2 * (p - G.plo[d]);
                ff[t1] = 2 * (a - G.plo[t1]) + e1;
                ff[t2] = 2 * (b - G.plo[t2]) + e2;
                m += 0.25 * uf[ff[0] + (long long)mf[0] * (ff[1] + (long long)mf[1] * ff[2])];
            }
        uc[face[0] + (long long)mc[0] * (face[1] + (long long)mc[1] * face[2])] = m;
    }
}

// max |D(beta0 U) - beta0 Sbar - c| over the unknowns (the divergence in place in dc, df)
__global__ void comp_divcheck_kernel(CompGeom G, const double *__restrict__ dc, const double *__restrict__ df,
                                     const double *__restrict__ bc, const double *__restrict__ sc,
                                     const double *__restrict__ bf, const double *__restrict__ sf,
                                     const SolveState *st, double *part, int nbc) {
    const bool fine = blockIdx.x >= nbc;
    const long long N = fine ? (long long)G.nf[0] * G.nf[1] * G.nf[2] : (long long)G.n[0] * G.n[1] * G.n[2];
    const int b0 = fine ? blockIdx.x - nbc : blockIdx.x, nb = fine ? gridDim.x - nbc : nbc;
    const double cm = st->mean;
    double mx = 0.0, z1 = 0.0, z2 = 0.0;
    for (long long q = b0 * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)nb * blockDim.x) {
        double x;
        if (fine) {
            x = df[q] - bf[q] * sf[q] - cm;
        } else {
            int c[3];
            coarse_ijk(G, q, c);
            if (in_patch(G, c)) continue;
            x = dc[q] - bc[q] * sc[q] - cm;
        }
        mx = nmax(mx, fabs(x));
    }
    block_red3(mx, z1, z2);
    if (threadIdx.x == 0) part[3 * blockIdx.x] = mx;
}

mx_status make_comp(mx_ctx *c, const mx_geom *geom, const int plo[3], const int phi[3], CompGeom &G) {
    mx_status st = check_geom(c, geom, false);
    if (st) return st;
    if (!plo || !phi) return set_err(c, MX_ERR_ARG, "composite: null patch box");
    for (int d = 0; d < 3; d++) {
        if (!(plo[d] >= 1 && phi[d] <= geom->n[d] - 1 && phi[d] - plo[d] >= 1))
            return set_err(c, MX_ERR_ARG,
                           "composite: the patch must keep one coarse cell from every domain face and be one cell thick");
        G.n[d] = geom->n[d];
        G.lo[d] = geom->lo[d];
        G.hi[d] = geom->hi[d];
        G.plo[d] = plo[d];
        G.phi[d] = phi[d];
        G.nf[d] = 2 * (phi[d] - plo[d]);
    }
    G.H = geom->dx;
    G.h = 0.5 * geom->dx;
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    return MX_OK;
}

}  // namespace

extern "C" mx_status mx_composite_apply(mx_ctx *c, const mx_geom *geom, const int plo[3], const int phi[3],
                                        const double *rho_c, const double *beta0_c, const double *rho_f,
                                        const double *beta0_f, const double *phi_c, const double *phi_f,
                                        double *out_c, double *out_f) {
    if (!c) return MX_ERR_ARG;
    CompGeom G;
    mx_status st = make_comp(c, geom, plo, phi, G);
    if (st) return st;
    if (!rho_c || !beta0_c || !rho_f || !beta0_f || !phi_c || !phi_f || !out_c || !out_f)
        return set_err(c, MX_ERR_ARG, "composite_apply: null array");
    const long long Nc = (long long)G.n[0] * G.n[1] * G.n[2], Nf = (long long)G.nf[0] * G.nf[1] * G.nf[2];
    comp_apply_coarse_kernel<<<red_blocks(Nc), 256, 0, c->stream>>>(G, rho_c, beta0_c, rho_f, beta0_f, phi_c, phi_f,
                                                                     out_c);
    comp_apply_fine_kernel<<<red_blocks(Nf), 256, 0, c->stream>>>(G, rho_c, beta0_c, rho_f, beta0_f, phi_c, phi_f,
                                                                   out_f);
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

extern "C" mx_status mx_composite_divergence(mx_ctx *c, const mx_geom *geom, const int plo[3], const int phi[3],
                                             const double *ux_c, const double *uy_c, const double *uz_c,
                                             const double *ux_f, const double *uy_f, const double *uz_f,
                                             const double *beta0_c, const double *beta0_f, double *out_c,
                                             double *out_f) {
    if (!c) return MX_ERR_ARG;
    CompGeom G;
    mx_status st = make_comp(c, geom, plo, phi, G);
    if (st) return st;
    if (!ux_c || !uy_c || !uz_c || !ux_f || !uy_f || !uz_f || !beta0_c || !beta0_f || !out_c || !out_f)
        return set_err(c, MX_ERR_ARG, "composite_divergence: null array");
    const long long Nc = (long long)G.n[0] * G.n[1] * G.n[2], Nf = (long long)G.nf[0] * G.nf[1] * G.nf[2];
    comp_div_coarse_kernel<<<red_blocks(Nc), 256, 0, c->stream>>>(G, ux_c, uy_c, uz_c, ux_f, uy_f, uz_f, beta0_c,
                                                                   beta0_f, out_c);
    comp_div_fine_kernel<<<red_blocks(Nf), 256, 0, c->stream>>>(G, ux_f, uy_f, uz_f, beta0_c, beta0_f, out_f);
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

// ---- composite projection (mx_mac_project_composite) ------------------------------------
// Refinement on the composite residual: r = f - L phi (FP64, the exact composite
// operator with face coefficients computed once per call), then per iteration a
// coarse correction (one FP32 V-cycle of the whole coarse grid; its right-hand
// side the coarse residual on uncovered cells and the mean of the eight fine
// residuals on covered ones, its coefficients from rho, beta0 with the covered
// cells replaced by their fine means), added to the uncovered coarse cells and,
// piecewise constant, to the patch; the fine residual again; a fine correction
// (one FP32 V-cycle of the patch with phi = 0 beyond its faces, the boundary
// faces weighted 8/15 b as the ghost weighs the boundary cell with the coarse
// correction held), added to the patch; the composite residual and its norm.
// The loop runs as one conditional CUDA graph (or from the host), stopping when
// the FP64 composite residual meets the tolerance.
namespace {
struct CompPlan {
    CompGeom G;
    int singular = 0;
    MacPlan *pc = nullptr, *pf = nullptr;
    void *mem = nullptr;
    double *fc, *rcb, *rm, *bm, *ff, *rfb;
    CompCoefs B;
    // the refinement loop's graph and what it was captured with
    cudaGraphExec_t graph = nullptr;
    const void *k_pc = nullptr, *k_pf = nullptr, *k_part = nullptr;
    int k_nu1 = -1, k_nu2 = -1, k_bot = -1, k_zcap = -1;
    ~CompPlan() {
        if (graph) cudaGraphExecDestroy(graph);
        if (mem) cudaFree(mem);
        if (pc) free_mac_plan(pc);
        if (pf) free_mac_plan(pf);
    }
};

bool same_comp(const CompGeom &a, const CompGeom &b) {
    for (int d = 0; d < 3; d++)
        if (a.n[d] != b.n[d] || a.lo[d] != b.lo[d] || a.hi[d] != b.hi[d] || a.plo[d] != b.plo[d] || a.phi[d] != b.phi[d])
            return false;
    return a.H == b.H;
}

// the context's composite plan for G (one kept: the last geometry)
CompPlan *get_comp_plan(mx_ctx *c, const CompGeom &G, const mx_geom *geom, mx_status *st) {
    *st = MX_OK;
    CompPlan *P = (CompPlan *)c->comp;
    if (P && same_comp(P->G, G)) return P;
    if (P) {
        cudaStreamSynchronize(c->stream);
        delete P;
        c->comp = nullptr;
    }
    P = new CompPlan();
    P->G = G;
    const DGeom gc = make_dgeom(geom);
    DGeom gf;
    for (int d = 0; d < 3; d++) {
        gf.n[d] = G.nf[d];
        gf.lo[d] = gf.hi[d] = MX_BC_DIRICHLET;
    }
    gf.nxy = (long long)gf.n[0] * gf.n[1];
    gf.N = gf.nxy * gf.n[2];
    gf.h = G.h;
    P->singular = geom_singular(gc);
    P->pc = create_mac_plan(c, gc, MX_PREC_MIXED, st);
    if (P->pc) P->pf = create_mac_plan(c, gf, MX_PREC_MIXED, st);
    if (!P->pc || !P->pf) {
        delete P;
        return nullptr;
    }
    const long long Nc = gc.N, Nf = gf.N;
    long long nface_c[3], nface_f[3], tot = 4 * Nc + 2 * Nf;
    for (int d = 0; d < 3; d++) {
        nface_c[d] = (Nc / G.n[d]) * (G.n[d] + 1);
        nface_f[d] = (Nf / G.nf[d]) * (G.nf[d] + 1);
        tot += nface_c[d] + nface_f[d];
    }
    if (cudaMalloc(&P->mem, sizeof(double) * tot) != cudaSuccess) {
        cudaGetLastError();
        P->mem = nullptr;
        delete P;
        *st = set_err(c, MX_ERR_OOM, "mac_project_composite: workspace cudaMalloc failed");
        return nullptr;
    }
    double *x = (double *)P->mem;
    P->fc = x;
    P->rcb = x + Nc;
    P->rm = x + 2 * Nc;
    P->bm = x + 3 * Nc;
    P->ff = x + 4 * Nc;
    P->rfb = P->ff + Nf;
    x = P->rfb + Nf;
    double *bcoef[6];
    for (int d = 0; d < 3; d++) {
        bcoef[d] = x;
        x += nface_c[d];
    }
    for (int d = 0; d < 3; d++) {
        bcoef[3 + d] = x;
        x += nface_f[d];
    }
    for (int d = 0; d < 3; d++) {
        P->B.c[d] = bcoef[d];
        P->B.f[d] = bcoef[3 + d];
    }
    c->comp = P;
    return P;
}

// one refinement iteration after the composite residual: the two corrections,
// then the residual and the convergence decision
void comp_body(cudaStream_t s, mx_ctx *c, CompPlan &P, double *phi_c, double *phi_f, const mx_opts &o, int zcap) {
    const CompGeom &G = P.G;
    const long long Nf = (long long)G.nf[0] * G.nf[1] * G.nf[2];
    const int nbc = gs_blocks((long long)G.n[0] * G.n[1] * G.n[2]), nbf = gs_blocks(Nf), nb = nbc + nbf;
    Hier<float> &HC = P.pc->H32, &HF = P.pf->H32;
    SolveState *dst = c->state;
    double *part = c->partials;
    comp_coarse_rhs_kernel<<<nbc, 256, 0, s>>>(G, P.rcb, P.rfb, dst, HC.lev[0].f);
    vcycle(s, HC, o.nu1, o.nu2, o.bottom_iters, P.singular, nullptr, 0, zcap);
    comp_coarse_update_kernel<<<nb, 256, 0, s>>>(G, phi_c, phi_f, HC.lev[0].e, dst, nbc);
    comp_resid_fine_kernel<<<nbf, 256, 0, s>>>(G, P.B, phi_c, phi_f, P.ff, P.rfb, nullptr);
    comp_fine_rhs_kernel<<<nbf, 256, 0, s>>>(Nf, P.rfb, dst, HF.lev[0].f);
    vcycle(s, HF, o.nu1, o.nu2, o.bottom_iters, 0, nullptr, 0, zcap);
    comp_fine_update_kernel<<<nbf, 256, 0, s>>>(Nf, phi_f, HF.lev[0].e, dst);
    comp_resid_coarse_kernel<<<nbc, 256, 0, s>>>(G, P.B, phi_c, phi_f, P.fc, P.rcb, part);
    comp_resid_fine_kernel<<<nbf, 256, 0, s>>>(G, P.B, phi_c, phi_f, P.ff, P.rfb, part + 3 * nbc);
    comp_decide_kernel<<<1, 1024, 0, s>>>(part, nb, dst);
}
}  // namespace

void destroy_comp_plan(mx_ctx *c) {
    delete (CompPlan *)c->comp;
    c->comp = nullptr;
}

extern "C" mx_status mx_mac_project_composite(mx_ctx *c, const mx_geom *geom, const int plo[3], const int phi[3],
                                              double *ux_c, double *uy_c, double *uz_c, const double *rho_c,
                                              const double *beta0_c, const double *sbar_c, double *phi_c,
                                              double *ux_f, double *uy_f, double *uz_f, const double *rho_f,
                                              const double *beta0_f, const double *sbar_f, double *phi_f,
                                              const mx_opts *opts, mx_info *info) {
    if (!c) return MX_ERR_ARG;
    CompGeom G;
    mx_status st = make_comp(c, geom, plo, phi, G);
    if (st) return st;
    if (!ux_c || !uy_c || !uz_c || !rho_c || !beta0_c || !sbar_c || !phi_c || !ux_f || !uy_f || !uz_f || !rho_f ||
        !beta0_f || !sbar_f || !phi_f)
        return set_err(c, MX_ERR_ARG, "mac_project_composite: null array");
    mx_opts o;
    if ((st = check_opts(c, opts, o))) return st;
    if (o.prec != MX_PREC_MIXED || o.krylov || o.smoother)
        return set_err(c, MX_ERR_ARG, "mac_project_composite: prec must be MX_PREC_MIXED, krylov and smoother 0");
    if (o.nu1 == 0 && o.nu2 == 0) o.nu1 = o.nu2 = 2;
    const int zcap = o.tile_z ? o.tile_z : 8;
    cudaStream_t s = c->stream;
    const long long Nc = (long long)G.n[0] * G.n[1] * G.n[2], Nf = (long long)G.nf[0] * G.nf[1] * G.nf[2];
    const int nbc = gs_blocks(Nc), nbf = gs_blocks(Nf), nb = nbc + nbf;
    if ((st = ensure_partials(c, nb))) return st;
    CompPlan *Pp = get_comp_plan(c, G, geom, &st);
    if (!Pp) return st;
    CompPlan &P = *Pp;
    const int singular = P.singular;
    double *part = c->partials;
    SolveState *dst = c->state;
    MX_CUDA(c, cudaEventRecord(c->ev0, s));
    SolveState init = {};
    init.tol = o.rel_tol;
    init.maxit = std::min(o.max_outer, o.max_vcycles);
    init.best = INFINITY;
    *c->hstate = init;
    MX_CUDA(c, cudaMemcpyAsync(dst, c->hstate, sizeof(SolveState), cudaMemcpyHostToDevice, s));

    // face coefficients of the composite operator and the correction operators
    double *uc[3] = {ux_c, uy_c, uz_c}, *uf[3] = {ux_f, uy_f, uz_f};
    for (int d = 0; d < 3; d++) {
        comp_coef_coarse_kernel<<<nbc, 256, 0, s>>>(G, d, (double *)P.B.c[d], rho_c, beta0_c);
        comp_coef_fine_kernel<<<nbf, 256, 0, s>>>(G, d, (double *)P.B.f[d], rho_c, beta0_c, rho_f, beta0_f);
    }
    comp_coarse_fields_kernel<<<nbc, 256, 0, s>>>(G, rho_c, beta0_c, rho_f, beta0_f, P.rm, P.bm);
    setup_coefficients_on(s, *P.pc, P.rm, P.bm);
    Hier<float> &HF = P.pf->H32;
    k_mac_coeffs_df(s, HF.lev[0], P.pf->D, rho_f, beta0_f, nullptr);
    comp_patch_bnd_kernel<<<nbf, 256, 0, s>>>(HF.lev[0], float(4.0 / 15.0));
    for (int l = 0; l + 1 < HF.nlev; l++) k_coarsen_coeffs(s, HF.lev[l], HF.lev[l + 1]);

    // right-hand side, mean removal, scale
    comp_div_coarse_kernel<<<nbc, 256, 0, s>>>(G, ux_c, uy_c, uz_c, ux_f, uy_f, uz_f, beta0_c, beta0_f, P.fc);
    comp_div_fine_kernel<<<nbf, 256, 0, s>>>(G, ux_f, uy_f, uz_f, beta0_c, beta0_f, P.ff);
    comp_rhs_kernel<<<nb, 256, 0, s>>>(G, P.fc, P.ff, beta0_c, sbar_c, beta0_f, sbar_f, part, nbc);
    comp_rhs_final_kernel<<<1, 1024, 0, s>>>(part, nb, dst, singular && o.remove_mean);
    if (singular && !o.remove_mean) {
        MX_CUDA(c, cudaMemcpyAsync(c->hstate, dst, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        MX_CUDA(c, cudaStreamSynchronize(s));
        if (std::fabs(c->hstate->aux) > 1e-12 * c->hstate->fnorm) {
            if (info) {
                std::memset(info, 0, sizeof(*info));
                info->status = MX_ERR_INCOMPAT;
            }
            return set_err(c, MX_ERR_INCOMPAT, "singular problem: right-hand side has non-zero mean and remove_mean = 0");
        }
    }
    if (singular && o.remove_mean) {
        comp_sub_mean_kernel<<<nb, 256, 0, s>>>(G, P.fc, P.ff, dst, part, nbc);
        comp_rmax_kernel<<<1, 1024, 0, s>>>(part, nb, &dst->fnorm);
    }
    comp_scale_kernel<<<1, 1, 0, s>>>(dst);
    if (!o.use_initial_guess) {
        MX_CUDA(c, cudaMemsetAsync(phi_c, 0, sizeof(double) * Nc, s));
        MX_CUDA(c, cudaMemsetAsync(phi_f, 0, sizeof(double) * Nf, s));
    }

    // first residual, then the refinement loop (a conditional graph, or from the host)
    comp_resid_coarse_kernel<<<nbc, 256, 0, s>>>(G, P.B, phi_c, phi_f, P.fc, P.rcb, part);
    comp_resid_fine_kernel<<<nbf, 256, 0, s>>>(G, P.B, phi_c, phi_f, P.ff, P.rfb, part + 3 * nbc);
    comp_decide_kernel<<<1, 1024, 0, s>>>(part, nb, dst);
    MX_CUDA(c, cudaMemcpyAsync(c->hstate, dst, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    MX_CUDA(c, cudaStreamSynchronize(s));
    if (!c->hstate->done) {
        if (o.use_graph) {
            if (!P.graph || P.k_pc != phi_c || P.k_pf != phi_f || P.k_part != part || P.k_nu1 != o.nu1 ||
                P.k_nu2 != o.nu2 || P.k_bot != o.bottom_iters || P.k_zcap != zcap) {
                if (P.graph) {
                    cudaGraphExecDestroy(P.graph);
                    P.graph = nullptr;
                }
                st = capture_while_graph(c, &P.graph, [&](cudaStream_t cs) { comp_body(cs, c, P, phi_c, phi_f, o, zcap); });
                if (st) return st;
                P.k_pc = phi_c;
                P.k_pf = phi_f;
                P.k_part = part;
                P.k_nu1 = o.nu1;
                P.k_nu2 = o.nu2;
                P.k_bot = o.bottom_iters;
                P.k_zcap = zcap;
            }
            MX_CUDA(c, cudaGraphLaunch(P.graph, s));
        } else {
            for (;;) {
                comp_body(s, c, P, phi_c, phi_f, o, zcap);
                MX_CUDA(c, cudaMemcpyAsync(c->hstate, dst, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
                MX_CUDA(c, cudaStreamSynchronize(s));
                if (c->hstate->done) break;
            }
        }
    }

    // normalisation (zero volume-weighted mean of the unknowns when singular), the
    // covered coarse phi, the velocity correction on both levels, the check
    if (singular) {
        comp_phi_sum_kernel<<<nb, 256, 0, s>>>(G, phi_c, phi_f, part, nbc);
        comp_phi_mean_kernel<<<1, 1024, 0, s>>>(part, nb, &dst->aux);
        comp_phi_fine_shift_kernel<<<nbf, 256, 0, s>>>(Nf, phi_f, &dst->aux);
    }
    comp_phi_coarse_final_kernel<<<nbc, 256, 0, s>>>(G, phi_c, phi_f, singular ? &dst->aux : nullptr);
    for (int d = 0; d < 3; d++) {
        comp_correct_coarse_kernel<<<nbc, 256, 0, s>>>(G, d, uc[d], phi_c, rho_c);
        comp_correct_fine_kernel<<<nbf, 256, 0, s>>>(G, d, uf[d], phi_c, phi_f, rho_c, rho_f);
    }
    for (int d = 0; d < 3; d++) comp_face_mean_kernel<<<nbc, 256, 0, s>>>(G, d, uc[d], uf[d]);
    comp_div_coarse_kernel<<<nbc, 256, 0, s>>>(G, ux_c, uy_c, uz_c, ux_f, uy_f, uz_f, beta0_c, beta0_f, P.rcb);
    comp_div_fine_kernel<<<nbf, 256, 0, s>>>(G, ux_f, uy_f, uz_f, beta0_c, beta0_f, P.rfb);
    comp_divcheck_kernel<<<nb, 256, 0, s>>>(G, P.rcb, P.rfb, beta0_c, sbar_c, beta0_f, sbar_f, dst, part, nbc);
    comp_rmax_kernel<<<1, 1024, 0, s>>>(part, nb, &dst->div_err);
    MX_CUDA(c, cudaEventRecord(c->ev1, s));
    MX_CUDA(c, cudaMemcpyAsync(c->hstate, dst, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    MX_CUDA(c, cudaStreamSynchronize(s));
    MX_CUDA(c, cudaGetLastError());
    const SolveState &hs = *c->hstate;
    if (info) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        info->outer_iters = hs.iter;
        info->vcycles = 2 * hs.iter;
        info->rel_resid = hs.fnorm > 0 ? hs.rnorm / hs.fnorm : hs.rnorm;
        info->rel_resid_l2 = 0.0;
        info->div_err_linf = hs.div_err;
        info->rhs_mean_removed = hs.mean;
        info->rhs_linf = hs.fnorm;
        info->ms = ms;
        info->status = hs.status;
    }
    if (hs.status != MX_OK) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "composite: no convergence, relative residual %.3e after %d iterations",
                      hs.rnorm / (hs.fnorm > 0 ? hs.fnorm : 1.0), hs.iter);
        return set_err(c, (mx_status)hs.status, buf);
    }
    return MX_OK;
}
