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
// FP64, one thread per cell: the operator and divergence of a composite
// solve, checked element by element against the oracle; the composite solver
// itself is not built on them yet.
#include <cmath>

#include "mx_internal.cuh"
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

__global__ void comp_apply_coarse_kernel(CompGeom G, const double *__restrict__ rc, const double *__restrict__ bc,
                                         const double *__restrict__ rf, const double *__restrict__ bf,
                                         const double *__restrict__ pc, const double *__restrict__ pf,
                                         double *__restrict__ out) {
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
        out[q] = acc;
    }
}

__global__ void comp_apply_fine_kernel(CompGeom G, const double *__restrict__ rc, const double *__restrict__ bc,
                                       const double *__restrict__ rf, const double *__restrict__ bf,
                                       const double *__restrict__ pc, const double *__restrict__ pf,
                                       double *__restrict__ out) {
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
        out[q] = acc;
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
