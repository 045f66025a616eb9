// Velocity split (Appendix A): U = U~ + w0 e_r.  U~ is projected with the
// constraint div(beta0 U~) = beta0 (S - Sbar), Sbar the lateral average of S, and
// w0 solves div(beta0 w0 e_r) = beta0 (Sbar - psi) in one dimension:
//     Q_0 = 0,  Q_{j+1} = Q_j + V_j beta0_j src_j,   w0_e = Q_e / (A_e beta0e_e),
// planar A = 1, V_j = r_{j+1} - r_j; spherical A = r^2, V_j = (r_{j+1}^3 - r_j^3)/3;
// beta0 on an interior edge is the mean of its two cells, on the last edge the last
// cell's; beyond an optional cutoff edge A w0 is held constant.
//
// w0 e_r on the MAC faces: planar, z-face k takes w0_k (the base-state cells are the
// cell layers).  Spherical, the centre on the corner c: a d-face sits at integer
// offset a along d and half-integer offsets along the other two axes, so
// 4 r^2 / dx^2 = K = 4 a^2 + B^2 + E^2 with B, E odd integers.  The factor
// dx w0(r) / r is tabulated once per K (K is 2 mod 4, so a quarter of the integers
// up to the largest; FP64, w0 linear in r between edges, A w0 held beyond the last
// edge) and every face takes u += tab[K >> 2] a: one FP64 FMA per face.
#include <algorithm>
#include <cmath>

#include "mx_internal.cuh"

namespace {

constexpr int W0_THREADS = 1024;
constexpr long long MAX_TAB = 1LL << 26;

__device__ __forceinline__ double shell(int sph, double r0, double r1) {
    return sph ? (r1 * r1 * r1 - r0 * r0 * r0) / 3.0 : r1 - r0;
}

// inclusive scan over the warp's lanes, a fixed shuffle pattern (deterministic)
__device__ __forceinline__ double warp_scan(double v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// one CTA: per-thread contiguous chunks, their sums scanned in thread order (lanes
// within a warp, then the warps' totals)
__global__ void __launch_bounds__(W0_THREADS) w0_kernel(int sph, int nr, const double *__restrict__ re,
                                                        const double *__restrict__ b, const double *__restrict__ src,
                                                        int cutoff, double *__restrict__ w0) {
    __shared__ double wsum[W0_THREADS / 32];
    const int chunk = (nr + W0_THREADS - 1) / W0_THREADS;
    const int j0 = min(nr, (int)threadIdx.x * chunk), j1 = min(nr, j0 + chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s = 0.0;
    for (int j = j0; j < j1; j++) s += shell(sph, re[j], re[j + 1]) * b[j] * src[j];
    const double incl = warp_scan(s);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const double wi = warp_scan(wsum[lane]);
        wsum[lane] = wi - wsum[lane];  // exclusive: the warps before this one
    }
    __syncthreads();
    double Q = wsum[warp] + (incl - s);  // everything before this thread's chunk
    if (threadIdx.x == 0) w0[0] = 0.0;
    for (int j = j0; j < j1; j++) {
        Q += shell(sph, re[j], re[j + 1]) * b[j] * src[j];
        const double be = j + 1 < nr ? 0.5 * (b[j] + b[j + 1]) : b[j];
        const double r1 = re[j + 1];
        w0[j + 1] = Q / ((sph ? r1 * r1 : 1.0) * be);
    }
    if (cutoff < 0 || cutoff >= nr) return;
    __syncthreads();  // orders the w0 writes above before the reads below (same CTA)
    const double wc = w0[cutoff], rc = re[cutoff];
    for (int e = cutoff + 1 + threadIdx.x; e <= nr; e += W0_THREADS) {
        const double r = re[e];
        w0[e] = sph ? wc * (rc * rc) / (r * r) : wc;
    }
}

// tab[q] = dx w0(r_K) / r_K for K = 4q + 2, r_K = (dx / 2) sqrt(K): a face's K is
// 2 mod 4 (two odd squares sum to 2 mod 8, 4 a^2 is 0 or 4 mod 8)
__global__ void w0_table_kernel(long long qmax, double dx, int nr, const double *__restrict__ re,
                                const double *__restrict__ w0, double *__restrict__ tab) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q > qmax) return;
    const long long K = 4 * q + 2;
    const double r = 0.5 * dx * sqrt((double)K);
    double w;
    if (r >= re[nr]) {
        const double rl = re[nr];
        w = w0[nr] * (rl * rl) / (r * r);
    } else if (r <= re[0]) {
        w = w0[0];
    } else {  // the edge interval (re[e], re[e + 1]] holding r
        int lo = 0, hi = nr - 1;  // smallest e with re[e + 1] >= r
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (re[mid + 1] >= r) hi = mid;
            else lo = mid + 1;
        }
        const double t = (r - re[lo]) / (re[lo + 1] - re[lo]);
        w = w0[lo] + t * (w0[lo + 1] - w0[lo]);
    }
    tab[q] = dx * w / r;
}

// u += tab[K] a on the D-faces (array m0 x m1 x m2, x fastest)
template <int D>
__global__ void w0_faces_kernel(int m0, int m1, int m2, int c0, int c1, int c2, const double *__restrict__ tab,
                                double *__restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= m0 || j >= m1) return;
#pragma unroll 4
    for (int k = blockIdx.z; k < m2; k += gridDim.z) {
        // integer offset along D, odd half-offsets (times 2) along the others
        const long long x = D == 0 ? (long long)(i - c0) : 2LL * (i - c0) + 1;
        const long long y = D == 1 ? (long long)(j - c1) : 2LL * (j - c1) + 1;
        const long long z = D == 2 ? (long long)(k - c2) : 2LL * (k - c2) + 1;
        const long long a = D == 0 ? x : (D == 1 ? y : z);
        const long long K = (D == 0 ? 4 * x * x : x * x) + (D == 1 ? 4 * y * y : y * y) + (D == 2 ? 4 * z * z : z * z);
        const long long f = i + (long long)m0 * (j + (long long)m1 * k);
        u[f] = fma(__ldg(tab + (K >> 2)), (double)a, u[f]);  // K = 4q + 2
    }
}

// planar: z-face k takes w0_k
__global__ void w0_planar_faces_kernel(long long nxy, const double *__restrict__ w0, double *__restrict__ uz) {
    const long long k = blockIdx.y;
    const double w = w0[k];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nxy; q += (long long)gridDim.x * blockDim.x)
        uz[k * nxy + q] += w;
}

// largest K over the faces of direction d
long long kmax_dir(const mx_geom *g, const int c[3], int d) {
    long long s = 0;
    for (int e = 0; e < 3; e++) {
        long long lo, hi;
        if (e == d) {  // faces 0..n_e, integer offsets, counted 4 a^2
            lo = -(long long)c[e];
            hi = (long long)g->n[e] - c[e];
            s += 4 * std::max(lo * lo, hi * hi);
        } else {  // cells 0..n_e - 1, odd offsets 2(j - c) + 1
            lo = 1 - 2LL * c[e];
            hi = 2LL * (g->n[e] - 1 - c[e]) + 1;
            s += std::max(lo * lo, hi * hi);
        }
    }
    return s;
}

mx_status grow(mx_ctx *c, void **buf, size_t *bytes, size_t need, const char *what) {
    if (need <= *bytes) return MX_OK;
    if (*buf) {
        cudaStreamSynchronize(c->stream);
        cudaFree(*buf);
    }
    *buf = nullptr;
    *bytes = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, MX_ERR_OOM, std::string(what) + ": scratch allocation failed");
    }
    *bytes = need;
    return MX_OK;
}

}  // namespace

void destroy_split_scratch(mx_ctx *c) {
    if (c->split_tab) cudaFree(c->split_tab);
    if (c->split_cells) cudaFree(c->split_cells);
    c->split_tab = c->split_cells = nullptr;
    c->split_tab_bytes = c->split_cells_bytes = 0;
}

extern "C" {

mx_status mx_w0_integrate(mx_ctx *c, int spherical, int nr, const double *r_edge, const double *beta0,
                          const double *src, int cutoff, double *w0) {
    if (!c) return MX_ERR_ARG;
    if (nr < 1 || !r_edge || !beta0 || !src || !w0) return set_err(c, MX_ERR_ARG, "w0_integrate: null array or nr < 1");
    if (cutoff < -1 || cutoff > nr) return set_err(c, MX_ERR_ARG, "w0_integrate: cutoff outside [-1, nr]");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    w0_kernel<<<1, W0_THREADS, 0, c->stream>>>(spherical ? 1 : 0, nr, r_edge, beta0, src, cutoff, w0);
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

mx_status mx_add_w0_faces(mx_ctx *c, const mx_geom *geom, int spherical, const int corner[3], int nr,
                          const double *r_edge, const double *w0, double *ux, double *uy, double *uz) {
    if (!c) return MX_ERR_ARG;
    mx_status st = check_geom(c, geom, false);
    if (st) return st;
    if (nr < 1 || !w0 || !uz || (spherical && (!ux || !uy || !r_edge || !corner)))
        return set_err(c, MX_ERR_ARG, "add_w0_faces: null array or nr < 1");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    const int n0 = geom->n[0], n1 = geom->n[1], n2 = geom->n[2];
    if (!spherical) {
        if (nr < n2) return set_err(c, MX_ERR_ARG, "add_w0_faces: planar needs nr >= n2 (w0 on the z faces)");
        const long long nxy = (long long)n0 * n1;
        const long long gx = std::min((nxy + 255) / 256, 64LL);
        w0_planar_faces_kernel<<<dim3((unsigned)gx, n2 + 1), 256, 0, c->stream>>>(nxy, w0, uz);
        MX_CUDA(c, cudaGetLastError());
        return MX_OK;
    }
    for (int d = 0; d < 3; d++)
        if (corner[d] < -(1 << 20) || corner[d] > (1 << 20)) return set_err(c, MX_ERR_ARG, "add_w0_faces: corner out of range");
    long long kmax = 0;
    for (int d = 0; d < 3; d++) kmax = std::max(kmax, kmax_dir(geom, corner, d));
    const long long qmax = kmax >> 2;  // entries for K = 2, 6, ..., kmax
    if (qmax + 1 > MAX_TAB) return set_err(c, MX_ERR_ARG, "add_w0_faces: corner too far from the box (radius table)");
    if ((st = grow(c, &c->split_tab, &c->split_tab_bytes, (size_t)(qmax + 1) * sizeof(double), "add_w0_faces")))
        return st;
    double *tab = (double *)c->split_tab;
    w0_table_kernel<<<(unsigned)((qmax + 256) / 256), 256, 0, c->stream>>>(qmax, geom->dx, nr, r_edge, w0, tab);
    const dim3 blk(128, 2);
    auto grid = [&](int m0, int m1, int m2) {
        return dim3((m0 + 127) / 128, (m1 + 1) / 2, std::min(m2, 32));
    };
    w0_faces_kernel<0><<<grid(n0 + 1, n1, n2), blk, 0, c->stream>>>(n0 + 1, n1, n2, corner[0], corner[1], corner[2],
                                                                    tab, ux);
    w0_faces_kernel<1><<<grid(n0, n1 + 1, n2), blk, 0, c->stream>>>(n0, n1 + 1, n2, corner[0], corner[1], corner[2],
                                                                    tab, uy);
    w0_faces_kernel<2><<<grid(n0, n1, n2 + 1), blk, 0, c->stream>>>(n0, n1, n2 + 1, corner[0], corner[1], corner[2],
                                                                    tab, uz);
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

mx_status mx_subtract_lateral_average(mx_ctx *c, const mx_geom *geom, int spherical, const int corner[3],
                                      const double *S, double *out) {
    if (!c) return MX_ERR_ARG;
    mx_status st = check_geom(c, geom, false);
    if (st) return st;
    if (!S || !out || (spherical && !corner)) return set_err(c, MX_ERR_ARG, "subtract_lateral_average: null array");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    return base_subtract_average(c, geom, spherical, corner, S, out);
}

mx_status mx_mac_project_split(mx_ctx *c, const mx_geom *geom, int spherical, const int corner[3], double *ux,
                               double *uy, double *uz, const double *rho, const double *beta0, const double *S,
                               int nr, const double *r_edge, const double *w0, double *phi, const mx_opts *opts,
                               mx_info *info) {
    if (!c) return MX_ERR_ARG;
    mx_status st = check_geom(c, geom, false);
    if (st) return st;
    if (!S) return set_err(c, MX_ERR_ARG, "mac_project_split: null S");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    const size_t ncell = (size_t)geom->n[0] * geom->n[1] * geom->n[2];
    if ((st = grow(c, &c->split_cells, &c->split_cells_bytes, ncell * sizeof(double), "mac_project_split"))) return st;
    double *bracket = (double *)c->split_cells;
    if ((st = base_subtract_average(c, geom, spherical, corner, S, bracket))) return st;
    const mx_status solve = mx_mac_project(c, geom, ux, uy, uz, rho, beta0, bracket, phi, opts, info);
    if (solve != MX_OK && solve != MX_ERR_NOCONV) return solve;
    if ((st = mx_add_w0_faces(c, geom, spherical, corner, nr, r_edge, w0, ux, uy, uz))) return st;
    MX_CUDA(c, cudaStreamSynchronize(c->stream));
    return solve;
}

}  // extern "C"
