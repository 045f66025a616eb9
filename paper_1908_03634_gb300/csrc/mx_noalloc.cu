// mx_residual_noalloc: the FP64 MAC residual r = f - L phi and its max norm
// without allocating anything, for callers that cannot call cudaMalloc (for
// example code running inside a caller-managed memory pool or arena, or
// callers that forbid allocation on their hot path).  The face coefficients are
// computed on the fly from rho and beta0, and the per-block partial maxima
// live in a file-scope device array of fixed size that every GPU loading the
// library holds until the process exits.
#include <atomic>
#include <cmath>
#include <mutex>

#include "mx_stencil.cuh"

constexpr int NA_MAX_TILES = 65536;  // one partial per 32 x 8 x 8 tile: up to 2^27 cells (512^3)

// [0, NA_MAX_TILES): block maxima; [NA_MAX_TILES]: the reduced norm
static __device__ __align__(256) double na_scratch[NA_MAX_TILES + 1];

// Effective coefficient of the low face of cell c along d (periodic average,
// wall 0, Dirichlet 2 beta0/rho), computed exactly as the stored coefficients.
__device__ __forceinline__ double na_lo_face(const DGeom &g, int d, int idx, long long c, long long stride,
                                             const double *rho, const double *beta0) {
    if (idx > 0) return (beta0[c - stride] + beta0[c]) / (rho[c - stride] + rho[c]);
    if (gper(g, d)) {
        const long long o = c + (long long)(g.n[d] - 1) * stride;
        return (beta0[o] + beta0[c]) / (rho[o] + rho[c]);
    }
    return g.lo[d] == MX_BC_DIRICHLET ? 2.0 * (beta0[c] / rho[c]) : 0.0;
}

__device__ __forceinline__ double na_hi_face(const DGeom &g, int d, int idx, long long c, long long stride,
                                             const double *rho, const double *beta0) {
    if (idx + 1 < g.n[d]) return (beta0[c] + beta0[c + stride]) / (rho[c] + rho[c + stride]);
    if (gper(g, d)) {
        const long long o = c - (long long)(g.n[d] - 1) * stride;
        return (beta0[c] + beta0[o]) / (rho[c] + rho[o]);
    }
    return g.hi[d] == MX_BC_DIRICHLET ? 2.0 * (beta0[c] / rho[c]) : 0.0;
}

__global__ void na_residual_kernel(DGeom g, const double *__restrict__ rho, const double *__restrict__ beta0,
                                   const double *__restrict__ phi, const double *__restrict__ f,
                                   double *__restrict__ r, double *part, double ih2) {
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + ZC, g.n[2]);
        for (int k = k0; k < k1; k++) {
            const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
            double b[6], v[6];
            b[0] = na_lo_face(g, 0, i, c, 1, rho, beta0);
            b[1] = na_hi_face(g, 0, i, c, 1, rho, beta0);
            b[2] = na_lo_face(g, 1, j, c, g.n[0], rho, beta0);
            b[3] = na_hi_face(g, 1, j, c, g.n[0], rho, beta0);
            b[4] = na_lo_face(g, 2, k, c, g.nxy, rho, beta0);
            b[5] = na_hi_face(g, 2, k, c, g.nxy, rho, beta0);
            nb_vals(g, phi, i, j, k, c, v);
            const double rr = f[c] - flux_sum(b, v, phi[c]) * ih2;
            r[c] = rr;
            mx = nmax(mx, fabs(rr));
        }
    }
    block_red3(mx, s2, s1);
    if (flat_tid() == 0) part[flat_bid()] = mx;
}

__global__ void na_reduce_kernel(double *part, int nb) {
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) mx = nmax(mx, part[q]);
    block_red3(mx, s2, s1);
    if (threadIdx.x == 0) part[NA_MAX_TILES] = mx;
}

// Device address of the scratch array, looked up once per device (under a lock,
// so that threads making their first call at the same time do not race).  The
// address belongs to the device's primary context: a cudaDeviceReset discards
// it, and this library must then be unloaded and loaded again.
static std::atomic<double *> na_ptr[64];
static std::mutex na_mu;

static double *na_scratch_addr(int dev) {
    double *p = na_ptr[dev].load(std::memory_order_acquire);
    if (p) return p;
    std::lock_guard<std::mutex> lock(na_mu);
    p = na_ptr[dev].load(std::memory_order_relaxed);
    if (!p) {
        if (cudaGetSymbolAddress((void **)&p, na_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        na_ptr[dev].store(p, std::memory_order_release);
    }
    return p;
}

extern "C" mx_status mx_residual_noalloc(const mx_geom *geom, const double *rho, const double *beta0,
                                         const double *phi, const double *f, double *r, double *rnorm_linf,
                                         void *cuda_stream) {
    if (!geom || !rho || !beta0 || !phi || !f || !r) return MX_ERR_ARG;
    if (check_geom(nullptr, geom, false) != MX_OK) return MX_ERR_ARG;
    const DGeom g = make_dgeom(geom);
    const dim3 grid = stencil_grid(g);
    const long long nb = (long long)grid.x * grid.y * grid.z;
    // more tiles than the fixed scratch holds, or a grid beyond the launch limits
    if (nb > NA_MAX_TILES || grid.y > 65535 || grid.z > 65535) return MX_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MX_ERR_CUDA;
    double *part = na_scratch_addr(dev);  // the first call on a device looks it up
    if (!part) return MX_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    na_residual_kernel<<<grid, dim3(SX, SY), 0, s>>>(g, rho, beta0, phi, f, r, part, 1.0 / (g.h * g.h));
    na_reduce_kernel<<<1, 1024, 0, s>>>(part, int(nb));
    if (cudaGetLastError() != cudaSuccess) return MX_ERR_CUDA;
    if (rnorm_linf) {
        if (cudaMemcpyAsync(rnorm_linf, part + NA_MAX_TILES, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return MX_ERR_CUDA;
    }
    return MX_OK;
}
