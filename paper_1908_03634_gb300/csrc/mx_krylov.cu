// Flexible conjugate gradients, FCG(1), around the FP32 V-cycle: the mixed MAC
// solve with mx_opts::krylov = 1.
//
// The system is L phi = f of the MAC projection (Eq. div1, div2; Appendix A),
// -L symmetric positive (semi)definite.  Iteration k
// holds r = f - L phi as rhat = r / scale (FP32; the V-cycle's right-hand side)
// and e = V(rhat), the V-cycle's correction.  Then
//   beta = -(e . q_prev) / (p_prev . q_prev)      (0 when restarting)
//   p    = e + beta p_prev,   q = h^2 L p          (FP32 stencil, hi coefficients)
//   t    = scale h^2 (p . rhat) / (p . q)          (exact line search along p)
//   phi += t p in double-float, followed by the residual of the new phi
//   (k_df_resid), so the loop's accuracy is that of iterative refinement.
// beta makes p conjugate (in the -L inner product) to the previous direction:
// Notay's flexible CG truncated to one direction (SIAM J. Sci. Comput. 22,
// 2000), which does not need the preconditioner to be symmetric or fixed (the
// sweeps run red then black on both sides of the coarse correction, and the
// bottom solve is BiCGStab).  With p = e exact (t = scale, beta = 0) the step
// is the refinement step.  The directions and q are FP32: they set the step
// sizes only, never the residual that decides convergence.
//
// Storage: two direction buffers alternating with the V-cycle count (a tile's
// halo is staged from the previous direction while other tiles write the new
// one) and q, written in place (only the next iteration's dot product reads it).
#include <cstdint>

#include "mx_krylov.cuh"
#include "mx_stencil.cuh"

namespace {

constexpr int KX = 32, KY = 8, KZ = 8;
constexpr int KHX = KX + 2, KHY = KY + 2, KHZ = KZ + 2;
constexpr int K_THREADS = 256;

__device__ __forceinline__ int kmap(int u, int n, bool per) {
    if (u >= 0 && u < n) return u;
    if (!per || u < -1 || u > n) return -1;
    return u < 0 ? u + n : u - n;
}

// per-block partials (0, e . q_prev, 0); nothing is read on a restart
template <bool VEC>
__global__ void __launch_bounds__(256) kry_dot_kernel(const float *__restrict__ e, const float *__restrict__ q,
                                                      long long n, const SolveState *st, double *part) {
    float s = 0.f;
    if (!st->kry_restart) {
        const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        const long long stride = (long long)gridDim.x * blockDim.x;
        long long done = 0;
        if (VEC) {
            const long long n4 = n >> 2;
            const float4 *__restrict__ e4 = reinterpret_cast<const float4 *>(e);
            const float4 *__restrict__ q4 = reinterpret_cast<const float4 *>(q);
            for (long long i = t0; i < n4; i += stride) {
                const float4 a = e4[i], b = q4[i];
                s = fmaf(a.x, b.x, s);
                s = fmaf(a.y, b.y, s);
                s = fmaf(a.z, b.z, s);
                s = fmaf(a.w, b.w, s);
            }
            done = n4 << 2;
        }
        for (long long i = done + t0; i < n; i += stride) s = fmaf(e[i], q[i], s);
    }
    float z0 = 0.f, z2 = 0.f;
    block_red3f(z0, s, z2);
    if (threadIdx.x == 0) {
        double *p = part + 3 * blockIdx.x;
        p[0] = 0.0;
        p[1] = double(s);
        p[2] = 0.0;
    }
}

__global__ void kry_beta_kernel(const double *part, int nb, SolveState *st) {
    double a, b, c;
    reduce_partials3(part, nb, a, b, c);
    if (flat_tid() == 0) {
        double beta = 0.0;
        if (!st->kry_restart) {
            beta = -b / st->kry_pq;
            if (!isfinite(beta)) beta = 0.0;
        }
        st->kry_beta = beta;
    }
}

// p = e + beta p_prev staged with a one-cell halo (zero outside the box on
// non-periodic axes, as the stored boundary coefficients expect), written to
// the buffer of this iteration; q = h^2 L p; partials (0, p . q, p . rhat).
__global__ void __launch_bounds__(K_THREADS) kry_dir_kernel(Level<float> L, const float *__restrict__ e,
                                                            float *p0, float *p1, float *__restrict__ q,
                                                            const SolveState *st, double *part) {
    __shared__ float sp[KHZ][KHY][KHX];
    const DGeom &g = L.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const bool px = gper(g, 0), py = gper(g, 1), pz = gper(g, 2);
    const int x0 = blockIdx.x * KX, y0 = blockIdx.y * KY, z0 = blockIdx.z * KZ;
    const int tid = threadIdx.x;
    const bool odd = st->iter & 1;
    float *__restrict__ pn = odd ? p1 : p0;
    const float *__restrict__ po = odd ? p0 : p1;
    const bool restart = st->kry_restart != 0;
    const float beta = float(st->kry_beta);
    for (int t = tid; t < KHX * KHY * KHZ; t += K_THREADS) {
        const int ax = t % KHX, ay = (t / KHX) % KHY, az = t / (KHX * KHY);
        const int lx = kmap(x0 - 1 + ax, nx, px), ly = kmap(y0 - 1 + ay, ny, py), lz = kmap(z0 - 1 + az, nz, pz);
        float v = 0.f;
        if (lx >= 0 && ly >= 0 && lz >= 0) {
            const long long c = lx + (long long)nx * (ly + (long long)ny * lz);
            v = e[c];
            if (!restart) v = fmaf(beta, po[c], v);
        }
        sp[az][ay][ax] = v;
    }
    __syncthreads();
    float spq = 0.f, spr = 0.f;
    for (int t = tid; t < KX * KY * KZ; t += K_THREADS) {
        const int ix = t % KX, iy = (t / KX) % KY, iz = t / (KX * KY);
        const int i = x0 + ix, j = y0 + iy, k = z0 + iz;
        if (i >= nx || j >= ny || k >= nz) continue;
        const long long c = i + (long long)nx * (j + (long long)ny * k);
        const int ax = ix + 1, ay = iy + 1, az = iz + 1;
        const float pc = sp[az][ay][ax];
        pn[c] = pc;
        // high-side faces: the neighbour's low face, the periodic image, or the boundary plane
        const float be = i + 1 < nx ? L.bx[c + 1] : (px ? L.bx[c - (nx - 1)] : L.hx[j + (long long)ny * k]);
        const float bn = j + 1 < ny ? L.by[c + nx]
                                    : (py ? L.by[c - (long long)(ny - 1) * nx] : L.hy[i + (long long)nx * k]);
        const float bt = k + 1 < nz ? L.bz[c + g.nxy]
                                    : (pz ? L.bz[c - (long long)(nz - 1) * g.nxy] : L.hz[i + (long long)nx * j]);
        float qv = L.bx[c] * (sp[az][ay][ax - 1] - pc);
        qv = fmaf(be, sp[az][ay][ax + 1] - pc, qv);
        qv = fmaf(L.by[c], sp[az][ay - 1][ax] - pc, qv);
        qv = fmaf(bn, sp[az][ay + 1][ax] - pc, qv);
        qv = fmaf(L.bz[c], sp[az - 1][ay][ax] - pc, qv);
        qv = fmaf(bt, sp[az + 1][ay][ax] - pc, qv);
        q[c] = qv;
        spq = fmaf(pc, qv, spq);
        spr = fmaf(pc, L.f[c], spr);
    }
    float z0f = 0.f;
    block_red3f(z0f, spq, spr);
    if (tid == 0) {
        double *p = part + 3 * flat_bid();
        p[0] = 0.0;
        p[1] = double(spq);
        p[2] = double(spr);
    }
}

// the line-search step t into the update step of the residual kernel; a
// direction that is not a descent direction of the energy (p . q >= 0, or a
// non-finite sum) takes t = 0 and restarts from p = e
__global__ void kry_step_kernel(const double *part, int nb, SolveState *st, double h2) {
    double a, pq, pr;
    reduce_partials3(part, nb, a, pq, pr);
    if (flat_tid() == 0) {
        double t = 0.0;
        int restart = 1;
        if (pq < 0.0 && isfinite(pq) && isfinite(pr)) {
            t = st->scale * h2 * pr / pq;
            if (isfinite(t)) {
                restart = 0;
                st->kry_pq = pq;
            } else {
                t = 0.0;
            }
        }
        st->kry_restart = restart;
        const float th = __double2float_rn(t);
        st->upd_h = th;
        st->upd_l = __double2float_rn(t - double(th));
    }
}

}  // namespace

void k_kry_dot(cudaStream_t s, long long n, const float *e, const float *q, SolveState *st, double *partials) {
    const int nb = red_blocks(n);
    const bool vec = ((reinterpret_cast<uintptr_t>(e) | reinterpret_cast<uintptr_t>(q)) & 15) == 0;
    if (vec) kry_dot_kernel<true><<<nb, 256, 0, s>>>(e, q, n, st, partials);
    else kry_dot_kernel<false><<<nb, 256, 0, s>>>(e, q, n, st, partials);
    kry_beta_kernel<<<1, 1024, 0, s>>>(partials, nb, st);
}

void k_kry_dir(cudaStream_t s, const Level<float> &L0, const float *e, float *p0, float *p1, float *q,
               SolveState *st, double *partials) {
    const DGeom &g = L0.g;
    const dim3 grid((g.n[0] + KX - 1) / KX, (g.n[1] + KY - 1) / KY, (g.n[2] + KZ - 1) / KZ);
    kry_dir_kernel<<<grid, K_THREADS, 0, s>>>(L0, e, p0, p1, q, st, partials);
    kry_step_kernel<<<1, 1024, 0, s>>>(partials, int(grid.x * grid.y * grid.z), st, g.h * g.h);
}

int kry_dir_blocks(const DGeom &g) {
    return ((g.n[0] + KX - 1) / KX) * ((g.n[1] + KY - 1) / KY) * ((g.n[2] + KZ - 1) / KZ);
}
