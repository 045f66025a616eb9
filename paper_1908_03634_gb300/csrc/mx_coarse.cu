// The coarse end of the V-cycle in one CTA: every level of at most
// COARSE_MAX_CELLS cells, from the first such level down to the bottom solve and
// back up, with the corrections and right-hand sides held in shared memory.
// On these levels a grid-wide launch does a few microseconds of work, so one
// launch replaces the dozens of per-level launches (smoothing, restriction,
// BiCGStab bottom solve, prolongation) that would otherwise dominate.
#include <cstring>

#include "mx_coarse.cuh"
#include "mx_rbgs.cuh"
#include "mx_stencil.cuh"

constexpr int CT = 1024;  // threads of the coarse CTA

// Exact division of x < 2^16 by d < 2^16 as a multiply-high with the
// precomputed m = ceil(2^32 / d) (the error x (m - 2^32/d) / 2^32 stays below
// 1/d, so the floor is exact).
struct FastDiv {
    unsigned d, m;
};
inline FastDiv fast_div(unsigned d) { return FastDiv{d, unsigned(((1ull << 32) + d - 1) / d)}; }
__device__ __forceinline__ int fdiv(int x, FastDiv f) { return int(__umulhi(unsigned(x), f.m)); }

template <typename T>
struct CoarseArgs {
    int nl;                        // number of levels handled (the last is the bottom)
    Level<T> lev[COARSE_MAX_LEVELS];
    FastDiv d0[COARSE_MAX_LEVELS], d1[COARSE_MAX_LEVELS], dh[COARSE_MAX_LEVELS];  // n0, n1, n0/2
    int nu1, nu2, bot_iters, singular;
};

// cell (i, j, k) of index c of a level of at most 2^16 cells
__device__ __forceinline__ void cell_ijk(int c, FastDiv d0, FastDiv d1, int &i, int &j, int &k) {
    const int r = fdiv(c, d0);
    i = c - r * int(d0.d);
    k = fdiv(r, d1);
    j = r - k * int(d1.d);
}
__device__ __forceinline__ void cell_ijk(const DGeom &g, int c, int &i, int &j, int &k) {
    i = c % g.n[0];
    const int r = c / g.n[0];
    j = r % g.n[1];
    k = r / g.n[1];
}

// the 6 face coefficients and neighbour values of in-box cell (i,j,k) = c
// with 32-bit indexing (the same values as face_coefs / nb_vals)
template <typename T>
__device__ __forceinline__ void coefs_nbs(const Level<T> &L, const T *p, int i, int j, int k, int c, T b[6], T v[6]) {
    const DGeom &g = L.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxy = nx * ny;
    const bool px = gper(g, 0), py = gper(g, 1), pz = gper(g, 2);
    b[0] = L.bx[c];
    b[1] = (i + 1 < nx) ? L.bx[c + 1] : (px ? L.bx[c - (nx - 1)] : L.hx[j + ny * k]);
    b[2] = L.by[c];
    b[3] = (j + 1 < ny) ? L.by[c + nx] : (py ? L.by[c - (ny - 1) * nx] : L.hy[i + nx * k]);
    b[4] = L.bz[c];
    b[5] = (k + 1 < nz) ? L.bz[c + nxy] : (pz ? L.bz[c - (nz - 1) * nxy] : L.hz[i + nx * j]);
    v[0] = i > 0 ? p[c - 1] : (px ? p[c + nx - 1] : T(0));
    v[1] = i + 1 < nx ? p[c + 1] : (px ? p[c - (nx - 1)] : T(0));
    v[2] = j > 0 ? p[c - nx] : (py ? p[c + (ny - 1) * nx] : T(0));
    v[3] = j + 1 < ny ? p[c + nx] : (py ? p[c - (ny - 1) * nx] : T(0));
    v[4] = k > 0 ? p[c - nxy] : (pz ? p[c + (nz - 1) * nxy] : T(0));
    v[5] = k + 1 < nz ? p[c + nxy] : (pz ? p[c - (nz - 1) * nxy] : T(0));
}

// One colour of red-black Gauss-Seidel: with n0 even the threads walk the
// colour's cells only (pair m of row r: i = 2m + parity); otherwise all cells.
template <typename T>
__device__ void cta_colour(const Level<T> &L, T *e, const T *f, int colour, T h2, FastDiv d1, FastDiv dh) {
    const DGeom &g = L.g;
    const int n0 = g.n[0];
    if (n0 % 2 == 0) {
        const int nc = int(g.N) / 2;
        for (int t = threadIdx.x; t < nc; t += CT) {
            const int r = fdiv(t, dh);  // row j + n1 k
            const int m = t - r * int(dh.d);
            const int k = fdiv(r, d1);
            const int j = r - k * int(d1.d);
            const int i = 2 * m + ((j + k + colour) & 1);
            const int c = i + n0 * r;
            T b[6], v[6];
            coefs_nbs(L, e, i, j, k, c, b, v);
            e[c] = gs_update(b, v, f[c], h2);
        }
    } else {
        for (int c = threadIdx.x; c < g.N; c += CT) {
            int i, j, k;
            cell_ijk(g, c, i, j, k);
            if (((i + j + k) & 1) != colour) continue;
            T b[6], v[6];
            coefs_nbs(L, e, i, j, k, c, b, v);
            e[c] = gs_update(b, v, f[c], h2);
        }
    }
    __syncthreads();
}

template <typename T>
__device__ void cta_resid_restrict(const Level<T> &F, const T *ef, const T *ff, const DGeom &gc, T *fc, T *ec, T ih2,
                                   FastDiv c0, FastDiv c1) {
    const DGeom &g = F.g;
    for (int C = threadIdx.x; C < gc.N; C += CT) {
        int I, J, K;
        cell_ijk(C, c0, c1, I, J, K);
        T s = T(0);
        for (int dk = 0; dk < 2; dk++)
            for (int dj = 0; dj < 2; dj++)
                for (int di = 0; di < 2; di++) {
                    const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                    const int c = i + g.n[0] * (j + g.n[1] * k);
                    T b[6], v[6];
                    coefs_nbs(F, ef, i, j, k, c, b, v);
                    s += ff[c] - flux_sum(b, v, ef[c]) * ih2;
                }
        fc[C] = s * T(0.125);
        ec[C] = T(0);
    }
    __syncthreads();
}

template <typename T>
__device__ void cta_prolong(const DGeom &gc, const T *ec, const DGeom &g, T *ef, FastDiv d0, FastDiv d1) {
    for (int c = threadIdx.x; c < g.N; c += CT) {
        int i, j, k;
        cell_ijk(c, d0, d1, i, j, k);
        ef[c] += ec[(i >> 1) + gc.n[0] * ((j >> 1) + gc.n[1] * (k >> 1))];
    }
    __syncthreads();
}

// dot product accumulated in T (FP32 on the mixed path: the bottom solve only
// needs a 1e-4 reduction, and FP64 is slow on this part)
template <typename T>
__device__ T cta_dot(const T *a, const T *b, int n) {
    T s = T(0);
    for (int q = threadIdx.x; q < n; q += CT) s += a[q] * b[q];
    __shared__ T res;
    if constexpr (sizeof(T) == sizeof(float)) {
        float m = 0.f, z = 0.f;
        block_red3f(m, s, z);
    } else {
        double m = 0.0, z = 0.0;
        block_red3(m, s, z);
    }
    if (threadIdx.x == 0) res = s;
    __syncthreads();
    const T out = res;
    __syncthreads();
    return out;
}

template <typename T>
__device__ T cta_sum(const T *a, int n) {
    T s = T(0);
    for (int q = threadIdx.x; q < n; q += CT) s += a[q];
    __shared__ T res;
    if constexpr (sizeof(T) == sizeof(float)) {
        float m = 0.f, z = 0.f;
        block_red3f(m, s, z);
    } else {
        double m = 0.0, z = 0.0;
        block_red3(m, s, z);
    }
    if (threadIdx.x == 0) res = s;
    __syncthreads();
    const T out = res;
    __syncthreads();
    return out;
}

template <typename T>
__device__ void cta_apply(const Level<T> &L, const T *x, T *y, T ih2) {
    const DGeom &g = L.g;
    for (int c = threadIdx.x; c < g.N; c += CT) {
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        T b[6], v[6];
        coefs_nbs(L, x, i, j, k, c, b, v);
        y[c] = flux_sum(b, v, x[c]) * ih2;
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// BiCGStab on a bottom level of at most 32 cells by one warp: one cell per
// lane, dot products by shuffles, the operator's neighbour values through a
// shared-memory vector; no block barriers.
template <typename T>
__device__ void warp_bicgstab(const Level<T> &L, T *x, const T *f, T *pv, int iters, int singular, T ih2) {
    const int n = int(L.g.N), lane = threadIdx.x;
    const bool act = lane < n;
    int i = 0, j = 0, k = 0;
    T b[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    if (act) {
        cell_ijk(L.g, lane, i, j, k);
        face_coefs(L, i, j, k, lane, b);
    }
    auto apply = [&](T val) -> T {  // (L val)_lane, values exchanged through pv
        if (act) pv[lane] = val;
        __syncwarp();
        T y = T(0);
        if (act) {
            T v[6];
            nb_vals(L.g, (const T *)pv, i, j, k, lane, v);
            y = flux_sum(b, v, val) * ih2;
        }
        __syncwarp();
        return y;
    };
    T rhs = act ? f[lane] : T(0);
    if (singular) rhs -= warp_sum(rhs) / T(n);
    if (!act) rhs = T(0);
    T xv = T(0), r = rhs, r0 = rhs, p = T(0), v = T(0);
    const T bnorm2 = warp_sum(rhs * rhs);
    if (bnorm2 > T(0)) {
        const T tol2 = bnorm2 * T(1e-8);
        T rho = T(1), alpha = T(1), omega = T(1);
        for (int it = 0; it < iters; it++) {
            const T rho1 = warp_sum(r0 * r);
            if (rho1 == T(0) || omega == T(0)) break;
            const T beta = (rho1 / rho) * (alpha / omega);
            p = r + beta * (p - omega * v);
            v = apply(p);
            const T r0v = warp_sum(r0 * v);
            if (r0v == T(0)) break;
            alpha = rho1 / r0v;
            const T sv = r - alpha * v;
            if (warp_sum(sv * sv) <= tol2) {
                xv += alpha * p;
                break;
            }
            const T tv = apply(sv);
            const T tt = warp_sum(tv * tv), ts = warp_sum(tv * sv);
            omega = tt > T(0) ? ts / tt : T(0);
            xv += alpha * p + omega * sv;
            r = sv - omega * tv;
            rho = rho1;
            if (warp_sum(r * r) <= tol2) break;
        }
    }
    if (!act) xv = T(0);
    if (singular) xv -= warp_sum(xv) / T(n);
    if (act) x[lane] = xv;
}

// BiCGStab on L x = f (x starts at 0), projected onto mean-free vectors when
// the problem is singular; stops at relative residual 1e-4 or `iters`.
template <typename T>
__device__ void cta_bicgstab(const Level<T> &L, T *x, const T *f, T *scr, int iters, int singular, T ih2) {
    const int n = int(L.g.N);
    if (n <= 32) {
        if (threadIdx.x < 32) warp_bicgstab(L, x, f, scr, iters, singular, ih2);
        __syncthreads();
        return;
    }
    T *r = scr, *r0 = scr + n, *p = scr + 2 * n, *v = scr + 3 * n, *sv = scr + 4 * n, *tv = scr + 5 * n;
    const T mean = singular ? cta_sum(f, n) / T(n) : T(0);
    for (int q = threadIdx.x; q < n; q += CT) {
        const T b = f[q] - mean;
        x[q] = T(0);
        r[q] = b;
        r0[q] = b;
        p[q] = T(0);
        v[q] = T(0);
    }
    __syncthreads();
    const T bnorm2 = cta_dot(r, r, n);
    if (!(bnorm2 > T(0))) return;
    const T tol2 = bnorm2 * T(1e-8);  // 1e-4 relative: ample for a multigrid bottom solve
    T rho = T(1), alpha = T(1), omega = T(1);
    for (int it = 0; it < iters; it++) {
        const T rho1 = cta_dot(r0, r, n);
        if (rho1 == T(0) || omega == T(0)) break;
        const T beta = (rho1 / rho) * (alpha / omega);
        for (int q = threadIdx.x; q < n; q += CT) p[q] = r[q] + beta * (p[q] - omega * v[q]);
        __syncthreads();
        cta_apply(L, p, v, ih2);
        const T r0v = cta_dot(r0, v, n);
        if (r0v == T(0)) break;
        alpha = rho1 / r0v;
        for (int q = threadIdx.x; q < n; q += CT) sv[q] = r[q] - alpha * v[q];
        __syncthreads();
        const T ss = cta_dot(sv, sv, n);
        if (ss <= tol2) {
            for (int q = threadIdx.x; q < n; q += CT) x[q] += alpha * p[q];
            __syncthreads();
            break;
        }
        cta_apply(L, sv, tv, ih2);
        const T tt = cta_dot(tv, tv, n);
        const T ts = cta_dot(tv, sv, n);
        omega = tt > T(0) ? ts / tt : T(0);
        for (int q = threadIdx.x; q < n; q += CT) {
            x[q] += alpha * p[q] + omega * sv[q];
            r[q] = sv[q] - omega * tv[q];
        }
        __syncthreads();
        rho = rho1;
        const T rr = cta_dot(r, r, n);
        if (rr <= tol2) break;
    }
    if (singular) {
        const T mx = cta_sum(x, n) / T(n);
        for (int q = threadIdx.x; q < n; q += CT) x[q] -= mx;
        __syncthreads();
    }
}

template <typename T>
__device__ void coarse_body(const CoarseArgs<T> &A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *e[COARSE_MAX_LEVELS], *f[COARSE_MAX_LEVELS];
    size_t off = 0;
    for (int l = 0; l < A.nl; l++) {
        e[l] = sm + off;
        off += A.lev[l].g.N;
        f[l] = sm + off;
        off += A.lev[l].g.N;
    }
    T *scr = sm + off;  // 6 bottom vectors
    // right-hand side of the first level from global memory
    for (int c = threadIdx.x; c < A.lev[0].g.N; c += CT) {
        f[0][c] = A.lev[0].f[c];
        e[0][c] = T(0);
    }
    __syncthreads();
    const int nb = A.nl - 1;
    for (int l = 0; l < nb; l++) {
        const Level<T> &L = A.lev[l];
        const T h2 = T(L.g.h * L.g.h);
        for (int q = 0; q < A.nu1; q++) {
            cta_colour(L, e[l], f[l], 0, h2, A.d1[l], A.dh[l]);
            cta_colour(L, e[l], f[l], 1, h2, A.d1[l], A.dh[l]);
        }
        cta_resid_restrict(L, e[l], f[l], A.lev[l + 1].g, f[l + 1], e[l + 1], T(1) / T(L.g.h * L.g.h), A.d0[l + 1],
                           A.d1[l + 1]);
    }
    {
        const Level<T> &L = A.lev[nb];
        cta_bicgstab(L, e[nb], f[nb], scr, A.bot_iters, A.singular, T(1) / T(L.g.h * L.g.h));
    }
    for (int l = nb - 1; l >= 0; l--) {
        const Level<T> &L = A.lev[l];
        const T h2 = T(L.g.h * L.g.h);
        cta_prolong(A.lev[l + 1].g, e[l + 1], L.g, e[l], A.d0[l], A.d1[l]);
        for (int q = 0; q < A.nu2; q++) {
            cta_colour(L, e[l], f[l], 0, h2, A.d1[l], A.dh[l]);
            cta_colour(L, e[l], f[l], 1, h2, A.d1[l], A.dh[l]);
        }
    }
    for (int c = threadIdx.x; c < A.lev[0].g.N; c += CT) A.lev[0].e[c] = e[0][c];
}

template <typename T>
__global__ void __launch_bounds__(CT) coarse_vcycle_kernel(CoarseArgs<T> A) {
    pdl_trigger();
    pdl_wait();
    coarse_body(A);
}

// batched: one CTA per box (boxes already converged return at once)
__global__ void __launch_bounds__(CT) coarse_vcycle_batch_kernel(const CoarseArgs<float> *args, const SolveState *st) {
    if (st[blockIdx.x].done) return;
    coarse_body(args[blockIdx.x]);
}

template <typename T>
size_t coarse_smem_bytes(const Level<T> *levs, int nl) {
    size_t n = 0;
    for (int l = 0; l < nl; l++) n += 2 * (size_t)levs[l].g.N;
    n += 6 * (size_t)levs[nl - 1].g.N;
    return n * sizeof(T);
}

template <typename T>
bool coarse_fits(const Level<T> *levs, int nl) {
    return nl >= 1 && nl <= COARSE_MAX_LEVELS && levs[0].g.N <= COARSE_MAX_CELLS &&
           coarse_smem_bytes(levs, nl) <= COARSE_MAX_SMEM;
}

template <typename T>
void k_coarse_vcycle(cudaStream_t s, const Level<T> *levs, int nl, int nu1, int nu2, int bot_iters, int singular) {
    CoarseArgs<T> A;
    A.nl = nl;
    for (int l = 0; l < nl; l++) {
        A.lev[l] = levs[l];
        A.d0[l] = fast_div(levs[l].g.n[0]);
        A.d1[l] = fast_div(levs[l].g.n[1]);
        A.dh[l] = fast_div(levs[l].g.n[0] > 1 ? levs[l].g.n[0] / 2 : 1);
    }
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.bot_iters = bot_iters;
    A.singular = singular;
    const size_t smem = coarse_smem_bytes(levs, nl);
    launch_pdl(coarse_vcycle_kernel<T>, dim3(1), dim3(CT), smem, s, A);
}

// Allow the coarse kernels more than the default 48 KB of dynamic shared
// memory (called once per device, outside any stream capture).
cudaError_t coarse_init() {
    cudaError_t e = cudaFuncSetAttribute(coarse_vcycle_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         COARSE_MAX_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(coarse_vcycle_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, COARSE_MAX_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(coarse_vcycle_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                COARSE_MAX_SMEM);
}

size_t coarse_args_bytes() { return sizeof(CoarseArgs<float>); }

void coarse_fill_args(void *dst, const Level<float> *levs, int nl, int nu1, int nu2, int bot_iters, int singular) {
    CoarseArgs<float> A;
    std::memset(&A, 0, sizeof(A));
    A.nl = nl;
    for (int l = 0; l < nl; l++) {
        A.lev[l] = levs[l];
        A.d0[l] = fast_div(levs[l].g.n[0]);
        A.d1[l] = fast_div(levs[l].g.n[1]);
        A.dh[l] = fast_div(levs[l].g.n[0] > 1 ? levs[l].g.n[0] / 2 : 1);
    }
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.bot_iters = bot_iters;
    A.singular = singular;
    std::memcpy(dst, &A, sizeof(A));
}

size_t coarse_smem_bytes_f(const Level<float> *levs, int nl) { return coarse_smem_bytes(levs, nl); }

void k_coarse_vcycle_batch(cudaStream_t s, const void *dev_args, const SolveState *st, int nbox, size_t smem) {
    if (nbox > 0)
        coarse_vcycle_batch_kernel<<<nbox, CT, smem, s>>>((const CoarseArgs<float> *)dev_args, st);
}

template bool coarse_fits<float>(const Level<float> *, int);
template bool coarse_fits<double>(const Level<double> *, int);
template void k_coarse_vcycle<float>(cudaStream_t, const Level<float> *, int, int, int, int, int);
template void k_coarse_vcycle<double>(cudaStream_t, const Level<double> *, int, int, int, int, int);
