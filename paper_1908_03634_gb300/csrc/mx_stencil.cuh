// Device helpers shared by the cell-centred kernels: neighbour access with the
// boundary closures, the 7-point face-flux operator and block reductions.
#pragma once

#include "mx_internal.cuh"

// Coefficients of the 6 faces of cell (i,j,k): w, e, s, n, b, t (x-, x+, y-, y+, z-, z+).
template <typename T>
__device__ __forceinline__ void face_coefs(const Level<T> &L, int i, int j, int k, long long c, T b[6]) {
    const DGeom &g = L.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    b[0] = L.bx[c];
    b[1] = (i + 1 < nx) ? L.bx[c + 1] : (gper(g, 0) ? L.bx[c - (nx - 1)] : L.hx[j + (long long)ny * k]);
    b[2] = L.by[c];
    b[3] = (j + 1 < ny) ? L.by[c + nx] : (gper(g, 1) ? L.by[c - (long long)(ny - 1) * nx] : L.hy[i + (long long)nx * k]);
    b[4] = L.bz[c];
    b[5] = (k + 1 < nz) ? L.bz[c + g.nxy] : (gper(g, 2) ? L.bz[c - (long long)(nz - 1) * g.nxy] : L.hz[i + (long long)nx * j]);
}

// The corrected MAC face velocity U_f - q_f (phi_R - phi_L) (Appendix A's
// correction): face p of axis d between cells cl and cr (ci: the interior cell
// of a boundary face), phi = 0 outside a Dirichlet face, U = 0 on a wall face.
// One FP64 expression for every face kind, shared by the correction kernels.
__device__ __forceinline__ double corr_face_value(const DGeom &g, int d, int p, long long cl, long long cr,
                                                  long long ci, const double *__restrict__ phi, double q, double u) {
    const int n = g.n[d];
    const bool inner = (p > 0 && p < n) || gper(g, d);
    const int bc = p == 0 ? g.lo[d] : g.hi[d];
    const bool wall = !inner && bc != MX_BC_DIRICHLET;
    const double pr = (inner || p == 0) ? phi[inner ? cr : ci] : 0.0;
    const double pl = (inner || p != 0) ? phi[inner ? cl : ci] : 0.0;
    const double un = fma(-q, pr - pl, u);
    return wall ? 0.0 : un;
}

// The 6 neighbour values of cell (i,j,k); 0 beyond a non-periodic face.
template <typename T>
__device__ __forceinline__ void nb_vals(const DGeom &g, const T *p, int i, int j, int k, long long c, T v[6]) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    v[0] = i > 0 ? p[c - 1] : (gper(g, 0) ? p[c + nx - 1] : T(0));
    v[1] = i + 1 < nx ? p[c + 1] : (gper(g, 0) ? p[c - (nx - 1)] : T(0));
    v[2] = j > 0 ? p[c - nx] : (gper(g, 1) ? p[c + (long long)(ny - 1) * nx] : T(0));
    v[3] = j + 1 < ny ? p[c + nx] : (gper(g, 1) ? p[c - (long long)(ny - 1) * nx] : T(0));
    v[4] = k > 0 ? p[c - g.nxy] : (gper(g, 2) ? p[c + (long long)(nz - 1) * g.nxy] : T(0));
    v[5] = k + 1 < nz ? p[c + g.nxy] : (gper(g, 2) ? p[c - (long long)(nz - 1) * g.nxy] : T(0));
}

// h^2 (L p)_c = sum_faces b_f (p_nb - p_c)
template <typename T>
__device__ __forceinline__ T flux_sum(const T b[6], const T v[6], T pc) {
    T s = b[0] * (v[0] - pc);
    s += b[1] * (v[1] - pc);
    s += b[2] * (v[2] - pc);
    s += b[3] * (v[3] - pc);
    s += b[4] * (v[4] - pc);
    s += b[5] * (v[5] - pc);
    return s;
}

// 1/d in FP64 without the FP64 divide (which runs at 1/11 of the FMA rate on
// this part): a correctly rounded FP32 reciprocal refined by two Newton-Raphson
// steps r <- r + r (1 - d r); the result is within about 2 ulp of 1/d.
// Values outside the FP32 range fall back to the division.
static __device__ __noinline__ double rcp64_slow(double d) { return 1.0 / d; }
__device__ __forceinline__ double rcp64(double d) {
    const float df = __double2float_rn(d);
    const float rf = __frcp_rn(df);
    // out of line: an inlined, predicated division would occupy the FP64 pipe on every call
    if (!(fabsf(df) > 1e-37f && fabsf(df) < 1e37f)) return rcp64_slow(d);
    double r = double(rf);
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

__device__ __forceinline__ int flat_tid() {
    return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}
__device__ __forceinline__ int flat_bid() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// Block-wide (max, sum, sum) of three doubles; result valid in thread 0.
// Fixed shuffle order: deterministic.
__device__ __forceinline__ void block_red3(double &a, double &b, double &c) {
    __shared__ double sh[96];
    const int t = flat_tid();
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    for (int o = 16; o > 0; o >>= 1) {
        a = nmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int lane = t & 31, wid = t >> 5;
    if (lane == 0) {
        sh[wid] = a;
        sh[32 + wid] = b;
        sh[64 + wid] = c;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (nthr + 31) >> 5;
        a = lane < nw ? sh[lane] : 0.0;
        b = lane < nw ? sh[32 + lane] : 0.0;
        c = lane < nw ? sh[64 + lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a = nmax(a, __shfl_xor_sync(0xffffffffu, a, o));
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
    }
    __syncthreads();
}

// Block-wide (max, sum, sum) of three floats (FP32 shuffles; GB300 runs FP64
// at 1/64 of the FP32 rate, so hot kernels keep their partials in FP32 and only
// the one-block finalize kernels accumulate in FP64).  Result in thread 0.
__device__ __forceinline__ void block_red3f(float &a, float &b, float &c) {
    __shared__ float shf[96];
    const int t = flat_tid();
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    for (int o = 16; o > 0; o >>= 1) {
        a = nmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int lane = t & 31, wid = t >> 5;
    if (lane == 0) {
        shf[wid] = a;
        shf[32 + wid] = b;
        shf[64 + wid] = c;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (nthr + 31) >> 5;
        a = lane < nw ? shf[lane] : 0.f;
        b = lane < nw ? shf[32 + lane] : 0.f;
        c = lane < nw ? shf[64 + lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) {
            a = nmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
    }
    __syncthreads();
}

// Reduce nb partial triples (max, sum, sum) with one block; results in thread 0.
__device__ __forceinline__ void reduce_partials3(const double *p, int nb, double &a, double &b, double &c) {
    a = 0.0;
    b = 0.0;
    c = 0.0;
    for (int q = flat_tid(); q < nb; q += blockDim.x * blockDim.y * blockDim.z) {
        a = nmax(a, p[3 * q]);
        b += p[3 * q + 1];
        c += p[3 * q + 2];
    }
    block_red3(a, b, c);
}

// Launch shape of the cell-centred stencil kernels: (32 x 8) threads per block,
// each thread walking ZC cells in z.
constexpr int SX = 32, SY = 8, ZC = 8;
inline dim3 stencil_grid(const DGeom &g) {
    return dim3((g.n[0] + SX - 1) / SX, (g.n[1] + SY - 1) / SY, (g.n[2] + ZC - 1) / ZC);
}
// z-chunk for a level with bxy blocks per chunk of planes: `cap` planes per
// thread (8 unless tuned) on large levels, fewer (down to 1) until the grid
// has >= 16 blocks per SM, so small levels are not latency-bound on a few
// long-running blocks (at 4 per SM the 128^3 restriction ran 7% slower).
inline int zchunk(long long bxy, int nz, int cap = ZC) {
    int zc = cap;
    while (zc > 1 && bxy * ((nz + zc - 1) / zc) < 16 * 152) zc >>= 1;
    return zc;
}
inline dim3 stencil_grid_zc(const DGeom &g, int zc) {
    return dim3((g.n[0] + SX - 1) / SX, (g.n[1] + SY - 1) / SY, (g.n[2] + zc - 1) / zc);
}
inline int stencil_zc(const DGeom &g, int cap = ZC) {
    return zchunk((long long)((g.n[0] + SX - 1) / SX) * ((g.n[1] + SY - 1) / SY), g.n[2], cap);
}
inline int stencil_blocks(const DGeom &g) {
    dim3 d = stencil_grid(g);
    return int(d.x * d.y * d.z);
}
