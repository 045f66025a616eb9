// Nodal projection (Step 11; Eq. div3; Appendix A) on the GPU.
//
// phi lives on nodes; a periodic axis of n cells has n nodes, a wall axis n+1.
// The operator is the trilinear finite-element discretisation of
// div(sigma grad phi) with cell-centred sigma = beta0/rho and lumped node
// weights w (1 inside, 1/2 on a wall, ...).  On cubic cells the element
// stiffness couples a node only to the corners that differ from it in two or
// three indices (edge neighbours have coefficient 0), so
//     12 w h^2 (L phi)_n = sum_m c_m (phi_m - phi_n),
// over the 12 face-diagonal neighbours m (c_m = sum of sigma over the two cells
// holding both nodes) and the 8 body-diagonal ones (c_m = sigma of the one
// cell).  Gauss-Seidel with the four colours (i mod 2, j mod 2) updates nodes
// that are never coupled to each other.  Coarse levels: sigma averaged over 8
// cells, full-weighting restriction scaled by the node weights, trilinear
// prolongation.  The refinement loop runs in double-float as for the MAC solve.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mx_async.cuh"
#include "mx_dfmath.cuh"
#include "mx_solver.cuh"
#include "mx_stencil.cuh"

struct NGeom {
    int n[3];   // cells
    int m[3];   // nodes
    int per[3];
    long long N, M;  // cells, nodes
    double h;
};

template <typename T>
struct NLevel {
    NGeom g;
    T *sigma;     // cells
    T *f, *e, *r; // nodes (r: residual scratch of the restriction)
    T *e2;        // second correction buffer (the Chebyshev steps alternate e <-> e2)
};

struct NDF {             // double-float arrays of the finest level
    float *sh, *sl;      // sigma
    float *fh, *fl;      // 12 h^2 w f  (the scaled nodal RHS)
    float *ph, *pl;      // phi, buffer 0
    float *ph2, *pl2;    // phi, buffer 1: after k updates phi is in buffer k & 1
};
// the phi buffer after `it` updates
__device__ __forceinline__ const float *nd_phi_h(const NDF &D, int it) { return (it & 1) ? D.ph2 : D.ph; }
__device__ __forceinline__ const float *nd_phi_l(const NDF &D, int it) { return (it & 1) ? D.pl2 : D.pl; }

struct NodalPlan {
    NGeom g;
    int prec;
    void *mem = nullptr;
    int nlev = 0;
    NLevel<float> L32[MX_MAXLEV];
    NLevel<double> L64[MX_MAXLEV];
    NDF D;
    double *sigma64 = nullptr, *f64 = nullptr;
    float4 *cellp = nullptr;  // mixed: per cell beta0 (ux, uy, uz, Sbar) as double-float pairs (two float4)
    float *bot32 = nullptr;
    double *bot64 = nullptr;
    // CUDA graph of the refinement loop, keyed by what it was captured with
    cudaGraphExec_t graph = nullptr;
    const void *graph_phi = nullptr;
    int graph_nu1 = -1, graph_nu2 = -1, graph_bot = -1, graph_tilez = -1, graph_smoother = -1;
    long long last_use = 0;
};

static NGeom make_ngeom(const DGeom &d) {
    NGeom g;
    for (int a = 0; a < 3; a++) {
        g.n[a] = d.n[a];
        g.per[a] = d.lo[a] == MX_BC_PERIODIC;
        g.m[a] = d.n[a] + (g.per[a] ? 0 : 1);
    }
    g.N = (long long)g.n[0] * g.n[1] * g.n[2];
    g.M = (long long)g.m[0] * g.m[1] * g.m[2];
    g.h = d.h;
    return g;
}

static int nodal_levels(const NGeom &g0, NGeom *out) {
    int nl = 0;
    out[nl++] = g0;
    for (;;) {
        const NGeom &g = out[nl - 1];
        bool ok = nl < MX_MAXLEV;
        for (int a = 0; a < 3; a++) ok = ok && g.n[a] % 2 == 0 && g.n[a] >= 4;
        if (!ok) break;
        NGeom c = g;
        for (int a = 0; a < 3; a++) {
            c.n[a] = g.n[a] / 2;
            c.m[a] = c.n[a] + (c.per[a] ? 0 : 1);
        }
        c.N = (long long)c.n[0] * c.n[1] * c.n[2];
        c.M = (long long)c.m[0] * c.m[1] * c.m[2];
        c.h = 2.0 * g.h;
        out[nl++] = c;
    }
    return nl;
}

// ---- device helpers ------------------------------------------------------------------

__device__ __forceinline__ int cell_wrap(const NGeom &g, int d, int i) {  // -1: outside a wall
    if (i >= 0 && i < g.n[d]) return i;
    if (!g.per[d]) return -1;
    return i < 0 ? i + g.n[d] : i - g.n[d];
}
__device__ __forceinline__ int node_wrap(const NGeom &g, int d, int a) {
    if (a >= 0 && a < g.m[d]) return a;
    if (!g.per[d]) return -1;
    return a < 0 ? a + g.m[d] : a - g.m[d];
}
__device__ __forceinline__ long long nidx(const NGeom &g, int a, int b, int c) {
    return a + (long long)g.m[0] * (b + (long long)g.m[1] * c);
}
__device__ __forceinline__ long long cidx(const NGeom &g, int i, int j, int k) {
    return i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
}
// node weight: (number of cells touching the node)/8
__device__ __forceinline__ float node_w(const NGeom &g, int a, int b, int c) {
    float w = 1.f;
    if (!g.per[0] && (a == 0 || a == g.m[0] - 1)) w *= 0.5f;
    if (!g.per[1] && (b == 0 || b == g.m[1] - 1)) w *= 0.5f;
    if (!g.per[2] && (c == 0 || c == g.m[2] - 1)) w *= 0.5f;
    return w;
}
__device__ __forceinline__ void node_of(const NGeom &g, long long q, int &a, int &b, int &c) {
    const int qi = int(q);  // node counts are < 2^31 (checked on entry)
    a = qi % g.m[0];
    const int r = qi / g.m[0];
    b = r % g.m[1];
    c = r / g.m[1];
}

// sigma of the 8 cells around node (a,b,c): s[iz][iy][ix], index 0 = cell a-1, 1 = cell a
template <typename T>
__device__ __forceinline__ void cell_ring(const NGeom &g, const T *sig, int a, int b, int c, T s[2][2][2]) {
    for (int dz = 0; dz < 2; dz++) {
        const int k = cell_wrap(g, 2, c - 1 + dz);
        for (int dy = 0; dy < 2; dy++) {
            const int j = cell_wrap(g, 1, b - 1 + dy);
            for (int dx = 0; dx < 2; dx++) {
                const int i = cell_wrap(g, 0, a - 1 + dx);
                s[dz][dy][dx] = (i >= 0 && j >= 0 && k >= 0) ? sig[cidx(g, i, j, k)] : T(0);
            }
        }
    }
}

// Visit the 20 coupled neighbours of node (a,b,c): fn(coef, node index or -1)
template <typename T, typename F>
__device__ __forceinline__ void for_couplings(const NGeom &g, int a, int b, int c, const T s[2][2][2], F fn) {
    for (int oz = -1; oz <= 1; oz++)
        for (int oy = -1; oy <= 1; oy++)
            for (int ox = -1; ox <= 1; ox++) {
                const int nz_ = (ox != 0) + (oy != 0) + (oz != 0);
                if (nz_ < 2) continue;
                // cells holding both nodes: along an axis with offset o != 0 the one
                // cell on that side, along an axis with o == 0 both cells
                T coef = T(0);
                for (int dz = 0; dz < 2; dz++) {
                    if (oz != 0 && dz != (oz > 0)) continue;
                    for (int dy = 0; dy < 2; dy++) {
                        if (oy != 0 && dy != (oy > 0)) continue;
                        for (int dx = 0; dx < 2; dx++) {
                            if (ox != 0 && dx != (ox > 0)) continue;
                            coef += s[dz][dy][dx];
                        }
                    }
                }
                const int na = node_wrap(g, 0, a + ox), nb = node_wrap(g, 1, b + oy), nc = node_wrap(g, 2, c + oz);
                fn(coef, (na >= 0 && nb >= 0 && nc >= 0) ? nidx(g, na, nb, nc) : -1LL);
            }
}

// ---- setup: sigma = beta0/rho (FP64, then FP32 copy and double-float split) -----------

__global__ void nd_sigma_kernel(long long N, const double *__restrict__ rho, const double *__restrict__ beta0,
                                double *__restrict__ s64, float *__restrict__ s32, float *__restrict__ sl) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const double v = beta0[q] * rcp64(rho[q]);
        if (s64) s64[q] = v;
        if (s32) {
            const float hi = __double2float_rn(v);
            s32[q] = hi;
            if (sl) sl[q] = __double2float_rn(v - double(hi));
        }
    }
}

template <typename T>
__global__ void nd_coarsen_sigma_kernel(NLevel<T> F, NLevel<T> C) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < C.g.N; q += (long long)gridDim.x * blockDim.x) {
        const int I = int(q % C.g.n[0]), J = int((q / C.g.n[0]) % C.g.n[1]), K = int(q / ((long long)C.g.n[0] * C.g.n[1]));
        T s = T(0);
        for (int e = 0; e < 8; e++) s += F.sigma[cidx(F.g, 2 * I + (e & 1), 2 * J + ((e >> 1) & 1), 2 * K + ((e >> 2) & 1))];
        C.sigma[q] = s * T(0.125);
    }
}

// ---- RHS f = D(beta0 U) - Sbar_n, with weighted sums for the mean -----------------------

// Node columns (a, b) walk up c: the divergence at node (a,b,c) sums over the
// (up to) 8 touching cells, which form the cell layers k = c-1 and k = c.  Each
// layer's 4 cells are reduced once into
//   x = sum_j (beta0 U_x)(a, j) - (beta0 U_x)(a-1, j)   (cells on the +x side minus -x side)
//   y = sum_i (beta0 U_y)(i, b) - (beta0 U_y)(i, b-1)
//   z = sum   (beta0 U_z),  s = sum beta0 Sbar,  n = number of cells
// and node c combines layers c-1 and c: (D_n U) = (x + x' + y + y' + z' - z)/(4 h w),
// Sbar_n = (s + s')/n, with w = n/8 (the node weight) a power of two.
constexpr int NRZ = 16;  // nodes per thread along z in the node-column kernels

struct RhsLayer {
    double x, y, z, s;
    int n;
};

__device__ __forceinline__ RhsLayer rhs_layer(const NGeom &g, const double *__restrict__ ux,
                                              const double *__restrict__ uy, const double *__restrict__ uz,
                                              const double *__restrict__ beta0, const double *__restrict__ sbar,
                                              int i0, int i1, int j0, int j1, int k) {
    RhsLayer L = {0.0, 0.0, 0.0, 0.0, 0};
    const int kk = cell_wrap(g, 2, k);
    if (kk < 0) return L;
    for (int jj = 0; jj < 2; jj++) {
        const int j = jj ? j1 : j0;
        if (j < 0) continue;
        for (int ii = 0; ii < 2; ii++) {
            const int i = ii ? i1 : i0;
            if (i < 0) continue;
            const int c = i + g.n[0] * (j + g.n[1] * kk);
            const double bt = beta0[c];
            const double px = bt * ux[c], py = bt * uy[c];
            L.x += ii ? px : -px;
            L.y += jj ? py : -py;
            L.z = fma(bt, uz[c], L.z);
            L.s = fma(bt, sbar[c], L.s);
            L.n++;
        }
    }
    return L;
}

// f = D_n(beta0 U) - Sbar_n - cm (cm = the weighted mean when sub_mean), with
// per-block partials (max |f|, sum w f, sum w); f may be null (divergence check)
__global__ void nd_rhs_col_kernel(NGeom g, const double *__restrict__ ux, const double *__restrict__ uy,
                                  const double *__restrict__ uz, const double *__restrict__ beta0,
                                  const double *__restrict__ sbar, double *__restrict__ f, double *part, int sub_mean,
                                  const SolveState *st, double i4h) {
    double mx = 0.0, s1 = 0.0, s0 = 0.0;
    const int a = blockIdx.x * 32 + threadIdx.x, b = blockIdx.y * 8 + threadIdx.y;
    const int c0 = blockIdx.z * NRZ, c1 = min(c0 + NRZ, g.m[2]);
    if (a < g.m[0] && b < g.m[1]) {
        const double cm = sub_mean ? st->mean : 0.0;
        const int i0 = cell_wrap(g, 0, a - 1), i1 = cell_wrap(g, 0, a);
        const int j0 = cell_wrap(g, 1, b - 1), j1 = cell_wrap(g, 1, b);
        RhsLayer lo = rhs_layer(g, ux, uy, uz, beta0, sbar, i0, i1, j0, j1, c0 - 1);
        for (int c = c0; c < c1; c++) {
            const RhsLayer hi = rhs_layer(g, ux, uy, uz, beta0, sbar, i0, i1, j0, j1, c);
            const int cnt = lo.n + hi.n;  // 1, 2, 4 or 8
            const double ic = cnt == 8 ? 0.125 : cnt == 4 ? 0.25 : cnt == 2 ? 0.5 : 1.0;
            const double div = ((lo.x + hi.x) + (lo.y + hi.y)) + (hi.z - lo.z);
            const double v = div * (8.0 * i4h * ic) - (lo.s + hi.s) * ic - cm;
            const double w = 0.125 * cnt;
            if (f) f[a + g.m[0] * (b + g.m[1] * c)] = v;
            mx = nmax(mx, fabs(v));
            s1 = fma(w, v, s1);
            s0 += w;
            lo = hi;
        }
    }
    block_red3(mx, s1, s0);
    if (flat_tid() == 0) {
        double *p = part + 3 * flat_bid();
        p[0] = mx;
        p[1] = s1;
        p[2] = s0;
    }
}

static dim3 nd_node_grid(const NGeom &g) { return dim3((g.m[0] + 31) / 32, (g.m[1] + 7) / 8, (g.m[2] + NRZ - 1) / NRZ); }
static int nd_node_blocks(const NGeom &g) {
    const dim3 d = nd_node_grid(g);
    return int(d.x * d.y * d.z);
}

// stage 0: weighted mean; stage 1: norms of the final RHS + initial state
__global__ void nd_finalize_rhs_kernel(const double *part, int nb, SolveState *st, int remove_mean, int stage) {
    double a, b, c;
    reduce_partials3(part, nb, a, b, c);
    if (threadIdx.x == 0) {
        if (stage == 0) {
            st->mean = remove_mean ? b / c : 0.0;
            st->aux = b / c;
            st->fnorm = a;
        } else {
            st->fnorm = a;
            st->fnorm2 = 0.0;
            st->fsum = b;
            set_scale(st, a > 0.0 ? a : 1.0);
            st->best = INFINITY;
            st->iter = 0;
            st->done = 0;
            st->status = MX_OK;
        }
    }
}

// subtract the weighted mean, norms, and store 12 h^2 w f as double-float (mixed) or f (FP64)
__global__ void nd_rhs_final_kernel(NGeom g, double *__restrict__ f, const SolveState *st, float *__restrict__ fh,
                                    float *__restrict__ fl, double *part) {
    const double m = st->mean, h2 = g.h * g.h;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.M; q += (long long)gridDim.x * blockDim.x) {
        int a, b, c;
        node_of(g, q, a, b, c);
        const double v = f[q] - m;
        f[q] = v;
        if (fh) {
            const double sv = 12.0 * h2 * double(node_w(g, a, b, c)) * v;
            const float hi = __double2float_rn(sv);
            fh[q] = hi;
            fl[q] = __double2float_rn(sv - double(hi));
        }
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

// ---- multigrid kernels (T = float or double) -----------------------------------------

// coarse f = full-weighting restriction of the fine residual (node weights):
// f_C = (1/(8 w_C)) sum_n P(n, C) w_n r_n; coarse e = 0.  One coarse node column
// per thread, marched in z: the 3 x 3 fine neighbourhood of plane 2C + 1 is kept
// for the next coarse plane (where it is plane 2C' - 1); the in-plane positions
// and weights are computed once per column.  Every weight is a power of two, so
// each term is exact; they are summed in the order oz, oy, ox.
template <typename T>
__global__ void __launch_bounds__(256) nd_restrict_march_kernel(NLevel<T> F, NLevel<T> C, int zc) {
    pdl_trigger();
    pdl_wait();
    const NGeom &g = F.g, &gc = C.g;
    const int A = blockIdx.x * 32 + threadIdx.x, B = blockIdx.y * 8 + threadIdx.y;
    if (A >= gc.m[0] || B >= gc.m[1]) return;
    const int C0 = blockIdx.z * zc, C1 = min(C0 + zc, gc.m[2]);
    int fa[3], fb[3];
    float wx[3], wy[3];
    for (int o = 0; o < 3; o++) {
        fa[o] = node_wrap(g, 0, 2 * A + o - 1);
        fb[o] = node_wrap(g, 1, 2 * B + o - 1);
        wx[o] = (o != 1 ? 0.5f : 1.f) * ((fa[o] >= 0 && !g.per[0] && (fa[o] == 0 || fa[o] == g.m[0] - 1)) ? 0.5f : 1.f);
        wy[o] = (o != 1 ? 0.5f : 1.f) * ((fb[o] >= 0 && !g.per[1] && (fb[o] == 0 || fb[o] == g.m[1] - 1)) ? 0.5f : 1.f);
    }
    const float wxyC = ((!gc.per[0] && (A == 0 || A == gc.m[0] - 1)) ? 0.5f : 1.f) *
                       ((!gc.per[1] && (B == 0 || B == gc.m[1] - 1)) ? 0.5f : 1.f);
    T v[3][3][3];  // [oz][oy][ox]
    auto load = [&](int c, T p[3][3]) {
        const int cz = node_wrap(g, 2, c);
        for (int y = 0; y < 3; y++)
            for (int x = 0; x < 3; x++)
                p[y][x] = (cz >= 0 && fa[x] >= 0 && fb[y] >= 0) ? F.r[nidx(g, fa[x], fb[y], cz)] : T(0);
    };
    T n1[3][3], n2[3][3];  // the next coarse plane's fine planes, loaded a plane ahead
    load(2 * C0 - 1, v[0]);
    load(2 * C0, v[1]);
    load(2 * C0 + 1, v[2]);
    for (int Cz = C0; Cz < C1; Cz++) {
        if (Cz + 1 < C1) {
            load(2 * Cz + 2, n1);
            load(2 * Cz + 3, n2);
        }
        T acc = T(0);
        for (int oz = 0; oz < 3; oz++) {
            const int cz = node_wrap(g, 2, 2 * Cz + oz - 1);
            if (cz < 0) continue;
            const float wz = (oz != 1 ? 0.5f : 1.f) * ((!g.per[2] && (cz == 0 || cz == g.m[2] - 1)) ? 0.5f : 1.f);
            for (int oy = 0; oy < 3; oy++) {
                if (fb[oy] < 0) continue;
                for (int ox = 0; ox < 3; ox++) {
                    if (fa[ox] < 0) continue;
                    // the offset factors times the fine node's weight
                    acc += T(wx[ox] * wy[oy] * wz) * v[oz][oy][ox];
                }
            }
        }
        const long long Q = nidx(gc, A, B, Cz);
        const float wC = wxyC * ((!gc.per[2] && (Cz == 0 || Cz == gc.m[2] - 1)) ? 0.5f : 1.f);
        C.f[Q] = acc / (T(8) * T(wC));
        C.e[Q] = T(0);
        for (int y = 0; y < 3; y++)
            for (int x = 0; x < 3; x++) {
                v[0][y][x] = v[2][y][x];
                v[1][y][x] = n1[y][x];
                v[2][y][x] = n2[y][x];
            }
    }
}

// e_fine += trilinear interpolation of e_coarse (out non-null: out = e_fine +
// it), one fine node column per thread, marched in z: the in-plane parents and
// weights are computed once per column and the parents' values of a coarse
// plane are loaded once for the (up to three) fine planes that use them; the
// terms (every weight a power of two) are added coarse plane by plane, then
// along y, then x.
template <typename T>
__global__ void __launch_bounds__(256) nd_prolong_march_kernel(NLevel<T> C, NLevel<T> F, T *out, int zc) {
    pdl_trigger();
    pdl_wait();
    const NGeom &g = F.g, &gc = C.g;
    const int a = blockIdx.x * 32 + threadIdx.x, b = blockIdx.y * 8 + threadIdx.y;
    if (a >= g.m[0] || b >= g.m[1]) return;
    const int c0 = blockIdx.z * zc, c1 = min(c0 + zc, g.m[2]);
    int ia[2], ib[2], na, nb;
    T wa[2], wb[2];
    auto par = [&](int x, int d, int *ix, T *w, int &cnt) {
        if ((x & 1) == 0) {
            ix[0] = ix[1] = x / 2;
            w[0] = T(1);
            w[1] = T(0);
            cnt = 1;
        } else {
            ix[0] = (x - 1) / 2;
            ix[1] = (x + 1) / 2;
            if (gc.per[d] && ix[1] == gc.m[d]) ix[1] = 0;
            w[0] = w[1] = T(0.5);
            cnt = 2;
        }
    };
    par(a, 0, ia, wa, na);
    par(b, 1, ib, wb, nb);
    // the parents' values of coarse plane Cz: p[v][t]
    auto load = [&](int Cz, T p[2][2]) {
        for (int v = 0; v < 2; v++)
            for (int t = 0; t < 2; t++) p[v][t] = (v < nb && t < na) ? C.e[nidx(gc, ia[t], ib[v], Cz)] : T(0);
    };
    auto terms = [&](T &s, const T p[2][2], T wc) {
        for (int v = 0; v < nb; v++)
            for (int t = 0; t < na; t++) s += wa[t] * wb[v] * wc * p[v][t];
    };
    // fine planes in pairs (2C, 2C + 1): 2C takes coarse plane C, 2C + 1 the planes C
    // and C + 1 (wrapped); the next pair's fine values and coarse plane are loaded
    // before this pair's stores
    auto upper = [&](int c) {
        int Cu = (c + 1) / 2;
        if (gc.per[2] && Cu == gc.m[2]) Cu = 0;
        return Cu;
    };
    T lo[2][2], hi[2][2], nhi[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
    load(c0 / 2, lo);  // c0 is even
    T ne0 = F.e[nidx(g, a, b, c0)], ne1 = T(0);
    if (c0 + 1 < c1) {
        ne1 = F.e[nidx(g, a, b, c0 + 1)];
        load(upper(c0 + 1), nhi);
    }
    for (int c = c0; c < c1; c += 2) {
        const T e0 = ne0, e1 = ne1;
        for (int v = 0; v < 2; v++)
            for (int t = 0; t < 2; t++) hi[v][t] = nhi[v][t];
        if (c + 2 < c1) {
            ne0 = F.e[nidx(g, a, b, c + 2)];
            if (c + 3 < c1) {
                ne1 = F.e[nidx(g, a, b, c + 3)];
                load(upper(c + 3), nhi);
            }
        }
        const long long q = nidx(g, a, b, c);
        T s0 = T(0);
        terms(s0, lo, T(1));
        if (out) out[q] = e0 + s0;
        else F.e[q] = e0 + s0;
        if (c + 1 < c1) {
            const long long q1 = q + (long long)g.m[0] * g.m[1];
            T s1 = T(0);
            terms(s1, lo, T(0.5));
            terms(s1, hi, T(0.5));
            if (out) out[q1] = e1 + s1;
            else F.e[q1] = e1 + s1;
        }
        for (int v = 0; v < 2; v++)
            for (int t = 0; t < 2; t++) lo[v][t] = hi[v][t];
    }
}

static int nd_xfer_zc(const NGeom &g) {
    const long long bxy = (long long)((g.m[0] + 31) / 32) * ((g.m[1] + 7) / 8);
    int zc = 32;
    while (zc > 2 && bxy * ((g.m[2] + zc - 1) / zc) < 8 * 152) zc >>= 1;
    return zc;
}


// y = L x
template <typename T>
__device__ void nd_apply_one(const NLevel<T> &L, const T *x, T *y, long long q) {
    const NGeom &g = L.g;
    int a, b, c;
    node_of(g, q, a, b, c);
    T s[2][2][2];
    cell_ring(g, L.sigma, a, b, c, s);
    T num = T(0), den = T(0);
    for_couplings(g, a, b, c, s, [&](T coef, long long m) {
        if (m >= 0) num += coef * x[m];
        den += coef;
    });
    y[q] = (num - den * x[q]) / (T(12) * T(node_w(g, a, b, c)) * T(g.h * g.h));
}

template <typename T>
__global__ void nd_apply_kernel(NLevel<T> L, const T *x, T *y) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < L.g.M; q += (long long)gridDim.x * blockDim.x)
        nd_apply_one(L, x, y, q);
}

// BiCGStab on the coarsest nodal level (one CTA).  The nodal operator is
// symmetric in the w-weighted inner product; singular problems (no Dirichlet
// nodes) are projected onto weighted-mean-free vectors.
constexpr int NBT = 256;

template <typename T>
__device__ T nd_wdot(const NGeom &g, const T *a, const T *b, int weighted) {
    float acc = 0.f, m = 0.f, z = 0.f;
    for (int q = threadIdx.x; q < g.M; q += NBT) {
        int x, y, zz;
        node_of(g, q, x, y, zz);
        const float w = weighted ? node_w(g, x, y, zz) : 1.f;
        acc += w * float(a[q]) * float(b[q]);
    }
    block_red3f(m, acc, z);
    __shared__ float res;
    if (threadIdx.x == 0) res = acc;
    __syncthreads();
    const T out = T(res);
    __syncthreads();
    return out;
}

template <typename T>
__device__ void nd_wmean0(const NGeom &g, T *x) {
    float acc = 0.f, ws = 0.f, m = 0.f;
    for (int q = threadIdx.x; q < g.M; q += NBT) {
        int a, b, c;
        node_of(g, q, a, b, c);
        const float w = node_w(g, a, b, c);
        acc += w * float(x[q]);
        ws += w;
    }
    block_red3f(m, acc, ws);
    __shared__ float mean;
    if (threadIdx.x == 0) mean = acc / ws;
    __syncthreads();
    for (int q = threadIdx.x; q < g.M; q += NBT) x[q] -= T(mean);
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(NBT) nd_bottom_kernel(NLevel<T> L, T *scr, int iters) {
    pdl_trigger();
    pdl_wait();
    const NGeom &g = L.g;
    const int n = int(g.M);
    T *x = L.e, *r = scr, *r0 = scr + n, *p = scr + 2 * n, *v = scr + 3 * n, *sv = scr + 4 * n, *tv = scr + 5 * n;
    for (int q = threadIdx.x; q < n; q += NBT) r[q] = L.f[q];
    __syncthreads();
    nd_wmean0(g, r);  // compatibility (all nodal problems here are singular)
    for (int q = threadIdx.x; q < n; q += NBT) {
        x[q] = T(0);
        r0[q] = r[q];
        p[q] = T(0);
        v[q] = T(0);
    }
    __syncthreads();
    const T bnorm2 = nd_wdot(g, r, r, 1);
    if (!(bnorm2 > T(0))) return;
    const T tol2 = bnorm2 * T(1e-8);
    T rho = T(1), alpha = T(1), omega = T(1);
    for (int it = 0; it < iters; it++) {
        const T rho1 = nd_wdot(g, r0, r, 1);
        if (rho1 == T(0) || omega == T(0)) break;
        const T beta = (rho1 / rho) * (alpha / omega);
        for (int q = threadIdx.x; q < n; q += NBT) p[q] = r[q] + beta * (p[q] - omega * v[q]);
        __syncthreads();
        for (int q = threadIdx.x; q < n; q += NBT) nd_apply_one(L, p, v, q);
        __syncthreads();
        const T r0v = nd_wdot(g, r0, v, 1);
        if (r0v == T(0)) break;
        alpha = rho1 / r0v;
        for (int q = threadIdx.x; q < n; q += NBT) sv[q] = r[q] - alpha * v[q];
        __syncthreads();
        if (nd_wdot(g, sv, sv, 1) <= tol2) {
            for (int q = threadIdx.x; q < n; q += NBT) x[q] += alpha * p[q];
            __syncthreads();
            break;
        }
        for (int q = threadIdx.x; q < n; q += NBT) nd_apply_one(L, sv, tv, q);
        __syncthreads();
        const T tt = nd_wdot(g, tv, tv, 1), ts = nd_wdot(g, tv, sv, 1);
        omega = tt > T(0) ? ts / tt : T(0);
        for (int q = threadIdx.x; q < n; q += NBT) {
            x[q] += alpha * p[q] + omega * sv[q];
            r[q] = sv[q] - omega * tv[q];
        }
        __syncthreads();
        rho = rho1;
        if (nd_wdot(g, r, r, 1) <= tol2) break;
    }
    nd_wmean0(g, x);
}

// ---- column-marching kernels ------------------------------------------------------------
// A thread owns one (a, b) node column and walks up a z-chunk, keeping the
// 3x3 neighbourhood of nodes of planes c-1, c, c+1 and the 2x2 cells below and
// above plane c in registers, so each node costs 9 node and 4 cell loads.
// One colour (a mod 2, b mod 2) is a set of whole columns, and nodes of one
// column are never coupled (edge neighbours), so a column can be updated in
// place while it is walked.

// In-plane offsets of a node column's 3 x 3 node neighbourhood and 2 x 2 cell
// neighbourhood (-1: beyond a wall), computed once per column so each plane of
// the march costs one plane base plus the loads.
struct ColMap {
    int no[3][3];  // node (a-1+x, b-1+y): offset within a node plane
    int co[2][2];  // cell (a-1+x, b-1+y): offset within a cell plane
};

__device__ __forceinline__ ColMap col_map(const NGeom &g, int a, int b) {
    ColMap m;
    for (int y = 0; y < 3; y++) {
        const int nb = node_wrap(g, 1, b - 1 + y);
        for (int x = 0; x < 3; x++) {
            const int na = node_wrap(g, 0, a - 1 + x);
            m.no[y][x] = (na >= 0 && nb >= 0) ? na + g.m[0] * nb : -1;
        }
    }
    for (int y = 0; y < 2; y++) {
        const int cb = cell_wrap(g, 1, b - 1 + y);
        for (int x = 0; x < 2; x++) {
            const int ca = cell_wrap(g, 0, a - 1 + x);
            m.co[y][x] = (ca >= 0 && cb >= 0) ? ca + g.n[0] * cb : -1;
        }
    }
    return m;
}

template <typename T>
__device__ __forceinline__ void load_node_plane(const NGeom &g, const ColMap &m, const T *e, int c, T p[3][3]) {
    const int cz = node_wrap(g, 2, c);
    const T *pl = e + (cz >= 0 ? cz : 0) * (g.m[0] * g.m[1]);
    for (int y = 0; y < 3; y++)
        for (int x = 0; x < 3; x++) p[y][x] = (cz >= 0 && m.no[y][x] >= 0) ? pl[m.no[y][x]] : T(0);
}

template <typename T>
__device__ __forceinline__ void load_cell_plane(const NGeom &g, const ColMap &m, const T *sig, int k, T s[2][2]) {
    const int kz = cell_wrap(g, 2, k);
    const T *pl = sig + (kz >= 0 ? kz : 0) * (g.n[0] * g.n[1]);
    for (int y = 0; y < 2; y++)
        for (int x = 0; x < 2; x++) s[y][x] = (kz >= 0 && m.co[y][x] >= 0) ? pl[m.co[y][x]] : T(0);
}

// sum_m c_m e_m and sum_m c_m for node (.., .., c) from the planes below (pm),
// at (p0) and above (pp) and the cells below (sl) and above (sh) the node
template <typename T>
__device__ __forceinline__ void couplings(const T pm[3][3], const T p0[3][3], const T pp[3][3], const T sl[2][2],
                                          const T sh[2][2], T &num, T &den) {
    num = T(0);
    // face diagonals in the xy plane: both z cells
    for (int y = 0; y < 2; y++)
        for (int x = 0; x < 2; x++) num += (sl[y][x] + sh[y][x]) * p0[2 * y][2 * x];
    // face diagonals in xz (oy = 0): both y cells; in yz (ox = 0): both x cells
    for (int x = 0; x < 2; x++) {
        num += (sl[0][x] + sl[1][x]) * pm[1][2 * x];
        num += (sh[0][x] + sh[1][x]) * pp[1][2 * x];
    }
    for (int y = 0; y < 2; y++) {
        num += (sl[y][0] + sl[y][1]) * pm[2 * y][1];
        num += (sh[y][0] + sh[y][1]) * pp[2 * y][1];
    }
    // body diagonals: one cell each
    for (int y = 0; y < 2; y++)
        for (int x = 0; x < 2; x++) {
            num += sl[y][x] * pm[2 * y][2 * x];
            num += sh[y][x] * pp[2 * y][2 * x];
        }
    den = T(4) * (((sl[0][0] + sl[0][1]) + (sl[1][0] + sl[1][1])) + ((sh[0][0] + sh[0][1]) + (sh[1][0] + sh[1][1])));
}

constexpr int NCZ = 16;  // z-chunk of the column kernels

template <typename T, int MODE>  // MODE 0: Gauss-Seidel on one colour, 1: residual r = f - L e
__global__ void nd_col_kernel(NLevel<T> L, int colour, int ncol_x, int ncol_y, int nzc) {
    pdl_trigger();
    pdl_wait();
    const NGeom &g = L.g;
    const int cx = colour & 1, cy = colour >> 1;
    const int tx = blockIdx.x * blockDim.x + threadIdx.x;
    const int ty = blockIdx.y;
    if (tx >= ncol_x || ty >= ncol_y) return;
    const int a = MODE == 0 ? 2 * tx + cx : tx, b = MODE == 0 ? 2 * ty + cy : ty;
    if (a >= g.m[0] || b >= g.m[1]) return;
    const int c0 = blockIdx.z * nzc, c1 = min(c0 + nzc, g.m[2]);
    const ColMap m = col_map(g, a, b);
    const T h2 = T(g.h * g.h);
    const float wxy = ((!g.per[0] && (a == 0 || a == g.m[0] - 1)) ? 0.5f : 1.f) *
                      ((!g.per[1] && (b == 0 || b == g.m[1] - 1)) ? 0.5f : 1.f);
    T pm[3][3], p0[3][3], pp[3][3], sl[2][2], sh[2][2];
    load_node_plane(g, m, L.e, c0 - 1, pm);
    load_node_plane(g, m, L.e, c0, p0);
    load_cell_plane(g, m, L.sigma, c0 - 1, sl);
    for (int c = c0; c < c1; c++) {
        load_node_plane(g, m, L.e, c + 1, pp);
        load_cell_plane(g, m, L.sigma, c, sh);
        T num, den;
        couplings(pm, p0, pp, sl, sh, num, den);
        const float w = wxy * ((!g.per[2] && (c == 0 || c == g.m[2] - 1)) ? 0.5f : 1.f);
        const long long q = nidx(g, a, b, c);
        if (MODE == 0) {
            if (den > T(0)) L.e[q] = (num - T(12) * T(w) * h2 * L.f[q]) / den;
        } else {
            L.r[q] = L.f[q] - (num - den * p0[1][1]) / (T(12) * T(w) * h2);
        }
        for (int y = 0; y < 3; y++)
            for (int x = 0; x < 3; x++) {
                pm[y][x] = p0[y][x];
                p0[y][x] = pp[y][x];
            }
        for (int y = 0; y < 2; y++)
            for (int x = 0; x < 2; x++) sl[y][x] = sh[y][x];
    }
}

// z-chunk of a column launch with bxy blocks per chunk: NCZ nodes per thread
// on large levels, fewer (down to 1) until there are >= 8 blocks per SM, so
// small levels are not latency-bound on a few long columns.
static int nd_zchunk(long long bxy, int m2, int cap) {
    int zc = cap;
    while (zc > 1 && bxy * ((m2 + zc - 1) / zc) < 8 * 152) zc >>= 1;
    return zc;
}

template <typename T>
static void k_nd_gs(cudaStream_t s, const NLevel<T> &L, int colour, int zcap) {
    const int cx = colour & 1, cy = colour >> 1;
    const int ncx = (L.g.m[0] - cx + 1) / 2, ncy = (L.g.m[1] - cy + 1) / 2;
    const int zc = nd_zchunk((long long)((ncx + 63) / 64) * ncy, L.g.m[2], zcap);
    dim3 grid((ncx + 63) / 64, ncy, (L.g.m[2] + zc - 1) / zc);
    launch_pdl(nd_col_kernel<T, 0>, grid, dim3(64), 0, s, L, colour, ncx, ncy, zc);
}

template <typename T, int MODE>
static void k_nd_tile(cudaStream_t s, const NLevel<T> &L, const T *ein, T *eout, T omega, int zcap);
// levels at least this many nodes wide take the tiled kernels (x is covered by
// one tile width per block; narrower levels keep the column kernels)
constexpr int ND_TILE_MIN = 32;
static bool nd_tiled(const NGeom &g);

template <typename T>
static void k_nd_residual(cudaStream_t s, const NLevel<T> &L, int zcap) {
    if (nd_tiled(L.g)) {
        k_nd_tile<T, 1>(s, L, L.e, (T *)nullptr, T(0), zcap);
        return;
    }
    const int zc = nd_zchunk((long long)((L.g.m[0] + 63) / 64) * L.g.m[1], L.g.m[2], zcap);
    dim3 grid((L.g.m[0] + 63) / 64, L.g.m[1], (L.g.m[2] + zc - 1) / zc);
    launch_pdl(nd_col_kernel<T, 1>, grid, dim3(64), 0, s, L, 0, L.g.m[0], L.g.m[1], zc);
}

// One Chebyshev smoothing step e_out = e_in + w D^-1 (f - L e_in), D the diagonal of
// L (its coefficient sum: 12 w h^2 (L e)_n = sum_m c_m (e_m - e_n)), node columns
// marched in z like the colour kernel; zero = 1: e_in is identically 0 (not read).
// The updated nodes go to a second buffer (the stencil reads old neighbours).
template <typename T>
__global__ void nd_cheb_kernel(NLevel<T> L, const T *__restrict__ ein, T *__restrict__ eout, T omega, int zero,
                               int nzc) {
    pdl_trigger();
    pdl_wait();
    const NGeom &g = L.g;
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a >= g.m[0] || b >= g.m[1]) return;
    const int c0 = blockIdx.z * nzc, c1 = min(c0 + nzc, g.m[2]);
    const ColMap m = col_map(g, a, b);
    const T h2 = T(g.h * g.h);
    const float wxy = ((!g.per[0] && (a == 0 || a == g.m[0] - 1)) ? 0.5f : 1.f) *
                      ((!g.per[1] && (b == 0 || b == g.m[1] - 1)) ? 0.5f : 1.f);
    T pm[3][3], p0[3][3], pp[3][3], sl[2][2], sh[2][2];
    for (int y = 0; y < 3; y++)
        for (int x = 0; x < 3; x++) pm[y][x] = p0[y][x] = pp[y][x] = T(0);
    if (!zero) {
        load_node_plane(g, m, ein, c0 - 1, pm);
        load_node_plane(g, m, ein, c0, p0);
    }
    load_cell_plane(g, m, L.sigma, c0 - 1, sl);
    for (int c = c0; c < c1; c++) {
        if (!zero) load_node_plane(g, m, ein, c + 1, pp);
        load_cell_plane(g, m, L.sigma, c, sh);
        T num, den;
        couplings(pm, p0, pp, sl, sh, num, den);
        const float w = wxy * ((!g.per[2] && (c == 0 || c == g.m[2] - 1)) ? 0.5f : 1.f);
        const long long q = nidx(g, a, b, c);
        const T e0 = p0[1][1];
        eout[q] = den > T(0) ? e0 + omega * ((num - den * e0) - T(12) * T(w) * h2 * L.f[q]) / den : e0;
        for (int y = 0; y < 3; y++)
            for (int x = 0; x < 3; x++) {
                pm[y][x] = p0[y][x];
                p0[y][x] = pp[y][x];
            }
        for (int y = 0; y < 2; y++)
            for (int x = 0; x < 2; x++) sl[y][x] = sh[y][x];
    }
}

// ---- out-of-place stencil passes, tiled in x-y and marched in z ----------------------
// A block of TBX x TTY threads owns a TBX x TNY tile of node columns (each
// thread two y-adjacent columns, sharing their neighbourhood loads) over nzc
// planes.  Step k of the march (node plane c0 + k) needs node plane c0 + k + 1
// (with its one-node halo: periodic images, zeros beyond a wall), cell layer
// c0 + k of sigma (with its halo) and f at plane c0 + k: one "stage", copied
// global -> shared by cp.async (element copies, zero-filled where there is no
// node or cell) into a ring of ND_NS slots, ND_NS - 1 stages ahead of the step
// that reads it, so the DRAM latency hides behind three planes of arithmetic;
// one barrier per plane.  Each thread keeps its 4 x 3 x 3 node and 3 x 2 x 2
// cell neighbourhood in registers, rotated by unrolling the march six planes
// deep.
// MODE 0: Chebyshev step eout = e + omega D^-1 (f - L e) (e = ein); MODE 2: the
// same from e = 0 (no node is read); MODE 1: residual L.r = L.f - L e (ein =
// L.e).  The couplings are the column
// kernels' (same terms, same order); the step divides with the fast FP32
// division and the residual multiplies by 1 / (12 w h^2).
constexpr int TBX = 32, TTY = 8, TNT = TBX * TTY, TNY = 2 * TTY;
constexpr int THX = TBX + 2, THN = THX * (TNY + 2);  // node plane with halo
constexpr int TCX = TBX + 1, TCN = TCX * (TNY + 1);  // cell layer with halo
constexpr int ND_NS = 4;                             // ring slots
constexpr int ND_HS = 3;                             // halo slots of each kind per thread
static_assert(THN <= ND_HS * TNT && TCN <= ND_HS * TNT, "halo slots per thread");

__device__ __forceinline__ float nd_fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double nd_fdiv(double a, double b) { return a / b; }


template <typename T>
struct NdStage {
    T p[THN];  // node plane
    T s[TCN];  // cell layer
    T f[TNY * TBX];  // f of the tile's nodes
};

// couplings() of the node in rows R..R+2 of a 4-row neighbourhood (same terms,
// same order)
template <int R, typename T>
__device__ __forceinline__ void couplings_r(const T pm[4][3], const T p0[4][3], const T pp[4][3], const T sl[3][2],
                                            const T sh[3][2], T &num, T &den) {
    num = T(0);
    for (int y = 0; y < 2; y++)
        for (int x = 0; x < 2; x++) num += (sl[R + y][x] + sh[R + y][x]) * p0[R + 2 * y][2 * x];
    for (int x = 0; x < 2; x++) {
        num += (sl[R][x] + sl[R + 1][x]) * pm[R + 1][2 * x];
        num += (sh[R][x] + sh[R + 1][x]) * pp[R + 1][2 * x];
    }
    for (int y = 0; y < 2; y++) {
        num += (sl[R + y][0] + sl[R + y][1]) * pm[R + 2 * y][1];
        num += (sh[R + y][0] + sh[R + y][1]) * pp[R + 2 * y][1];
    }
    for (int y = 0; y < 2; y++)
        for (int x = 0; x < 2; x++) {
            num += sl[R + y][x] * pm[R + 2 * y][2 * x];
            num += sh[R + y][x] * pp[R + 2 * y][2 * x];
        }
    den = T(4) * (((sl[R][0] + sl[R][1]) + (sl[R + 1][0] + sl[R + 1][1])) +
                  ((sh[R][0] + sh[R][1]) + (sh[R + 1][0] + sh[R + 1][1])));
}

template <typename T, int MODE>
__global__ void __launch_bounds__(TNT, sizeof(T) == 4 ? 3 : 1)
    nd_tile_kernel(NLevel<T> L, const T *__restrict__ ein, T *__restrict__ eout, T omega, int nzc) {
    pdl_trigger();
    pdl_wait();
    extern __shared__ __align__(16) unsigned char nd_smem[];
    NdStage<T> *st = reinterpret_cast<NdStage<T> *>(nd_smem);
    const NGeom &g = L.g;
    const int tid = threadIdx.x, tx = tid % TBX, ty = tid / TBX;
    const int a0 = blockIdx.x * TBX, b0 = blockIdx.y * TNY;
    const int a = a0 + tx, b = b0 + 2 * ty;  // this thread's nodes: (a, b) and (a, b + 1)
    const bool own0 = a < g.m[0] && b < g.m[1], own1 = a < g.m[0] && b + 1 < g.m[1];
    const int c0 = blockIdx.z * nzc, c1 = min(c0 + nzc, g.m[2]);
    const int np = g.m[0] * g.m[1], ncp = g.n[0] * g.n[1];  // 32-bit indices: M, N < 2^31 (host check)
    // the tile's halo slots reach at most one node or cell past either end of
    // the nodes the tile owns, which one periodic wrap maps into the box;
    // beyond a wall or past that reach nw / cw give -1
    auto nw = [&](int d, int x) { return x > g.m[d] ? -1 : node_wrap(g, d, x); };
    auto cw = [&](int d, int x) { return x > g.m[d] - 1 ? -1 : cell_wrap(g, d, x); };
    // per slot: the in-plane offset; slots 0 and 1 exist for every thread.
    // A node beyond a wall couples only through cells beyond that wall, whose
    // sigma is zero-filled (cmask bit clear: a 0-byte copy), so its slot may
    // hold any finite node: it copies node 0 of the plane (the products are +-0
    // either way, and adding a zero leaves the sum's bits unchanged).
    static_assert(THN >= 2 * TNT && TCN >= 2 * TNT, "two full slot rows");
    int no[ND_HS], co[ND_HS], cmask = 0;
    for (int k = 0; k < ND_HS; k++) {
        const int sl = tid + k * TNT;
        no[k] = co[k] = 0;
        if (sl < THN) {
            const int na = nw(0, a0 - 1 + sl % THX), nb = nw(1, b0 - 1 + sl / THX);
            if (na >= 0 && nb >= 0) no[k] = na + g.m[0] * nb;
        }
        if (sl < TCN) {
            const int ca = cw(0, a0 - 1 + sl % TCX), cb = cw(1, b0 - 1 + sl / TCX);
            if (ca >= 0 && cb >= 0) {
                co[k] = ca + g.n[0] * cb;
                cmask |= 1 << k;
            }
        }
    }
    const bool slot2n = tid + 2 * TNT < THN, slot2c = tid + 2 * TNT < TCN;
    const int qa = own0 ? a + g.m[0] * b : 0;  // this thread's first node at plane 0
    // stage k: node plane c0 + 1 + k, cell layer c0 + k, f at plane c0 + k; any
    // part outside [c0 - 1, c1] (planes), [c0 - 1, c1 - 1] (layers) or
    // [c0, c1 - 1] (f) is not copied (nothing reads it)
    auto issue = [&](int k) {
        NdStage<T> &S = st[(k + 2) % ND_NS];
        const int c = c0 + 1 + k, kl = c0 + k;
        if (MODE != 2 && c <= c1) {
            const int cz = node_wrap(g, 2, c);  // beyond a z wall: any plane (see above)
            const T *base = ein + (cz >= 0 ? cz * np : 0);
            cp_async_el(&S.p[tid], base + no[0], (int)sizeof(T));
            cp_async_el(&S.p[tid + TNT], base + no[1], (int)sizeof(T));
            if (slot2n) cp_async_el(&S.p[tid + 2 * TNT], base + no[2], (int)sizeof(T));
        }
        if (kl >= c0 - 1 && kl <= c1 - 1) {
            const int kz = cell_wrap(g, 2, kl);
            const T *base = L.sigma + (kz >= 0 ? kz * ncp : 0);
            const int m = kz >= 0 ? cmask : 0;
            cp_async_el(&S.s[tid], base + co[0], (m & 1) ? (int)sizeof(T) : 0);
            cp_async_el(&S.s[tid + TNT], base + co[1], (m & 2) ? (int)sizeof(T) : 0);
            if (slot2c) cp_async_el(&S.s[tid + 2 * TNT], base + co[2], (m & 4) ? (int)sizeof(T) : 0);
        }
        if (kl >= c0 && kl < c1) {
            if (own0) cp_async_el(&S.f[2 * ty * TBX + tx], L.f + (qa + kl * np), (int)sizeof(T));
            if (own1) cp_async_el(&S.f[(2 * ty + 1) * TBX + tx], L.f + (qa + g.m[0] + kl * np), (int)sizeof(T));
        }
        cp_async_commit();
    };
    auto get_nodes = [&](int k, T p[4][3]) {
        const T *sp = st[(k + 2) % ND_NS].p + 2 * ty * THX + tx;
        for (int y = 0; y < 4; y++)
            for (int x = 0; x < 3; x++) p[y][x] = MODE == 2 ? T(0) : sp[y * THX + x];
    };
    auto get_cells = [&](int k, T s[3][2]) {
        const T *sc = st[(k + 2) % ND_NS].s + 2 * ty * TCX + tx;
        for (int y = 0; y < 3; y++)
            for (int x = 0; x < 2; x++) s[y][x] = sc[y * TCX + x];
    };
    const T h2 = T(g.h * g.h);
    const float wx = (!g.per[0] && (a == 0 || a == g.m[0] - 1)) ? 0.5f : 1.f;
    const float wy0 = (!g.per[1] && (b == 0 || b == g.m[1] - 1)) ? 0.5f : 1.f;
    const float wy1 = (!g.per[1] && (b + 1 == 0 || b + 1 == g.m[1] - 1)) ? 0.5f : 1.f;
    const T f12a = T(12) * T(wx * wy0) * h2, f12b = T(12) * T(wx * wy1) * h2;  // 12 w h^2 off the z walls
    const T inva = T(1) / f12a, invb = T(1) / f12b;
    T P0[4][3], P1[4][3], P2[4][3], S0[3][2], S1[3][2];
    // prologue: stages -2 (plane c0 - 1) and -1 (plane c0, layer c0 - 1) into
    // registers; then stages 0, 1, 2 in flight
    issue(-2);
    issue(-1);
    cp_async_wait<0>();
    __syncthreads();
    get_nodes(-2, P0);
    get_nodes(-1, P1);
    get_cells(-1, S0);
    __syncthreads();
    issue(0);
    issue(1);
    issue(2);
    auto one = [&](int R, const T num, const T den, const T e0, const T f, const T f12, const T inv, bool wall,
                   int q) {
        if (MODE != 1) {
            const T t = (num - den * e0) - (wall ? T(0.5) * f12 : f12) * f;
            eout[q] = den > T(0) ? e0 + nd_fdiv(omega * t, den) : e0;
        } else {
            L.r[q] = f - (num - den * e0) * (wall ? T(2) * inv : inv);
        }
    };
    auto step = [&](int k, T pm[4][3], T p0[4][3], T pp[4][3], T sl[3][2], T sh[3][2]) {
        cp_async_wait<2>();  // this thread's copies of stage k
        __syncthreads();     // everyone's; and stage k - 1 is free for stage k + 3
        get_nodes(k, pp);
        get_cells(k, sh);
        const int c = c0 + k;
        const bool wall = !g.per[2] && (c == 0 || c == g.m[2] - 1);
        const T *fs = st[(k + 2) % ND_NS].f + 2 * ty * TBX + tx;
        const int q = qa + c * np;
        if (own0) {
            T num, den;
            couplings_r<0>(pm, p0, pp, sl, sh, num, den);
            one(0, num, den, p0[1][1], fs[0], f12a, inva, wall, q);
        }
        if (own1) {
            T num, den;
            couplings_r<1>(pm, p0, pp, sl, sh, num, den);
            one(1, num, den, p0[2][1], fs[TBX], f12b, invb, wall, q + g.m[0]);
        }
        issue(k + 3);
    };
    const int nk = c1 - c0;
    for (int k = 0; k < nk; k += 6) {
        step(k, P0, P1, P2, S0, S1);
        if (k + 1 >= nk) break;
        step(k + 1, P1, P2, P0, S1, S0);
        if (k + 2 >= nk) break;
        step(k + 2, P2, P0, P1, S0, S1);
        if (k + 3 >= nk) break;
        step(k + 3, P0, P1, P2, S1, S0);
        if (k + 4 >= nk) break;
        step(k + 4, P1, P2, P0, S0, S1);
        if (k + 5 >= nk) break;
        step(k + 5, P2, P0, P1, S1, S0);
    }
    cp_async_wait<0>();  // no copy outlives the block
}

template <typename T, int MODE>
static void k_nd_tile(cudaStream_t s, const NLevel<T> &L, const T *ein, T *eout, T omega, int zcap) {
    const long long bxy = (long long)((L.g.m[0] + TBX - 1) / TBX) * ((L.g.m[1] + TNY - 1) / TNY);
    // deep chunks (the halo planes are re-read once per chunk), halved until the
    // grid fills every SM a few times over
    int zc = 4 * (zcap > 0 ? zcap : NCZ);
    while (zc > 4 && bxy * ((L.g.m[2] + zc - 1) / zc) < 4 * 3 * 152) zc >>= 1;
    dim3 grid((L.g.m[0] + TBX - 1) / TBX, (L.g.m[1] + TNY - 1) / TNY, (L.g.m[2] + zc - 1) / zc);
    const size_t smem = sizeof(NdStage<T>) * ND_NS;  // FP64: above the 48 KB default, opted in
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(nd_tile_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_pdl(nd_tile_kernel<T, MODE>, grid, dim3(TNT), smem, s, L, ein, eout, omega, zc);
}

// the tiled kernels index with 32-bit integers
static bool nd_tiled(const NGeom &g) { return g.m[0] >= ND_TILE_MIN && g.M < (1LL << 31) && g.N < (1LL << 31); }

template <typename T>
static void k_nd_cheb(cudaStream_t s, const NLevel<T> &L, const T *ein, T *eout, T omega, int zcap) {
    if (nd_tiled(L.g)) {
        if (ein) k_nd_tile<T, 0>(s, L, ein, eout, omega, zcap);
        else k_nd_tile<T, 2>(s, L, ein, eout, omega, zcap);
        return;
    }
    const int zc = nd_zchunk((long long)((L.g.m[0] + 63) / 64) * L.g.m[1], L.g.m[2], zcap);
    dim3 grid((L.g.m[0] + 63) / 64, L.g.m[1], (L.g.m[2] + zc - 1) / zc);
    launch_pdl(nd_cheb_kernel<T>, grid, dim3(64), 0, s, L, ein, eout, omega, ein ? 0 : 1, zc);
}

// weights of a degree-m Chebyshev smoother: the inverses of the roots of the
// degree-m Chebyshev polynomial mapped onto [lo, hi] of the spectrum of D^-1 L,
// largest root first.  The error factor prod_k (1 - lambda / root_k) is at most
// 1 / T_m((hi + lo) / (hi - lo)) on [lo, hi] and at most 1 on [0, lo].
static void cheb_weights(int m, double lo, double hi, double *w) {
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < m; k++) {
        const double lam = 0.5 * (hi + lo) + 0.5 * (hi - lo) * std::cos(pi * (2 * k + 1) / (2.0 * m));
        w[k] = 1.0 / lam;
    }
}
// The interval.  hi: the operator is the trilinear finite-element Laplacian
// sum_cells sigma_c K_c, and each cell matrix K_c (8 x 8) has eigenvalues
// {0, h/2, h/3, h/6} (tensor products of the 1-D stiffness and mass matrices)
// and diagonal h/3, so v'K_c v <= 1.5 v'diag(K_c) v; summing over cells with
// sigma_c > 0 gives lambda_max(D^-1 L) <= 1.5 for any coefficient field (on the
// coarser levels too, which are rediscretised).  lo: the smoother's share of the
// spectrum; the modes below it are left to the coarse grid (0.4 converged in
// the fewest V-cycles on the stratified workloads at 192^3..512^3).
constexpr double CHEB_LO = 0.4, CHEB_HI = 1.5;

// ---- double-float residual of the refinement loop ------------------------------------
__device__ __forceinline__ void ts2(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// phi + scale e in double-float: the update of the refinement loop
__device__ __forceinline__ void nd_df_axpy(float ph, float pl, float ev, float sh, float sl, float &oh, float &ol) {
    const float t = sh * ev;
    const float te = fmaf(sh, ev, -t) + sl * ev;
    float h, e1;
    ts2(ph, t, h, e1);
    const float l = pl + (te + e1);
    ts2(h, l, oh, ol);
}

// phi (buffer it & 1) = phi (buffer (it - 1) & 1) + scale e, it = the update count
// (the column residual's geometries; the tiled residual applies the update itself)
__global__ void nd_df_update_kernel(NDF D, long long M, const float *__restrict__ e, const SolveState *st) {
    pdl_trigger();
    pdl_wait();
    const float sh = st->scale_h, sl = st->scale_l;
    const int it = st->iter;
    const float *__restrict__ xh = nd_phi_h(D, it - 1), *__restrict__ xl = nd_phi_l(D, it - 1);
    float *__restrict__ yh = (it & 1) ? D.ph2 : D.ph, *__restrict__ yl = (it & 1) ? D.pl2 : D.pl;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < M; q += (long long)gridDim.x * blockDim.x)
        nd_df_axpy(xh[q], xl[q], e[q], sh, sl, yh[q], yl[q]);
}

// The first residual of a mixed solve from phi = 0: every coupling term of
// the residual kernels is exactly +0 there, so the residual is f.  It is formed
// node by node with their final expression and node weights (bit for bit
// their rhat; the norms differ only in the grouping of the sums, and the
// convergence decision reads the max), and phi's double-float buffer is
// zeroed in the same pass.
__global__ void nd_df_resid_zero_kernel(NLevel<float> L0, NDF D, const SolveState *st, double *part) {
    const NGeom &g = L0.g;
    const float inv = st->inv_scale_f;
    const float ih2 = float(1.0 / (g.h * g.h));
    const long long mxy = (long long)g.m[0] * g.m[1];
    float mx = 0.f, s2 = 0.f, s1 = 0.f;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.M; q += (long long)gridDim.x * blockDim.x) {
        const int c = int(q / mxy), r = int(q - c * mxy);
        const int b = r / g.m[0], a = r - b * g.m[0];
        const float wxy = ((!g.per[0] && (a == 0 || a == g.m[0] - 1)) ? 0.5f : 1.f) *
                          ((!g.per[1] && (b == 0 || b == g.m[1] - 1)) ? 0.5f : 1.f);
        const bool wall = !g.per[2] && (c == 0 || c == g.m[2] - 1);
        const float sc = wall ? ih2 / (12.f * (wxy * 0.5f)) : ih2 / (12.f * wxy);
        float Rh, Re;
        ts2(D.fh[q], -0.f, Rh, Re);
        Re += D.fl[q] - 0.f;
        const float R = Rh + Re;  // 12 w h^2 r
        const float rh = R * sc * inv;
        L0.f[q] = rh;
        D.ph[q] = 0.f;
        D.pl[q] = 0.f;
        mx = nmaxf(mx, fabsf(rh));
        s2 = fmaf(rh, rh, s2);
        s1 += rh;
    }
    block_red3f(mx, s2, s1);
    if (threadIdx.x == 0) {
        double *p = part + 3 * blockIdx.x;
        p[0] = double(mx);
        p[1] = double(s2);
        p[2] = double(s1);
    }
}

// ---- column-marching residuals of the refinement loop -------------------------------

// acc += coef * (q - p) in double-float, coef = (kh, kl), q = (qh, ql), p = (ch, cl)
__device__ __forceinline__ void df_acc(float kh, float kl, float qh, float ql, float ch, float cl, float &Sh,
                                       float &Se) {
    float dh, de;
    ts2(qh, -ch, dh, de);
    de += ql - cl;
    const float th = kh * dh;
    float te = fmaf(kh, dh, -th);
    te = fmaf(kh, de, te);
    te = fmaf(kl, dh, te);
    float s, e1;
    ts2(Sh, th, s, e1);
    Sh = s;
    Se += e1 + te;
}
// (a + b) in double-float from two double-float values
__device__ __forceinline__ void df_add2(float ah, float al, float bh, float bl, float &sh, float &sl) {
    float e;
    ts2(ah, bh, sh, e);
    sl = e + (al + bl);
}

__device__ __forceinline__ void load_df_plane(const NGeom &g, const ColMap &m, const float *hi, const float *lo, int c,
                                              float ph[3][3], float pl[3][3]) {
    const int cz = node_wrap(g, 2, c);
    const int base = (cz >= 0 ? cz : 0) * (g.m[0] * g.m[1]);
    for (int y = 0; y < 3; y++)
        for (int x = 0; x < 3; x++) {
            const bool ok = cz >= 0 && m.no[y][x] >= 0;
            const int q = base + (ok ? m.no[y][x] : 0);
            ph[y][x] = ok ? hi[q] : 0.f;
            pl[y][x] = ok ? lo[q] : 0.f;
        }
}
__device__ __forceinline__ void load_df_cells(const NGeom &g, const ColMap &m, const float *hi, const float *lo, int k,
                                              float sh[2][2], float sl[2][2]) {
    const int kz = cell_wrap(g, 2, k);
    const int base = (kz >= 0 ? kz : 0) * (g.n[0] * g.n[1]);
    for (int y = 0; y < 2; y++)
        for (int x = 0; x < 2; x++) {
            const bool ok = kz >= 0 && m.co[y][x] >= 0;
            const int q = base + (ok ? m.co[y][x] : 0);
            sh[y][x] = ok ? hi[q] : 0.f;
            sl[y][x] = ok ? lo[q] : 0.f;
        }
}

// 12 w h^2 r = 12 w h^2 f - sum_m c_m (phi_m - phi_n) in double-float, node
// columns marched in z; rhat = r / scale in FP32 with norm partials per block
__global__ void nd_df_col_resid_kernel(NLevel<float> L0, NDF D, const SolveState *st, double *part) {
    pdl_trigger();
    pdl_wait();
    const NGeom &g = L0.g;
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    const int c0 = blockIdx.z * NCZ, c1 = min(c0 + NCZ, g.m[2]);
    const float inv = st->inv_scale_f;
    const float ih2 = float(1.0 / (g.h * g.h));
    float mx = 0.f, s2 = 0.f, s1 = 0.f;
    const float *__restrict__ xh = nd_phi_h(D, st->iter), *__restrict__ xl = nd_phi_l(D, st->iter);
    if (a < g.m[0]) {
        const ColMap m = col_map(g, a, b);
        const float wxy = ((!g.per[0] && (a == 0 || a == g.m[0] - 1)) ? 0.5f : 1.f) *
                          ((!g.per[1] && (b == 0 || b == g.m[1] - 1)) ? 0.5f : 1.f);
        float pmh[3][3], pml[3][3], p0h[3][3], p0l[3][3], pph[3][3], ppl[3][3];
        float slh[2][2], sll[2][2], shh[2][2], shl[2][2];
        load_df_plane(g, m, xh, xl, c0 - 1, pmh, pml);
        load_df_plane(g, m, xh, xl, c0, p0h, p0l);
        load_df_cells(g, m, D.sh, D.sl, c0 - 1, slh, sll);
        for (int c = c0; c < c1; c++) {
            load_df_plane(g, m, xh, xl, c + 1, pph, ppl);
            load_df_cells(g, m, D.sh, D.sl, c, shh, shl);
            const float ch = p0h[1][1], cl = p0l[1][1];
            float Sh = 0.f, Se = 0.f, kh, kl;
            for (int y = 0; y < 2; y++)
                for (int x = 0; x < 2; x++) {
                    df_add2(slh[y][x], sll[y][x], shh[y][x], shl[y][x], kh, kl);
                    df_acc(kh, kl, p0h[2 * y][2 * x], p0l[2 * y][2 * x], ch, cl, Sh, Se);
                    df_acc(slh[y][x], sll[y][x], pmh[2 * y][2 * x], pml[2 * y][2 * x], ch, cl, Sh, Se);
                    df_acc(shh[y][x], shl[y][x], pph[2 * y][2 * x], ppl[2 * y][2 * x], ch, cl, Sh, Se);
                }
            for (int x = 0; x < 2; x++) {
                df_add2(slh[0][x], sll[0][x], slh[1][x], sll[1][x], kh, kl);
                df_acc(kh, kl, pmh[1][2 * x], pml[1][2 * x], ch, cl, Sh, Se);
                df_add2(shh[0][x], shl[0][x], shh[1][x], shl[1][x], kh, kl);
                df_acc(kh, kl, pph[1][2 * x], ppl[1][2 * x], ch, cl, Sh, Se);
            }
            for (int y = 0; y < 2; y++) {
                df_add2(slh[y][0], sll[y][0], slh[y][1], sll[y][1], kh, kl);
                df_acc(kh, kl, pmh[2 * y][1], pml[2 * y][1], ch, cl, Sh, Se);
                df_add2(shh[y][0], shl[y][0], shh[y][1], shl[y][1], kh, kl);
                df_acc(kh, kl, pph[2 * y][1], ppl[2 * y][1], ch, cl, Sh, Se);
            }
            const long long q = nidx(g, a, b, c);
            float Rh, Re;
            ts2(D.fh[q], -Sh, Rh, Re);
            Re += D.fl[q] - Se;
            const float R = Rh + Re;  // 12 w h^2 r
            const float w = wxy * ((!g.per[2] && (c == 0 || c == g.m[2] - 1)) ? 0.5f : 1.f);
            const float rh = R * (ih2 / (12.f * w)) * inv;
            L0.f[q] = rh;
            mx = nmaxf(mx, fabsf(rh));
            s2 = fmaf(rh, rh, s2);
            s1 += rh;
            for (int y = 0; y < 3; y++)
                for (int x = 0; x < 3; x++) {
                    pmh[y][x] = p0h[y][x];
                    pml[y][x] = p0l[y][x];
                    p0h[y][x] = pph[y][x];
                    p0l[y][x] = ppl[y][x];
                }
            for (int y = 0; y < 2; y++)
                for (int x = 0; x < 2; x++) {
                    slh[y][x] = shh[y][x];
                    sll[y][x] = shl[y][x];
                }
        }
    }
    block_red3f(mx, s2, s1);
    if (threadIdx.x == 0) {
        double *p = part + 3 * (blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z));
        p[0] = double(mx);
        p[1] = double(s2);
        p[2] = double(s1);
    }
}

// The double-float residual tiled like nd_tile_kernel (one node per thread,
// a 32 x 8 tile of columns, the halo planes of phi (hi, lo), the cell layers of
// sigma (hi, lo) and f (hi, lo) staged by cp.async in a ring of ND_NS slots):
// the couplings, their order and the final scaling are the column kernel's, so
// the result is the same bit for bit; the sums of sigma over the two cells of
// an upper face (x-z and y-z pairs) are kept for the next plane, where they are
// the lower face's.
constexpr int DBX = 32, DBY = 8, DNT = DBX * DBY;
constexpr int DHX = DBX + 2, DHN = DHX * (DBY + 2);
constexpr int DCX = DBX + 1, DCN = DCX * (DBY + 1);
static_assert(DHN <= 2 * DNT && DCN <= 2 * DNT && DHN > DNT && DCN > DNT, "two halo slots per thread");

struct NdDfStage {
    float ph[DHN], pl[DHN];
    float sh[DCN], sl[DCN];
    float fh[DNT], fl[DNT];
    float e[DHN];  // the update direction at the staged nodes (UPDATE)
};

static int nd_df_zchunk(const NGeom &g) {
    const long long bxy = (long long)((g.m[0] + DBX - 1) / DBX) * ((g.m[1] + DBY - 1) / DBY);
    int zc = 64;
    while (zc > 4 && bxy * ((g.m[2] + zc - 1) / zc) < 4 * 2 * 152) zc >>= 1;
    return zc;
}
static dim3 nd_df_tile_grid(const NGeom &g) {
    const int zc = nd_df_zchunk(g);
    return dim3((g.m[0] + DBX - 1) / DBX, (g.m[1] + DBY - 1) / DBY, (g.m[2] + zc - 1) / zc);
}

// UPDATE: phi after it = st->iter updates is formed here from buffer (it - 1) & 1
// and e = L0.e, node by node as nd_df_update_kernel does (the same arithmetic),
// staged for the residual and written to buffer it & 1 at the block's own nodes;
// without UPDATE the residual reads buffer it & 1.
template <bool UPDATE>
__global__ void __launch_bounds__(DNT, 2)
    nd_df_tile_resid_kernel(NLevel<float> L0, NDF D, const SolveState *st, double *part, int nzc) {
    pdl_trigger();
    pdl_wait();
    extern __shared__ __align__(16) unsigned char nd_smem[];
    NdDfStage *sg = reinterpret_cast<NdDfStage *>(nd_smem);
    const NGeom &g = L0.g;
    const int tid = threadIdx.x, tx = tid % DBX, ty = tid / DBX;
    const int a0 = blockIdx.x * DBX, b0 = blockIdx.y * DBY;
    const int a = a0 + tx, b = b0 + ty;
    const bool own = a < g.m[0] && b < g.m[1];
    const int c0 = blockIdx.z * nzc, c1 = min(c0 + nzc, g.m[2]);
    const int np = g.m[0] * g.m[1], ncp = g.n[0] * g.n[1];
    // halo slots (see nd_tile_kernel): nodes beyond a wall read node 0 of the
    // plane (their couplings' sigma is zero-filled), cells beyond one are zero
    auto nw = [&](int d, int x) { return x > g.m[d] ? -1 : node_wrap(g, d, x); };
    auto cw = [&](int d, int x) { return x > g.m[d] - 1 ? -1 : cell_wrap(g, d, x); };
    int no[2], co[2], cmask = 0;
    for (int k = 0; k < 2; k++) {
        const int sl = tid + k * DNT;
        no[k] = co[k] = 0;
        if (sl < DHN) {
            const int na = nw(0, a0 - 1 + sl % DHX), nb = nw(1, b0 - 1 + sl / DHX);
            if (na >= 0 && nb >= 0) no[k] = na + g.m[0] * nb;
        }
        if (sl < DCN) {
            const int ca = cw(0, a0 - 1 + sl % DCX), cb = cw(1, b0 - 1 + sl / DCX);
            if (ca >= 0 && cb >= 0) {
                co[k] = ca + g.n[0] * cb;
                cmask |= 1 << k;
            }
        }
    }
    const bool slot1n = tid + DNT < DHN, slot1c = tid + DNT < DCN;
    const int qa = own ? a + g.m[0] * b : 0;
    const int it = st->iter;
    const float *__restrict__ xh = nd_phi_h(D, UPDATE ? it - 1 : it), *__restrict__ xl = nd_phi_l(D, UPDATE ? it - 1 : it);
    float *__restrict__ yh = (it & 1) ? D.ph2 : D.ph, *__restrict__ yl = (it & 1) ? D.pl2 : D.pl;
    const float uh = st->scale_h, ul = st->scale_l;
    // halo slots at the block's own nodes (the updated phi is written there)
    bool wr[2];
    for (int k = 0; k < 2; k++) {
        const int sl = tid + k * DNT, sx = sl % DHX - 1, sy = sl / DHX - 1;
        wr[k] = sl < DHN && sx >= 0 && sx < DBX && sy >= 0 && sy < DBY && a0 + sx < g.m[0] && b0 + sy < g.m[1];
    }
    // stage k: phi plane c0 + 1 + k, sigma layer c0 + k, f at plane c0 + k
    auto issue = [&](int k) {
        NdDfStage &S = sg[(k + 2) % ND_NS];
        const int c = c0 + 1 + k, kl = c0 + k;
        if (c <= c1) {
            const int cz = node_wrap(g, 2, c);
            const int o = cz >= 0 ? cz * np : 0;
            cp_async_el(&S.ph[tid], xh + o + no[0], 4);
            cp_async_el(&S.pl[tid], xl + o + no[0], 4);
            if (UPDATE) cp_async_el(&S.e[tid], L0.e + o + no[0], 4);
            if (slot1n) {
                cp_async_el(&S.ph[tid + DNT], xh + o + no[1], 4);
                cp_async_el(&S.pl[tid + DNT], xl + o + no[1], 4);
                if (UPDATE) cp_async_el(&S.e[tid + DNT], L0.e + o + no[1], 4);
            }
        }
        if (kl >= c0 - 1 && kl <= c1 - 1) {
            const int kz = cell_wrap(g, 2, kl);
            const int o = kz >= 0 ? kz * ncp : 0;
            const int m = kz >= 0 ? cmask : 0;
            cp_async_el(&S.sh[tid], D.sh + o + co[0], (m & 1) ? 4 : 0);
            cp_async_el(&S.sl[tid], D.sl + o + co[0], (m & 1) ? 4 : 0);
            if (slot1c) {
                cp_async_el(&S.sh[tid + DNT], D.sh + o + co[1], (m & 2) ? 4 : 0);
                cp_async_el(&S.sl[tid + DNT], D.sl + o + co[1], (m & 2) ? 4 : 0);
            }
        }
        if (own && kl >= c0 && kl < c1) {
            cp_async_el(&S.fh[tid], D.fh + qa + kl * np, 4);
            cp_async_el(&S.fl[tid], D.fl + qa + kl * np, 4);
        }
        cp_async_commit();
    };
    // the update at this thread's halo slots of stage k (phi plane c0 + 1 + k),
    // written out where the slot is one of the block's own nodes of [c0, c1)
    auto update = [&](int k) {
        NdDfStage &S = sg[(k + 2) % ND_NS];
        const int c = c0 + 1 + k;
        const bool wplane = c >= c0 && c < c1;
        const long long o = (long long)c * np;
        for (int j = 0; j < 2; j++) {
            const int sl = tid + j * DNT;
            if (j == 1 && !slot1n) break;
            float h, l;
            nd_df_axpy(S.ph[sl], S.pl[sl], S.e[sl], uh, ul, h, l);
            S.ph[sl] = h;
            S.pl[sl] = l;
            if (wplane && wr[j]) {
                yh[o + no[j]] = h;
                yl[o + no[j]] = l;
            }
        }
    };
    auto get_nodes = [&](int k, float h[3][3], float l[3][3]) {
        const NdDfStage &S = sg[(k + 2) % ND_NS];
        const int o = ty * DHX + tx;
        for (int y = 0; y < 3; y++)
            for (int x = 0; x < 3; x++) {
                h[y][x] = S.ph[o + y * DHX + x];
                l[y][x] = S.pl[o + y * DHX + x];
            }
    };
    auto get_cells = [&](int k, float h[2][2], float l[2][2]) {
        const NdDfStage &S = sg[(k + 2) % ND_NS];
        const int o = ty * DCX + tx;
        for (int y = 0; y < 2; y++)
            for (int x = 0; x < 2; x++) {
                h[y][x] = S.sh[o + y * DCX + x];
                l[y][x] = S.sl[o + y * DCX + x];
            }
    };
    const float inv = st->inv_scale_f;
    const float ih2 = float(1.0 / (g.h * g.h));
    const float wxy = ((!g.per[0] && (a == 0 || a == g.m[0] - 1)) ? 0.5f : 1.f) *
                      ((!g.per[1] && (b == 0 || b == g.m[1] - 1)) ? 0.5f : 1.f);
    const float sc_in = ih2 / (12.f * wxy), sc_wall = ih2 / (12.f * (wxy * 0.5f));
    float mx = 0.f, s2 = 0.f, s1 = 0.f;
    float PH0[3][3], PL0[3][3], PH1[3][3], PL1[3][3], PH2[3][3], PL2[3][3];
    float SH0[2][2], SL0[2][2], SH1[2][2], SL1[2][2];
    float xzh[2], xzl[2], yzh[2], yzl[2];  // lower-face sigma pair sums of the current plane
    issue(-2);
    issue(-1);
    cp_async_wait<0>();
    __syncthreads();
    if (UPDATE) {
        update(-2);
        update(-1);
        __syncthreads();
    }
    get_nodes(-2, PH0, PL0);
    get_nodes(-1, PH1, PL1);
    get_cells(-1, SH0, SL0);
    __syncthreads();
    for (int x = 0; x < 2; x++) df_add2(SH0[0][x], SL0[0][x], SH0[1][x], SL0[1][x], xzh[x], xzl[x]);
    for (int y = 0; y < 2; y++) df_add2(SH0[y][0], SL0[y][0], SH0[y][1], SL0[y][1], yzh[y], yzl[y]);
    issue(0);
    issue(1);
    issue(2);
    auto step = [&](int k, float pmh[3][3], float pml[3][3], float p0h[3][3], float p0l[3][3], float pph[3][3],
                    float ppl[3][3], float slh[2][2], float sll[2][2], float shh[2][2], float shl[2][2]) {
        cp_async_wait<2>();
        __syncthreads();
        if (UPDATE) {
            update(k);
            __syncthreads();
        }
        get_nodes(k, pph, ppl);
        get_cells(k, shh, shl);
        const int c = c0 + k;
        const NdDfStage &S = sg[(k + 2) % ND_NS];
        const float ch = p0h[1][1], cl = p0l[1][1];
        float Sh = 0.f, Se = 0.f, kh, kl;
        for (int y = 0; y < 2; y++)
            for (int x = 0; x < 2; x++) {
                df_add2(slh[y][x], sll[y][x], shh[y][x], shl[y][x], kh, kl);
                df_acc(kh, kl, p0h[2 * y][2 * x], p0l[2 * y][2 * x], ch, cl, Sh, Se);
                df_acc(slh[y][x], sll[y][x], pmh[2 * y][2 * x], pml[2 * y][2 * x], ch, cl, Sh, Se);
                df_acc(shh[y][x], shl[y][x], pph[2 * y][2 * x], ppl[2 * y][2 * x], ch, cl, Sh, Se);
            }
        for (int x = 0; x < 2; x++) {
            df_acc(xzh[x], xzl[x], pmh[1][2 * x], pml[1][2 * x], ch, cl, Sh, Se);
            df_add2(shh[0][x], shl[0][x], shh[1][x], shl[1][x], kh, kl);
            df_acc(kh, kl, pph[1][2 * x], ppl[1][2 * x], ch, cl, Sh, Se);
            xzh[x] = kh;
            xzl[x] = kl;
        }
        for (int y = 0; y < 2; y++) {
            df_acc(yzh[y], yzl[y], pmh[2 * y][1], pml[2 * y][1], ch, cl, Sh, Se);
            df_add2(shh[y][0], shl[y][0], shh[y][1], shl[y][1], kh, kl);
            df_acc(kh, kl, pph[2 * y][1], ppl[2 * y][1], ch, cl, Sh, Se);
            yzh[y] = kh;
            yzl[y] = kl;
        }
        if (own) {
            const int q = qa + c * np;
            float Rh, Re;
            ts2(S.fh[tid], -Sh, Rh, Re);
            Re += S.fl[tid] - Se;
            const float R = Rh + Re;  // 12 w h^2 r
            const bool wall = !g.per[2] && (c == 0 || c == g.m[2] - 1);
            const float rh = R * (wall ? sc_wall : sc_in) * inv;
            L0.f[q] = rh;
            mx = nmaxf(mx, fabsf(rh));
            s2 = fmaf(rh, rh, s2);
            s1 += rh;
        }
        issue(k + 3);
    };
    const int nk = c1 - c0;
    for (int k = 0; k < nk; k += 6) {
        step(k, PH0, PL0, PH1, PL1, PH2, PL2, SH0, SL0, SH1, SL1);
        if (k + 1 >= nk) break;
        step(k + 1, PH1, PL1, PH2, PL2, PH0, PL0, SH1, SL1, SH0, SL0);
        if (k + 2 >= nk) break;
        step(k + 2, PH2, PL2, PH0, PL0, PH1, PL1, SH0, SL0, SH1, SL1);
        if (k + 3 >= nk) break;
        step(k + 3, PH0, PL0, PH1, PL1, PH2, PL2, SH1, SL1, SH0, SL0);
        if (k + 4 >= nk) break;
        step(k + 4, PH1, PL1, PH2, PL2, PH0, PL0, SH0, SL0, SH1, SL1);
        if (k + 5 >= nk) break;
        step(k + 5, PH2, PL2, PH0, PL0, PH1, PL1, SH1, SL1, SH0, SL0);
    }
    cp_async_wait<0>();
    block_red3f(mx, s2, s1);
    if (threadIdx.x == 0) {
        double *p = part + 3 * (blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z));
        p[0] = double(mx);
        p[1] = double(s2);
        p[2] = double(s1);
    }
}

static dim3 nd_col_grid(const NGeom &g) { return dim3((g.m[0] + 63) / 64, g.m[1], (g.m[2] + NCZ - 1) / NCZ); }
static int nd_col_blocks(const NGeom &g) {
    const dim3 d = nd_col_grid(g);
    return int(d.x * d.y * d.z);
}

// FP64 residual r = f - L phi (plain FP64 path and mx_residual), columns marched in z
__global__ void nd_col_resid64_kernel(NLevel<double> L, const double *__restrict__ phi, const double *__restrict__ f,
                                      double *__restrict__ rout, double *__restrict__ rhat, const SolveState *st,
                                      double *part) {
    const NGeom &g = L.g;
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    const int c0 = blockIdx.z * NCZ, c1 = min(c0 + NCZ, g.m[2]);
    const double inv = st ? st->inv_scale : 1.0;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    if (a < g.m[0]) {
        const ColMap m = col_map(g, a, b);
        const double wxy = ((!g.per[0] && (a == 0 || a == g.m[0] - 1)) ? 0.5 : 1.0) *
                           ((!g.per[1] && (b == 0 || b == g.m[1] - 1)) ? 0.5 : 1.0);
        double pm[3][3], p0[3][3], pp[3][3], sl[2][2], sh[2][2];
        load_node_plane(g, m, phi, c0 - 1, pm);
        load_node_plane(g, m, phi, c0, p0);
        load_cell_plane(g, m, L.sigma, c0 - 1, sl);
        for (int c = c0; c < c1; c++) {
            load_node_plane(g, m, phi, c + 1, pp);
            load_cell_plane(g, m, L.sigma, c, sh);
            // differences from the centre keep the cancellation exact in FP64
            double dm[3][3], d0[3][3], dp[3][3];
            for (int y = 0; y < 3; y++)
                for (int x = 0; x < 3; x++) {
                    dm[y][x] = pm[y][x] - p0[1][1];
                    d0[y][x] = p0[y][x] - p0[1][1];
                    dp[y][x] = pp[y][x] - p0[1][1];
                }
            double num, den;
            couplings(dm, d0, dp, sl, sh, num, den);
            const double w = wxy * ((!g.per[2] && (c == 0 || c == g.m[2] - 1)) ? 0.5 : 1.0);
            const long long q = nidx(g, a, b, c);
            const double r = f[q] - num / (12.0 * w * g.h * g.h);
            if (rout) rout[q] = r;
            if (rhat) rhat[q] = r * inv;
            mx = nmax(mx, fabs(r));
            s2 += r * r;
            s1 += r;
            for (int y = 0; y < 3; y++)
                for (int x = 0; x < 3; x++) {
                    pm[y][x] = p0[y][x];
                    p0[y][x] = pp[y][x];
                }
            for (int y = 0; y < 2; y++)
                for (int x = 0; x < 2; x++) sl[y][x] = sh[y][x];
        }
    }
    block_red3(mx, s2, s1);
    if (threadIdx.x == 0) {
        double *p = part + 3 * (blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z));
        p[0] = mx;
        p[1] = s2;
        p[2] = s1;
    }
}

__global__ void nd_update64_kernel(double *phi, const double *e, const SolveState *st, long long M) {
    const double sc = st->scale;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < M; q += (long long)gridDim.x * blockDim.x)
        phi[q] += sc * e[q];
}

__global__ void nd_split_kernel(const double *__restrict__ x, float *__restrict__ hi, float *__restrict__ lo,
                                long long M) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < M; q += (long long)gridDim.x * blockDim.x) {
        const float h = __double2float_rn(x[q]);
        hi[q] = h;
        lo[q] = __double2float_rn(x[q] - double(h));
    }
}

// r = f - L phi with L phi from the FP32 operator (mx_residual, mixed precision)
__global__ void nd_resid32_kernel(const double *__restrict__ f, const float *__restrict__ lphi, double *__restrict__ r,
                                  long long M, double *part) {
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < M; q += (long long)gridDim.x * blockDim.x) {
        const double v = double(float(f[q]) - lphi[q]);
        r[q] = v;
        mx = nmax(mx, fabs(v));
    }
    block_red3(mx, s2, s1);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = mx;
        part[3 * blockIdx.x + 1] = s2;
        part[3 * blockIdx.x + 2] = s1;
    }
}


// weighted mean of phi -> st->aux, then subtraction
__global__ void nd_wsum_kernel(NGeom g, const double *x, double *part) {
    double s1 = 0.0, s0 = 0.0, m = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.M; q += (long long)gridDim.x * blockDim.x) {
        int a, b, c;
        node_of(g, q, a, b, c);
        const double w = node_w(g, a, b, c);
        s1 += w * x[q];
        s0 += w;
    }
    block_red3(m, s1, s0);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = 0.0;
        part[3 * blockIdx.x + 1] = s1;
        part[3 * blockIdx.x + 2] = s0;
    }
}
__global__ void nd_wmean_finalize_kernel(const double *part, int nb, double *dst) {
    double a, b, c;
    reduce_partials3(part, nb, a, b, c);
    if (threadIdx.x == 0) *dst = b / c;
}

// U -= G phi / rho at cell centres
// U -= G_c phi / rho per cell: (G_c phi)_d = (1/(4h)) sum of the 4 d-edges of
// the cell.  Cell columns walk up k and reuse the top face's nodes as the next
// cell's bottom face.
__global__ void nd_correct_kernel(NGeom g, const double *__restrict__ rho, const double *__restrict__ phi,
                                  double *__restrict__ ux, double *__restrict__ uy, double *__restrict__ uz,
                                  double i4h) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int k0 = blockIdx.z * NRZ, k1 = min(k0 + NRZ, g.n[2]);
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int a1 = (g.per[0] && i + 1 == g.m[0]) ? 0 : i + 1;
    const int b1 = (g.per[1] && j + 1 == g.m[1]) ? 0 : j + 1;
    const int m01 = g.m[0] * g.m[1];
    const int o00 = i + g.m[0] * j, o10 = a1 + g.m[0] * j, o01 = i + g.m[0] * b1, o11 = a1 + g.m[0] * b1;
    auto face = [&](int c, double p[4]) {
        const int cc = (g.per[2] && c == g.m[2]) ? 0 : c;
        const double *q = phi + (long long)m01 * cc;
        p[0] = q[o00];
        p[1] = q[o10];
        p[2] = q[o01];
        p[3] = q[o11];
    };
    double lo[4], hi[4];
    face(k0, lo);
    for (int k = k0; k < k1; k++) {
        face(k + 1, hi);
        const double gx = ((lo[1] - lo[0]) + (lo[3] - lo[2]) + (hi[1] - hi[0]) + (hi[3] - hi[2])) * i4h;
        const double gy = ((lo[2] - lo[0]) + (lo[3] - lo[1]) + (hi[2] - hi[0]) + (hi[3] - hi[1])) * i4h;
        const double gz = ((hi[0] - lo[0]) + (hi[1] - lo[1]) + (hi[2] - lo[2]) + (hi[3] - lo[3])) * i4h;
        const int c = i + g.n[0] * (j + g.n[1] * k);
        const double ir = rcp64(rho[c]);
        ux[c] -= gx * ir;
        uy[c] -= gy * ir;
        uz[c] -= gz * ir;
        for (int e = 0; e < 4; e++) lo[e] = hi[e];
    }
}

// ---- mixed precision: setup and finish in double-float arithmetic ----------------------
// FP64 inputs are split into double-float pairs by integer bit operations and
// the arithmetic runs on the FP32 pipe (GB300 executes FP64 at 1/58 of the
// FP32 rate); results written as FP64 are formed from their pairs with one
// FP64 addition.

// sigma = beta0 / rho as (hi, lo)
__global__ void nd_sigma_df_kernel(long long N, const double *__restrict__ rho, const double *__restrict__ beta0,
                                   float *__restrict__ s32, float *__restrict__ sl) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const dfloat v = df_div(df_split(beta0[q]), df_split(rho[q]));
        s32[q] = v.h;
        sl[q] = v.l;
    }
}

struct RhsLayerDF {
    dfloat x, y, z, s;
    int n;
};

// The products beta0 (ux, uy, uz, Sbar) of every cell in double-float, formed once
// per cell (the node gather below adds them; forming them inside the gather did
// the same work for each of the cell's four node columns): P[2c] = (beta0 ux,
// beta0 uy), P[2c+1] = (beta0 uz, beta0 Sbar), each as (hi, lo).
__device__ __forceinline__ void cell_products(const double *__restrict__ ux, const double *__restrict__ uy,
                                              const double *__restrict__ uz, const double *__restrict__ beta0,
                                              const double *__restrict__ sbar, long long c, float4 *__restrict__ P) {
    const dfloat bt = df_split(beta0[c]);
    const dfloat px = df_mul(bt, df_split(ux[c])), py = df_mul(bt, df_split(uy[c]));
    const dfloat pz = df_mul(bt, df_split(uz[c])), ps = df_mul(bt, df_split(sbar[c]));
    P[2 * c] = make_float4(px.h, px.l, py.h, py.l);
    P[2 * c + 1] = make_float4(pz.h, pz.l, ps.h, ps.l);
}
__global__ void nd_cell_prod_kernel(long long N, const double *__restrict__ ux, const double *__restrict__ uy,
                                    const double *__restrict__ uz, const double *__restrict__ beta0,
                                    const double *__restrict__ sbar, float4 *__restrict__ P) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x)
        cell_products(ux, uy, uz, beta0, sbar, q, P);
}
// rhs_layer_df from the formed products: the same additions in the same order
__device__ __forceinline__ RhsLayerDF rhs_layer_pre(const NGeom &g, const float4 *__restrict__ P, int i0, int i1,
                                                    int j0, int j1, int k) {
    RhsLayerDF L = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, 0};
    const int kk = cell_wrap(g, 2, k);
    if (kk < 0) return L;
    for (int jj = 0; jj < 2; jj++) {
        const int j = jj ? j1 : j0;
        if (j < 0) continue;
        for (int ii = 0; ii < 2; ii++) {
            const int i = ii ? i1 : i0;
            if (i < 0) continue;
            const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * kk);
            const float4 a = P[2 * c], b = P[2 * c + 1];
            const dfloat px = {a.x, a.y}, py = {a.z, a.w}, pz = {b.x, b.y}, ps = {b.z, b.w};
            L.x = df_add(L.x, ii ? px : df_neg(px));
            L.y = df_add(L.y, jj ? py : df_neg(py));
            L.z = df_add(L.z, pz);
            L.s = df_add(L.s, ps);
            L.n++;
        }
    }
    return L;
}

__device__ __forceinline__ dfloat df_scale(dfloat a, float p2) { return dfloat{a.h * p2, a.l * p2}; }  // p2 = 2^k

// the gather of nd_rhs_col_kernel in double-float: f (may be null) as (fh, fl),
// partials (max |f|, sum w f, sum w); i4h8 = 8/(4h)
__global__ void nd_rhs_col_df_kernel(NGeom g, const float4 *__restrict__ P, float *__restrict__ fh,
                                     float *__restrict__ fl, double *part, int sub_mean, const SolveState *st,
                                     dfloat i4h8) {
    float s0 = 0.f;
    dfloat mx = {0.f, 0.f}, s1 = {0.f, 0.f};
    const int a = blockIdx.x * 32 + threadIdx.x, b = blockIdx.y * 8 + threadIdx.y;
    const int c0 = blockIdx.z * NRZ, c1 = min(c0 + NRZ, g.m[2]);
    if (a < g.m[0] && b < g.m[1]) {
        const dfloat cm = sub_mean ? df_split(st->mean) : dfloat{0.f, 0.f};
        const int i0 = cell_wrap(g, 0, a - 1), i1 = cell_wrap(g, 0, a);
        const int j0 = cell_wrap(g, 1, b - 1), j1 = cell_wrap(g, 1, b);
        RhsLayerDF lo = rhs_layer_pre(g, P, i0, i1, j0, j1, c0 - 1);
        for (int c = c0; c < c1; c++) {
            const RhsLayerDF hi = rhs_layer_pre(g, P, i0, i1, j0, j1, c);
            const int cnt = lo.n + hi.n;  // 1, 2, 4 or 8
            const float ic = cnt == 8 ? 0.125f : cnt == 4 ? 0.25f : cnt == 2 ? 0.5f : 1.f;
            const dfloat div = df_add(df_add(df_add(lo.x, hi.x), df_add(lo.y, hi.y)), df_sub(hi.z, lo.z));
            const dfloat v = df_sub(df_sub(df_mul(div, df_scale(i4h8, ic)), df_scale(df_add(lo.s, hi.s), ic)), cm);
            const float w = 0.125f * cnt;
            if (fh) {
                const int q = a + g.m[0] * (b + g.m[1] * c);
                fh[q] = v.h;
                fl[q] = v.l;
            }
            df_absmax(mx, v);
            s1 = df_add(s1, df_scale(v, w));
            s0 += w;
            lo = hi;
        }
    }
    double pa = df_to_double(mx), pb = df_to_double(s1), pc = s0;
    block_red3(pa, pb, pc);
    if (flat_tid() == 0) {
        double *p = part + 3 * flat_bid();
        p[0] = pa;
        p[1] = pb;
        p[2] = pc;
    }
}

// f <- 12 h^2 w (f - mean) in double-float; partials (max, sum^2, sum) of f - mean
__global__ void nd_rhs_final_df_kernel(NGeom g, const SolveState *st, dfloat h2x12, float *__restrict__ fh,
                                       float *__restrict__ fl, double *part) {
    const dfloat m = df_split(st->mean);
    dfloat mx = {0.f, 0.f}, s1 = {0.f, 0.f};
    float s2 = 0.f;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.M; q += (long long)gridDim.x * blockDim.x) {
        int a, b, c;
        node_of(g, q, a, b, c);
        const dfloat v = df_sub(dfloat{fh[q], fl[q]}, m);
        const dfloat sv = df_mul(df_scale(h2x12, node_w(g, a, b, c)), v);
        fh[q] = sv.h;
        fl[q] = sv.l;
        df_absmax(mx, v);
        s2 = fmaf(v.h, v.h, s2);
        s1 = df_add(s1, v);
    }
    double pa = df_to_double(mx), pb = s2, pc = df_to_double(s1);
    block_red3(pa, pb, pc);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = pa;
        part[3 * blockIdx.x + 1] = pb;
        part[3 * blockIdx.x + 2] = pc;
    }
}

// phi (double) from its double-float pair, with partials (0, sum w phi, sum w)
__global__ void nd_df_final_sum_kernel(NGeom g, NDF D, const SolveState *st, double *__restrict__ phi, double *part) {
    const float *__restrict__ xh = nd_phi_h(D, st->iter), *__restrict__ xl = nd_phi_l(D, st->iter);
    dfloat s1 = {0.f, 0.f};
    float s0 = 0.f;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.M; q += (long long)gridDim.x * blockDim.x) {
        int a, b, c;
        node_of(g, q, a, b, c);
        const dfloat v = {xh[q], xl[q]};
        phi[q] = df_to_double(v);
        const float w = node_w(g, a, b, c);
        s1 = df_add(s1, df_scale(v, w));
        s0 += w;
    }
    double pa = 0.0, pb = df_to_double(s1), pc = s0;
    block_red3(pa, pb, pc);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = pa;
        part[3 * blockIdx.x + 1] = pb;
        part[3 * blockIdx.x + 2] = pc;
    }
}

// U -= G_c phi / rho per cell from phi's double-float pair (the weighted mean
// of phi cancels in the edge differences), in double-float
// (also forms the cell products of the corrected U for the divergence check)
__global__ void nd_correct_df_kernel(NGeom g, const double *__restrict__ rho, NDF D, const SolveState *st,
                                     double *__restrict__ ux, double *__restrict__ uy, double *__restrict__ uz,
                                     dfloat i4h, const double *__restrict__ beta0, const double *__restrict__ sbar,
                                     float4 *__restrict__ P) {
    const float *__restrict__ xh = nd_phi_h(D, st->iter), *__restrict__ xl = nd_phi_l(D, st->iter);
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int k0 = blockIdx.z * NRZ, k1 = min(k0 + NRZ, g.n[2]);
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int a1 = (g.per[0] && i + 1 == g.m[0]) ? 0 : i + 1;
    const int b1 = (g.per[1] && j + 1 == g.m[1]) ? 0 : j + 1;
    const int m01 = g.m[0] * g.m[1];
    const int o00 = i + g.m[0] * j, o10 = a1 + g.m[0] * j, o01 = i + g.m[0] * b1, o11 = a1 + g.m[0] * b1;
    auto face = [&](int c, dfloat p[4]) {
        const int cc = (g.per[2] && c == g.m[2]) ? 0 : c;
        const int base = m01 * cc;
        p[0] = dfloat{xh[base + o00], xl[base + o00]};
        p[1] = dfloat{xh[base + o10], xl[base + o10]};
        p[2] = dfloat{xh[base + o01], xl[base + o01]};
        p[3] = dfloat{xh[base + o11], xl[base + o11]};
    };
    dfloat lo[4], hi[4];
    face(k0, lo);
    for (int k = k0; k < k1; k++) {
        face(k + 1, hi);
        const dfloat gx = df_add(df_add(df_sub(lo[1], lo[0]), df_sub(lo[3], lo[2])),
                                 df_add(df_sub(hi[1], hi[0]), df_sub(hi[3], hi[2])));
        const dfloat gy = df_add(df_add(df_sub(lo[2], lo[0]), df_sub(lo[3], lo[1])),
                                 df_add(df_sub(hi[2], hi[0]), df_sub(hi[3], hi[1])));
        const dfloat gz = df_add(df_add(df_sub(hi[0], lo[0]), df_sub(hi[1], lo[1])),
                                 df_add(df_sub(hi[2], lo[2]), df_sub(hi[3], lo[3])));
        const int c = i + g.n[0] * (j + g.n[1] * k);
        const dfloat f = df_div(i4h, df_split(rho[c]));  // 1/(4 h rho)
        ux[c] = df_to_double(df_sub(df_split(ux[c]), df_mul(gx, f)));
        uy[c] = df_to_double(df_sub(df_split(uy[c]), df_mul(gy, f)));
        uz[c] = df_to_double(df_sub(df_split(uz[c]), df_mul(gz, f)));
        cell_products(ux, uy, uz, beta0, sbar, c, P);
        for (int e = 0; e < 4; e++) lo[e] = hi[e];
    }
}

static dfloat df_host(double v) {
    dfloat r;
    r.h = float(v);
    r.l = float(v - double(r.h));
    return r;
}

// ---- host side -------------------------------------------------------------------------

static bool same_ngeom(const NGeom &a, const NGeom &b) {
    for (int d = 0; d < 3; d++)
        if (a.n[d] != b.n[d] || a.per[d] != b.per[d]) return false;
    return a.h == b.h;
}

static void carve_nodal(Bump &b, NodalPlan &P) {
    NGeom gs[MX_MAXLEV];
    P.nlev = nodal_levels(P.g, gs);
    for (int l = 0; l < P.nlev; l++) {
        if (P.prec == MX_PREC_MIXED) {
            P.L32[l].g = gs[l];
            P.L32[l].sigma = b.take<float>(gs[l].N);
            P.L32[l].f = b.take<float>(gs[l].M);
            P.L32[l].e = b.take<float>(gs[l].M);
            P.L32[l].r = b.take<float>(gs[l].M);
            P.L32[l].e2 = b.take<float>(gs[l].M);
        } else {
            P.L64[l].g = gs[l];
            P.L64[l].sigma = b.take<double>(gs[l].N);
            P.L64[l].f = b.take<double>(gs[l].M);
            P.L64[l].e = b.take<double>(gs[l].M);
            P.L64[l].r = b.take<double>(gs[l].M);
            P.L64[l].e2 = b.take<double>(gs[l].M);
        }
    }
    const long long Mb = gs[P.nlev - 1].M;
    if (P.prec == MX_PREC_MIXED) {
        P.bot32 = b.take<float>(6 * Mb);
        P.D.sh = P.L32[0].sigma;
        P.D.sl = b.take<float>(P.g.N);
        P.D.fh = b.take<float>(P.g.M);
        P.D.fl = b.take<float>(P.g.M);
        P.D.ph = b.take<float>(P.g.M);
        P.D.pl = b.take<float>(P.g.M);
        P.D.ph2 = b.take<float>(P.g.M);
        P.D.pl2 = b.take<float>(P.g.M);
        P.cellp = b.take<float4>(2 * P.g.N);
        P.sigma64 = nullptr;
    } else {
        P.bot64 = b.take<double>(6 * Mb);
        P.sigma64 = P.L64[0].sigma;
    }
    P.f64 = b.take<double>(P.g.M);
}

static void free_nodal_plan(NodalPlan *p) {
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->mem) cudaFree(p->mem);
    delete p;
}

static NodalPlan *get_nodal_plan(mx_ctx *c, const NGeom &g, int prec, mx_status *st) {
    const dim3 tg = nd_df_tile_grid(g);
    *st = ensure_partials(c, std::max<long long>(std::max(152 * 8, nd_col_blocks(g)), (long long)tg.x * tg.y * tg.z));
    if (*st) return nullptr;
    for (NodalPlan *p : c->nplans)
        if (p->prec == prec && same_ngeom(p->g, g)) {
            p->last_use = ++c->use_counter;
            return p;
        }
    if (c->nplans.size() >= 2) {
        auto it = std::min_element(c->nplans.begin(), c->nplans.end(),
                                   [](NodalPlan *a, NodalPlan *b) { return a->last_use < b->last_use; });
        cudaStreamSynchronize(c->stream);
        free_nodal_plan(*it);
        c->nplans.erase(it);
    }
    NodalPlan *P = new NodalPlan();
    P->g = g;
    P->prec = prec;
    Bump dry{nullptr, 0};
    carve_nodal(dry, *P);
    if (cudaMalloc(&P->mem, dry.off + 256) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        *st = set_err(c, MX_ERR_OOM, "nodal plan cudaMalloc failed");
        return nullptr;
    }
    Bump real{(char *)P->mem, 0};
    carve_nodal(real, *P);
    P->last_use = ++c->use_counter;
    c->nplans.push_back(P);
    return P;
}

void destroy_nodal_plans(mx_ctx *c) {
    for (NodalPlan *p : c->nplans) free_nodal_plan(p);
    c->nplans.clear();
}

static int nblk(long long n) { return red_blocks(n); }

// Chebyshev: pre-smoothing from e = 0 starts writing in the buffer that leaves the
// result in e; post-smoothing starts from the prolonged e, put in e2 (the
// prolongation writes out of place) when the step count is odd, in e otherwise,
// so every level's final correction is in e as with the colour sweeps.
template <typename T>
static void nd_vcycle(cudaStream_t s, NLevel<T> *L, int nl, T *bot, int nu1, int nu2, int bot_iters, mx_ctx *pc,
                      int zcap, int cheb = 0) {
    double w1[16], w2[16];
    if (cheb) {
        // one Chebyshev polynomial of degree nu1 + nu2 per V-cycle, its roots split:
        // post-smoothing takes the nu2 largest, pre-smoothing the nu1 smallest (of
        // the splits tried -- this one, the reverse, alternating -- the one that
        // converged in the fewest V-cycles)
        double w[32];
        cheb_weights(nu1 + nu2, CHEB_LO, CHEB_HI, w);
        for (int k = 0; k < nu2; k++) w2[k] = w[k];
        for (int k = 0; k < nu1; k++) w1[k] = w[nu2 + k];
    }
    prof_begin(pc, s, MX_PH_UPDATE);
    if (!cheb) cudaMemsetAsync(L[0].e, 0, sizeof(T) * L[0].g.M, s);
    prof_end(pc, s, MX_PH_UPDATE, cheb ? 0 : 1);
    for (int l = 0; l < nl - 1; l++) {
        if (l == 0) prof_begin(pc, s, MX_PH_SMOOTH_FINE);
        if (cheb) {
            T *bufs[2] = {L[l].e, L[l].e2};
            int o = nu1 % 2 == 1 ? 0 : 1;
            const T *in = nullptr;
            for (int q = 0; q < nu1; q++) {
                k_nd_cheb(s, L[l], in, bufs[o], T(w1[q]), zcap);
                in = bufs[o];
                o ^= 1;
            }
        } else {
            for (int q = 0; q < nu1; q++)
                for (int col = 0; col < 4; col++) k_nd_gs(s, L[l], col, zcap);
        }
        if (l == 0) {
            prof_end(pc, s, MX_PH_SMOOTH_FINE, cheb ? nu1 : 4 * nu1);
            prof_begin(pc, s, MX_PH_RESTRICT_FINE);
        }
        k_nd_residual(s, L[l], zcap);
        {
            const NGeom &gc = L[l + 1].g;
            const int zc = nd_xfer_zc(gc);
            launch_pdl(nd_restrict_march_kernel<T>, dim3((gc.m[0] + 31) / 32, (gc.m[1] + 7) / 8, (gc.m[2] + zc - 1) / zc),
                       dim3(32, 8), 0, s, L[l], L[l + 1], zc);
        }
        if (l == 0) {
            prof_end(pc, s, MX_PH_RESTRICT_FINE, 2);
            prof_begin(pc, s, MX_PH_COARSE);
        }
    }
    if (nl == 1) prof_begin(pc, s, MX_PH_COARSE);
    launch_pdl(nd_bottom_kernel<T>, dim3(1), dim3(NBT), 0, s, L[nl - 1], bot, bot_iters);
    if (nl == 1) prof_end(pc, s, MX_PH_COARSE, 1);
    for (int l = nl - 2; l >= 0; l--) {
        if (l == 0) {
            prof_end(pc, s, MX_PH_COARSE, 0);
            prof_begin(pc, s, MX_PH_PROLONG_FINE);
        }
        const bool odd = cheb && nu2 % 2 == 1;
        {
            const NGeom &gf = L[l].g;
            const int zc = nd_xfer_zc(gf);
            launch_pdl(nd_prolong_march_kernel<T>, dim3((gf.m[0] + 31) / 32, (gf.m[1] + 7) / 8, (gf.m[2] + zc - 1) / zc),
                       dim3(32, 8), 0, s, L[l + 1], L[l], odd ? L[l].e2 : (T *)nullptr, zc);
        }
        if (l == 0) {
            prof_end(pc, s, MX_PH_PROLONG_FINE, 1);
            prof_begin(pc, s, MX_PH_SMOOTH_FINE);
        }
        if (cheb) {
            T *in = odd ? L[l].e2 : L[l].e;
            for (int q = 0; q < nu2; q++) {
                T *out = in == L[l].e ? L[l].e2 : L[l].e;
                k_nd_cheb(s, L[l], (const T *)in, out, T(w2[q]), zcap);
                in = out;
            }
        } else {
            for (int q = 0; q < nu2; q++)
                for (int col = 3; col >= 0; col--) k_nd_gs(s, L[l], col, zcap);
        }
        if (l == 0) prof_end(pc, s, MX_PH_SMOOTH_FINE, cheb ? nu2 : 4 * nu2);
    }
}

static mx_status nodal_setup(mx_ctx *c, NodalPlan &P, const double *rho, const double *beta0) {
    cudaStream_t s = c->stream;
    const NGeom &g = P.g;
    if (P.prec == MX_PREC_MIXED) {
        nd_sigma_df_kernel<<<nblk(g.N), 256, 0, s>>>(g.N, rho, beta0, P.L32[0].sigma, P.D.sl);
        for (int l = 0; l + 1 < P.nlev; l++)
            nd_coarsen_sigma_kernel<float><<<nblk(P.L32[l + 1].g.N), 256, 0, s>>>(P.L32[l], P.L32[l + 1]);
    } else {
        nd_sigma_kernel<<<nblk(g.N), 256, 0, s>>>(g.N, rho, beta0, P.L64[0].sigma, nullptr, nullptr);
        for (int l = 0; l + 1 < P.nlev; l++)
            nd_coarsen_sigma_kernel<double><<<nblk(P.L64[l + 1].g.N), 256, 0, s>>>(P.L64[l], P.L64[l + 1]);
    }
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

extern "C" mx_status mx_nodal_project(mx_ctx *c, const mx_geom *geom, double *ux, double *uy, double *uz,
                                      const double *rho, const double *beta0, const double *sbar, double *phi,
                                      const mx_opts *opts, mx_info *info) {
    if (!c) return MX_ERR_ARG;
    mx_status st = check_geom(c, geom, true);
    if (st) return st;
    if (!ux || !uy || !uz || !rho || !beta0 || !sbar || !phi) return set_err(c, MX_ERR_ARG, "nodal_project: null array");
    mx_opts o;
    if (opts) o = *opts;
    else mx_default_opts(&o);
    if (!(o.rel_tol >= 0.0) || o.max_outer < 0 || o.nu1 < 0 || o.nu2 < 0 || o.nu1 > 16 || o.nu2 > 16 ||
        o.bottom_iters < 1 || (o.prec != MX_PREC_FP64 && o.prec != MX_PREC_MIXED) ||
        !(o.tile_z == 0 || o.tile_z == 1 || o.tile_z == 2 || o.tile_z == 4 || o.tile_z == 8 || o.tile_z == 16) ||
        (o.smoother != 0 && o.smoother != 1))
        return set_err(c, MX_ERR_ARG, "invalid options");
    if (o.krylov) return set_err(c, MX_ERR_ARG, "nodal: krylov = 1 is for MAC solves");
    tune_apply(c, MX_OP_NODAL, geom, o);
    if (o.nu1 < 1 || o.nu2 < 1) return set_err(c, MX_ERR_ARG, "nodal: nu1 and nu2 must be >= 1 (or both 0)");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    const NGeom g = make_ngeom(make_dgeom(geom));
    NodalPlan *P = get_nodal_plan(c, g, o.prec, &st);
    if (!P) return st;
    cudaStream_t s = c->stream;
    const int nb = nblk(g.M);
    MX_CUDA(c, cudaEventRecord(c->ev0, s));
    SolveState init = {};
    init.tol = o.rel_tol;
    init.maxit = std::min(o.max_outer, o.max_vcycles);
    *c->hstate = init;
    MX_CUDA(c, cudaMemcpyAsync(c->state, c->hstate, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    prof_begin(c, s, MX_PH_SETUP);
    if ((st = nodal_setup(c, *P, rho, beta0))) return st;
    const bool mixed = o.prec == MX_PREC_MIXED;
    if (mixed) {
        nd_cell_prod_kernel<<<nblk(g.N), 256, 0, s>>>(g.N, ux, uy, uz, beta0, sbar, P->cellp);
        nd_rhs_col_df_kernel<<<nd_node_grid(g), dim3(32, 8), 0, s>>>(g, P->cellp, P->D.fh, P->D.fl, c->partials, 0,
                                                                    c->state, df_host(2.0 / g.h));
    } else
        nd_rhs_col_kernel<<<nd_node_grid(g), dim3(32, 8), 0, s>>>(g, ux, uy, uz, beta0, sbar, P->f64, c->partials, 0,
                                                                 c->state, 0.25 / g.h);
    nd_finalize_rhs_kernel<<<1, 1024, 0, s>>>(c->partials, nd_node_blocks(g), c->state, o.remove_mean, 0);
    if (!o.remove_mean) {
        MX_CUDA(c, cudaMemcpyAsync(c->hstate, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        MX_CUDA(c, cudaStreamSynchronize(s));
        if (std::fabs(c->hstate->aux) > 1e-12 * c->hstate->fnorm) {
            if (info) {
                std::memset(info, 0, sizeof(*info));
                info->status = MX_ERR_INCOMPAT;
            }
            return set_err(c, MX_ERR_INCOMPAT, "nodal: right-hand side has non-zero weighted mean and remove_mean = 0");
        }
    }
    if (mixed)
        nd_rhs_final_df_kernel<<<nb, 256, 0, s>>>(g, c->state, df_host(12.0 * g.h * g.h), P->D.fh, P->D.fl,
                                                  c->partials);
    else
        nd_rhs_final_kernel<<<nb, 256, 0, s>>>(g, P->f64, c->state, nullptr, nullptr, c->partials);
    nd_finalize_rhs_kernel<<<1, 1024, 0, s>>>(c->partials, nb, c->state, 0, 1);
    if (mixed) {
        if (o.use_initial_guess) nd_split_kernel<<<nb, 256, 0, s>>>(phi, P->D.ph, P->D.pl, g.M);
        // else phi = 0 is set by the first residual's pass
    } else if (!o.use_initial_guess) {
        MX_CUDA(c, cudaMemsetAsync(phi, 0, sizeof(double) * g.M, s));
    }
    prof_end(c, s, MX_PH_SETUP, 0);
    const int zcap = o.tile_z ? o.tile_z : NCZ;
    // refinement loop: residual, then while not converged {V-cycle, update, residual}
    // (upd: the tiled double-float residual also applies the loop's update)
    const bool tiled = mixed && nd_tiled(g);
    auto residual = [&](cudaStream_t ss, mx_ctx *pc, bool upd) {
        prof_begin(pc, ss, MX_PH_RESID64);
        int nparts = nd_col_blocks(g);
        if (tiled) {
            const dim3 grid = nd_df_tile_grid(g);
            nparts = int(grid.x * grid.y * grid.z);
            auto kern = upd ? nd_df_tile_resid_kernel<true> : nd_df_tile_resid_kernel<false>;
            launch_pdl(kern, grid, dim3(DNT), sizeof(NdDfStage) * ND_NS, ss, P->L32[0], P->D,
                       (const SolveState *)c->state, c->partials, nd_df_zchunk(g));
        } else if (mixed) {
            launch_pdl(nd_df_col_resid_kernel, nd_col_grid(g), dim3(64), 0, ss, P->L32[0], P->D,
                       (const SolveState *)c->state, c->partials);
        } else {
            nd_col_resid64_kernel<<<nd_col_grid(g), 64, 0, ss>>>(P->L64[0], phi, P->f64, nullptr, P->L64[0].f,
                                                                 c->state, c->partials);
        }
        k_finalize_residual(ss, c->partials, nparts, c->state, mixed ? 1 : 0);
        prof_end(pc, ss, MX_PH_RESID64, 2);
    };
    auto step = [&](cudaStream_t ss, mx_ctx *pc) {
        if (mixed) {
            nd_vcycle<float>(ss, P->L32, P->nlev, P->bot32, o.nu1, o.nu2, o.bottom_iters, pc, zcap, o.smoother);
            if (!tiled) {
                prof_begin(pc, ss, MX_PH_UPDATE);
                launch_pdl(nd_df_update_kernel, dim3(nb), dim3(256), 0, ss, P->D, (long long)g.M,
                           (const float *)P->L32[0].e, (const SolveState *)c->state);
                prof_end(pc, ss, MX_PH_UPDATE, 1);
            }
        } else {
            nd_vcycle<double>(ss, P->L64, P->nlev, P->bot64, o.nu1, o.nu2, o.bottom_iters, pc, zcap, o.smoother);
            prof_begin(pc, ss, MX_PH_UPDATE);
            nd_update64_kernel<<<nb, 256, 0, ss>>>(phi, P->L64[0].e, c->state, g.M);
            prof_end(pc, ss, MX_PH_UPDATE, 1);
        }
        residual(ss, pc, tiled);
    };
    if (mixed && !o.use_initial_guess) {
        prof_begin(c, s, MX_PH_RESID64);
        nd_df_resid_zero_kernel<<<nb, 256, 0, s>>>(P->L32[0], P->D, (const SolveState *)c->state, c->partials);
        k_finalize_residual(s, c->partials, nb, c->state, 1);
        prof_end(c, s, MX_PH_RESID64, 2);
    } else {
        residual(s, c, false);
    }
    MX_CUDA(c, cudaMemcpyAsync(c->hstate, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    MX_CUDA(c, cudaStreamSynchronize(s));
    prof_flush(c);
    if (!c->hstate->done) {
        if (o.use_graph && !c->prof) {
            // the FP64 loop updates phi in place; the mixed loop never touches it
            const void *kphi = mixed ? nullptr : (const void *)phi;
            if (!P->graph || P->graph_phi != kphi || P->graph_nu1 != o.nu1 || P->graph_nu2 != o.nu2 ||
                P->graph_bot != o.bottom_iters || P->graph_tilez != o.tile_z || P->graph_smoother != o.smoother) {
                if (P->graph) {
                    cudaGraphExecDestroy(P->graph);
                    P->graph = nullptr;
                }
                if ((st = capture_while_graph(c, &P->graph, [&](cudaStream_t cs) { step(cs, nullptr); }))) return st;
                P->graph_phi = kphi;
                P->graph_nu1 = o.nu1;
                P->graph_nu2 = o.nu2;
                P->graph_bot = o.bottom_iters;
                P->graph_tilez = o.tile_z;
                P->graph_smoother = o.smoother;
            }
            MX_CUDA(c, cudaGraphLaunch(P->graph, s));
        } else {
            do {
                step(s, c);
                MX_CUDA(c, cudaMemcpyAsync(c->hstate, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
                MX_CUDA(c, cudaStreamSynchronize(s));
                prof_flush(c);
            } while (!c->hstate->done);
        }
    }
    prof_begin(c, s, MX_PH_FINISH);
    // phi with its weighted mean removed, U -= G_c phi / rho, the divergence check
    const dim3 cgrid((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, (g.n[2] + NRZ - 1) / NRZ);
    if (mixed) {
        nd_df_final_sum_kernel<<<nb, 256, 0, s>>>(g, P->D, c->state, phi, c->partials);
    } else {
        nd_wsum_kernel<<<nb, 256, 0, s>>>(g, phi, c->partials);
    }
    nd_wmean_finalize_kernel<<<1, 1024, 0, s>>>(c->partials, nb, &c->state->aux);
    k_sub_scalar(s, g.M, phi, &c->state->aux);
    if (mixed)
        nd_correct_df_kernel<<<cgrid, dim3(32, 8), 0, s>>>(g, rho, P->D, c->state, ux, uy, uz, df_host(0.25 / g.h),
                                                          beta0, sbar, P->cellp);
    else nd_correct_kernel<<<cgrid, dim3(32, 8), 0, s>>>(g, rho, phi, ux, uy, uz, 0.25 / g.h);
    // divergence of the projected velocity minus Sbar_n minus c: the RHS gather with the mean subtracted
    if (mixed)
        nd_rhs_col_df_kernel<<<nd_node_grid(g), dim3(32, 8), 0, s>>>(g, P->cellp, nullptr, nullptr, c->partials, 1,
                                                                    c->state, df_host(2.0 / g.h));
    else
        nd_rhs_col_kernel<<<nd_node_grid(g), dim3(32, 8), 0, s>>>(g, ux, uy, uz, beta0, sbar, nullptr, c->partials,
                                                                 1, c->state, 0.25 / g.h);
    k_finalize_max(s, c->partials, nd_node_blocks(g), &c->state->div_err);
    prof_end(c, s, MX_PH_FINISH, 6);
    MX_CUDA(c, cudaEventRecord(c->ev1, s));
    MX_CUDA(c, cudaMemcpyAsync(c->hstate, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    MX_CUDA(c, cudaStreamSynchronize(s));
    MX_CUDA(c, cudaGetLastError());
    const SolveState &hs = *c->hstate;
    if (info) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        info->outer_iters = hs.iter;
        info->vcycles = hs.iter;
        info->rel_resid = hs.fnorm > 0 ? hs.rnorm / hs.fnorm : hs.rnorm;
        info->rel_resid_l2 = 0.0;
        info->div_err_linf = hs.div_err;
        info->rhs_mean_removed = hs.mean;
        info->rhs_linf = hs.fnorm;
        info->ms = ms;
        info->status = hs.status;
    }
    if (hs.status != MX_OK) return set_err(c, (mx_status)hs.status, "nodal: no convergence");
    return MX_OK;
}

// mx_apply_op / mx_residual for the nodal operator
mx_status nodal_apply(mx_ctx *c, const mx_geom *geom, int prec, const double *rho, const double *beta0,
                      const double *phi, const double *f, double *out, double *rnorm) {
    const NGeom g = make_ngeom(make_dgeom(geom));
    mx_status st;
    NodalPlan *P = get_nodal_plan(c, g, prec, &st);
    if (!P) return st;
    cudaStream_t s = c->stream;
    if ((st = nodal_setup(c, *P, rho, beta0))) return st;
    const int nb = nblk(g.M);
    if (prec == MX_PREC_FP64) {
        if (f) {
            nd_col_resid64_kernel<<<nd_col_grid(g), 64, 0, s>>>(P->L64[0], phi, f, out, nullptr, nullptr, c->partials);
            if (rnorm) k_finalize_max(s, c->partials, nd_col_blocks(g), &c->state->rnorm);
        } else {
            nd_apply_kernel<double><<<nb, 256, 0, s>>>(P->L64[0], phi, out);
        }
    } else {
        NLevel<float> &l0 = P->L32[0];
        k_cast<float>(s, g.M, phi, l0.e);
        nd_apply_kernel<float><<<nb, 256, 0, s>>>(l0, l0.e, l0.f);
        if (f) {
            nd_resid32_kernel<<<nb, 256, 0, s>>>(f, l0.f, out, g.M, c->partials);
            if (rnorm) k_finalize_max(s, c->partials, nb, &c->state->rnorm);
        } else {
            k_uncast<float>(s, g.M, l0.f, out);
        }
    }
    if (rnorm) {
        MX_CUDA(c, cudaMemcpyAsync(c->hstate, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        MX_CUDA(c, cudaStreamSynchronize(s));
        *rnorm = c->hstate->rnorm;
    }
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

