// Outer (iterative-refinement) loop of the mixed-precision MAC solve in
// double-float arithmetic: each double-precision quantity of the loop (phi, the
// right-hand side and the face coefficients) is held as an unevaluated sum of
// two floats hi + lo (|lo| <= ulp(hi)/2, about 48 significant bits), and the
// residual r = f - L phi and the update phi += s e are evaluated with the
// error-free transformations TwoSum (Knuth) and FMA-based TwoProd (Dekker).
// GB300 executes FP64 at 1/58 of its FP32 rate, so an FP64 residual is bound
// by the FP64 pipe while these kernels stay bound by memory bandwidth.
//
// Accuracy: the RHS is the FP64 value rounded to 48 bits (relative 2^-48) and
// the coefficients are within a few 2^-48; the residual of the stored phi is
// computed with an error of a few 2^-48 relative to the largest flux term, far
// below the 1e-10 relative residual the loop converges to.
#include "mx_async.cuh"
#include "mx_df.cuh"
#include "mx_dfmath.cuh"
#include "mx_stencil.cuh"

// ---- error-free transformations -------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {  // |a| >= |b|
    s = a + b;
    e = b - (s - a);
}
__device__ __forceinline__ void split_double(double x, float &hi, float &lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - double(hi));
}

// ---- coefficients b = (beta0_L + beta0_R)/(rho_L + rho_R) in double-float,
// stored as hi (the FP32 level-0 array) + lo, and (q non-null) the correction
// factors q = 2/(h (rho_L + rho_R)) as FP64; a Dirichlet face uses the interior
// cell: b = 2 beta0/rho, q = 2/(h rho).  Both come from one double-float
// reciprocal of the face's rho sum (a few 2^-48 relative).  rho and beta0 are
// split into double-float once per cell: the split goes to the +x neighbour by
// warp shuffle and to the +y neighbour through shared memory, and the column
// carries the cell below; so every thread of the block runs the plane loop. ----
__device__ __forceinline__ dfloat df_recip(dfloat a) {
    const float r0 = __frcp_rn(a.h);
    float e = fmaf(-a.h, r0, 1.0f);
    e = fmaf(-a.l, r0, e);
    return df_norm(r0, r0 * e);
}

__global__ void mac_coeffs_df_kernel(Level<float> L, DFArrays D, FaceQ Q, const double *__restrict__ rho,
                                     const double *__restrict__ beta0, dfloat ih2x) {
    __shared__ dfloat sr[2][SY][SX], sbt[2][SY][SX];
    const DGeom &g = L.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.x * SX + tx, j = blockIdx.y * SY + ty;
    const int k0 = blockIdx.z * ZC;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long nxy = g.nxy;
    const int k1 = min(k0 + ZC, nz);
    const bool act = i < nx && j < ny;
    const bool wq = Q.x != nullptr;
    const dfloat zero = {0.f, 0.f};
    auto store = [&](float *bh, float *bl, double *qd, long long o, dfloat b, dfloat q) {
        bh[o] = b.h;
        bl[o] = b.l;
        if (wq) qd[o] = df_to_double(q);
    };
    auto face = [&](dfloat rl, dfloat bl, dfloat rr, dfloat br, dfloat &b, dfloat &q) {
        const dfloat inv = df_recip(df_add(rl, rr));
        b = df_mul(df_add(bl, br), inv);
        q = df_mul(ih2x, inv);
    };
    auto own = [&](int bc, dfloat r, dfloat be, dfloat &b, dfloat &q) {
        if (bc == MX_BC_DIRICHLET) {
            const dfloat inv = df_recip(r);
            b = df_mul(df_add(be, be), inv);
            q = df_mul(ih2x, inv);
        } else {
            b = zero;
            q = zero;
        }
    };
    long long c = act ? i + (long long)nx * (j + (long long)ny * k0) : 0;
    dfloat rc = zero, bc = zero, rdn = zero, bdn = zero;
    if (act) {
        rc = df_split(rho[c]);
        bc = df_split(beta0[c]);
        // the cell below the first one (its wrap image when periodic)
        if (k0 > 0 || gper(g, 2)) {
            const long long cd = k0 > 0 ? c - nxy : c + (long long)(nz - 1) * nxy;
            rdn = df_split(rho[cd]);
            bdn = df_split(beta0[cd]);
        }
    }
    int buf = 0;
    for (int k = k0; k < k1; k++, c += nxy, buf ^= 1) {
        sr[buf][ty][tx] = rc;
        sbt[buf][ty][tx] = bc;
        dfloat rw, bw;
        rw.h = __shfl_up_sync(0xffffffffu, rc.h, 1);
        rw.l = __shfl_up_sync(0xffffffffu, rc.l, 1);
        bw.h = __shfl_up_sync(0xffffffffu, bc.h, 1);
        bw.l = __shfl_up_sync(0xffffffffu, bc.l, 1);
        __syncthreads();
        if (act) {
            dfloat b, q;
            if (i > 0 || gper(g, 0)) {
                if (tx == 0) {
                    const long long cl = i > 0 ? c - 1 : c + nx - 1;
                    rw = df_split(rho[cl]);
                    bw = df_split(beta0[cl]);
                }
                face(rw, bw, rc, bc, b, q);
            } else {
                own(g.lo[0], rc, bc, b, q);
            }
            store(L.bx, D.bxl, Q.x, c, b, q);
            D.b0h[c] = bc.h;
            D.b0l[c] = bc.l;
            if (j > 0 || gper(g, 1)) {
                dfloat rs, bs;
                if (ty > 0) {
                    rs = sr[buf][ty - 1][tx];
                    bs = sbt[buf][ty - 1][tx];
                } else {
                    const long long cs = j > 0 ? c - nx : c + (long long)(ny - 1) * nx;
                    rs = df_split(rho[cs]);
                    bs = df_split(beta0[cs]);
                }
                face(rs, bs, rc, bc, b, q);
            } else {
                own(g.lo[1], rc, bc, b, q);
            }
            store(L.by, D.byl, Q.y, c, b, q);
            if (k > 0 || gper(g, 2)) face(rdn, bdn, rc, bc, b, q);
            else own(g.lo[2], rc, bc, b, q);
            store(L.bz, D.bzl, Q.z, c, b, q);
            if (i == nx - 1 && L.hx) {
                own(g.hi[0], rc, bc, b, q);
                store(L.hx, D.hxl, Q.hx, j + (long long)ny * k, b, q);
            }
            if (j == ny - 1 && L.hy) {
                own(g.hi[1], rc, bc, b, q);
                store(L.hy, D.hyl, Q.hy, i + (long long)nx * k, b, q);
            }
            if (k == nz - 1 && L.hz) {
                own(g.hi[2], rc, bc, b, q);
                store(L.hz, D.hzl, Q.hz, i + (long long)nx * j, b, q);
            }
            rdn = rc;
            bdn = bc;
            if (k + 1 < k1) {
                rc = df_split(rho[c + nxy]);
                bc = df_split(beta0[c + nxy]);
            }
        }
    }
}

void k_mac_coeffs_df(cudaStream_t s, const Level<float> &L0, const DFArrays &D, const double *rho,
                     const double *beta0, const FaceQ *q) {
    const double v = 2.0 / L0.g.h;
    dfloat ih2x;
    ih2x.h = float(v);
    ih2x.l = float(v - double(ih2x.h));
    mac_coeffs_df_kernel<<<stencil_grid(L0.g), dim3(SX, SY), 0, s>>>(L0, D, q ? *q : FaceQ{}, rho, beta0, ih2x);
}

// ---- RHS f = D(beta0 U) - beta0 Sbar in double-float ----------------------------
// The FP64 inputs U and Sbar are split into double-float (integer bit
// operations), beta0 comes split from the coefficient pass (b0h, b0l), the
// divergence is evaluated with double-float arithmetic on the FP32 pipe, and f
// is stored as a double-float pair (fh, fl); no FP64 arithmetic per cell.
// Face flux times 2: (beta0_L + beta0_R) U_f inside and across periodic faces,
// (beta0_in + beta0_in) U_f on a Dirichlet face, 0 on a wall (operands are
// selected, then one expression is evaluated); the factor 1/(2h) is applied
// once per cell.
// The cells of a thread's column, plane by plane.  Along x the warp's lanes
// are neighbouring cells: a cell's beta0 split goes to its +x neighbour by
// shuffle and its x-low face flux back as that neighbour's x-high flux, so
// every x face is evaluated once (lane 31, and the cell on the box's high x
// edge, evaluate their own high face).  The y faces are evaluated per cell,
// and the z-high flux with the split above carries to the next plane.  The
// arithmetic per face is the same wherever it is evaluated.  Every lane of a
// warp calls this (act = false outside the box): the shuffles take the warp.
template <typename F>
__device__ __forceinline__ void df_div_block(const DGeom &g, const double *__restrict__ ux,
                                             const double *__restrict__ uy, const double *__restrict__ uz,
                                             const float *__restrict__ b0h, const float *__restrict__ b0l,
                                             const double *__restrict__ sbar, int i, int j, int k0, int k1,
                                             dfloat hih, F fn) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long nxy = g.nxy;
    static_assert(SX == 32, "one warp per row of the block");
    const int lane = threadIdx.x;
    const bool act = i < nx && j < ny;
    const bool px = gper(g, 0), py = gper(g, 1), pz = gper(g, 2);
    const dfloat zero = {0.f, 0.f};
    auto B = [&](long long q) { return dfloat{b0h[q], b0l[q]}; };
    // twice the flux at face p of axis d from the split beta0 of its low (bl)
    // and high (bh) cells: the face mean inside and across periodic faces, the
    // interior cell's value on a Dirichlet face, 0 on a wall
    auto flux2 = [&](int d, int p, dfloat bl, dfloat bh, double u) -> dfloat {
        dfloat a = bl, b = bh;
        if (!((p > 0 && p < g.n[d]) || gper(g, d))) {
            const int bc = p == 0 ? g.lo[d] : g.hi[d];
            a = bc == MX_BC_DIRICHLET ? (p == 0 ? bh : bl) : zero;
            b = a;
        }
        return df_mul(df_add(a, b), df_split(u));
    };
    long long c = act ? i + (long long)nx * (j + (long long)ny * k0) : 0;
    dfloat bo = zero, fzl = zero;
    if (act) {
        bo = B(c);
        const dfloat bd = k0 > 0 ? B(c - nxy) : (pz ? B(c + (long long)(nz - 1) * nxy) : zero);
        fzl = flux2(2, k0, bd, bo, uz[c]);
    }
    for (int k = k0; k < k1; k++, c += nxy) {
        dfloat bw;
        bw.h = __shfl_up_sync(0xffffffffu, bo.h, 1);
        bw.l = __shfl_up_sync(0xffffffffu, bo.l, 1);
        const long long fx = i + (long long)(nx + 1) * (j + (long long)ny * k);
        dfloat fxl = zero;
        if (act) {
            if (lane == 0) bw = i > 0 ? B(c - 1) : (px ? B(c + nx - 1) : zero);
            fxl = flux2(0, i, bw, bo, ux[fx]);
        }
        dfloat fxh;
        fxh.h = __shfl_down_sync(0xffffffffu, fxl.h, 1);
        fxh.l = __shfl_down_sync(0xffffffffu, fxl.l, 1);
        if (act) {
            if (lane == SX - 1 || i + 1 >= nx) {
                const dfloat be = i + 1 < nx ? B(c + 1) : (px ? B(c - (nx - 1)) : zero);
                fxh = flux2(0, i + 1, bo, be, ux[fx + 1]);
            }
            const long long fy = i + (long long)nx * (j + (long long)(ny + 1) * k);
            const dfloat bs = j > 0 ? B(c - nx) : (py ? B(c + (long long)(ny - 1) * nx) : zero);
            const dfloat bn = j + 1 < ny ? B(c + nx)
                                         : (py ? B(c - (long long)(ny - 1) * nx) : zero);
            const dfloat fyl = flux2(1, j, bs, bo, uy[fy]);
            const dfloat fyh = flux2(1, j + 1, bo, bn, uy[fy + nx]);
            const dfloat bu = k + 1 < nz ? B(c + nxy)
                                         : (pz ? B(c - (long long)(nz - 1) * nxy) : zero);
            const dfloat fzh = flux2(2, k + 1, bo, bu, uz[c + nxy]);
            const dfloat div = df_add(df_add(df_sub(fxh, fxl), df_sub(fyh, fyl)), df_sub(fzh, fzl));
            fn(c, df_sub(df_mul(div, hih), df_mul(bo, df_split(sbar[c]))));
            fzl = fzh;
            bo = bu;
        }
    }
}

// per-block partials (max |x|, sum x^2, sum x) from per-thread double-float max
// and sum and a float sum of squares
__device__ __forceinline__ void df_partials(dfloat mx, float s2, dfloat s1, double *p) {
    double a = df_to_double(mx), b = s2, c = df_to_double(s1);
    block_red3(a, b, c);
    if (flat_tid() == 0) {
        p[0] = a;
        p[1] = b;
        p[2] = c;
    }
}

__global__ void __launch_bounds__(SX *SY, 5) mac_rhs_df_kernel(DGeom g, const double *__restrict__ ux, const double *__restrict__ uy,
                                  const double *__restrict__ uz, const float *__restrict__ b0h,
                                  const float *__restrict__ b0l, const double *__restrict__ sbar,
                                  float *__restrict__ fh, float *__restrict__ fl, double *part, dfloat hih) {
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    dfloat mx = {0.f, 0.f}, s1 = {0.f, 0.f};
    float s2 = 0.f;
    df_div_block(g, ux, uy, uz, b0h, b0l, sbar, i, j, k0, min(k0 + ZC, g.n[2]), hih, [&](long long c, dfloat v) {
            fh[c] = v.h;
            fl[c] = v.l;
            df_absmax(mx, v);
            s2 = fmaf(v.h, v.h, s2);
            s1 = df_add(s1, v);
        });
    df_partials(mx, s2, s1, part + 3 * flat_bid());
}

// max |D(beta0 U) - beta0 Sbar - c| of the projected velocity
__global__ void __launch_bounds__(SX *SY, 5) mac_divcheck_df_kernel(DGeom g, const double *__restrict__ ux, const double *__restrict__ uy,
                                       const double *__restrict__ uz, const float *__restrict__ b0h,
                                       const float *__restrict__ b0l, const double *__restrict__ sbar,
                                       const SolveState *st, double *part, dfloat hih) {
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    const dfloat cm = df_split(st->mean);
    dfloat mx = {0.f, 0.f};
    df_div_block(g, ux, uy, uz, b0h, b0l, sbar, i, j, k0, min(k0 + ZC, g.n[2]), hih,
                 [&](long long, dfloat v) { df_absmax(mx, df_sub(v, cm)); });
    df_partials(mx, 0.f, dfloat{0.f, 0.f}, part + 3 * flat_bid());
}

static dfloat df_const(double v) {
    dfloat r;
    r.h = float(v);
    r.l = float(v - double(r.h));
    return r;
}

void k_mac_rhs_df(cudaStream_t s, const DGeom &g, const double *ux, const double *uy, const double *uz,
                  const double *sbar, const DFArrays &D, double *partials) {
    mac_rhs_df_kernel<<<stencil_grid(g), dim3(SX, SY), 0, s>>>(g, ux, uy, uz, D.b0h, D.b0l, sbar, D.fh, D.fl,
                                                               partials, df_const(0.5 / g.h));
}

void k_mac_divcheck_df(cudaStream_t s, const DGeom &g, const double *ux, const double *uy, const double *uz,
                       const double *sbar, const DFArrays &D, const SolveState *st, double *partials) {
    mac_divcheck_df_kernel<<<stencil_grid(g), dim3(SX, SY), 0, s>>>(g, ux, uy, uz, D.b0h, D.b0l, sbar, st, partials,
                                                                    df_const(0.5 / g.h));
}

// ---- f <- f - mean, stored as h^2 f; norms of f - mean --------------------------------
__global__ void sub_mean_scale_kernel(long long n, const SolveState *st, dfloat h2, float *__restrict__ fh,
                                      float *__restrict__ fl, double *part) {
    const dfloat m = df_split(st->mean);
    dfloat mx = {0.f, 0.f}, s1 = {0.f, 0.f};
    float s2 = 0.f;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const dfloat v = df_sub(dfloat{fh[q], fl[q]}, m);
        const dfloat w = df_mul(v, h2);
        fh[q] = w.h;
        fl[q] = w.l;
        df_absmax(mx, v);
        s2 = fmaf(v.h, v.h, s2);
        s1 = df_add(s1, v);
    }
    df_partials(mx, s2, s1, part + 3 * blockIdx.x);
}

void k_sub_mean_scale(cudaStream_t s, const DGeom &g, const SolveState *st, const DFArrays &D, double *partials,
                      int nb) {
    sub_mean_scale_kernel<<<nb, RED_THREADS, 0, s>>>(g.N, st, df_const(g.h * g.h), D.fh, D.fl, partials);
}

// ---- phi conversions ----------------------------------------------------------------
__global__ void df_from_double_kernel(const double *__restrict__ x, float *__restrict__ hi, float *__restrict__ lo,
                                      long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        split_double(x[q], hi[q], lo[q]);
}
__global__ void df_to_double_kernel(const float *__restrict__ hi, const float *__restrict__ lo, double *__restrict__ x,
                                    long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        x[q] = double(hi[q]) + double(lo[q]);
}
void k_df_from_double(cudaStream_t s, long long n, const double *x, const DFArrays &D) {
    df_from_double_kernel<<<red_blocks(n), 256, 0, s>>>(x, D.ph, D.pl, n);
}
void k_df_to_double(cudaStream_t s, long long n, const DFArrays &D, double *x) {
    df_to_double_kernel<<<red_blocks(n), 256, 0, s>>>(D.ph, D.pl, x, n);
}

// ---- update phi += scale * e --------------------------------------------------------
__global__ void df_update_kernel(float *__restrict__ ph, float *__restrict__ pl, const float *__restrict__ e,
                                 const SolveState *st, long long n) {
    float sh, sl;
    split_double(st->scale, sh, sl);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const float ev = e[q];
        const float t = sh * ev;
        const float te = fmaf(sh, ev, -t) + sl * ev;
        float h, e1;
        two_sum(ph[q], t, h, e1);
        const float l = pl[q] + (te + e1);
        float nh, nl;
        two_sum(h, l, nh, nl);
        ph[q] = nh;
        pl[q] = nl;
    }
}

void k_df_update(cudaStream_t s, const DGeom &g, const DFArrays &D, const float *e, const SolveState *st) {
    df_update_kernel<<<red_blocks(g.N), 256, 0, s>>>(D.ph, D.pl, e, st, g.N);
}

// ---- residual r = f - L phi in double-float; rhat = r / scale (FP32) ---------------
// One flux term: acc += b * (p_nb - p_c), all in double-float.
__device__ __forceinline__ void df_term(float bh, float bl, float qh, float ql, float ch, float cl, float &Sh,
                                        float &Se) {
    float dh, de;
    two_sum(qh, -ch, dh, de);
    de += ql - cl;
    const float th = bh * dh;
    float te = fmaf(bh, dh, -th);
    te = fmaf(bh, de, te);
    te = fmaf(bl, dh, te);
    float s, e1;
    two_sum(Sh, th, s, e1);
    Sh = s;
    Se += e1 + te;
}

// phi += sc * e in double-float (sc = (sh, sl))
__device__ __forceinline__ void df_axpy(float &ph, float &pl, float sh, float sl, float ev) {
    const float t = sh * ev;
    const float te = fmaf(sh, ev, -t) + sl * ev;
    float h, e1;
    two_sum(ph, t, h, e1);
    const float l = pl + (te + e1);
    two_sum(h, l, ph, pl);
}

// Tile of the residual kernel: owned cells plus a 1-cell halo of phi in shared memory.
constexpr int DX = 32, DY = 8, DZ = 8;
constexpr int DHX = DX + 2, DHY = DY + 2, DHZ = DZ + 2;
constexpr int DF_THREADS = 256;

__device__ __forceinline__ int df_map(int u, int n, bool per) {
    if (u >= 0 && u < n) return u;
    if (!per || u < -1 || u > n) return -1;
    return u < 0 ? u + n : u - n;
}

// UPDATE: phi_new = phi_old + step * e is formed while staging (for the halo
// too, from the same inputs, so neighbouring tiles agree bit for bit), written
// to the other phi buffer, and the residual is taken of phi_new.  The two phi
// buffers alternate with the V-cycle count held on the device.
template <bool UPDATE>
__device__ __forceinline__ void df_resid_body(const Level<float> &L, const DFArrays &D, const float *__restrict__ e,
                                              const SolveState *st, float ih2, double *p, int bx, int by, int bz) {
    __shared__ float sh_[DHZ][DHY][DHX], sl_[DHZ][DHY][DHX];
    const DGeom &g = L.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const bool px = gper(g, 0), py = gper(g, 1), pz = gper(g, 2);
    const int x0 = bx * DX, y0 = by * DY, z0 = bz * DZ;
    const int tid = threadIdx.x;
    const int it = st->iter;
    const int src = UPDATE ? ((it - 1) & 1) : (it & 1), dst = it & 1;
    const float *__restrict__ sph = src ? D.ph2 : D.ph;
    const float *__restrict__ spl = src ? D.pl2 : D.pl;
    float *__restrict__ dph = dst ? D.ph2 : D.ph;
    float *__restrict__ dpl = dst ? D.pl2 : D.pl;
    float sch = 0.f, scl = 0.f;
    if (UPDATE) {
        sch = st->upd_h;
        scl = st->upd_l;
    }
    for (int q = tid; q < DHX * DHY * DHZ; q += DF_THREADS) {
        const int ax = q % DHX, ay = (q / DHX) % DHY, az = q / (DHX * DHY);
        const int lx = df_map(x0 - 1 + ax, nx, px), ly = df_map(y0 - 1 + ay, ny, py), lz = df_map(z0 - 1 + az, nz, pz);
        float h = 0.f, l = 0.f;
        if (lx >= 0 && ly >= 0 && lz >= 0) {
            const long long c = lx + (long long)nx * (ly + (long long)ny * lz);
            h = sph[c];
            l = spl[c];
            if (UPDATE) df_axpy(h, l, sch, scl, e[c]);
        }
        sh_[az][ay][ax] = h;
        sl_[az][ay][ax] = l;
    }
    __syncthreads();
    const float c_hat = ih2 * st->inv_scale_f;
    float mx = 0.f, s2f = 0.f, s1f = 0.f;
    for (int q = tid; q < DX * DY * DZ; q += DF_THREADS) {
        const int ix = q % DX, iy = (q / DX) % DY, iz = q / (DX * DY);
        const int i = x0 + ix, j = y0 + iy, k = z0 + iz;
        if (i >= nx || j >= ny || k >= nz) continue;
        const long long c = i + (long long)nx * (j + (long long)ny * k);
        const int ax = ix + 1, ay = iy + 1, az = iz + 1;
        const float ch = sh_[az][ay][ax], cl = sl_[az][ay][ax];
        if (UPDATE) {
            dph[c] = ch;
            dpl[c] = cl;
        }
        // high-side face coefficients: the neighbour's low face, or the boundary plane
        float beh, bel, bnh, bnl, bth, btl;
        if (i + 1 < nx) { beh = L.bx[c + 1]; bel = D.bxl[c + 1]; }
        else if (px) { beh = L.bx[c - (nx - 1)]; bel = D.bxl[c - (nx - 1)]; }
        else { const long long q2 = j + (long long)ny * k; beh = L.hx[q2]; bel = D.hxl[q2]; }
        if (j + 1 < ny) { bnh = L.by[c + nx]; bnl = D.byl[c + nx]; }
        else if (py) { const long long o = c - (long long)(ny - 1) * nx; bnh = L.by[o]; bnl = D.byl[o]; }
        else { const long long q2 = i + (long long)nx * k; bnh = L.hy[q2]; bnl = D.hyl[q2]; }
        if (k + 1 < nz) { bth = L.bz[c + g.nxy]; btl = D.bzl[c + g.nxy]; }
        else if (pz) { const long long o = c - (long long)(nz - 1) * g.nxy; bth = L.bz[o]; btl = D.bzl[o]; }
        else { const long long q2 = i + (long long)nx * j; bth = L.hz[q2]; btl = D.hzl[q2]; }
        float Sh = 0.f, Se = 0.f;
        df_term(L.bx[c], D.bxl[c], sh_[az][ay][ax - 1], sl_[az][ay][ax - 1], ch, cl, Sh, Se);
        df_term(beh, bel, sh_[az][ay][ax + 1], sl_[az][ay][ax + 1], ch, cl, Sh, Se);
        df_term(L.by[c], D.byl[c], sh_[az][ay - 1][ax], sl_[az][ay - 1][ax], ch, cl, Sh, Se);
        df_term(bnh, bnl, sh_[az][ay + 1][ax], sl_[az][ay + 1][ax], ch, cl, Sh, Se);
        df_term(L.bz[c], D.bzl[c], sh_[az - 1][ay][ax], sl_[az - 1][ay][ax], ch, cl, Sh, Se);
        df_term(bth, btl, sh_[az + 1][ay][ax], sl_[az + 1][ay][ax], ch, cl, Sh, Se);
        // R = h^2 f - S
        float Rh, Re;
        two_sum(D.fh[c], -Sh, Rh, Re);
        Re += D.fl[c] - Se;
        const float R = Rh + Re;
        const float rh = R * c_hat;  // r / scale: O(1), so its FP32 norms neither over- nor underflow
        L.f[c] = rh;
        mx = nmaxf(mx, fabsf(rh));
        s2f = fmaf(rh, rh, s2f);
        s1f += rh;
    }
    block_red3f(mx, s2f, s1f);
    if (tid == 0) {
        p[0] = double(mx);
        p[1] = double(s2f);
        p[2] = double(s1f);
    }
}

// e_odd (may be null): the update direction when the V-cycle count is odd
// (FCG keeps its two directions in alternating buffers)
template <bool UPDATE>
__global__ void __launch_bounds__(DF_THREADS)
    df_resid_tile_kernel(Level<float> L, DFArrays D, const float *__restrict__ e, const float *__restrict__ e_odd,
                         const SolveState *st, float ih2, double *part) {
    pdl_trigger();
    pdl_wait();
    const float *ee = (UPDATE && e_odd && (st->iter & 1)) ? e_odd : e;
    df_resid_body<UPDATE>(L, D, ee, st, ih2, part + 3 * flat_bid(), blockIdx.x, blockIdx.y, blockIdx.z);
}

// batched: work[blockIdx.x] = (box, bx, by, bz); the box's partials start at boxes[box].part_off
template <bool UPDATE>
__global__ void __launch_bounds__(DF_THREADS)
    df_resid_batch_kernel(const DFBox *boxes, const int4 *work, const SolveState *st, double *part) {
    const int4 w = work[blockIdx.x];
    if (st[w.x].done) return;
    const DFBox &B = boxes[w.x];
    const Level<float> L = B.L0;
    const DFArrays D = B.D;
    const DGeom &g = L.g;
    const int nbx = (g.n[0] + DX - 1) / DX, nby = (g.n[1] + DY - 1) / DY;
    double *p = part + 3 * ((long long)B.part_off + w.y + nbx * (w.z + nby * w.w));
    df_resid_body<UPDATE>(L, D, UPDATE ? L.e : nullptr, &st[w.x], float(1.0 / (g.h * g.h)), p, w.y, w.z, w.w);
}

// ---- the same residual as a z-march --------------------------------------------
// A block of 32 x 8 threads owns a 32 x 8 tile of cell columns over nzc planes.
// Step k (cell plane c0 + k) reads one "stage" (this block's slice of the
// inputs, copied global -> shared by cp.async into a ring of DM_NS slots, two
// stages ahead): the old phi (hi, lo) and e of plane c0 + k + 1 with a one-cell
// x-y halo (zero beyond a wall), the x and y face coefficients (hi, lo) of plane
// c0 + k with the tile's high faces, the low z faces of plane c0 + k (stage k + 1
// gives the high ones) and h^2 f.  phi_new = phi + step e is formed once per
// staged value (into one of two shared planes) and once more by each thread for
// its own column, so a column's z neighbours stay in registers.  The flux terms,
// their order and the update arithmetic are the tile kernel's: the results are
// the same bit for bit.  32-bit indices (N < 2^31, checked by the caller).
constexpr int DM_X = 32, DM_Y = 8, DM_T = DM_X * DM_Y;
constexpr int DM_HX = DM_X + 2, DM_HN = DM_HX * (DM_Y + 2);  // phi plane with halo
constexpr int DM_BXX = DM_X + 1, DM_BXN = DM_BXX * DM_Y;    // x faces (with the tile's high column)
constexpr int DM_BYN = DM_X * (DM_Y + 1);                   // y faces (with the tile's high row)
constexpr int DM_NS = 4;
static_assert(DM_HN <= 2 * DM_T && DM_BXN <= 2 * DM_T && DM_BYN <= 2 * DM_T, "two slots per thread");
// The wide variant (n_x a multiple of 4) stages whole rows in 16-byte chunks:
// the phi plane from x0 - 4 (pitch 40), the x faces from x0 (pitch 36).
constexpr int DW_PX = 40, DW_PN = DW_PX * (DM_Y + 2);
constexpr int DW_BXP = 36, DW_BXN = DW_BXP * DM_Y;
constexpr int DW_ITEMS = 100 + 72 + 72 + 64 + 64;  // chunk positions: phi, x faces, y faces, z faces, f
static_assert(DW_ITEMS <= 2 * DM_T, "two chunk items per thread");

struct DmStage {
    float ph[DW_PN], pl[DW_PN], pe[DW_PN];
    float bxh[DW_BXN], bxl[DW_BXN];
    float byh[DM_BYN], byl[DM_BYN];
    float bzh[DM_T], bzl[DM_T];
    float fh[DM_T], fl[DM_T];
};
static_assert(DW_PN >= DM_HN && DW_BXN >= DM_BXN && (DW_PN % 4) == 0 && (DW_BXN % 4) == 0 && (DM_BYN % 4) == 0,
              "both layouts fit; 16-byte aligned arrays");
struct DmShared {
    DmStage st[DM_NS];
    float ch[2][DW_PN], cl[2][DW_PN];  // phi_new of plane c0 + k (buffer k & 1)
};

static int df_march_zchunk(const DGeom &g) {
    const long long bxy = (long long)((g.n[0] + DM_X - 1) / DM_X) * ((g.n[1] + DM_Y - 1) / DM_Y);
    int zc = 64;
    while (zc > 4 && bxy * ((g.n[2] + zc - 1) / zc) < 4 * 3 * 152) zc >>= 1;
    return zc;
}
static dim3 df_march_grid(const DGeom &g) {
    const int zc = df_march_zchunk(g);
    return dim3((g.n[0] + DM_X - 1) / DM_X, (g.n[1] + DM_Y - 1) / DM_Y, (g.n[2] + zc - 1) / zc);
}
static bool df_march_ok(const DGeom &g) { return g.n[0] >= DM_X && g.N < (1LL << 31); }
static bool df_march_wide(const DGeom &g) { return g.n[0] % 4 == 0; }

// one block's march: tile (bx, by), z-chunk bz of nzc planes; partials to p
template <bool UPDATE, bool WIDE>
__device__ __forceinline__ void df_march_body(const Level<float> &L, const DFArrays &D, const float *__restrict__ e,
                                              const float *__restrict__ e_odd, const SolveState *st, float ih2,
                                              double *p, int bx, int by, int bz, int nzc) {
    extern __shared__ __align__(16) unsigned char dm_smem[];
    DmShared &sm = *reinterpret_cast<DmShared *>(dm_smem);
    const DGeom &g = L.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxy = nx * ny;
    const bool px = gper(g, 0), py = gper(g, 1), pz = gper(g, 2);
    const int tid = threadIdx.x, tx = tid % DM_X, ty = tid / DM_X;
    const int x0 = bx * DM_X, y0 = by * DM_Y;
    const int i = x0 + tx, j = y0 + ty;
    const bool own = i < nx && j < ny;
    const int c0 = bz * nzc, c1 = min(c0 + nzc, nz);
    const int nk = c1 - c0;
    const int it = st->iter;
    const int src = UPDATE ? ((it - 1) & 1) : (it & 1), dst = it & 1;
    const float *__restrict__ sph = src ? D.ph2 : D.ph;
    const float *__restrict__ spl = src ? D.pl2 : D.pl;
    float *__restrict__ dph = dst ? D.ph2 : D.ph;
    float *__restrict__ dpl = dst ? D.pl2 : D.pl;
    const float *__restrict__ ee = (UPDATE && e_odd && (it & 1)) ? e_odd : e;
    float sch = 0.f, scl = 0.f;
    if (UPDATE) {
        sch = st->upd_h;
        scl = st->upd_l;
    }
    // this thread's slots.  phi: in-plane offset (po, bit k of pmask: a cell
    // there).  x faces: kind 1 = bx at (offset, plane stride nxy), kind 2 = the
    // high plane hx at (offset, plane stride ny), 0 = no copy; y faces alike
    // (hy: plane stride nx).
    constexpr int PX = WIDE ? DW_PX : DM_HX, XO = WIDE ? 4 : 1, BXP = WIDE ? DW_BXP : DM_BXX;
    int po[2], xo[2], yo[2], pmask = 0, xk = 0, yk = 0;
    // wide: this thread's chunk items (wtyp: 0 phi, 1 x faces, 2 y faces, 3 z
    // faces, 4 f; wkind: 0 none (phi: zero fill), 1 main array, 2 high boundary
    // plane; wdst: float offset in the stage array; woff: in-plane offset)
    int wtyp[2] = {-1, -1}, wkind[2] = {0, 0}, wdst[2] = {0, 0}, woff[2] = {0, 0};
    for (int s = 0; s < 2 && WIDE; s++) {
        const int q = tid + s * DM_T;
        if (q >= DW_ITEMS) break;
        if (q < 100) {  // phi: 10 rows x 10 chunks from x0 - 4
            const int yy = q / 10, cc = q % 10, xs = x0 - 4 + 4 * cc;
            const int ly = df_map(y0 - 1 + yy, ny, py);
            const int lx = (xs >= 0 && xs + 4 <= nx) ? xs : (xs == -4 && px) ? nx - 4 : (xs == nx && px) ? 0 : -1;
            wtyp[s] = 0;
            wdst[s] = yy * DW_PX + 4 * cc;
            wkind[s] = (lx >= 0 && ly >= 0) ? 1 : 0;
            woff[s] = wkind[s] ? lx + nx * ly : 0;
        } else if (q < 172) {  // x faces: 8 rows x 9 chunks from x0
            const int r = q - 100, yy = r / 9, cc = r % 9, x = x0 + 4 * cc, y = y0 + yy;
            wtyp[s] = 1;
            wdst[s] = yy * DW_BXP + 4 * cc;
            if (y < ny && x + 4 <= nx) {
                wkind[s] = 1;
                woff[s] = x + nx * y;
            } else if (y < ny && x == nx) {
                wkind[s] = px ? 1 : 2;  // periodic: the row's first faces; else hx (one face)
                woff[s] = px ? nx * y : y;
            }
        } else if (q < 244) {  // y faces: 9 rows x 8 chunks
            const int r = q - 172, yy = r / 8, cc = r % 8, x = x0 + 4 * cc, y = y0 + yy;
            wtyp[s] = 2;
            wdst[s] = yy * DM_X + 4 * cc;
            if (x < nx && y < ny) {
                wkind[s] = 1;
                woff[s] = x + nx * y;
            } else if (x < nx && y == ny) {
                wkind[s] = py ? 1 : 2;
                woff[s] = x;
            }
        } else {  // z faces or f: 8 rows x 8 chunks of the tile
            const int r = q < 308 ? q - 244 : q - 308, yy = r / 8, cc = r % 8, x = x0 + 4 * cc, y = y0 + yy;
            wtyp[s] = q < 308 ? 3 : 4;
            wdst[s] = yy * DM_X + 4 * cc;
            wkind[s] = (x < nx && y < ny) ? 1 : 0;
            woff[s] = wkind[s] ? x + nx * y : 0;
        }
    }
    for (int s = 0; s < 2 && !WIDE; s++) {
        const int q = tid + s * DM_T;
        po[s] = xo[s] = yo[s] = 0;
        if (q < DM_HN) {
            const int lx = df_map(x0 - 1 + q % DM_HX, nx, px), ly = df_map(y0 - 1 + q / DM_HX, ny, py);
            if (lx >= 0 && ly >= 0) {
                po[s] = lx + nx * ly;
                pmask |= 1 << s;
            }
        }
        if (q < DM_BXN) {
            const int x = x0 + q % DM_BXX, y = y0 + q / DM_BXX;
            if (y < ny && x < nx) {
                xo[s] = x + nx * y;
                xk |= 1 << (2 * s);
            } else if (y < ny && x == nx) {
                if (px) {
                    xo[s] = nx * y;
                    xk |= 1 << (2 * s);
                } else {
                    xo[s] = y;
                    xk |= 2 << (2 * s);
                }
            }
        }
        if (q < DM_BYN) {
            const int x = x0 + q % DM_X, y = y0 + q / DM_X;
            if (x < nx && y < ny) {
                yo[s] = x + nx * y;
                yk |= 1 << (2 * s);
            } else if (x < nx && y == ny) {
                if (py) {
                    yo[s] = x;
                    yk |= 1 << (2 * s);
                } else {
                    yo[s] = x;
                    yk |= 2 << (2 * s);
                }
            }
        }
    }
    const bool slot1 = tid + DM_T < DM_HN, slot1x = tid + DM_T < DM_BXN, slot1y = tid + DM_T < DM_BYN;
    const int oc = own ? i + nx * j : 0;  // own column, in-plane
    // stage k: phi raw of plane c0 + k + 1 (k in [-2, nk - 1]); faces and f of
    // plane c0 + k (k in [0, nk - 1]); low z faces of plane c0 + k (k in [0, nk])
    auto issue_wide = [&](int k) {
        DmStage &S = sm.st[(k + 2) % DM_NS];
        const int c = c0 + k;
        for (int s = 0; s < 2; s++) {
            const int t = wtyp[s], kd = wkind[s], d = wdst[s], o = woff[s];
            if (t == 0) {
                if (k <= nk - 1) {
                    const int p = df_map(c0 + k + 1, nz, pz);
                    const int n = (p >= 0 && kd) ? 16 : 0;
                    const int base = (p >= 0 && kd) ? p * nxy + o : 0;
                    cp_async16(&S.ph[d], sph + base, n);
                    cp_async16(&S.pl[d], spl + base, n);
                    if (UPDATE) cp_async16(&S.pe[d], ee + base, n);
                }
            } else if (t == 1) {
                if (k >= 0 && k <= nk - 1 && kd == 1) {
                    cp_async16(&S.bxh[d], L.bx + c * nxy + o, 16);
                    cp_async16(&S.bxl[d], D.bxl + c * nxy + o, 16);
                } else if (k >= 0 && k <= nk - 1 && kd == 2) {
                    cp_async_el(&S.bxh[d], L.hx + c * ny + o, 4);
                    cp_async_el(&S.bxl[d], D.hxl + c * ny + o, 4);
                }
            } else if (t == 2) {
                if (k >= 0 && k <= nk - 1 && kd) {
                    const float *hh = kd == 1 ? L.by + c * nxy : L.hy + c * nx;
                    const float *hl = kd == 1 ? D.byl + c * nxy : D.hyl + c * nx;
                    cp_async16(&S.byh[d], hh + o, 16);
                    cp_async16(&S.byl[d], hl + o, 16);
                }
            } else if (t == 3) {
                if (k >= 0 && k <= nk && kd) {
                    const float *hh = c < nz ? L.bz + c * nxy : (pz ? L.bz : L.hz);
                    const float *hl = c < nz ? D.bzl + c * nxy : (pz ? D.bzl : D.hzl);
                    cp_async16(&S.bzh[d], hh + o, 16);
                    cp_async16(&S.bzl[d], hl + o, 16);
                }
            } else if (t == 4) {
                if (k >= 0 && k <= nk - 1 && kd) {
                    cp_async16(&S.fh[d], D.fh + c * nxy + o, 16);
                    cp_async16(&S.fl[d], D.fl + c * nxy + o, 16);
                }
            }
        }
        cp_async_commit();
    };
    auto issue = [&](int k) {
        if (WIDE) {
            issue_wide(k);
            return;
        }
        DmStage &S = sm.st[(k + 2) % DM_NS];
        if (k <= nk - 1) {
            const int p = df_map(c0 + k + 1, nz, pz);
            const int base = p >= 0 ? p * nxy : 0;
            const int m = p >= 0 ? pmask : 0;
            for (int s = 0; s < 2; s++) {
                if (s == 1 && !slot1) break;
                const int q = tid + s * DM_T, n = ((m >> s) & 1) ? 4 : 0;
                cp_async_el(&S.ph[q], sph + base + po[s], n);
                cp_async_el(&S.pl[q], spl + base + po[s], n);
                if (UPDATE) cp_async_el(&S.pe[q], ee + base + po[s], n);
            }
        }
        const int c = c0 + k;
        if (k >= 0 && k <= nk - 1) {
            for (int s = 0; s < 2; s++) {
                const int q = tid + s * DM_T;
                const int kx = (xk >> (2 * s)) & 3, ky = (yk >> (2 * s)) & 3;
                if (kx && (s == 0 || slot1x)) {
                    const float *hh = kx == 1 ? L.bx + c * nxy : L.hx + c * ny;
                    const float *hl = kx == 1 ? D.bxl + c * nxy : D.hxl + c * ny;
                    cp_async_el(&S.bxh[q], hh + xo[s], 4);
                    cp_async_el(&S.bxl[q], hl + xo[s], 4);
                }
                if (ky && (s == 0 || slot1y)) {
                    const float *hh = ky == 1 ? L.by + c * nxy : L.hy + c * nx;
                    const float *hl = ky == 1 ? D.byl + c * nxy : D.hyl + c * nx;
                    cp_async_el(&S.byh[q], hh + yo[s], 4);
                    cp_async_el(&S.byl[q], hl + yo[s], 4);
                }
            }
            if (own) {
                cp_async_el(&S.fh[tid], D.fh + c * nxy + oc, 4);
                cp_async_el(&S.fl[tid], D.fl + c * nxy + oc, 4);
            }
        }
        if (k >= 0 && k <= nk && own) {
            if (c < nz) {
                cp_async_el(&S.bzh[tid], L.bz + c * nxy + oc, 4);
                cp_async_el(&S.bzl[tid], D.bzl + c * nxy + oc, 4);
            } else if (pz) {  // the top face of the last plane: plane 0's low face
                cp_async_el(&S.bzh[tid], L.bz + oc, 4);
                cp_async_el(&S.bzl[tid], D.bzl + oc, 4);
            } else {          // or the high boundary plane
                cp_async_el(&S.bzh[tid], L.hz + oc, 4);
                cp_async_el(&S.bzl[tid], D.hzl + oc, 4);
            }
        }
        cp_async_commit();
    };
    auto newval = [&](const DmStage &S, int q, float &h, float &l) {
        h = S.ph[q];
        l = S.pl[q];
        if (UPDATE) df_axpy(h, l, sch, scl, S.pe[q]);
    };
    auto convert = [&](const DmStage &S, int b) {  // this thread's window slots of the stage's plane into buffer b
        for (int s = 0; s < 2; s++) {
            if (s == 1 && !slot1) break;
            const int q = tid + s * DM_T;                           // the 34 x 10 window around the tile
            const int w = (q / DM_HX) * PX + (q % DM_HX) + XO - 1;  // its place in the staged plane
            float h, l;
            newval(S, w, h, l);
            sm.ch[b][w] = h;
            sm.cl[b][w] = l;
        }
    };
    const int qo = (ty + 1) * PX + tx + XO;  // own column in the halo plane
    float pmh, pml, p0h, p0l;
    issue(-2);
    issue(-1);
    cp_async_wait<0>();
    __syncthreads();
    newval(sm.st[0], qo, pmh, pml);  // plane c0 - 1
    newval(sm.st[1], qo, p0h, p0l);  // plane c0
    if (UPDATE && own) {
        dph[c0 * nxy + oc] = p0h;
        dpl[c0 * nxy + oc] = p0l;
    }
    convert(sm.st[1], 0);
    __syncthreads();
    issue(0);
    issue(1);
    issue(2);
    const float c_hat = ih2 * st->inv_scale_f;
    float mx = 0.f, s2f = 0.f, s1f = 0.f;
    for (int k = 0; k < nk; k++) {
        cp_async_wait<1>();  // stages k and k + 1
        __syncthreads();
        const DmStage &S = sm.st[(k + 2) % DM_NS];
        const DmStage &S1 = sm.st[(k + 3) % DM_NS];
        float puh, pul;
        newval(S, qo, puh, pul);  // plane c0 + k + 1, own column
        const int c = c0 + k;
        if (UPDATE && own && c + 1 < c1) {
            dph[(c + 1) * nxy + oc] = puh;
            dpl[(c + 1) * nxy + oc] = pul;
        }
        if (k + 1 < nk) convert(S, (k + 1) & 1);
        if (own) {
            const float *h = sm.ch[k & 1], *l = sm.cl[k & 1];
            const int bxq = ty * BXP + tx, byq = ty * DM_X + tx;
            float Sh = 0.f, Se = 0.f;
            df_term(S.bxh[bxq], S.bxl[bxq], h[qo - 1], l[qo - 1], p0h, p0l, Sh, Se);
            df_term(S.bxh[bxq + 1], S.bxl[bxq + 1], h[qo + 1], l[qo + 1], p0h, p0l, Sh, Se);
            df_term(S.byh[byq], S.byl[byq], h[qo - PX], l[qo - PX], p0h, p0l, Sh, Se);
            df_term(S.byh[byq + DM_X], S.byl[byq + DM_X], h[qo + PX], l[qo + PX], p0h, p0l, Sh, Se);
            df_term(S.bzh[tid], S.bzl[tid], pmh, pml, p0h, p0l, Sh, Se);
            df_term(S1.bzh[tid], S1.bzl[tid], puh, pul, p0h, p0l, Sh, Se);
            float Rh, Re;
            two_sum(S.fh[tid], -Sh, Rh, Re);
            Re += S.fl[tid] - Se;
            const float R = Rh + Re;
            const float rh = R * c_hat;
            L.f[c * nxy + oc] = rh;
            mx = nmaxf(mx, fabsf(rh));
            s2f = fmaf(rh, rh, s2f);
            s1f += rh;
        }
        issue(k + 3);
        pmh = p0h;
        pml = p0l;
        p0h = puh;
        p0l = pul;
    }
    cp_async_wait<0>();
    block_red3f(mx, s2f, s1f);
    if (tid == 0) {
        p[0] = double(mx);
        p[1] = double(s2f);
        p[2] = double(s1f);
    }
}

template <bool UPDATE, bool WIDE>
__global__ void __launch_bounds__(DM_T, 3)
    df_march_kernel(Level<float> L, DFArrays D, const float *__restrict__ e, const float *__restrict__ e_odd,
                    const SolveState *st, float ih2, double *part, int nzc) {
    pdl_trigger();
    pdl_wait();
    df_march_body<UPDATE, WIDE>(L, D, e, e_odd, st, ih2, part + 3 * flat_bid(), blockIdx.x, blockIdx.y, blockIdx.z,
                                nzc);
}

// batched: work[blockIdx.x] = (box, bx, by, z-chunk) over each box's march grid;
// the box's partials start at boxes[box].part_off (block bx + nbx (by + nby bz))
template <bool UPDATE, bool WIDE>
__global__ void __launch_bounds__(DM_T, 3)
    df_march_batch_kernel(const DFBox *boxes, const int4 *work, const SolveState *st, double *part) {
    const int4 w = work[blockIdx.x];
    if (st[w.x].done) return;
    const DFBox &B = boxes[w.x];
    const Level<float> L = B.L0;
    const DFArrays D = B.D;
    const DGeom &g = L.g;
    const int nbx = (g.n[0] + DM_X - 1) / DM_X, nby = (g.n[1] + DM_Y - 1) / DM_Y;
    double *p = part + 3 * ((long long)B.part_off + w.y + nbx * (w.z + nby * w.w));
    df_march_body<UPDATE, WIDE>(L, D, UPDATE ? L.e : nullptr, nullptr, &st[w.x], float(1.0 / (g.h * g.h)), p, w.y, w.z,
                                w.w, B.zc);
}

dim3 df_resid_grid(const DGeom &g) {
    return dim3((g.n[0] + DX - 1) / DX, (g.n[1] + DY - 1) / DY, (g.n[2] + DZ - 1) / DZ);
}

int df_resid_blocks(const DGeom &g) {
    return ((g.n[0] + DX - 1) / DX) * ((g.n[1] + DY - 1) / DY) * ((g.n[2] + DZ - 1) / DZ);
}

void k_df_resid_batch(cudaStream_t s, const DFBox *boxes, const int4 *work, int nwork, const SolveState *st,
                      double *partials, int update, int march) {
    if (nwork <= 0) return;
    if (march) {
        const size_t smem = sizeof(DmShared);
        auto go = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<nwork, DM_T, smem, s>>>(boxes, work, st, partials);
        };
        if (march == 2) {
            if (update) go(df_march_batch_kernel<true, true>);
            else go(df_march_batch_kernel<false, true>);
        } else {
            if (update) go(df_march_batch_kernel<true, false>);
            else go(df_march_batch_kernel<false, false>);
        }
        return;
    }
    if (update) df_resid_batch_kernel<true><<<nwork, DF_THREADS, 0, s>>>(boxes, work, st, partials);
    else df_resid_batch_kernel<false><<<nwork, DF_THREADS, 0, s>>>(boxes, work, st, partials);
}

dim3 df_resid_batch_grid(const DGeom &g, int march, int *zc) {
    if (march) {
        // deep chunks: the blocks of all boxes fill the GPU together, so no box
        // needs to be cut finer (each chunk re-reads two halo planes)
        *zc = 64;
        return dim3((g.n[0] + DM_X - 1) / DM_X, (g.n[1] + DM_Y - 1) / DM_Y, (g.n[2] + 63) / 64);
    }
    *zc = 0;
    return df_resid_grid(g);
}
int df_march_usable(const DGeom &g) { return df_march_ok(g) ? (df_march_wide(g) ? 2 : 1) : 0; }

int k_df_resid(cudaStream_t s, const Level<float> &L0, const DFArrays &D, const float *e, const SolveState *st,
               double *partials, const float *e_odd) {
    const DGeom &g = L0.g;
    const float ih2 = float(1.0 / (g.h * g.h));
    if (df_march_ok(g)) {
        const dim3 grid = df_march_grid(g);
        const int zc = df_march_zchunk(g);
        const size_t smem = sizeof(DmShared);
        auto go = [&](auto kern, const float *ea, const float *eb) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            launch_pdl(kern, grid, dim3(DM_T), smem, s, L0, D, ea, eb, st, ih2, partials, zc);
        };
        const bool wide = df_march_wide(g);
        if (e) {
            if (wide) go(df_march_kernel<true, true>, e, e_odd);
            else go(df_march_kernel<true, false>, e, e_odd);
        } else {
            if (wide) go(df_march_kernel<false, true>, (const float *)nullptr, (const float *)nullptr);
            else go(df_march_kernel<false, false>, (const float *)nullptr, (const float *)nullptr);
        }
        return int(grid.x * grid.y * grid.z);
    }
    dim3 grid((g.n[0] + DX - 1) / DX, (g.n[1] + DY - 1) / DY, (g.n[2] + DZ - 1) / DZ);
    if (e) launch_pdl(df_resid_tile_kernel<true>, grid, dim3(DF_THREADS), 0, s, L0, D, e, e_odd, st, ih2, partials);
    else launch_pdl(df_resid_tile_kernel<false>, grid, dim3(DF_THREADS), 0, s, L0, D, (const float *)nullptr,
                    (const float *)nullptr, st, ih2, partials);
    return int(grid.x * grid.y * grid.z);
}

int df_resid_parts(const DGeom &g) {
    if (df_march_ok(g)) {
        const dim3 d = df_march_grid(g);
        return int(d.x * d.y * d.z);
    }
    return df_resid_blocks(g);
}

// The first residual of a solve from phi = 0 is f itself: rhat = (h^2 f) c_hat
// evaluated as the residual kernel would (every flux term is exactly 0 there),
// so the results are bit-identical without the stencil pass; partials on
// df_resid_blocks blocks like the residual kernel's.
__global__ void df_resid_zero_kernel(long long n, const float *__restrict__ fh, const float *__restrict__ fl,
                                     float *__restrict__ rhat, const SolveState *st, float ih2, double *part) {
    const float c_hat = ih2 * st->inv_scale_f;
    float mx = 0.f, s2f = 0.f, s1f = 0.f;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        float Rh, Re;
        two_sum(fh[q], -0.f, Rh, Re);
        Re += fl[q] - 0.f;
        const float rh = (Rh + Re) * c_hat;
        rhat[q] = rh;
        mx = nmaxf(mx, fabsf(rh));
        s2f = fmaf(rh, rh, s2f);
        s1f += rh;
    }
    block_red3f(mx, s2f, s1f);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = double(mx);
        part[3 * blockIdx.x + 1] = double(s2f);
        part[3 * blockIdx.x + 2] = double(s1f);
    }
}

// The same over the batched residual's work list: the entries of box b are the
// contiguous run starting at its part_off, so entry r of the run covers cells
// r * 256 + t, r * 256 + t + cnt[b] * 256, ... and writes partial part_off + r,
// the slot the stencil kernel's block of that entry writes.  It also sets the
// box's phi buffer 0 (the one the first update reads) to zero.
__global__ void __launch_bounds__(256) df_resid_zero_batch_kernel(const DFBox *boxes, const int4 *work,
                                                                  const int *cnt, const SolveState *st,
                                                                  double *part) {
    const int4 w = work[blockIdx.x];
    const DFBox &B = boxes[w.x];
    const DGeom &g = B.L0.g;
    const long long r = (long long)blockIdx.x - B.part_off, step = (long long)cnt[w.x] * 256;
    float *__restrict__ ph = B.D.ph, *__restrict__ pl = B.D.pl;
    if (st[w.x].done) {  // converged at the start (f = 0): phi = 0 only
        for (long long q = r * 256 + threadIdx.x; q < g.N; q += step) {
            ph[q] = 0.f;
            pl[q] = 0.f;
        }
        return;
    }
    const float *__restrict__ fh = B.D.fh, *__restrict__ fl = B.D.fl;
    float *__restrict__ rhat = B.L0.f;
    const float c_hat = float(1.0 / (g.h * g.h)) * st[w.x].inv_scale_f;
    float mx = 0.f, s2f = 0.f, s1f = 0.f;
    for (long long q = r * 256 + threadIdx.x; q < g.N; q += step) {
        float Rh, Re;
        two_sum(fh[q], -0.f, Rh, Re);
        Re += fl[q] - 0.f;
        const float rh = (Rh + Re) * c_hat;
        rhat[q] = rh;
        ph[q] = 0.f;
        pl[q] = 0.f;
        mx = nmaxf(mx, fabsf(rh));
        s2f = fmaf(rh, rh, s2f);
        s1f += rh;
    }
    block_red3f(mx, s2f, s1f);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = double(mx);
        part[3 * blockIdx.x + 1] = double(s2f);
        part[3 * blockIdx.x + 2] = double(s1f);
    }
}

void k_df_resid_zero_batch(cudaStream_t s, const DFBox *boxes, const int4 *work, int nwork, const int *cnt,
                           const SolveState *st, double *partials) {
    if (nwork > 0) df_resid_zero_batch_kernel<<<nwork, 256, 0, s>>>(boxes, work, cnt, st, partials);
}

void k_df_resid_zero(cudaStream_t s, const Level<float> &L0, const DFArrays &D, const SolveState *st, double *partials) {
    const DGeom &g = L0.g;
    df_resid_zero_kernel<<<df_resid_blocks(g), DF_THREADS, 0, s>>>(g.N, D.fh, D.fl, L0.f, st, float(1.0 / (g.h * g.h)),
                                                                  partials);
}

// final phi (double) from the current double-float buffer (selected by the
// V-cycle count), formed from the float bit patterns with one FP64 addition,
// with per-block partials (0, sum phi, 0) for the mean
__global__ void df_final_kernel(DFArrays D, const SolveState *st, double *__restrict__ x, long long n,
                                double *part) {
    const int b = st->iter & 1;
    const float *__restrict__ hi = b ? D.ph2 : D.ph;
    const float *__restrict__ lo = b ? D.pl2 : D.pl;
    dfloat s1 = {0.f, 0.f};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const dfloat v = {hi[q], lo[q]};
        x[q] = df_to_double(v);
        if (part) s1 = df_add(s1, v);
    }
    if (part) {
        double a = 0.0, sum = df_to_double(s1), c = 0.0;
        block_red3(a, sum, c);
        if (threadIdx.x == 0) {
            double *p = part + 3 * blockIdx.x;
            p[0] = a;
            p[1] = sum;
            p[2] = c;
        }
    }
}

void k_df_final(cudaStream_t s, long long n, const DFArrays &D, const SolveState *st, double *x, double *partials) {
    df_final_kernel<<<red_blocks(n), 256, 0, s>>>(D, st, x, n, partials);
}
