// Outer (iterative-refinement) loop of the mixed-precision MAC solve in
// double-float arithmetic: each double-precision quantity of the loop (phi, the
// right-hand side and the face coefficients) is held as an unevaluated sum of
// two floats hi + lo (|lo| <= ulp(hi)/2, about 48 significant bits), and the
// residual r = f - L phi and the update phi += s e are evaluated with the
// error-free transformations TwoSum (Knuth) and FMA-based TwoProd (Dekker).
// GB300 executes FP64 at 1/58 of its FP32 rate, so an FP64 residual is bound
// by the FP64 pipe while these kernels stay bound by memory bandwidth.
//
// Accuracy: the coefficients and RHS are the FP64 values rounded to 48 bits
// (relative 2^-48); the residual of the stored phi is computed with an error of
// a few 2^-48 relative to the largest flux term, far below the 1e-10 relative
// residual the loop converges to.
#include "mx_df.cuh"
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

// ---- coefficients: FP64 face values, stored as hi (the FP32 level-0 array) + lo
__device__ __forceinline__ double face_b(const double *beta0, const double *rho, long long cl, long long cr) {
    return (beta0[cl] + beta0[cr]) / (rho[cl] + rho[cr]);
}

__global__ void mac_coeffs_df_kernel(Level<float> L, DFArrays D, const double *__restrict__ rho,
                                     const double *__restrict__ beta0) {
    const DGeom &g = L.g;
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int k1 = min(k0 + ZC, nz);
    for (int k = k0; k < k1; k++) {
        const long long c = i + (long long)nx * (j + (long long)ny * k);
        const double own = 2.0 * (beta0[c] / rho[c]);  // a Dirichlet face's effective coefficient
        double bx, by, bz;
        if (i > 0) bx = face_b(beta0, rho, c - 1, c);
        else if (gper(g, 0)) bx = face_b(beta0, rho, c + nx - 1, c);
        else bx = g.lo[0] == MX_BC_DIRICHLET ? own : 0.0;
        if (j > 0) by = face_b(beta0, rho, c - nx, c);
        else if (gper(g, 1)) by = face_b(beta0, rho, c + (long long)(ny - 1) * nx, c);
        else by = g.lo[1] == MX_BC_DIRICHLET ? own : 0.0;
        if (k > 0) bz = face_b(beta0, rho, c - g.nxy, c);
        else if (gper(g, 2)) bz = face_b(beta0, rho, c + (long long)(nz - 1) * g.nxy, c);
        else bz = g.lo[2] == MX_BC_DIRICHLET ? own : 0.0;
        split_double(bx, L.bx[c], D.bxl[c]);
        split_double(by, L.by[c], D.byl[c]);
        split_double(bz, L.bz[c], D.bzl[c]);
        if (i == nx - 1 && L.hx) {
            const long long q = j + (long long)ny * k;
            split_double(g.hi[0] == MX_BC_DIRICHLET ? own : 0.0, L.hx[q], D.hxl[q]);
        }
        if (j == ny - 1 && L.hy) {
            const long long q = i + (long long)nx * k;
            split_double(g.hi[1] == MX_BC_DIRICHLET ? own : 0.0, L.hy[q], D.hyl[q]);
        }
        if (k == nz - 1 && L.hz) {
            const long long q = i + (long long)nx * j;
            split_double(g.hi[2] == MX_BC_DIRICHLET ? own : 0.0, L.hz[q], D.hzl[q]);
        }
    }
}

void k_mac_coeffs_df(cudaStream_t s, const Level<float> &L0, const DFArrays &D, const double *rho,
                     const double *beta0) {
    mac_coeffs_df_kernel<<<stencil_grid(L0.g), dim3(SX, SY), 0, s>>>(L0, D, rho, beta0);
}

// ---- RHS: f <- f - mean, stored as h^2 f in double-float; norms of f ------------
__global__ void sub_mean_split_kernel(const double *__restrict__ f, long long n, const SolveState *st, double h2,
                                      float *__restrict__ fh, float *__restrict__ fl, double *part) {
    const double m = st->mean;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const double v = f[q] - m;
        split_double(v * h2, fh[q], fl[q]);
        mx = fmax(mx, fabs(v));
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

void k_sub_mean_split(cudaStream_t s, const DGeom &g, const double *f, const SolveState *st, const DFArrays &D,
                      double *partials, int nb) {
    sub_mean_split_kernel<<<nb, RED_THREADS, 0, s>>>(f, g.N, st, g.h * g.h, D.fh, D.fl, partials);
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

__global__ void df_resid_kernel(Level<float> L, DFArrays D, const SolveState *st, float ih2, double *part) {
    const DGeom &g = L.g;
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    const float c_hat = float(double(ih2) * st->inv_scale);
    float mx = 0.f, s2f = 0.f, s1f = 0.f;
    if (i < g.n[0] && j < g.n[1]) {
        const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
        const int k1 = min(k0 + ZC, nz);
        for (int k = k0; k < k1; k++) {
            const long long c = i + (long long)nx * (j + (long long)ny * k);
            // neighbour indices (valid array positions; out-of-box neighbours read as 0)
            const bool hw = i > 0 || gper(g, 0), he = i + 1 < nx || gper(g, 0);
            const bool hs = j > 0 || gper(g, 1), hn = j + 1 < ny || gper(g, 1);
            const bool hb = k > 0 || gper(g, 2), ht = k + 1 < nz || gper(g, 2);
            const long long cw = i > 0 ? c - 1 : c + nx - 1, ce = i + 1 < nx ? c + 1 : c - (nx - 1);
            const long long cs = j > 0 ? c - nx : c + (long long)(ny - 1) * nx;
            const long long cn = j + 1 < ny ? c + nx : c - (long long)(ny - 1) * nx;
            const long long cb = k > 0 ? c - g.nxy : c + (long long)(nz - 1) * g.nxy;
            const long long ct = k + 1 < nz ? c + g.nxy : c - (long long)(nz - 1) * g.nxy;
            // high-side face coefficients: the neighbour's low face, or the boundary plane
            float beh, bel, bnh, bnl, bth, btl;
            if (i + 1 < nx || gper(g, 0)) { beh = L.bx[ce]; bel = D.bxl[ce]; }
            else { const long long q = j + (long long)ny * k; beh = L.hx[q]; bel = D.hxl[q]; }
            if (j + 1 < ny || gper(g, 1)) { bnh = L.by[cn]; bnl = D.byl[cn]; }
            else { const long long q = i + (long long)nx * k; bnh = L.hy[q]; bnl = D.hyl[q]; }
            if (k + 1 < nz || gper(g, 2)) { bth = L.bz[ct]; btl = D.bzl[ct]; }
            else { const long long q = i + (long long)nx * j; bth = L.hz[q]; btl = D.hzl[q]; }
            const float ch = D.ph[c], cl = D.pl[c];
            float Sh = 0.f, Se = 0.f;
            df_term(L.bx[c], D.bxl[c], hw ? D.ph[cw] : 0.f, hw ? D.pl[cw] : 0.f, ch, cl, Sh, Se);
            df_term(beh, bel, he ? D.ph[ce] : 0.f, he ? D.pl[ce] : 0.f, ch, cl, Sh, Se);
            df_term(L.by[c], D.byl[c], hs ? D.ph[cs] : 0.f, hs ? D.pl[cs] : 0.f, ch, cl, Sh, Se);
            df_term(bnh, bnl, hn ? D.ph[cn] : 0.f, hn ? D.pl[cn] : 0.f, ch, cl, Sh, Se);
            df_term(L.bz[c], D.bzl[c], hb ? D.ph[cb] : 0.f, hb ? D.pl[cb] : 0.f, ch, cl, Sh, Se);
            df_term(bth, btl, ht ? D.ph[ct] : 0.f, ht ? D.pl[ct] : 0.f, ch, cl, Sh, Se);
            // R = h^2 f - S
            float Rh, Re;
            two_sum(D.fh[c], -Sh, Rh, Re);
            Re += D.fl[c] - Se;
            const float R = Rh + Re;
            L.f[c] = R * c_hat;
            const float r = R * ih2;
            mx = fmaxf(mx, fabsf(r));
            s2f = fmaf(r, r, s2f);
            s1f += r;
        }
    }
    double dm = double(mx), s2 = double(s2f), s1 = double(s1f);
    block_red3(dm, s2, s1);
    if (flat_tid() == 0) {
        double *p = part + 3 * flat_bid();
        p[0] = dm;
        p[1] = s2;
        p[2] = s1;
    }
}

void k_df_resid(cudaStream_t s, const Level<float> &L0, const DFArrays &D, const SolveState *st, double *partials) {
    const float ih2 = float(1.0 / (L0.g.h * L0.g.h));
    df_resid_kernel<<<stencil_grid(L0.g), dim3(SX, SY), 0, s>>>(L0, D, st, ih2, partials);
}
