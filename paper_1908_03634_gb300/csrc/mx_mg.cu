// Cell-centred geometric multigrid kernels (MAC projection solve, Appendix A):
// red-black Gauss-Seidel, residual + 8-cell-average restriction,
// piecewise-constant prolongation, coefficient coarsening, a single-CTA
// BiCGStab bottom solve, and the FP64 residual / update of the refinement loop.
// Templated on the V-cycle precision T (float for the mixed-precision path,
// double for the plain FP64 path).
#include "mx_rbgs.cuh"
#include "mx_stencil.cuh"

// ------------------------------------------------------------------------------
// coefficients

template <typename T>
__global__ void coarsen_coeffs_kernel(Level<T> F, Level<T> Cl) {
    const long long C = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (C >= Cl.g.N) return;
    const int nxc = Cl.g.n[0], nyc = Cl.g.n[1];
    const int I = int(C % nxc), J = int((C / nxc) % nyc), K = int(C / ((long long)nxc * nyc));
    const int nxf = F.g.n[0], nyf = F.g.n[1];
    auto fc = [&](int i, int j, int k) { return (long long)i + (long long)nxf * ((long long)j + (long long)nyf * k); };
    const int i = 2 * I, j = 2 * J, k = 2 * K;
    Cl.bx[C] = T(0.25) * ((F.bx[fc(i, j, k)] + F.bx[fc(i, j + 1, k)]) + (F.bx[fc(i, j, k + 1)] + F.bx[fc(i, j + 1, k + 1)]));
    Cl.by[C] = T(0.25) * ((F.by[fc(i, j, k)] + F.by[fc(i + 1, j, k)]) + (F.by[fc(i, j, k + 1)] + F.by[fc(i + 1, j, k + 1)]));
    Cl.bz[C] = T(0.25) * ((F.bz[fc(i, j, k)] + F.bz[fc(i + 1, j, k)]) + (F.bz[fc(i, j + 1, k)] + F.bz[fc(i + 1, j + 1, k)]));
    if (I == 0 && Cl.hx) {  // high-x boundary plane, indexed (j, k)
        Cl.hx[J + (long long)nyc * K] = T(0.25) * ((F.hx[j + (long long)nyf * k] + F.hx[j + 1 + (long long)nyf * k]) +
                                                   (F.hx[j + (long long)nyf * (k + 1)] + F.hx[j + 1 + (long long)nyf * (k + 1)]));
    }
    if (J == 0 && Cl.hy) {  // high-y plane, indexed (i, k)
        Cl.hy[I + (long long)nxc * K] = T(0.25) * ((F.hy[i + (long long)nxf * k] + F.hy[i + 1 + (long long)nxf * k]) +
                                                   (F.hy[i + (long long)nxf * (k + 1)] + F.hy[i + 1 + (long long)nxf * (k + 1)]));
    }
    if (K == 0 && Cl.hz) {  // high-z plane, indexed (i, j)
        Cl.hz[I + (long long)nxc * J] = T(0.25) * ((F.hz[i + (long long)nxf * j] + F.hz[i + 1 + (long long)nxf * j]) +
                                                   (F.hz[i + (long long)nxf * (j + 1)] + F.hz[i + 1 + (long long)nxf * (j + 1)]));
    }
}

template <typename T>
void k_coarsen_coeffs(cudaStream_t s, const Level<T> &fine, const Level<T> &coarse) {
    const long long n = coarse.g.N;
    coarsen_coeffs_kernel<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(fine, coarse);
}

__global__ void round_coeffs_kernel(const double *a, float *b, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        b[q] = float(a[q]);
}

void k_round_coeffs(cudaStream_t s, const Level<double> &src, const Level<float> &dst) {
    const DGeom &g = src.g;
    const long long N = g.N;
    const int nb = red_blocks(N);
    round_coeffs_kernel<<<nb, 256, 0, s>>>(src.bx, dst.bx, N);
    round_coeffs_kernel<<<nb, 256, 0, s>>>(src.by, dst.by, N);
    round_coeffs_kernel<<<nb, 256, 0, s>>>(src.bz, dst.bz, N);
    if (src.hx) round_coeffs_kernel<<<64, 256, 0, s>>>(src.hx, dst.hx, (long long)g.n[1] * g.n[2]);
    if (src.hy) round_coeffs_kernel<<<64, 256, 0, s>>>(src.hy, dst.hy, (long long)g.n[0] * g.n[2]);
    if (src.hz) round_coeffs_kernel<<<64, 256, 0, s>>>(src.hz, dst.hz, (long long)g.n[0] * g.n[1]);
}

// ------------------------------------------------------------------------------
// FP64 residual of the refinement loop: r = f - L phi, handed to the correction
// solve as rhat = r / scale (in T), with block partials of max|r|, sum r^2, sum r.

template <typename T>
__global__ void residual64_kernel(Level<double> L, const double *__restrict__ phi, const double *__restrict__ f,
                                  T *__restrict__ rhat, const SolveState *st, double *part, double ih2) {
    const DGeom &g = L.g;
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    const double inv = st->inv_scale;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + ZC, g.n[2]);
        for (int k = k0; k < k1; k++) {
            const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
            double b[6], v[6];
            face_coefs(L, i, j, k, c, b);
            nb_vals(g, phi, i, j, k, c, v);
            const double r = f[c] - flux_sum(b, v, phi[c]) * ih2;
            rhat[c] = T(r * inv);
            mx = nmax(mx, fabs(r));
            s2 += r * r;
            s1 += r;
        }
    }
    block_red3(mx, s2, s1);
    if (flat_tid() == 0) {
        double *p = part + 3 * flat_bid();
        p[0] = mx;
        p[1] = s2;
        p[2] = s1;
    }
}

template <typename T>
void k_residual64(cudaStream_t s, const Level<double> &L64, const double *phi, const double *f, T *rhat,
                  const SolveState *st, double *partials, int nb) {
    (void)nb;
    const double ih2 = 1.0 / (L64.g.h * L64.g.h);
    residual64_kernel<T><<<stencil_grid(L64.g), dim3(SX, SY), 0, s>>>(L64, phi, f, rhat, st, partials, ih2);
}

// Convergence control of the refinement loop: one thread decides from the
// reduced norms (a = max, b = sum of squares, c = sum).
__device__ void decide(SolveState *st, double a, double b, double c) {
    st->rnorm = a;
    st->rnorm2 = sqrt(b);
    st->rsum = c;
    const int k = st->iter;
    const bool conv = a <= st->tol * st->fnorm;
    if (!isfinite(b) || !isfinite(a)) {
        st->status = MX_ERR_NOCONV;
        st->done = 1;
    } else if (conv) {
        st->status = MX_OK;
        st->done = 1;
    } else if (k >= st->maxit) {
        st->status = MX_ERR_NOCONV;
        st->done = 1;
    } else if (k > 3 && a > 1e3 * st->best) {
        st->status = MX_ERR_NOCONV;  // residual growth: divergence
        st->done = 1;
    } else {
        st->done = 0;
        st->iter = k + 1;
    }
    if (a < st->best) st->best = a;
}

__global__ void finalize_residual_kernel(const double *part, int nb, SolveState *st, int scaled) {
    pdl_trigger();
    pdl_wait();
    double a, b, c;
    reduce_partials3(part, nb, a, b, c);
    if (flat_tid() == 0) {
        if (scaled) {  // partials of r / scale
            const double sc = st->scale;
            a *= sc;
            b *= sc * sc;
            c *= sc;
        }
        decide(st, a, b, c);
    }
}

void k_finalize_residual(cudaStream_t s, const double *partials, int nb, SolveState *st, int scaled) {
    launch_pdl(finalize_residual_kernel, dim3(1), dim3(1024), 0, s, partials, nb, st, scaled);
}

// one block per box: partials [off[b], off[b] + cnt[b]) of r / scale; boxes
// already done skipped this residual and stay as they are
__global__ void finalize_residual_batch_kernel(const double *part, const int *off, const int *cnt, SolveState *st) {
    const int b = blockIdx.x;
    if (st[b].done) return;
    double a, s2, s1;
    reduce_partials3(part + 3 * (long long)off[b], cnt[b], a, s2, s1);
    if (threadIdx.x == 0) {
        const double sc = st[b].scale;
        decide(&st[b], a * sc, s2 * sc * sc, s1 * sc);
    }
}

void k_finalize_residual_batch(cudaStream_t s, const double *partials, const int *off, const int *cnt, SolveState *st,
                               int nbox) {
    finalize_residual_batch_kernel<<<nbox, 256, 0, s>>>(partials, off, cnt, st);
}

template <typename T>
__global__ void update_kernel(double *__restrict__ phi, const T *__restrict__ e, const SolveState *st, long long n) {
    const double sc = st->scale;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        phi[q] += sc * double(e[q]);
}

template <typename T>
void k_update(cudaStream_t s, const DGeom &g, double *phi, const T *e, const SolveState *st) {
    update_kernel<T><<<red_blocks(g.N), 256, 0, s>>>(phi, e, st, g.N);
}

// ------------------------------------------------------------------------------
// V-cycle kernels

// One colour of red-black Gauss-Seidel: cells with (i+j+k) % 2 == colour solve
// their row exactly with the other colour's current values.  zero = 1 (red
// pass of the first sweep from a zero initial guess): the black neighbours are
// taken as 0 without reading e.
template <typename T>
__device__ __forceinline__ void rbgs_body(const Level<T> &L, int colour, T h2, int zero, int bx, int by, int bz,
                                          int tx, int ty, int zc) {
    const DGeom &g = L.g;
    const int t = bx * SX + tx, j = by * SY + ty;
    const int k0 = bz * zc;
    if (j >= g.n[1]) return;
    const int k1 = min(k0 + zc, g.n[2]);
    for (int k = k0; k < k1; k++) {
        const int i = 2 * t + ((j + k + colour) & 1);
        if (i >= g.n[0]) continue;
        const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
        T b[6], v[6];
        face_coefs(L, i, j, k, c, b);
        if (zero) {
            for (int q = 0; q < 6; q++) v[q] = T(0);
        } else {
            nb_vals(g, L.e, i, j, k, c, v);
        }
        L.e[c] = gs_update(b, v, L.f[c], h2);
    }
}

// The black pass walks z downwards (blocks are dispatched in index order): it
// starts on the planes the red pass touched last, still in L2, and ends where the
// next red pass starts.  The cells of one colour update independently, so the
// order changes no result.
template <typename T>
__global__ void rbgs_kernel(Level<T> L, int colour, T h2, int zero, int zc) {
    pdl_trigger();
    pdl_wait();
    const int bz = colour ? gridDim.z - 1 - blockIdx.z : blockIdx.z;
    rbgs_body(L, colour, h2, zero, blockIdx.x, blockIdx.y, bz, threadIdx.x, threadIdx.y, zc);
}

dim3 rbgs_grid(const DGeom &g, int zc) {
    return dim3(((g.n[0] + 1) / 2 + SX - 1) / SX, (g.n[1] + SY - 1) / SY, (g.n[2] + zc - 1) / zc);
}
static int rbgs_zc(const DGeom &g, int cap) {
    return zchunk((long long)(((g.n[0] + 1) / 2 + SX - 1) / SX) * ((g.n[1] + SY - 1) / SY), g.n[2], cap);
}

// batched: work[blockIdx.x] = (box, bx, by, bz); level descriptors levs[box * MX_MAXLEV + level]
__global__ void rbgs_batch_kernel(const Level<float> *levs, const int4 *work, const SolveState *st, int level,
                                  int colour, int zero) {
    const int4 w = work[blockIdx.x];
    if (st[w.x].done) return;
    const Level<float> L = levs[w.x * MX_MAXLEV + level];
    rbgs_body(L, colour, float(L.g.h * L.g.h), zero, w.y, w.z, w.w, threadIdx.x, threadIdx.y, ZC);
}

void k_rbgs_batch(cudaStream_t s, const Level<float> *levs, const int4 *work, int nwork, const SolveState *st,
                  int level, int colour, int zero) {
    if (nwork > 0) rbgs_batch_kernel<<<nwork, dim3(SX, SY), 0, s>>>(levs, work, st, level, colour, zero);
}

template <typename T>
void k_rbgs(cudaStream_t s, const Level<T> &L, int colour, int zero, int zcap) {
    const DGeom &g = L.g;
    const int zc = rbgs_zc(g, zcap);
    launch_pdl(rbgs_kernel<T>, rbgs_grid(g, zc), dim3(SX, SY), 0, s, L, colour, T(g.h * g.h), zero, zc);
}

// Coarse RHS = average of the 8 fine residuals f - L e.
template <typename T>
__device__ __forceinline__ void resid_restrict_body(const Level<T> &F, const Level<T> &Cl, T ih2, int bx, int by,
                                                    int bz, int tx, int ty, int zc) {
    const DGeom &gc = Cl.g;
    const int I = bx * SX + tx, J = by * SY + ty;
    const int K0 = bz * zc;
    if (I >= gc.n[0] || J >= gc.n[1]) return;
    const DGeom &g = F.g;
    const int K1 = min(K0 + zc, gc.n[2]);
    for (int K = K0; K < K1; K++) {
        T s = T(0);
        for (int dk = 0; dk < 2; dk++)
            for (int dj = 0; dj < 2; dj++)
                for (int di = 0; di < 2; di++) {
                    const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                    const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
                    T b[6], v[6];
                    face_coefs(F, i, j, k, c, b);
                    nb_vals(g, F.e, i, j, k, c, v);
                    s += F.f[c] - flux_sum(b, v, F.e[c]) * ih2;
                }
        const long long C = I + (long long)gc.n[0] * (J + (long long)gc.n[1] * K);
        Cl.f[C] = s * T(0.125);
    }
}

// The same residual and restriction with one thread per fine cell column: a
// block of SX x SY threads covers a fine SX x SY tile (n_x and n_y even) and
// marches fine planes in pairs; each thread forms its cell's residual, and after
// each pair the thread at the even corner of each 2 x 2 x 2 group sums the eight
// values from shared memory in the order (dk, dj, di) of resid_restrict_body, so
// the coarse right-hand side is the same bit for bit.  Eight times as many
// threads as coarse cells: the load latency hides on the fine level, and the
// small levels fill the GPU.
template <typename T>
__device__ __forceinline__ void resid_restrict_fine_body(const Level<T> &F, const Level<T> &Cl, T ih2, int bx, int by,
                                                         int bz, int zcf) {
    __shared__ T sr[2][SY][SX];
    const DGeom &g = F.g, &gc = Cl.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = bx * SX + tx, j = by * SY + ty;
    const bool act = i < g.n[0] && j < g.n[1];
    const int k0 = bz * zcf, k1 = min(k0 + zcf, g.n[2]);  // k0 and zcf even
    for (int k = k0; k < k1; k++) {
        T r = T(0);
        if (act) {
            const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
            T b[6], v[6];
            face_coefs(F, i, j, k, c, b);
            nb_vals(g, F.e, i, j, k, c, v);
            r = F.f[c] - flux_sum(b, v, F.e[c]) * ih2;
        }
        sr[k & 1][ty][tx] = r;
        if (k & 1) {
            __syncthreads();
            if (act && !(tx & 1) && !(ty & 1)) {
                T sum = T(0);
                for (int dk = 0; dk < 2; dk++)
                    for (int dj = 0; dj < 2; dj++)
                        for (int di = 0; di < 2; di++) sum += sr[dk][ty + dj][tx + di];
                const int I = i >> 1, J = j >> 1, K = k >> 1;
                Cl.f[I + (long long)gc.n[0] * (J + (long long)gc.n[1] * K)] = sum * T(0.125);
            }
            __syncthreads();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(SX *SY) resid_restrict_fine_kernel(Level<T> F, Level<T> Cl, T ih2, int zcf) {
    pdl_trigger();
    pdl_wait();
    resid_restrict_fine_body(F, Cl, ih2, blockIdx.x, blockIdx.y, blockIdx.z, zcf);
}

template <typename T>
__global__ void resid_restrict_kernel(Level<T> F, Level<T> Cl, T ih2, int zc) {
    pdl_trigger();
    pdl_wait();
    resid_restrict_body(F, Cl, ih2, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, threadIdx.y, zc);
}

__global__ void resid_restrict_batch_kernel(const Level<float> *levs, const int4 *work, const SolveState *st,
                                            int level) {
    const int4 w = work[blockIdx.x];
    if (st[w.x].done) return;
    const Level<float> F = levs[w.x * MX_MAXLEV + level];
    const Level<float> C = levs[w.x * MX_MAXLEV + level + 1];
    resid_restrict_body(F, C, float(1.0 / (F.g.h * F.g.h)), w.y, w.z, w.w, threadIdx.x, threadIdx.y, ZC);
}

// the fine-cell form over a work list of fine tiles (every box's level has even extents)
__global__ void __launch_bounds__(SX *SY) resid_restrict_fine_batch_kernel(const Level<float> *levs, const int4 *work,
                                                                          const SolveState *st, int level, int zcf) {
    const int4 w = work[blockIdx.x];
    if (st[w.x].done) return;
    const Level<float> F = levs[w.x * MX_MAXLEV + level];
    const Level<float> C = levs[w.x * MX_MAXLEV + level + 1];
    resid_restrict_fine_body(F, C, float(1.0 / (F.g.h * F.g.h)), w.y, w.z, w.w, zcf);
}

dim3 resid_restrict_fine_grid(const DGeom &fine, int zcf) {
    return dim3((fine.n[0] + SX - 1) / SX, (fine.n[1] + SY - 1) / SY, (fine.n[2] + zcf - 1) / zcf);
}

void k_resid_restrict_batch(cudaStream_t s, const Level<float> *levs, const int4 *work, int nwork,
                            const SolveState *st, int level, int zcf) {
    if (nwork <= 0) return;
    if (zcf > 0)
        resid_restrict_fine_batch_kernel<<<nwork, dim3(SX, SY), 0, s>>>(levs, work, st, level, zcf);
    else
        resid_restrict_batch_kernel<<<nwork, dim3(SX, SY), 0, s>>>(levs, work, st, level);
}

template <typename T>
void k_resid_restrict(cudaStream_t s, const Level<T> &fine, const Level<T> &coarse, int zcap) {
    const double h = fine.g.h;
    const DGeom &g = fine.g;
    if (g.n[0] % 2 == 0 && g.n[1] % 2 == 0 && g.n[2] % 2 == 0) {
        // fine planes per block: even, halved until the grid fills the GPU a few times
        const long long bxy = (long long)((g.n[0] + SX - 1) / SX) * ((g.n[1] + SY - 1) / SY);
        int zcf = 16;
        while (zcf > 2 && bxy * ((g.n[2] + zcf - 1) / zcf) < 4 * 4 * 152) zcf >>= 1;
        const dim3 grid((g.n[0] + SX - 1) / SX, (g.n[1] + SY - 1) / SY, (g.n[2] + zcf - 1) / zcf);
        launch_pdl(resid_restrict_fine_kernel<T>, grid, dim3(SX, SY), 0, s, fine, coarse, T(1.0 / (h * h)), zcf);
        return;
    }
    const int zc = stencil_zc(coarse.g, zcap);
    launch_pdl(resid_restrict_kernel<T>, stencil_grid_zc(coarse.g, zc), dim3(SX, SY), 0, s, fine, coarse,
               T(1.0 / (h * h)), zc);
}

// e_fine += e_coarse(parent)
template <typename T>
__device__ __forceinline__ void prolong_body(const Level<T> &Cl, const Level<T> &F, int bx, int by, int bz, int tx,
                                             int ty, int zc) {
    const DGeom &g = F.g;
    const int i = bx * SX + tx, j = by * SY + ty;
    const int k0 = bz * zc;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int k1 = min(k0 + zc, g.n[2]);
    // four planes at a time: their loads are issued before any store (one plane
    // per iteration would make a chain of dependent round trips)
    for (int kb = k0; kb < k1; kb += 4) {
        T fe[4], ce[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int k = kb + q;
            if (k < k1) {
                const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
                const long long C = (i >> 1) + (long long)Cl.g.n[0] * ((j >> 1) + (long long)Cl.g.n[1] * (k >> 1));
                fe[q] = F.e[c];
                ce[q] = Cl.e[C];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int k = kb + q;
            if (k < k1) F.e[i + (long long)g.n[0] * (j + (long long)g.n[1] * k)] = fe[q] + ce[q];
        }
    }
}

template <typename T>
__global__ void prolong_kernel(Level<T> Cl, Level<T> F, int zc) {
    pdl_trigger();
    pdl_wait();
    prolong_body(Cl, F, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, threadIdx.y, zc);
}

__global__ void prolong_batch_kernel(const Level<float> *levs, const int4 *work, const SolveState *st, int level) {
    const int4 w = work[blockIdx.x];
    if (st[w.x].done) return;
    const Level<float> C = levs[w.x * MX_MAXLEV + level + 1];
    const Level<float> F = levs[w.x * MX_MAXLEV + level];
    prolong_body(C, F, w.y, w.z, w.w, threadIdx.x, threadIdx.y, ZC);
}

void k_prolong_batch(cudaStream_t s, const Level<float> *levs, const int4 *work, int nwork, const SolveState *st,
                     int level) {
    if (nwork > 0) prolong_batch_kernel<<<nwork, dim3(SX, SY), 0, s>>>(levs, work, st, level);
}

template <typename T>
void k_prolong(cudaStream_t s, const Level<T> &coarse, const Level<T> &fine, int zcap) {
    const int zc = stencil_zc(fine.g, zcap);
    launch_pdl(prolong_kernel<T>, stencil_grid_zc(fine.g, zc), dim3(SX, SY), 0, s, coarse, fine, zc);
}

// y = L x on a level (unscaled by nothing: true operator, 1/h^2 included)
template <typename T>
__global__ void apply_kernel(Level<T> L, const T *__restrict__ x, T *__restrict__ y, T ih2) {
    const DGeom &g = L.g;
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int k1 = min(k0 + ZC, g.n[2]);
    for (int k = k0; k < k1; k++) {
        const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
        T b[6], v[6];
        face_coefs(L, i, j, k, c, b);
        nb_vals(g, x, i, j, k, c, v);
        y[c] = flux_sum(b, v, x[c]) * ih2;
    }
}

template <typename T>
void k_apply(cudaStream_t s, const Level<T> &L, const T *phi, T *out) {
    const double h = L.g.h;
    apply_kernel<T><<<stencil_grid(L.g), dim3(SX, SY), 0, s>>>(L, phi, out, T(1.0 / (h * h)));
}

// ------------------------------------------------------------------------------
// Bottom solve: BiCGStab on the coarsest level, one CTA, fixed iteration cap.

constexpr int BOT_THREADS = 256;

template <typename T>
__device__ T bot_dot(const T *a, const T *b, int n) {
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += BOT_THREADS) s += double(a[q]) * double(b[q]);
    double m = 0.0, z = 0.0;
    block_red3(m, s, z);
    __shared__ double res;
    if (threadIdx.x == 0) res = s;
    __syncthreads();
    return T(res);
}

template <typename T>
__device__ void bot_apply(const Level<T> &L, const T *x, T *y, T ih2) {
    const DGeom &g = L.g;
    for (int c = threadIdx.x; c < g.N; c += BOT_THREADS) {
        const int i = c % g.n[0], j = (c / g.n[0]) % g.n[1], k = c / (g.n[0] * g.n[1]);
        T b[6], v[6];
        face_coefs(L, i, j, k, c, b);
        nb_vals(g, x, i, j, k, c, v);
        y[c] = flux_sum(b, v, x[c]) * ih2;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(BOT_THREADS) bottom_kernel(Level<T> L, T *scr, int iters, int singular, T ih2) {
    pdl_trigger();
    pdl_wait();
    const int n = int(L.g.N);
    T *x = L.e, *r = scr, *r0 = scr + n, *p = scr + 2 * n, *v = scr + 3 * n, *sv = scr + 4 * n, *tv = scr + 5 * n;
    T *bvec = scr + 6 * n;
    // right-hand side, projected onto mean-free vectors for singular problems
    T mean = T(0);
    if (singular) {
        double s = 0.0;
        for (int q = threadIdx.x; q < n; q += BOT_THREADS) s += double(L.f[q]);
        double m = 0.0, z = 0.0;
        block_red3(m, s, z);
        __shared__ double sm;
        if (threadIdx.x == 0) sm = s / n;
        __syncthreads();
        mean = T(sm);
    }
    for (int q = threadIdx.x; q < n; q += BOT_THREADS) {
        const T b = L.f[q] - mean;
        bvec[q] = b;
        x[q] = T(0);
        r[q] = b;
        r0[q] = b;
        p[q] = T(0);
        v[q] = T(0);
    }
    __syncthreads();
    const T bnorm2 = bot_dot(bvec, bvec, n);
    if (!(bnorm2 > T(0))) return;
    const T tol2 = bnorm2 * T(1e-8);  // 1e-4 relative: ample for a multigrid bottom solve
    T rho = T(1), alpha = T(1), omega = T(1);
    for (int it = 0; it < iters; it++) {
        const T rho1 = bot_dot(r0, r, n);
        if (rho1 == T(0) || omega == T(0)) break;
        const T beta = (rho1 / rho) * (alpha / omega);
        for (int q = threadIdx.x; q < n; q += BOT_THREADS) p[q] = r[q] + beta * (p[q] - omega * v[q]);
        __syncthreads();
        bot_apply(L, p, v, ih2);
        const T r0v = bot_dot(r0, v, n);
        if (r0v == T(0)) break;
        alpha = rho1 / r0v;
        for (int q = threadIdx.x; q < n; q += BOT_THREADS) sv[q] = r[q] - alpha * v[q];
        __syncthreads();
        const T ss = bot_dot(sv, sv, n);
        if (ss <= tol2) {
            for (int q = threadIdx.x; q < n; q += BOT_THREADS) x[q] += alpha * p[q];
            __syncthreads();
            break;
        }
        bot_apply(L, sv, tv, ih2);
        const T tt = bot_dot(tv, tv, n);
        const T ts = bot_dot(tv, sv, n);
        omega = tt > T(0) ? ts / tt : T(0);
        for (int q = threadIdx.x; q < n; q += BOT_THREADS) {
            x[q] += alpha * p[q] + omega * sv[q];
            r[q] = sv[q] - omega * tv[q];
        }
        __syncthreads();
        rho = rho1;
        const T rr = bot_dot(r, r, n);
        if (rr <= tol2) break;
    }
    if (singular) {
        double s = 0.0;
        for (int q = threadIdx.x; q < n; q += BOT_THREADS) s += double(x[q]);
        double m = 0.0, z = 0.0;
        block_red3(m, s, z);
        __shared__ double sm2;
        if (threadIdx.x == 0) sm2 = s / n;
        __syncthreads();
        const T mx = T(sm2);
        for (int q = threadIdx.x; q < n; q += BOT_THREADS) x[q] -= mx;
    }
}

template <typename T>
void k_bottom(cudaStream_t s, const Level<T> &L, T *scratch, int iters, int singular) {
    const double h = L.g.h;
    launch_pdl(bottom_kernel<T>, dim3(1), dim3(BOT_THREADS), 0, s, L, scratch, iters, singular, T(1.0 / (h * h)));
}

// ------------------------------------------------------------------------------
// small vector kernels

template <typename T>
__global__ void cast_kernel(const double *a, T *b, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        b[q] = T(a[q]);
}
template <typename T>
__global__ void uncast_kernel(const T *a, double *b, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        b[q] = double(a[q]);
}
template <typename T>
void k_cast(cudaStream_t s, long long n, const double *src, T *dst) {
    cast_kernel<T><<<red_blocks(n), 256, 0, s>>>(src, dst, n);
}
template <typename T>
void k_uncast(cudaStream_t s, long long n, const T *src, double *dst) {
    uncast_kernel<T><<<red_blocks(n), 256, 0, s>>>(src, dst, n);
}

__global__ void sum_partials_kernel(const double *x, long long n, double *part) {
    double s = 0.0, m = 0.0, z = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        s += x[q];
        m = nmax(m, fabs(x[q]));
    }
    block_red3(m, s, z);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = m;
        part[3 * blockIdx.x + 1] = s;
        part[3 * blockIdx.x + 2] = 0.0;
    }
}

void k_sum_partials(cudaStream_t s, const DGeom &g, const double *x, double *partials, int nb) {
    sum_partials_kernel<<<nb, RED_THREADS, 0, s>>>(x, g.N, partials);
}

// dst = scale * sum of the partial sums
__global__ void finalize_sum_kernel(const double *part, int nb, double *dst, double scale) {
    double a, b, c;
    reduce_partials3(part, nb, a, b, c);
    if (threadIdx.x == 0) *dst = b * scale;
}

void k_finalize_sum(cudaStream_t s, const double *partials, int nb, double *dst, double scale) {
    finalize_sum_kernel<<<1, 1024, 0, s>>>(partials, nb, dst, scale);
}

__global__ void sub_scalar_kernel(double *x, long long n, const double *val) {
    const double v = *val;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        x[q] -= v;
}

void k_sub_scalar(cudaStream_t s, long long n, double *x, const double *val) {
    sub_scalar_kernel<<<red_blocks(n), 256, 0, s>>>(x, n, val);
}

// plain FP64 residual r = f - L phi with norm partials (the mx_residual entry point)
__global__ void residual_plain_kernel(Level<double> L, const double *__restrict__ phi, const double *__restrict__ f,
                                      double *__restrict__ r, double *part, double ih2) {
    const DGeom &g = L.g;
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y;
    const int k0 = blockIdx.z * ZC;
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + ZC, g.n[2]);
        for (int k = k0; k < k1; k++) {
            const long long c = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
            double b[6], v[6];
            face_coefs(L, i, j, k, c, b);
            nb_vals(g, phi, i, j, k, c, v);
            const double rr = f[c] - flux_sum(b, v, phi[c]) * ih2;
            r[c] = rr;
            mx = nmax(mx, fabs(rr));
            s2 += rr * rr;
            s1 += rr;
        }
    }
    block_red3(mx, s2, s1);
    if (flat_tid() == 0) {
        double *p = part + 3 * flat_bid();
        p[0] = mx;
        p[1] = s2;
        p[2] = s1;
    }
}

void k_residual_plain(cudaStream_t s, const Level<double> &L, const double *phi, const double *f, double *r,
                      double *partials, int nb) {
    (void)nb;
    residual_plain_kernel<<<stencil_grid(L.g), dim3(SX, SY), 0, s>>>(L, phi, f, r, partials, 1.0 / (L.g.h * L.g.h));
}

// ------------------------------------------------------------------------------
// explicit instantiations
#define MX_INST(T)                                                                                               \
    template void k_coarsen_coeffs<T>(cudaStream_t, const Level<T> &, const Level<T> &);                        \
    template void k_residual64<T>(cudaStream_t, const Level<double> &, const double *, const double *, T *,      \
                                  const SolveState *, double *, int);                                            \
    template void k_update<T>(cudaStream_t, const DGeom &, double *, const T *, const SolveState *);            \
    template void k_rbgs<T>(cudaStream_t, const Level<T> &, int, int, int);                                      \
    template void k_resid_restrict<T>(cudaStream_t, const Level<T> &, const Level<T> &, int);                  \
    template void k_prolong<T>(cudaStream_t, const Level<T> &, const Level<T> &, int);                         \
    template void k_bottom<T>(cudaStream_t, const Level<T> &, T *, int, int);                                   \
    template void k_apply<T>(cudaStream_t, const Level<T> &, const T *, T *);                                   \
    template void k_cast<T>(cudaStream_t, long long, const double *, T *);                                       \
    template void k_uncast<T>(cudaStream_t, long long, const T *, double *);
MX_INST(float)
MX_INST(double)
