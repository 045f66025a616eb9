// Base-state mapping (Sec. 3.1): the lateral Average of a cell field onto the
// one-dimensional base state and the Fill of a base state onto the cells.
//
// Planar: the base state is aligned with the cell heights; Average is the
// arithmetic mean of each z plane (Fill is injection, mx_fill_base_state).
//
// Spherical, with the centre of the star on the cell corner c: the centre of
// cell (i, j, k) lies at (a + 1/2, b + 1/2, e + 1/2) dx from it, a = i - c0,
// b = j - c1, e = k - c2, so its radius is dx sqrt(0.75 + 2m) with
// m = T(a) + T(b) + T(e), T(a) = a (a + 1) / 2 (Eq. radii).  The irregular base
// state holds the mean over the cells of each m; its Fill reads bin m of every
// cell.  The uniform base state (radial cells (j + 1/2) dr) is filled by
// quadratic interpolation in r: all cells of a bin share their radius, so the
// interpolant is evaluated once per bin and gathered.  The Average onto the
// uniform base state interpolates the bin means quadratically.
//
// The radial Average runs without atomics, in a fixed order (deterministic):
//   1. fold: the rows (j, k) with equal s = T(b) + T(e) form a group; each CTA
//      sums the rows of its groups column by column (one pass over the field,
//      whole rows, coalesced) and folds the mirror columns a and -1 - a (equal
//      T) together into G[group][t], t = (a >= 0 ? a : -1 - a);
//   2. bins: bin m = s + T(t) sums G[group(s)][t] over t, one lane per bin.
// Sums are double-float on the FP32 pipe (GB300 runs FP64 at 1/58 of FP32); the
// fold adds row pairs in FP64 first, which moves about a third of the work to
// the otherwise idle FP64 pipe.  The fast passes keep their sums as float pairs
// and accept magnitudes 2^-73..2^97; a value outside raises a flag, and
// full-range passes (launched after them, returning at once otherwise) redo the
// Average with scaled double-float accumulators, FP64 for outliers, and doubles
// for the staged sums.  The planar Average works the same way.
#include <algorithm>
#include <cmath>

#include "mx_dfmath.cuh"
#include "mx_internal.cuh"

namespace {

constexpr int FOLD_THREADS = 256;
constexpr int BIN_THREADS = 256;
constexpr int MAX_RADIAL_PLANS = 4;

__host__ __device__ __forceinline__ long long tri(long long t) { return t * (t + 1) / 2; }

// t range of T(a) over a in [lo, hi]: t = a for a >= 0, -1 - a for a < 0
void t_range(long long lo, long long hi, long long &tmin, long long &tmax) {
    if (lo >= 0) {
        tmin = lo;
        tmax = hi;
    } else if (hi < 0) {
        tmin = -1 - hi;
        tmax = -1 - lo;
    } else {
        tmin = 0;
        tmax = std::max(hi, -1 - lo);
    }
}

}  // namespace

struct RadialPlan {
    int n[3], c[3];
    long long nbins, smin, smax, nne;
    int kmin, kmax, wt;  // column index t in [kmin, kmax], wt = kmax - kmin + 1
    int ngroups, nbatch, nrows;
    int *rows;           // row ids j + ny k, ordered by s
    int *gstart;         // first row of each group (ngroups + 1)
    int *grp;            // group of s (index s - smin), -1 where no row has that s
    int *bstart;         // first group of each fold batch (nbatch + 1)
    long long *count;    // cells per bin
    long long *gsv;      // s of each group
    int *nonempty;       // bins with cells, increasing
    double *G;           // folded column sums, t-major: G[t * ngroups + g]
    int gmax;            // most groups in one fold batch
    double *tab;         // per-bin values of the uniform fill
    double *avg_tmp;     // per-bin means (scratch of the velocity-split bracket)
    void *mem;
    long long last_use;
};

struct RadDev {
    int nx, ny, c0, c1, c2, kmin, kmax, wt, ngroups, gmax;
    long long nbins, smin, smax;
    const int *rows, *gstart, *grp, *bstart;
    const long long *count;
};

static RadDev rad_dev(const RadialPlan *p) {
    RadDev d;
    d.nx = p->n[0];
    d.ny = p->n[1];
    d.c0 = p->c[0];
    d.c1 = p->c[1];
    d.c2 = p->c[2];
    d.kmin = p->kmin;
    d.kmax = p->kmax;
    d.wt = p->wt;
    d.ngroups = p->ngroups;
    d.gmax = p->gmax;
    d.nbins = p->nbins;
    d.smin = p->smin;
    d.smax = p->smax;
    d.rows = p->rows;
    d.gstart = p->gstart;
    d.grp = p->grp;
    d.bstart = p->bstart;
    d.count = p->count;
    return d;
}

// ---------------------------------------------------------------------------------------
// kernels

// Double-float accumulator with deferred renormalisation: TwoSum of the high
// parts, the low parts and the TwoSum error gathered in l (tens of terms per
// accumulator, each below 2^-24 of the running sum, so l stays exact to about
// 2^-48 of it); norm() renormalises once at the end.
struct DfAcc {
    float h = 0.f, l = 0.f;
    __device__ __forceinline__ void add(dfloat x) {
        const float s = h + x.h;
        const float bb = s - h;
        l += ((h - (s - bb)) + (x.h - bb)) + x.l;
        h = s;
    }
    __device__ __forceinline__ dfloat norm() const { return df_norm(h, l); }
};


// Sums over the whole double range: a double-float accumulator on the FP32 pipe
// that holds the values scaled by 2^shift, the shift fixed by the first value
// (which lands at 2^0; the values of one accumulator, one column of a row group or
// one bin, share their radius and usually their magnitude).  Values within
// 2^-73..2^77 of the scale go through the double-float lane (its sums keep 2^50 of
// headroom below the FP32 range); others, subnormals and non-finite values are
// added in FP64, out of line.  Zeros are skipped.  Fields such as mass fractions
// (1e-30) or energies (1e50) stay on the fast lane.
static __device__ __noinline__ double wide_add(double a, double v) { return a + v; }
static __device__ __noinline__ double wide_total(double t, double x) { return t + x; }
struct WideAcc {
    DfAcc a;
    double x = 0.0;
    int shift = 1 << 20;  // unset
    __device__ __forceinline__ void add(double v) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        const unsigned E = (unsigned)(b >> 52) & 0x7ffu;
        if ((b << 1) == 0ull) return;
        if (shift == (1 << 20)) shift = (E == 0u || E == 0x7ffu) ? 0 : 1023 - (int)E;
        const unsigned Es = (unsigned)((int)E + shift);
        if (Es - 950u < 150u && E - 1u < 0x7feu) a.add(df_split_bits(b, Es));
        else x = wide_add(x, v);
    }
    __device__ __forceinline__ double total() const {
        double t = 0.0;
        if (shift != (1 << 20)) {  // 2^-shift (the first value's exponent), exact
            const double scale = __longlong_as_double((long long)(unsigned long long)(1023 - shift) << 52);
            t = df_to_double(a.norm()) * scale;
        }
        return x != 0.0 ? wide_total(t, x) : t;
    }
};

// df_split for the fast passes: magnitudes 2^-73..2^97 (sums of up to 2^27 of them
// stay below 2^124, inside the FP32 range of the pair's high part); zero gives
// (0, 0); any other value contributes nothing here and raises *wide (the
// full-range passes then redo the sum): once per thread (the flag `seen`), one
// atomic per warp, out of line (kept out of line, the common path compiles to a
// tighter loop).
static __device__ __noinline__ void mark_wide(int *wide) {
    const unsigned m = __activemask();
    if ((threadIdx.x & 31u) == (unsigned)(__ffs(m) - 1)) atomicOr(wide, 1);
}
__device__ __forceinline__ dfloat df_split_mark(double x, bool &seen, int *wide) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned E = (unsigned)(b >> 52) & 0x7ffu;
    if (E - 950u < 170u) return df_split_bits(b, E);
    if ((b << 1) != 0ull && !seen) {
        seen = true;
        mark_wide(wide);
    }
    return dfloat{0.f, 0.f};
}

// The same with the shift fixed in advance (uniform over a CTA): no per-value
// initialisation.  shift = 1023 - E0 puts values of exponent E0 at 2^0.
struct FixedWideAcc {
    DfAcc a;
    double x = 0.0;
    __device__ __forceinline__ void add(double v, int shift) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        const unsigned E = (unsigned)(b >> 52) & 0x7ffu;
        const unsigned Es = (unsigned)((int)E + shift);
        if (Es - 950u < 150u && E - 1u < 0x7feu) a.add(df_split_bits(b, Es));
        else if ((b << 1) != 0ull) x = wide_add(x, v);
    }
    __device__ __forceinline__ double total(int shift) const {
        const double scale = __longlong_as_double((long long)(unsigned long long)(1023 - shift) << 52);
        const double t = df_to_double(a.norm()) * scale;
        return x != 0.0 ? wide_total(t, x) : t;
    }
};

// shift placing the exponent of v at 2^0 (0 for zero, subnormal or non-finite v)
__device__ __forceinline__ int scale_shift(double v) {
    const unsigned E = (unsigned)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ffu;
    return (E == 0u || E == 0x7ffu) ? 0 : 1023 - (int)E;
}

// 1. fold, fast pass (magnitudes 2^-73..2^97; any other value raises *wide and
// the full-range pass below redoes the Average).  One CTA per batch of whole
// groups (at most gmax of them).  Each thread owns a column (V = 2: a column
// pair, 16-byte loads; n0 even, so every row starts on a 16-byte boundary) and
// walks all rows of the batch in rounds of 8 loads, across group boundaries (16
// loads in flight per thread, no barrier between groups).  At a group's last row
// the column sum goes to racc[group][column].  After one barrier the mirror
// columns a and -1 - a fold together and G is written t-major (G[t][g], runs of
// the batch's consecutive groups).
template <int V>
__global__ void __launch_bounds__(FOLD_THREADS, 4) rad_fold_kernel(const double *__restrict__ f, RadDev P,
                                                                   float2 *__restrict__ GT, int *__restrict__ wide) {
    extern __shared__ float2 racc[];
    bool seen = false;
    const int g0 = P.bstart[blockIdx.x], g1 = P.bstart[blockIdx.x + 1];
    const int R0 = P.gstart[g0], R1 = P.gstart[g1];
    const int nx = P.nx, nv = nx / V, wt = P.wt;
    for (int q = threadIdx.x; q < nv; q += blockDim.x) {
        DfAcc acc[V];
        int cur = g0, gend = P.gstart[g0 + 1];
        auto flush = [&]() {
#pragma unroll
            for (int w = 0; w < V; w++) {
                const dfloat a = acc[w].norm();
                racc[(long long)(cur - g0) * nx + q * V + w] = make_float2(a.h, a.l);
                acc[w] = DfAcc();
            }
            cur++;
            if (cur < g1) gend = P.gstart[cur + 1];
        };
        for (int r = R0; r < R1; r += 8) {
            double v[8][V];
#pragma unroll
            for (int u = 0; u < 8; u++) {
#pragma unroll
                for (int w = 0; w < V; w++) v[u][w] = 0.0;
                if (r + u < R1) {  // uniform over the CTA
                    const double *src = f + (long long)P.rows[r + u] * nx + (long long)q * V;
                    if constexpr (V == 2) {
                        const double2 t = __ldcs(reinterpret_cast<const double2 *>(src));
                        v[u][0] = t.x;
                        v[u][V - 1] = t.y;
                    } else {
                        v[u][0] = __ldcs(src);
                    }
                }
            }
            // rows of the same group add in FP64 pairs before the double-float
            // accumulation (moves about a third of the work to the FP64 pipe,
            // which the double-float operations leave idle); group boundaries are
            // uniform over the CTA, so are these branches
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                const int ra = r + u, rb = ra + 1;
                if (ra < R1) {
                    if (rb < gend) {  // both rows in the current group
#pragma unroll
                        for (int w = 0; w < V; w++) acc[w].add(df_split_mark(v[u][w] + v[u + 1][w], seen, wide));
                        if (rb + 1 == gend) flush();
                    } else {  // ra ends the group
#pragma unroll
                        for (int w = 0; w < V; w++) acc[w].add(df_split_mark(v[u][w], seen, wide));
                        flush();
                        if (rb < R1) {
#pragma unroll
                            for (int w = 0; w < V; w++) acc[w].add(df_split_mark(v[u + 1][w], seen, wide));
                            if (rb + 1 == gend) flush();
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    const int ng = g1 - g0;
    for (int e = threadIdx.x; e < ng * wt; e += blockDim.x) {
        const int t = e / ng, j = e - t * ng;
        const int k = P.kmin + t;
        const int i1 = P.c0 + k, i2 = P.c0 - 1 - k;  // a = k and a = -1 - k
        const float2 *ra = racc + (long long)j * nx;
        dfloat v{0.f, 0.f};
        if (i1 >= 0 && i1 < nx) v = dfloat{ra[i1].x, ra[i1].y};
        if (i2 >= 0 && i2 < nx) v = df_add(v, dfloat{ra[i2].x, ra[i2].y});
        GT[(long long)t * P.ngroups + g0 + j] = make_float2(v.h, v.l);
    }
}

// 1'. fold, full-range pass (returns at once unless the fast pass met a value
// outside its window): the fast fold's structure, with an accumulator scaled by
// a power of two fixed per CTA (FP64 for values far from it) and doubles for
// the column sums and G.
template <int V>
__global__ void __launch_bounds__(FOLD_THREADS, 4) rad_fold_wide_kernel(const double *__restrict__ f, RadDev P,
                                                                        double *__restrict__ GT,
                                                                        const int *__restrict__ wide) {
    if (*wide == 0) return;  // the fast pass covered every value
    extern __shared__ double raccw[];
    double *racc = raccw;
    const int g0 = P.bstart[blockIdx.x], g1 = P.bstart[blockIdx.x + 1];
    const int R0 = P.gstart[g0], R1 = P.gstart[g1];
    const int nx = P.nx, nv = nx / V, wt = P.wt;
    // the CTA's scale: the largest magnitude in the middle of its first row (one
    // warp's reduction, uniform over the CTA)
    __shared__ int s_shift;
    if (threadIdx.x < 32) {
        const int i = min(nx - 1, nx / 2 - 16 + (int)threadIdx.x);
        double m = fabs(f[(long long)P.rows[R0] * nx + max(0, i)]);
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) s_shift = scale_shift(m);
    }
    __syncthreads();
    const int shift = s_shift;
    for (int q = threadIdx.x; q < nv; q += blockDim.x) {
        FixedWideAcc acc[V];
        int cur = g0, gend = P.gstart[g0 + 1];
        auto flush = [&]() {
#pragma unroll
            for (int w = 0; w < V; w++) {
                racc[(long long)(cur - g0) * nx + q * V + w] = acc[w].total(shift);
                acc[w] = FixedWideAcc();
            }
            cur++;
            if (cur < g1) gend = P.gstart[cur + 1];
        };
        for (int r = R0; r < R1; r += 8) {
            double v[8][V];
#pragma unroll
            for (int u = 0; u < 8; u++) {
#pragma unroll
                for (int w = 0; w < V; w++) v[u][w] = 0.0;
                if (r + u < R1) {  // uniform over the CTA
                    const double *src = f + (long long)P.rows[r + u] * nx + (long long)q * V;
                    if constexpr (V == 2) {
                        const double2 t = __ldcs(reinterpret_cast<const double2 *>(src));
                        v[u][0] = t.x;
                        v[u][V - 1] = t.y;
                    } else {
                        v[u][0] = __ldcs(src);
                    }
                }
            }
            // rows of the same group add in FP64 pairs before the double-float
            // accumulation (moves about a third of the work to the FP64 pipe,
            // which the double-float operations leave idle); group boundaries are
            // uniform over the CTA, so are these branches
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                const int ra = r + u, rb = ra + 1;
                if (ra < R1) {
                    if (rb < gend) {  // both rows in the current group
#pragma unroll
                        for (int w = 0; w < V; w++) acc[w].add(v[u][w] + v[u + 1][w], shift);
                        if (rb + 1 == gend) flush();
                    } else {  // ra ends the group
#pragma unroll
                        for (int w = 0; w < V; w++) acc[w].add(v[u][w], shift);
                        flush();
                        if (rb < R1) {
#pragma unroll
                            for (int w = 0; w < V; w++) acc[w].add(v[u + 1][w], shift);
                            if (rb + 1 == gend) flush();
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    const int ng = g1 - g0;
    for (int e = threadIdx.x; e < ng * wt; e += blockDim.x) {
        const int t = e / ng, j = e - t * ng;
        const int k = P.kmin + t;
        const int i1 = P.c0 + k, i2 = P.c0 - 1 - k;  // a = k and a = -1 - k
        const double *ra = racc + (long long)j * nx;
        double v = 0.0;
        if (i1 >= 0 && i1 < nx) v = ra[i1];
        if (i2 >= 0 && i2 < nx) v += ra[i2];
        GT[(long long)t * P.ngroups + g0 + j] = v;
    }
}

// largest t >= 0 with T(t) <= x (-1 for x < 0), x < 2^31: a float estimate corrected
// with exact integer tests (the estimate is within one of the answer)
__device__ __forceinline__ long long floor_tinv(long long x) {
    if (x < 0) return -1;
    long long t = (long long)((sqrtf(8.0f * (float)x + 1.0f) - 1.0f) * 0.5f);
#pragma unroll
    for (int it = 0; it < 2; it++) {
        if (tri(t) > x) t--;
        else if (tri(t + 1) <= x) t++;
    }
    return t;
}

// 2. bins, fast pass (reads the fast fold's double-float G): a CTA per 32
// consecutive bins, lane = bin; the t range splits into one contiguous slice per
// warp (for each t the lanes read consecutive s in grp and neighbouring groups in
// GT[t][.]); the warps' partial sums combine in warp order.
constexpr int BIN_WARPS = BIN_THREADS / 32;
__global__ void __launch_bounds__(BIN_THREADS) rad_bin_kernel(RadDev P, const float2 *__restrict__ GT,
                                                              double *__restrict__ avg) {
    __shared__ float2 part[BIN_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long m0 = (long long)blockIdx.x * 32, m = m0 + lane;
    const long long mlast = min(m0 + 31, P.nbins - 1);
    const long long tlo = max((long long)P.kmin, floor_tinv(m0 - P.smax - 1) + 1);
    const long long thi = min((long long)P.kmax, floor_tinv(mlast - P.smin));
    const long long chunk = (thi - tlo + BIN_WARPS) / BIN_WARPS;  // ceil(nt / warps), nt may be 0
    const long long ta = tlo + w * chunk, tb = min(thi, ta + chunk - 1);
    DfAcc acc;
    if (ta <= tb) {
        // s = m - T(t) falls by t + 1 from t to t + 1; the G row advances by ngroups
        long long s = m - tri(ta);
        const float2 *gt = GT + (ta - P.kmin) * (long long)P.ngroups;
        const bool live = m < P.nbins;
        for (long long t = ta; t <= tb; t += 4) {
            int g[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                g[u] = (live && t + u <= tb && s >= P.smin && s <= P.smax) ? __ldg(P.grp + (s - P.smin)) : -1;
                s -= t + u + 1;
            }
            float2 v[4];
#pragma unroll
            for (int u = 0; u < 4; u++)
                v[u] = g[u] >= 0 ? __ldg(gt + (long long)u * P.ngroups + g[u]) : make_float2(0.f, 0.f);
            gt += 4LL * P.ngroups;
#pragma unroll
            for (int u = 0; u < 4; u++) acc.add(dfloat{v[u].x, v[u].y});
        }
    }
    const dfloat a = acc.norm();
    part[w][lane] = make_float2(a.h, a.l);
    __syncthreads();
    if (w == 0 && m < P.nbins) {
        dfloat sum{part[0][lane].x, part[0][lane].y};
        for (int q = 1; q < BIN_WARPS; q++) sum = df_add(sum, dfloat{part[q][lane].x, part[q][lane].y});
        const long long cnt = P.count[m];
        avg[m] = cnt ? df_to_double(sum) / (double)cnt : 0.0;
    }
}

// 2'. bins, full-range pass (after the full-range fold; returns at once unless
// flagged): as the fast bins, over the doubles of G with the wide accumulator.
__global__ void __launch_bounds__(BIN_THREADS) rad_bin_wide_kernel(RadDev P, const double *__restrict__ GT,
                                                                   const int *__restrict__ wide,
                                                                   double *__restrict__ avg) {
    if (*wide == 0) return;
    __shared__ double part[BIN_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long m0 = (long long)blockIdx.x * 32, m = m0 + lane;
    const long long mlast = min(m0 + 31, P.nbins - 1);
    const long long tlo = max((long long)P.kmin, floor_tinv(m0 - P.smax - 1) + 1);
    const long long thi = min((long long)P.kmax, floor_tinv(mlast - P.smin));
    const long long chunk = (thi - tlo + BIN_WARPS) / BIN_WARPS;  // ceil(nt / warps), nt may be 0
    const long long ta = tlo + w * chunk, tb = min(thi, ta + chunk - 1);
    WideAcc acc;
    if (ta <= tb) {
        // s = m - T(t) falls by t + 1 from t to t + 1; the G row advances by ngroups
        long long s = m - tri(ta);
        const double *gt = GT + (ta - P.kmin) * (long long)P.ngroups;
        const bool live = m < P.nbins;
        for (long long t = ta; t <= tb; t += 4) {
            int g[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                g[u] = (live && t + u <= tb && s >= P.smin && s <= P.smax) ? __ldg(P.grp + (s - P.smin)) : -1;
                s -= t + u + 1;
            }
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = g[u] >= 0 ? __ldg(gt + (long long)u * P.ngroups + g[u]) : 0.0;
            gt += 4LL * P.ngroups;
#pragma unroll
            for (int u = 0; u < 4; u++) acc.add(v[u]);
        }
    }
    part[w][lane] = acc.total();
    __syncthreads();
    if (w == 0 && m < P.nbins) {
        double sum = part[0][lane];
        for (int q = 1; q < BIN_WARPS; q++) sum += part[q][lane];
        const long long cnt = P.count[m];
        avg[m] = cnt ? sum / (double)cnt : 0.0;
    }
}

// Fill from per-bin values, out(i, j, k) = v[T(a) + s], s = T(b) + T(e): the rows of a
// group share s, so each group's row is gathered once (into smem) and stored to all
// its rows (16-byte streaming stores for V = 2).  SUB: out = src - v[m] instead
// (the bracket S - Sbar of the velocity split).
template <int V, bool SUB>
__global__ void __launch_bounds__(FOLD_THREADS) rad_fill_kernel(RadDev P, const long long *__restrict__ gs,
                                                                const double *__restrict__ v,
                                                                const double *__restrict__ src,
                                                                double *__restrict__ out) {
    extern __shared__ double rowv[];
    const int g0 = P.bstart[blockIdx.x], g1 = P.bstart[blockIdx.x + 1];
    const int nx = P.nx, nv = nx / V;
    for (int g = g0; g < g1; g++) {
        const long long s = gs[g];
        for (int i = threadIdx.x; i < nx; i += blockDim.x) rowv[i] = __ldg(v + tri((long long)(i - P.c0)) + s);
        __syncthreads();
        const int r0 = P.gstart[g], r1 = P.gstart[g + 1];
        for (int r = r0; r < r1; r++) {
            const long long base = (long long)P.rows[r] * nx;
            for (int q = threadIdx.x; q < nv; q += blockDim.x) {
                if constexpr (V == 2) {
                    double2 val = make_double2(rowv[2 * q], rowv[2 * q + 1]);
                    if constexpr (SUB) {
                        const double2 x = __ldcs(reinterpret_cast<const double2 *>(src + base) + q);
                        val = make_double2(x.x - val.x, x.y - val.y);
                    }
                    __stcs(reinterpret_cast<double2 *>(out + base) + q, val);
                } else {
                    double val = rowv[q];
                    if constexpr (SUB) val = __ldcs(src + base + q) - val;
                    __stcs(out + base + q, val);
                }
            }
        }
        __syncthreads();
    }
}

// 3-point Lagrange value at r, every operation rounded on its own (no contraction)
__device__ __forceinline__ double lagrange3_rn(double r, double x0, double y0, double x1, double y1, double x2,
                                               double y2) {
    const double a = __ddiv_rn(__dmul_rn(__dmul_rn(y0, __dsub_rn(r, x1)), __dsub_rn(r, x2)),
                               __dmul_rn(__dsub_rn(x0, x1), __dsub_rn(x0, x2)));
    const double b = __ddiv_rn(__dmul_rn(__dmul_rn(y1, __dsub_rn(r, x0)), __dsub_rn(r, x2)),
                               __dmul_rn(__dsub_rn(x1, x0), __dsub_rn(x1, x2)));
    const double c = __ddiv_rn(__dmul_rn(__dmul_rn(y2, __dsub_rn(r, x0)), __dsub_rn(r, x1)),
                               __dmul_rn(__dsub_rn(x2, x0), __dsub_rn(x2, x1)));
    return __dadd_rn(__dadd_rn(a, b), c);
}

__device__ __forceinline__ double bin_radius(long long m, double dx) {
    return __dmul_rn(dx, __dsqrt_rn(__dadd_rn(0.75, __dmul_rn(2.0, (double)m))));
}

// uniform fill, per bin: the quadratic through the radial cell centres jc-1, jc, jc+1,
// jc the radial cell holding r (kept one cell inside either end)
__global__ void rad_uniform_table_kernel(long long nbins, double dx, const double *__restrict__ prof, int nr,
                                         double dr, double *__restrict__ tab) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nbins) return;
    const double r = bin_radius(m, dx);
    long long jc = (long long)floor(__ddiv_rn(r, dr));
    jc = jc < 1 ? 1 : (jc > nr - 2 ? nr - 2 : jc);
    tab[m] = lagrange3_rn(r, __dmul_rn((double)jc - 0.5, dr), prof[jc - 1], __dmul_rn((double)jc + 0.5, dr),
                          prof[jc], __dmul_rn((double)jc + 1.5, dr), prof[jc + 1]);
}

// Average onto the uniform base state: at r = (j + 1/2) dr, the quadratic through the
// non-empty bin of radius nearest to r (the smaller on a tie) and its non-empty
// neighbours (kept one inside either end)
__global__ void rad_to_uniform_kernel(const int *__restrict__ ne, long long nne, double dx,
                                      const double *__restrict__ avg, int nr, double dr, double *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nr) return;
    const double r = __dmul_rn((double)j + 0.5, dr);
    long long lo = 0, hi = nne;  // first q with radius(ne[q]) >= r
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (bin_radius(ne[mid], dx) < r) lo = mid + 1;
        else hi = mid;
    }
    long long best;
    if (lo == 0) best = 0;
    else if (lo == nne) best = nne - 1;
    else {
        const double d0 = fabs(__dsub_rn(bin_radius(ne[lo - 1], dx), r));
        const double d1 = fabs(__dsub_rn(bin_radius(ne[lo], dx), r));
        best = d1 < d0 ? lo : lo - 1;
    }
    best = best < 1 ? 1 : (best > nne - 2 ? nne - 2 : best);
    const long long m0 = ne[best - 1], m1 = ne[best], m2 = ne[best + 1];
    out[j] = lagrange3_rn(r, bin_radius(m0, dx), avg[m0], bin_radius(m1, dx), avg[m1], bin_radius(m2, dx), avg[m2]);
}

// planar: per-(plane, chunk) sums, then one warp per plane
constexpr int PL_THREADS = 256;
__device__ __forceinline__ dfloat warp_df_sum(dfloat a) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const dfloat b{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
        a = df_add(a, b);
    }
    return a;
}
__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// Planar sums, fast pass (magnitudes 2^-73..2^97, else *wide is raised).  V = 2:
// 16-byte loads (n0 n1 even and a 16-byte aligned field); 4 loads in flight per
// thread; neighbouring values add in FP64 pairs, the pair sums in double-float
// (as in the radial fold); one double per block.
template <int V>
__global__ void __launch_bounds__(PL_THREADS) plane_sum_kernel(const double *__restrict__ f, long long nxy,
                                                               int nchunk, double *__restrict__ part,
                                                               int *__restrict__ wide) {
    __shared__ float2 ws[PL_THREADS / 32];
    bool seen = false;
    const long long nv = nxy / V;
    const long long len = (nv + nchunk - 1) / nchunk;
    const long long b0 = (long long)blockIdx.x * len, b1 = min(nv, b0 + len);
    const double *p = f + (long long)blockIdx.y * nxy;
    DfAcc acc;
    long long q = b0 + threadIdx.x;
    for (; q + 3 * PL_THREADS < b1; q += 4 * PL_THREADS) {
        double v[4][2];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if constexpr (V == 2) {
                const double2 t = __ldcs(reinterpret_cast<const double2 *>(p) + q + u * PL_THREADS);
                v[u][0] = t.x;
                v[u][1] = t.y;
            } else {
                v[u][0] = __ldcs(p + q + u * PL_THREADS);
            }
        }
        if constexpr (V == 2) {
#pragma unroll
            for (int u = 0; u < 4; u++) acc.add(df_split_mark(v[u][0] + v[u][1], seen, wide));
        } else {
            acc.add(df_split_mark(v[0][0] + v[1][0], seen, wide));
            acc.add(df_split_mark(v[2][0] + v[3][0], seen, wide));
        }
    }
    for (; q < b1; q += PL_THREADS) {
        if constexpr (V == 2) {
            const double2 t = __ldcs(reinterpret_cast<const double2 *>(p) + q);
            acc.add(df_split_mark(t.x + t.y, seen, wide));
        } else {
            acc.add(df_split_mark(__ldcs(p + q), seen, wide));
        }
    }
    dfloat a = warp_df_sum(acc.norm());
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = make_float2(a.h, a.l);
    __syncthreads();
    if (threadIdx.x == 0) {
        dfloat s{ws[0].x, ws[0].y};
        for (int w = 1; w < PL_THREADS / 32; w++) s = df_add(s, dfloat{ws[w].x, ws[w].y});
        part[(long long)blockIdx.y * nchunk + blockIdx.x] = df_to_double(s);
    }
}

// Full-range pass of the planar sums (runs when the fast pass set *wide).
// V = 2: 16-byte loads (n0 n1 even and a 16-byte aligned field); 4 loads in
// flight per thread; neighbouring values add in FP64 pairs, the pair sums in the
// wide double-float accumulator (as in the radial fold); per-thread totals reduce
// in FP64 (a few operations per thread)
template <int V>
__global__ void __launch_bounds__(PL_THREADS) plane_sum_wide_kernel(const double *__restrict__ f, long long nxy,
                                                                    int nchunk, double *__restrict__ part,
                                                                    const int *__restrict__ wide) {
    if (*wide == 0) return;
    __shared__ double ws[PL_THREADS / 32];
    const long long nv = nxy / V;
    const long long len = (nv + nchunk - 1) / nchunk;
    const long long b0 = (long long)blockIdx.x * len, b1 = min(nv, b0 + len);
    const double *p = f + (long long)blockIdx.y * nxy;
    WideAcc acc;
    long long q = b0 + threadIdx.x;
    for (; q + 3 * PL_THREADS < b1; q += 4 * PL_THREADS) {
        double v[4][2];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if constexpr (V == 2) {
                const double2 t = __ldcs(reinterpret_cast<const double2 *>(p) + q + u * PL_THREADS);
                v[u][0] = t.x;
                v[u][1] = t.y;
            } else {
                v[u][0] = __ldcs(p + q + u * PL_THREADS);
            }
        }
        if constexpr (V == 2) {
#pragma unroll
            for (int u = 0; u < 4; u++) acc.add(v[u][0] + v[u][1]);
        } else {
            acc.add(v[0][0] + v[1][0]);
            acc.add(v[2][0] + v[3][0]);
        }
    }
    for (; q < b1; q += PL_THREADS) {
        if constexpr (V == 2) {
            const double2 t = __ldcs(reinterpret_cast<const double2 *>(p) + q);
            acc.add(t.x + t.y);
        } else {
            acc.add(__ldcs(p + q));
        }
    }
    const double a = warp_sum(acc.total());
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = ws[0];
        for (int w = 1; w < PL_THREADS / 32; w++) t += ws[w];
        part[(long long)blockIdx.y * nchunk + blockIdx.x] = t;
    }
}

// out = S - prof[k] on plane k (grid: x over the plane, y over planes)
__global__ void plane_sub_kernel(const double *__restrict__ S, const double *__restrict__ prof, long long nxy,
                                 double *__restrict__ out) {
    const long long k = blockIdx.y;
    const double p = prof[k];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nxy; q += (long long)gridDim.x * blockDim.x)
        out[k * nxy + q] = S[k * nxy + q] - p;
}

__global__ void plane_final_kernel(const double *__restrict__ part, int nz, int nchunk, long long nxy,
                                   double *__restrict__ out) {
    const int k = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (k >= nz) return;
    double acc = 0.0;
    for (int c = threadIdx.x & 31; c < nchunk; c += 32) acc += part[(long long)k * nchunk + c];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) out[k] = acc / (double)nxy;
}

// ---------------------------------------------------------------------------------------
// plans (host)

static bool radial_ranges(const mx_geom *g, const int c[3], long long tmin[3], long long tmax[3], long long &nbins) {
    for (int d = 0; d < 3; d++) {
        if (g->n[d] < 1 || c[d] < -(1 << 20) || c[d] > (1 << 20)) return false;
        t_range(-(long long)c[d], (long long)g->n[d] - 1 - c[d], tmin[d], tmax[d]);
    }
    nbins = tri(tmax[0]) + tri(tmax[1]) + tri(tmax[2]) + 1;
    return nbins < (1LL << 31);
}

static void free_radial_plan(RadialPlan *p) {
    if (!p) return;
    if (p->mem) cudaFree(p->mem);
    delete p;
}

void destroy_radial_plans(mx_ctx *c) {
    for (RadialPlan *p : c->rplans) free_radial_plan(p);
    c->rplans.clear();
    if (c->base_tmp) cudaFree(c->base_tmp);
    c->base_tmp = nullptr;
    c->base_tmp_bytes = 0;
    if (c->base_flag) cudaFree(c->base_flag);
    c->base_flag = nullptr;
}

static mx_status get_radial_plan(mx_ctx *c, const mx_geom *geom, const int corner[3], RadialPlan **out) {
    for (RadialPlan *p : c->rplans)
        if (p->n[0] == geom->n[0] && p->n[1] == geom->n[1] && p->n[2] == geom->n[2] && p->c[0] == corner[0] &&
            p->c[1] == corner[1] && p->c[2] == corner[2]) {
            p->last_use = ++c->use_counter;
            *out = p;
            return MX_OK;
        }
    long long tmin[3], tmax[3], nbins;
    if (!radial_ranges(geom, corner, tmin, tmax, nbins))
        return set_err(c, MX_ERR_ARG, "radial: corner out of range or too many bins");
    const int nx = geom->n[0], ny = geom->n[1], nz = geom->n[2];
    if (nx > 12000) return set_err(c, MX_ERR_ARG, "radial: n[0] above 12000");  // row buffers in smem
    const long long nrows = (long long)ny * nz;
    if (nrows >= (1LL << 31)) return set_err(c, MX_ERR_ARG, "radial: too many rows");
    const long long smin = tri(tmin[1]) + tri(tmin[2]), smax = tri(tmax[1]) + tri(tmax[2]);
    const long long ns = smax - smin + 1;
    if (ns > (1LL << 26)) return set_err(c, MX_ERR_ARG, "radial: corner too far from the box");
    // rows grouped by s (counting sort, stable in the row id)
    std::vector<int> scount(ns + 1, 0), rows(nrows), grp(ns, -1), gstart;
    std::vector<long long> gs;
    for (long long r = 0; r < nrows; r++) {
        const long long j = r % ny, k = r / ny;
        scount[tri(j - corner[1]) + tri(k - corner[2]) - smin + 1]++;
    }
    for (long long s = 0; s < ns; s++) scount[s + 1] += scount[s];
    {
        std::vector<int> pos(scount.begin(), scount.end() - 1);
        for (long long r = 0; r < nrows; r++) {
            const long long j = r % ny, k = r / ny;
            rows[pos[tri(j - corner[1]) + tri(k - corner[2]) - smin]++] = int(r);
        }
    }
    for (long long s = 0; s < ns; s++)
        if (scount[s + 1] > scount[s]) {
            grp[s] = int(gstart.size());
            gstart.push_back(scount[s]);
            gs.push_back(s + smin);
        }
    const int ngroups = int(gstart.size());
    gstart.push_back(int(nrows));
    // fold batches: whole groups, about rb rows and at most gmax groups each (the
    // batch's column sums, gmax rows of n0 double-floats, stay in about 16 KB of
    // shared memory, so that shared memory does not limit the CTAs per SM)
    const long long rb = std::min(128LL, std::max(8LL, nrows / 4096));
    const int gmax = int(std::max(1LL, std::min(64LL, 2048LL / nx)));
    std::vector<int> bstart{0};
    for (int g = 0; g < ngroups; g++) {
        const long long in_batch = gstart[g] - gstart[bstart.back()];
        if (g > bstart.back() && (in_batch >= rb || g - bstart.back() >= gmax)) bstart.push_back(g);
    }
    bstart.push_back(ngroups);
    const int nbatch = int(bstart.size()) - 1;
    // cells per bin: rows of the group times the columns of each t
    const long long kmin = tmin[0], kmax = tmax[0], wt = kmax - kmin + 1;
    std::vector<long long> count(nbins, 0);
    for (int g = 0; g < ngroups; g++) {
        const long long nr = gstart[g + 1] - gstart[g];
        for (long long t = kmin; t <= kmax; t++) {
            const long long i1 = corner[0] + t, i2 = corner[0] - 1 - t;
            const long long mult = (i1 >= 0 && i1 < nx) + (i2 >= 0 && i2 < nx);
            count[gs[g] + tri(t)] += nr * mult;
        }
    }
    std::vector<int> ne;
    for (long long m = 0; m < nbins; m++)
        if (count[m] > 0) ne.push_back(int(m));
    RadialPlan *p = new RadialPlan();
    for (int d = 0; d < 3; d++) {
        p->n[d] = geom->n[d];
        p->c[d] = corner[d];
    }
    p->nbins = nbins;
    p->smin = smin;
    p->smax = smax;
    p->kmin = int(kmin);
    p->kmax = int(kmax);
    p->wt = int(wt);
    p->ngroups = ngroups;
    p->gmax = gmax;
    p->nbatch = nbatch;
    p->nrows = int(nrows);
    p->nne = (long long)ne.size();
    Bump b{nullptr, 0};
    auto carve = [&](Bump &bb) {
        p->rows = bb.take<int>(nrows);
        p->gstart = bb.take<int>(ngroups + 1);
        p->grp = bb.take<int>(ns);
        p->bstart = bb.take<int>(nbatch + 1);
        p->count = bb.take<long long>(nbins);
        p->gsv = bb.take<long long>(std::max(1, ngroups));
        p->nonempty = bb.take<int>(std::max<size_t>(1, ne.size()));
        p->G = bb.take<double>((size_t)ngroups * wt);
        p->tab = bb.take<double>(nbins);
        p->avg_tmp = bb.take<double>(nbins);
    };
    carve(b);
    if (cudaMalloc(&p->mem, b.off) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return set_err(c, MX_ERR_OOM, "radial: plan allocation failed");
    }
    Bump b2{(char *)p->mem, 0};
    carve(b2);
    cudaError_t e = cudaSuccess;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(p->rows, rows.data(), rows.size() * sizeof(int));
    up(p->gstart, gstart.data(), gstart.size() * sizeof(int));
    up(p->grp, grp.data(), grp.size() * sizeof(int));
    up(p->bstart, bstart.data(), bstart.size() * sizeof(int));
    up(p->count, count.data(), count.size() * sizeof(long long));
    up(p->gsv, gs.data(), gs.size() * sizeof(long long));
    up(p->nonempty, ne.data(), ne.size() * sizeof(int));
    if (e != cudaSuccess) {
        free_radial_plan(p);
        return set_err(c, MX_ERR_CUDA, std::string("radial: plan upload: ") + cudaGetErrorString(e));
    }
    if ((int)c->rplans.size() >= MAX_RADIAL_PLANS) {  // evict the least recently used
        auto it = std::min_element(c->rplans.begin(), c->rplans.end(),
                                   [](RadialPlan *a, RadialPlan *bb) { return a->last_use < bb->last_use; });
        cudaStreamSynchronize(c->stream);
        free_radial_plan(*it);
        c->rplans.erase(it);
    }
    p->last_use = ++c->use_counter;
    c->rplans.push_back(p);
    *out = p;
    return MX_OK;
}

// threads of the fold and fill CTAs: one per column pair of a row, 64 to 256
static int fold_threads(int nx) {
    const int nv = (nx + 1) / 2;
    return std::min(FOLD_THREADS, std::max(64, (nv + 31) / 32 * 32));
}

template <int V, bool SUB>
static mx_status launch_fill_t(mx_ctx *c, const RadialPlan *p, const double *v, const double *src, double *out) {
    const size_t smem = (size_t)p->n[0] * sizeof(double);
    if (smem > 48 * 1024)
        MX_CUDA(c, cudaFuncSetAttribute(rad_fill_kernel<V, SUB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    rad_fill_kernel<V, SUB><<<p->nbatch, fold_threads(p->n[0]), smem, c->stream>>>(rad_dev(p), p->gsv, v, src, out);
    return MX_OK;
}

// out = v[m] on every cell, or out = src - v[m] with src
static mx_status launch_fill(mx_ctx *c, const RadialPlan *p, const double *v, double *out,
                             const double *src = nullptr) {
    if (p->nbatch == 0) return MX_OK;
    // 16-byte accesses need an even row length and 16-byte aligned arrays
    const bool vec = p->n[0] % 2 == 0 && ((uintptr_t)out & 15) == 0 && ((uintptr_t)src & 15) == 0;
    if (src) return vec ? launch_fill_t<2, true>(c, p, v, src, out) : launch_fill_t<1, true>(c, p, v, src, out);
    return vec ? launch_fill_t<2, false>(c, p, v, src, out) : launch_fill_t<1, false>(c, p, v, src, out);
}

static mx_status check_corner_args(mx_ctx *c, const mx_geom *geom, const int corner[3]) {
    if (!c) return MX_ERR_ARG;
    mx_status st = check_geom(c, geom, false);
    if (st) return st;
    if (!corner) return set_err(c, MX_ERR_ARG, "radial: null corner");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    return MX_OK;
}

// the flag the fast passes set when a value lies outside their window (one int per
// context, cleared at the start of each Average)
static mx_status wide_flag(mx_ctx *c, int **flag) {
    if (!c->base_flag) {
        if (cudaMalloc(&c->base_flag, 256) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, MX_ERR_OOM, "average: flag allocation failed");
        }
    }
    *flag = (int *)c->base_flag;
    MX_CUDA(c, cudaMemsetAsync(*flag, 0, sizeof(int), c->stream));
    return MX_OK;
}

template <int V>
static mx_status launch_fold(mx_ctx *c, const RadialPlan *p, const double *field, int *flag, size_t smem, int nthr) {
    if (smem > 48 * 1024) {
        MX_CUDA(c, cudaFuncSetAttribute(rad_fold_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        MX_CUDA(c, cudaFuncSetAttribute(rad_fold_wide_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(smem)));
    }
    rad_fold_kernel<V><<<p->nbatch, nthr, smem, c->stream>>>(field, rad_dev(p), (float2 *)p->G, flag);
    return MX_OK;
}

// the radial Average into avg (nbins doubles): the fast passes, then the full-range
// passes, which return at once unless the fast fold flagged a value
static mx_status rad_average(mx_ctx *c, const RadialPlan *p, const double *field, double *avg) {
    if (p->nbatch == 0) return MX_OK;
    int *flag;
    mx_status st = wide_flag(c, &flag);
    if (st) return st;
    const bool vec = p->n[0] % 2 == 0 && ((uintptr_t)field & 15) == 0;  // 16-byte loads
    const size_t smem = (size_t)p->gmax * p->n[0] * sizeof(double);
    const int nthr = fold_threads(p->n[0]);
    const long long nb = (p->nbins + 31) / 32;
    if (vec) {
        if ((st = launch_fold<2>(c, p, field, flag, smem, nthr))) return st;
    } else {
        if ((st = launch_fold<1>(c, p, field, flag, smem, nthr))) return st;
    }
    rad_bin_kernel<<<(unsigned)nb, BIN_THREADS, 0, c->stream>>>(rad_dev(p), (const float2 *)p->G, avg);
    if (vec) rad_fold_wide_kernel<2><<<p->nbatch, nthr, smem, c->stream>>>(field, rad_dev(p), p->G, flag);
    else rad_fold_wide_kernel<1><<<p->nbatch, nthr, smem, c->stream>>>(field, rad_dev(p), p->G, flag);
    rad_bin_wide_kernel<<<(unsigned)nb, BIN_THREADS, 0, c->stream>>>(rad_dev(p), p->G, flag, avg);
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

// the plane means of field into prof (n2 doubles); scratch: nz * nchunk partial
// pairs, then n2 doubles (*prof_tmp, for callers that need a profile of their own)
static mx_status planar_average(mx_ctx *c, const mx_geom *geom, const double *field, double *prof,
                                double **prof_tmp = nullptr) {
    const long long nxy = (long long)geom->n[0] * geom->n[1];
    const int nz = geom->n[2];
    long long nchunk = std::min((nxy + 1023) / 1024, (2432LL + nz - 1) / nz);
    nchunk = std::max(1LL, nchunk);
    const size_t part_b = ((size_t)nz * nchunk * sizeof(double) + 255) & ~size_t(255);
    const size_t need = part_b + (size_t)nz * sizeof(double);
    if (need > c->base_tmp_bytes) {
        if (c->base_tmp) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->base_tmp);
        }
        c->base_tmp = nullptr;
        c->base_tmp_bytes = 0;
        if (cudaMalloc(&c->base_tmp, need) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, MX_ERR_OOM, "average_planar: scratch allocation failed");
        }
        c->base_tmp_bytes = need;
    }
    double *part = (double *)c->base_tmp;
    if (prof_tmp) *prof_tmp = prof = (double *)((char *)c->base_tmp + part_b);
    int *flag;
    mx_status st = wide_flag(c, &flag);
    if (st) return st;
    const dim3 grid((unsigned)nchunk, nz);
    if (nxy % 2 == 0 && ((uintptr_t)field & 15) == 0) {
        plane_sum_kernel<2><<<grid, PL_THREADS, 0, c->stream>>>(field, nxy, int(nchunk), part, flag);
        plane_sum_wide_kernel<2><<<grid, PL_THREADS, 0, c->stream>>>(field, nxy, int(nchunk), part, flag);
    } else {
        plane_sum_kernel<1><<<grid, PL_THREADS, 0, c->stream>>>(field, nxy, int(nchunk), part, flag);
        plane_sum_wide_kernel<1><<<grid, PL_THREADS, 0, c->stream>>>(field, nxy, int(nchunk), part, flag);
    }
    plane_final_kernel<<<(nz + 7) / 8, 256, 0, c->stream>>>(part, nz, int(nchunk), nxy, prof);
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

// out = S - Sbar, Sbar the lateral average of S filled back onto the cells (plane
// means, or the irregular radial means of the star centred on corner)
mx_status base_subtract_average(mx_ctx *c, const mx_geom *geom, int spherical, const int corner[3], const double *S,
                                double *out) {
    mx_status st;
    if (spherical) {
        RadialPlan *p;
        if ((st = get_radial_plan(c, geom, corner, &p))) return st;
        if ((st = rad_average(c, p, S, p->avg_tmp))) return st;
        if ((st = launch_fill(c, p, p->avg_tmp, out, S))) return st;
    } else {
        double *prof = nullptr;
        if ((st = planar_average(c, geom, S, nullptr, &prof))) return st;
        const long long nxy = (long long)geom->n[0] * geom->n[1];
        const long long gx = std::min((nxy + 255) / 256, 64LL);
        plane_sub_kernel<<<dim3((unsigned)gx, geom->n[2]), 256, 0, c->stream>>>(S, prof, nxy, out);
    }
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

// ---------------------------------------------------------------------------------------
// C ABI

extern "C" {

long long mx_radial_nbins(const mx_geom *geom, const int corner[3]) {
    if (!geom || !corner) return -1;
    long long tmin[3], tmax[3], nbins;
    if (!radial_ranges(geom, corner, tmin, tmax, nbins)) return -1;
    return nbins;
}

mx_status mx_average_planar(mx_ctx *c, const mx_geom *geom, const double *field, double *prof) {
    if (!c) return MX_ERR_ARG;
    mx_status st = check_geom(c, geom, false);
    if (st) return st;
    if (!field || !prof) return set_err(c, MX_ERR_ARG, "average_planar: null array");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    return planar_average(c, geom, field, prof);
}

mx_status mx_average_radial(mx_ctx *c, const mx_geom *geom, const int corner[3], const double *field,
                            long long nbins, double *avg, long long *count) {
    mx_status st = check_corner_args(c, geom, corner);
    if (st) return st;
    if (!field || !avg) return set_err(c, MX_ERR_ARG, "average_radial: null array");
    RadialPlan *p;
    if ((st = get_radial_plan(c, geom, corner, &p))) return st;
    if (nbins != p->nbins) return set_err(c, MX_ERR_ARG, "average_radial: nbins differs from mx_radial_nbins");
    if ((st = rad_average(c, p, field, avg))) return st;
    if (count)
        MX_CUDA(c, cudaMemcpyAsync(count, p->count, p->nbins * sizeof(long long), cudaMemcpyDeviceToDevice,
                                   c->stream));
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

mx_status mx_fill_radial(mx_ctx *c, const mx_geom *geom, const int corner[3], const double *base,
                         long long nbins, double *out) {
    mx_status st = check_corner_args(c, geom, corner);
    if (st) return st;
    if (!base || !out) return set_err(c, MX_ERR_ARG, "fill_radial: null array");
    RadialPlan *p;
    if ((st = get_radial_plan(c, geom, corner, &p))) return st;
    if (nbins != p->nbins) return set_err(c, MX_ERR_ARG, "fill_radial: nbins differs from mx_radial_nbins");
    if ((st = launch_fill(c, p, base, out))) return st;
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

mx_status mx_radial_to_uniform(mx_ctx *c, const mx_geom *geom, const int corner[3], const double *avg, int nr,
                               double dr, double *prof) {
    mx_status st = check_corner_args(c, geom, corner);
    if (st) return st;
    if (!avg || !prof) return set_err(c, MX_ERR_ARG, "radial_to_uniform: null array");
    if (nr < 1 || !(dr > 0.0)) return set_err(c, MX_ERR_ARG, "radial_to_uniform: needs nr >= 1 and dr > 0");
    RadialPlan *p;
    if ((st = get_radial_plan(c, geom, corner, &p))) return st;
    if (p->nne < 3) return set_err(c, MX_ERR_ARG, "radial_to_uniform: fewer than 3 non-empty radii");
    rad_to_uniform_kernel<<<(nr + 127) / 128, 128, 0, c->stream>>>(p->nonempty, p->nne, geom->dx, avg, nr, dr,
                                                                    prof);
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

mx_status mx_fill_uniform(mx_ctx *c, const mx_geom *geom, const int corner[3], const double *prof, int nr,
                          double dr, double *out) {
    mx_status st = check_corner_args(c, geom, corner);
    if (st) return st;
    if (!prof || !out) return set_err(c, MX_ERR_ARG, "fill_uniform: null array");
    if (nr < 3 || !(dr > 0.0)) return set_err(c, MX_ERR_ARG, "fill_uniform: needs nr >= 3 and dr > 0");
    RadialPlan *p;
    if ((st = get_radial_plan(c, geom, corner, &p))) return st;
    rad_uniform_table_kernel<<<(unsigned)((p->nbins + 255) / 256), 256, 0, c->stream>>>(p->nbins, geom->dx, prof,
                                                                                         nr, dr, p->tab);
    if ((st = launch_fill(c, p, p->tab, out))) return st;
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

}  // extern "C"
