// One full red-black Gauss-Seidel sweep (red cells, then black cells) of the
// FP32 correction equation L e = f in a single pass over memory.
//
// A block owns a TX x TY column tile and marches up a z-chunk.  The old e
// plane t+1 is staged in shared memory with a 2-cell halo (5-plane ring);
// red cells of plane t are updated on the tile plus a 1-cell halo (the halo is
// recomputed redundantly, so no block reads another block's output), then black
// cells of plane t-1 are updated on the tile from the new red values of planes
// t-2, t-1, t.  In z the pipeline lags by one plane: red(t) only reads black
// values that black(t-1) has not yet replaced.  The result goes to a second
// buffer (e_out), so overlapping halos never race.  Per cell the arithmetic is
// exactly that of the two-pass colour kernels (gs_update), so both produce
// bit-identical sweeps.
//
// Variants: ZERO = the input correction is identically 0 (first sweep of a
// V-cycle level: no read of e); PROLONG = the input is e + P e_coarse
// (piecewise-constant prolongation applied on load, the first sweep after the
// coarse-grid correction).
#include "mx_rbgs.cuh"
#include "mx_stencil.cuh"

constexpr int TX = 32, TY = 8;
constexpr int R1X = TX + 2, R1Y = TY + 2;  // tile + 1 halo: red updates
constexpr int R2X = TX + 4, R2Y = TY + 4;  // tile + 2 halo: staged old e
constexpr int NSLOT = 5;
constexpr int RB_THREADS = ((R1X * R1Y + 31) / 32) * 32;  // 352
constexpr int ZCH = 32;                                    // longest z-chunk per block

// Map an unwrapped coordinate u of a tile position to a cell index, or -1 when
// the position holds no cell: beyond a non-periodic wall, or farther than
// `reach` cells past the end of the box (tiles wider than a small coarse level
// must not wrap more than once).
__device__ __forceinline__ int map_coord(int u, int n, bool per, int reach) {
    if (u >= 0 && u < n) return u;
    if (!per || u < -reach || u >= n + reach) return -1;
    return u < 0 ? u + n : u - n;
}

// Coefficients and right-hand side of one cell (the row of L e = f).
struct RowData {
    float b[6];
    float f;
};

__device__ __forceinline__ void load_row(const Level<float> &L, int gx, int gy, int gz, RowData &r) {
    const DGeom &g = L.g;
    const long long c = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * gz);
    face_coefs(L, gx, gy, gz, c, r.b);
    r.f = L.f[c];
}

template <int MODE>
__global__ void __launch_bounds__(RB_THREADS, 3)
    rbgs_fused_kernel(Level<float> L, const float *__restrict__ ein, float *__restrict__ eout,
                      const float *__restrict__ ecoarse, int ncx, int ncy, float h2, int zch) {
    __shared__ float slot[NSLOT][R2Y][R2X];
    const DGeom &g = L.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const bool px_ = gper(g, 0), py_ = gper(g, 1), pz_ = gper(g, 2);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zch, z1 = min(z0 + zch, nz);
    const int tid = threadIdx.x;

    // this thread's R1 position
    const bool active = tid < R1X * R1Y;
    const int rx = active ? tid % R1X : 0, ry = active ? tid / R1X : 0;
    const int gxu = x0 - 1 + rx, gyu = y0 - 1 + ry;  // unwrapped (colour parity)
    const int gx = map_coord(gxu, nx, px_, 1), gy = map_coord(gyu, ny, py_, 1);
    const bool inplane = active && gx >= 0 && gy >= 0;
    // owned cells: inside the tile and inside the box (unwrapped)
    const bool interior = inplane && rx >= 1 && rx <= TX && ry >= 1 && ry <= TY && gxu < nx && gyu < ny;
    const int qx = rx + 1, qy = ry + 1;  // position in the R2 slot

    // the (at most two) R2 positions this thread stages, fixed for all planes
    const int q0 = tid, q1 = tid + RB_THREADS;
    int lx0 = -1, ly0 = -1, lx1 = -1, ly1 = -1;
    if (q0 < R2X * R2Y) {
        lx0 = map_coord(x0 - 2 + q0 % R2X, nx, px_, 2);
        ly0 = map_coord(y0 - 2 + q0 / R2X, ny, py_, 2);
    }
    if (q1 < R2X * R2Y) {
        lx1 = map_coord(x0 - 2 + q1 % R2X, nx, px_, 2);
        ly1 = map_coord(y0 - 2 + q1 / R2X, ny, py_, 2);
    }
    auto fetch1 = [&](int lx, int ly, int gz) -> float {
        float v = 0.f;
        if (MODE != RB_ZERO && gz >= 0 && lx >= 0 && ly >= 0) {
            v = ein[lx + (long long)nx * (ly + (long long)ny * gz)];
            if (MODE == RB_PROLONG)
                v += ecoarse[(lx >> 1) + (long long)ncx * ((ly >> 1) + (long long)ncy * (gz >> 1))];
        }
        return v;
    };
    float pre0 = 0.f, pre1 = 0.f;  // staged values of the next plane, in flight
    auto fetch_plane = [&](int t) {
        const int gz = map_coord(t, nz, pz_, 2);
        pre0 = fetch1(lx0, ly0, gz);
        pre1 = fetch1(lx1, ly1, gz);
    };
    auto store_plane = [&](int t) {
        const int sl = ((t % NSLOT) + NSLOT) % NSLOT;
        if (q0 < R2X * R2Y) slot[sl][q0 / R2X][q0 % R2X] = pre0;
        if (q1 < R2X * R2Y) slot[sl][q1 / R2X][q1 % R2X] = pre1;
    };

    // Rows of the two updates of the thread's next busy iteration t
    // ((gxu+gyu+t) even): red at plane t, black at plane t-1.  A thread is busy
    // every other plane; the rows are loaded right after its previous busy
    // iteration, so the loads overlap two barriers.
    RowData red_row, black_row;
    auto busy = [&](int t) { return ((gxu + gyu + t) & 1) == 0; };
    auto prefetch_rows = [&](int t) {
        const int gz = map_coord(t, nz, pz_, 1);
        if (inplane && gz >= 0) load_row(L, gx, gy, gz, red_row);
        if (interior && t - 1 >= z0 && t - 1 < z1) load_row(L, gx, gy, t - 1, black_row);
    };

    fetch_plane(z0 - 2);
    store_plane(z0 - 2);
    fetch_plane(z0 - 1);
    store_plane(z0 - 1);
    fetch_plane(z0);
    const int tfirst = z0 - 1;
    prefetch_rows(busy(tfirst) ? tfirst : tfirst + 1);
    for (int t = tfirst; t <= z1; t++) {
        store_plane(t + 1);
        if (t + 2 <= z1 + 1) fetch_plane(t + 2);
        __syncthreads();
        if (!busy(t)) continue;  // rows of iteration t+1 are already in flight
        const int st = ((t % NSLOT) + NSLOT) % NSLOT;
        const int sm = ((t - 1) % NSLOT + NSLOT) % NSLOT;
        const int sp = ((t + 1) % NSLOT + NSLOT) % NSLOT;
        const int gz = map_coord(t, nz, pz_, 1);
        // red cell of plane t (tile + 1 halo)
        if (inplane && gz >= 0) {
            float v[6];
            v[0] = slot[st][qy][qx - 1];
            v[1] = slot[st][qy][qx + 1];
            v[2] = slot[st][qy - 1][qx];
            v[3] = slot[st][qy + 1][qx];
            v[4] = slot[sm][qy][qx];
            v[5] = slot[sp][qy][qx];
            const float er = gs_update(red_row.b, v, red_row.f, h2);
            slot[st][qy][qx] = er;
            if (interior && t >= z0 && t < z1) eout[gx + (long long)nx * (gy + (long long)ny * t)] = er;  // final
        }
        // plane t-1 of the tile is final: its black cell here, its red cell was
        // computed by this thread one iteration ago
        const int tb = t - 1;
        if (interior && tb >= z0 && tb < z1) {
            const long long c = gx + (long long)nx * (gy + (long long)ny * tb);
            const int s2 = ((tb - 1) % NSLOT + NSLOT) % NSLOT;
            float v[6];
            v[0] = slot[sm][qy][qx - 1];
            v[1] = slot[sm][qy][qx + 1];
            v[2] = slot[sm][qy - 1][qx];
            v[3] = slot[sm][qy + 1][qx];
            v[4] = slot[s2][qy][qx];
            v[5] = slot[st][qy][qx];
            eout[c] = gs_update(black_row.b, v, black_row.f, h2);
        }
        prefetch_rows(t + 2);  // the thread's next busy iteration
    }
}

void k_rbgs_fused(cudaStream_t s, const Level<float> &L, const float *ein, float *eout, int mode,
                  const Level<float> *coarse) {
    const DGeom &g = L.g;
    // z-chunk: long chunks amortise the redundant halo planes, short ones give
    // small levels enough blocks (>= ~4 per SM)
    const long long cols = (long long)((g.n[0] + TX - 1) / TX) * ((g.n[1] + TY - 1) / TY);
    int zch = ZCH;
    while (zch > 4 && cols * ((g.n[2] + zch - 1) / zch) < 4 * 152) zch /= 2;
    dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + zch - 1) / zch);
    const float h2 = float(g.h * g.h);
    const float *ec = coarse ? coarse->e : nullptr;
    const int ncx = coarse ? coarse->g.n[0] : 0, ncy = coarse ? coarse->g.n[1] : 0;
    if (mode == RB_ZERO)
        rbgs_fused_kernel<RB_ZERO><<<grid, RB_THREADS, 0, s>>>(L, ein, eout, ec, ncx, ncy, h2, zch);
    else if (mode == RB_PROLONG)
        rbgs_fused_kernel<RB_PROLONG><<<grid, RB_THREADS, 0, s>>>(L, ein, eout, ec, ncx, ncy, h2, zch);
    else
        rbgs_fused_kernel<RB_PLAIN><<<grid, RB_THREADS, 0, s>>>(L, ein, eout, ec, ncx, ncy, h2, zch);
}
