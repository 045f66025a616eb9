// One full red-black Gauss-Seidel sweep (red cells, then black cells) of the
// FP32 correction equation L e = f in a single pass over memory.
//
// A block owns a TX x TY column tile of cells and marches up a z-chunk of ZB
// planes.  It keeps the last planes of the old e (tile plus a 2-cell halo in x
// and y) in a ring of shared-memory planes.  At plane p it updates the red
// cells of the tile plus a 1-cell ring (the ring is recomputed redundantly, so
// no block reads another block's output), then the black cells of plane p-1
// from those new red values, and writes plane p-1 of the tile to a second
// buffer (e_out), so halos shared by neighbouring blocks never race.  The
// chunk recomputes the red cells of the plane below and above it.  Per cell
// the arithmetic is exactly that of the two-pass colour kernels (gs_update),
// so both produce bit-identical sweeps.
//
// Variants: ZERO = the input correction is identically 0 (first sweep of a
// V-cycle level: no read of e); PROLONG = the input is e + P e_coarse
// (piecewise-constant prolongation applied on load, the first sweep after the
// coarse-grid correction).
//
// Requirements (checked by rbgs_fused_ok): n_x even, so that cell pairs
// (2m, 2m+1) are float2-aligned and a periodic wrap maps pairs to pairs, and
// every periodic extent >= 2 (halo positions wrap at most once).
#include "mx_rbgs.cuh"
#include "mx_stencil.cuh"

constexpr int TX = 64, TY = 8, ZB = 16;        // owned cells of a block: TX x TY x ZB
constexpr int PW = TX + 4, PH = TY + 4;        // staged plane: +2 halo in x and y
constexpr int NSLOT = 5;                       // planes p-2 .. p+2 in flight
constexpr int RB_THREADS = 32 * TY;            // one warp per row, two cells per lane
constexpr int LOAD_ITEMS = PH * (PW / 2);      // float2 loads per plane
constexpr int LOAD_PER_THREAD = (LOAD_ITEMS + RB_THREADS - 1) / RB_THREADS;
constexpr int RING_ITEMS = TX / 2 * 2 + 2 * TY;  // red pairs of the two ring rows + ring-column cells

// Map an unwrapped coordinate u (at most `reach` cells outside the box) to a
// cell index, or -1 when the position holds no cell (beyond a non-periodic face).
__device__ __forceinline__ int map_coord(int u, int n, bool per, int reach) {
    if (u >= 0 && u < n) return u;
    if (!per || u < -reach || u >= n + reach) return -1;
    return u < 0 ? u + n : u - n;
}

// b[6] of an in-box cell with 32-bit indexing (the same values face_coefs reads).
__device__ __forceinline__ void coefs32(const Level<float> &L, int nx, int ny, int nz, int nxy, bool px, bool py,
                                        bool pz, int i, int j, int k, int c, float b[6]) {
    b[0] = __ldg(L.bx + c);
    b[1] = (i + 1 < nx) ? __ldg(L.bx + c + 1) : (px ? __ldg(L.bx + c - (nx - 1)) : __ldg(L.hx + j + ny * k));
    b[2] = __ldg(L.by + c);
    b[3] = (j + 1 < ny) ? __ldg(L.by + c + nx) : (py ? __ldg(L.by + c - (ny - 1) * nx) : __ldg(L.hy + i + nx * k));
    b[4] = __ldg(L.bz + c);
    b[5] = (k + 1 < nz) ? __ldg(L.bz + c + nxy) : (pz ? __ldg(L.bz + c - (nz - 1) * nxy) : __ldg(L.hz + i + nx * j));
}

// Fixed per-thread description of one cell column position of the tile:
// in-box coordinates (or gx < 0 when the position holds no cell) and its
// staged position.
struct ColPos {
    int gx, gy, ax, ay;
};

__device__ __forceinline__ ColPos col_pos(int ux, int uy, int x0, int y0, int nx, int ny, bool px, bool py) {
    ColPos c;
    c.gx = map_coord(ux, nx, px, 1);
    c.gy = map_coord(uy, ny, py, 1);
    if (c.gy < 0) c.gx = -1;
    c.ax = ux - x0 + 2;
    c.ay = uy - y0 + 2;
    return c;
}

template <int MODE>
__global__ void __launch_bounds__(RB_THREADS, 4)
    rbgs_march_kernel(Level<float> L, const float *__restrict__ ein, float *__restrict__ eout,
                      const float *__restrict__ ecoarse, int ncx, int ncy, float h2) {
    pdl_trigger();
    pdl_wait();
    __shared__ __align__(16) float sp[NSLOT][PH][PW];
    const DGeom &g = L.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxy = nx * ny;
    const bool px = gper(g, 0), py = gper(g, 1), pz = gper(g, 2);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, k0 = blockIdx.z * ZB;
    const int xe = min(x0 + TX, nx), ye = min(y0 + TY, ny), k1 = min(k0 + ZB, nz);
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5, tid = threadIdx.x;
    const float *__restrict__ f = L.f;

    // staging of one plane of the old e (tile + 2 halo): this thread's float2
    // items, as an in-plane global offset (-1: no cell) and a staged offset
    int ld_xy[LOAD_PER_THREAD], ld_s[LOAD_PER_THREAD], ld_c[LOAD_PER_THREAD];
#pragma unroll
    for (int r = 0; r < LOAD_PER_THREAD; r++) {
        const int q = tid + r * RB_THREADS;
        const int ay = q / (PW / 2), m = q % (PW / 2);
        const int gy = map_coord(y0 - 2 + ay, ny, py, 2), gx = map_coord(x0 - 2 + 2 * m, nx, px, 2);
        const bool ok = q < LOAD_ITEMS && gx >= 0 && gy >= 0;
        ld_xy[r] = ok ? gx + nx * gy : -1;
        ld_s[r] = q < LOAD_ITEMS ? ay * PW + 2 * m : -1;
        ld_c[r] = ok ? (gx >> 1) + ncx * (gy >> 1) : 0;
    }
    float2 pre[LOAD_PER_THREAD];
    auto fetch = [&](int p) {
        const int gz = map_coord(p, nz, pz, 2);
#pragma unroll
        for (int r = 0; r < LOAD_PER_THREAD; r++) {
            float2 v = make_float2(0.f, 0.f);
            if (MODE != RB_ZERO && gz >= 0 && ld_xy[r] >= 0) {
                v = __ldg(reinterpret_cast<const float2 *>(ein + ld_xy[r] + nxy * gz));
                if (MODE == RB_PROLONG) {
                    const float ec = __ldg(ecoarse + ld_c[r] + ncx * ncy * (gz >> 1));
                    v.x += ec;
                    v.y += ec;
                }
            }
            pre[r] = v;
        }
    };
    auto store = [&](int p) {
        float *plane = &sp[(p + 2 * NSLOT) % NSLOT][0][0];
#pragma unroll
        for (int r = 0; r < LOAD_PER_THREAD; r++)
            if (ld_s[r] >= 0) *reinterpret_cast<float2 *>(plane + ld_s[r]) = pre[r];
    };

    // this thread's interior pair (both parities) and ring item
    const int row_y = y0 + ly, pair_x = x0 + 2 * lx;
    const bool pair_in = row_y < ye && pair_x < xe;
    const ColPos in0 = col_pos(pair_x, row_y, x0, y0, nx, ny, px, py);
    const ColPos in1 = col_pos(pair_x + 1, row_y, x0, y0, nx, ny, px, py);
    // ring: a red pair of ring row y0-1 or ye (kind 1), or a cell of ring
    // column x0-1 or xe (kind 2), the latter red only on planes of one parity
    int ring_kind = 0, rux = 0, ruy = 0;
    if (tid < TX) {
        const int top = tid >= TX / 2;
        rux = x0 + 2 * (top ? tid - TX / 2 : tid);
        ruy = top ? ye : y0 - 1;
        ring_kind = rux < xe ? 1 : 0;
    } else if (tid < RING_ITEMS) {
        const int r = tid - TX, right = r >= TY;
        ruy = y0 + (right ? r - TY : r);
        rux = right ? xe : x0 - 1;
        ring_kind = ruy < ye ? 2 : 0;
    }
    const ColPos rg0 = col_pos(rux, ruy, x0, y0, nx, ny, px, py);
    const ColPos rg1 = col_pos(rux + 1, ruy, x0, y0, nx, ny, px, py);

    // red (or black) update of the cell at P on plane gz; returns the new value
    auto update = [&](const ColPos &P, int gz, int sm, int s0, int s1) -> float {
        const int c = P.gx + nx * P.gy + nxy * gz;
        float b[6], v[6];
        coefs32(L, nx, ny, nz, nxy, px, py, pz, P.gx, P.gy, gz, c, b);
        const float fc = __ldg(f + c);
        const int ax = P.ax, ay = P.ay;
        v[0] = sp[s0][ay][ax - 1];
        v[1] = sp[s0][ay][ax + 1];
        v[2] = sp[s0][ay - 1][ax];
        v[3] = sp[s0][ay + 1][ax];
        v[4] = sp[sm][ay][ax];
        v[5] = sp[s1][ay][ax];
        return gs_update(b, v, fc, h2);
    };

    // prologue: planes k0-2 .. k0-1 staged, k0 in flight
    fetch(k0 - 2);
    store(k0 - 2);
    fetch(k0 - 1);
    store(k0 - 1);
    fetch(k0);
    for (int p = k0 - 1; p <= k1; p++) {
        store(p + 1);
        if (p + 2 <= k1 + 1) fetch(p + 2);
        __syncthreads();
        const int s0 = (p + 2 * NSLOT) % NSLOT, sm = (p - 1 + 2 * NSLOT) % NSLOT, s1 = (p + 1) % NSLOT;
        // red cells of plane p: tile + 1-cell ring (no corners); (x + y + z) even
        const int gz = map_coord(p, nz, pz, 1);
        if (gz >= 0) {
            if (pair_in) {
                const ColPos &P = ((row_y + p) & 1) ? in1 : in0;
                sp[s0][P.ay][P.ax] = update(P, gz, sm, s0, s1);
            }
            if (ring_kind == 1) {
                const ColPos &P = ((ruy + p) & 1) ? rg1 : rg0;
                if (P.gx >= 0) sp[s0][P.ay][P.ax] = update(P, gz, sm, s0, s1);
            } else if (ring_kind == 2 && ((rux + ruy + p) & 1) == 0 && rg0.gx >= 0) {
                sp[s0][rg0.ay][rg0.ax] = update(rg0, gz, sm, s0, s1);
            }
        }
        __syncthreads();
        // black cells of plane q = p-1 (inside the chunk), then write the pair
        const int q = p - 1;
        if (q >= k0 && q < k1 && pair_in) {
            const int sq = (q + 2 * NSLOT) % NSLOT, sqm = (q - 1 + 2 * NSLOT) % NSLOT;
            const int odd = (row_y + q + 1) & 1;  // black cell = pair_x + odd
            const ColPos &P = odd ? in1 : in0;
            const float nb = update(P, q, sqm, sq, s0);
            const float nr = sp[sq][P.ay][P.ax + (odd ? -1 : 1)];
            float2 *dst = reinterpret_cast<float2 *>(eout + in0.gx + nx * row_y + nxy * q);
            *dst = odd ? make_float2(nr, nb) : make_float2(nb, nr);
        }
    }
}

bool rbgs_fused_ok(const DGeom &g) {
    if (g.n[0] % 2) return false;
    for (int d = 0; d < 3; d++)
        if (gper(g, d) && g.n[d] < 2) return false;
    return true;
}

void k_rbgs_fused(cudaStream_t s, const Level<float> &L, const float *ein, float *eout, int mode,
                  const Level<float> *coarse) {
    const DGeom &g = L.g;
    dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + ZB - 1) / ZB);
    const float h2 = float(g.h * g.h);
    const float *ec = coarse ? coarse->e : nullptr;
    const int ncx = coarse ? coarse->g.n[0] : 0, ncy = coarse ? coarse->g.n[1] : 0;
    auto k = mode == RB_ZERO ? rbgs_march_kernel<RB_ZERO>
             : mode == RB_PROLONG ? rbgs_march_kernel<RB_PROLONG> : rbgs_march_kernel<RB_PLAIN>;
    launch_pdl(k, grid, dim3(RB_THREADS), 0, s, L, ein, eout, ec, ncx, ncy, h2);
}
