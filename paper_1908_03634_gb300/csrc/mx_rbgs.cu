// One full red-black Gauss-Seidel sweep (red cells, then black cells) of the
// FP32 correction equation L e = f in a single pass over memory.
//
// A block owns a BX x BY x BZ tile.  It stages the old e on the tile plus a
// 2-cell halo in shared memory (all loads issued at once), updates the red
// cells of the tile plus a 1-cell halo (the halo is recomputed redundantly, so
// no block reads another block's output), then the black cells of the tile
// from those new red values, and writes the tile to a second buffer (e_out),
// so overlapping halos never race.  Per cell the arithmetic is exactly that of
// the two-pass colour kernels (gs_update): both produce bit-identical sweeps.
//
// Variants: ZERO = the input correction is identically 0 (first sweep of a
// V-cycle level: no read of e); PROLONG = the input is e + P e_coarse
// (piecewise-constant prolongation applied on load, the first sweep after the
// coarse-grid correction).
#include "mx_rbgs.cuh"
#include "mx_stencil.cuh"

constexpr int BX = 32, BY = 8, BZ = 8;                 // owned cells
constexpr int EX = BX + 4, EY = BY + 4, EZ = BZ + 4;   // staged e: +2 halo
constexpr int RX = BX + 2, RY = BY + 2, RZ = BZ + 2;   // red updates: +1 halo
constexpr int RB_THREADS = 256;

// Map an unwrapped coordinate u of a tile position to a cell index, or -1 when
// the position holds no cell: beyond a non-periodic wall, or farther than
// `reach` cells past the end of the box (tiles wider than a small level must
// not wrap more than once).
__device__ __forceinline__ int map_coord(int u, int n, bool per, int reach) {
    if (u >= 0 && u < n) return u;
    if (!per || u < -reach || u >= n + reach) return -1;
    return u < 0 ? u + n : u - n;
}

template <int MODE>
__global__ void __launch_bounds__(RB_THREADS, 6)
    rbgs_tile_kernel(Level<float> L, const float *__restrict__ ein, float *__restrict__ eout,
                     const float *__restrict__ ecoarse, int ncx, int ncy, float h2) {
    __shared__ float se[EZ][EY][EX];
    const DGeom &g = L.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const bool px = gper(g, 0), py = gper(g, 1), pz = gper(g, 2);
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * BZ;
    const int tid = threadIdx.x;

    // 1. stage e (tile + 2 halo)
    for (int q = tid; q < EX * EY * EZ; q += RB_THREADS) {
        const int ax = q % EX, ay = (q / EX) % EY, az = q / (EX * EY);
        float v = 0.f;
        if (MODE != RB_ZERO) {
            const int lx = map_coord(x0 - 2 + ax, nx, px, 2), ly = map_coord(y0 - 2 + ay, ny, py, 2);
            const int lz = map_coord(z0 - 2 + az, nz, pz, 2);
            if (lx >= 0 && ly >= 0 && lz >= 0) {
                v = ein[lx + (long long)nx * (ly + (long long)ny * lz)];
                if (MODE == RB_PROLONG)
                    v += ecoarse[(lx >> 1) + (long long)ncx * ((ly >> 1) + (long long)ncy * (lz >> 1))];
            }
        }
        se[az][ay][ax] = v;
    }
    __syncthreads();

    // 2. red cells of the tile + 1 halo; a red cell reads only black (old) values
    constexpr int PAIRS = RX / 2;  // 17 red cells per row of 34
    for (int q = tid; q < PAIRS * RY * RZ; q += RB_THREADS) {
        const int pr = q % PAIRS, row = q / PAIRS;
        const int ry = row % RY, rz = row / RY;
        const int gyu = y0 - 1 + ry, gzu = z0 - 1 + rz;
        const int rx = 2 * pr + ((x0 - 1 + gyu + gzu) & 1);  // (gxu + gyu + gzu) even
        const int gxu = x0 - 1 + rx;
        const int gx = map_coord(gxu, nx, px, 1), gy = map_coord(gyu, ny, py, 1), gz = map_coord(gzu, nz, pz, 1);
        if (gx < 0 || gy < 0 || gz < 0) continue;
        const long long c = gx + (long long)nx * (gy + (long long)ny * gz);
        float b[6], v[6];
        face_coefs(L, gx, gy, gz, c, b);
        const int ax = rx + 1, ay = ry + 1, az = rz + 1;
        v[0] = se[az][ay][ax - 1];
        v[1] = se[az][ay][ax + 1];
        v[2] = se[az][ay - 1][ax];
        v[3] = se[az][ay + 1][ax];
        v[4] = se[az - 1][ay][ax];
        v[5] = se[az + 1][ay][ax];
        se[az][ay][ax] = gs_update(b, v, L.f[c], h2);
    }
    __syncthreads();

    // 3. black cells of the tile from the new red values; write the tile
    for (int q = tid; q < BX * BY * BZ; q += RB_THREADS) {
        const int ix = q % BX, iy = (q / BX) % BY, iz = q / (BX * BY);
        const int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
        if (gx >= nx || gy >= ny || gz >= nz) continue;
        const long long c = gx + (long long)nx * (gy + (long long)ny * gz);
        const int ax = ix + 2, ay = iy + 2, az = iz + 2;
        if (((gx + gy + gz) & 1) == 0) {
            eout[c] = se[az][ay][ax];
        } else {
            float b[6], v[6];
            face_coefs(L, gx, gy, gz, c, b);
            v[0] = se[az][ay][ax - 1];
            v[1] = se[az][ay][ax + 1];
            v[2] = se[az][ay - 1][ax];
            v[3] = se[az][ay + 1][ax];
            v[4] = se[az - 1][ay][ax];
            v[5] = se[az + 1][ay][ax];
            eout[c] = gs_update(b, v, L.f[c], h2);
        }
    }
}

void k_rbgs_fused(cudaStream_t s, const Level<float> &L, const float *ein, float *eout, int mode,
                  const Level<float> *coarse) {
    const DGeom &g = L.g;
    dim3 grid((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY, (g.n[2] + BZ - 1) / BZ);
    const float h2 = float(g.h * g.h);
    const float *ec = coarse ? coarse->e : nullptr;
    const int ncx = coarse ? coarse->g.n[0] : 0, ncy = coarse ? coarse->g.n[1] : 0;
    if (mode == RB_ZERO)
        rbgs_tile_kernel<RB_ZERO><<<grid, RB_THREADS, 0, s>>>(L, ein, eout, ec, ncx, ncy, h2);
    else if (mode == RB_PROLONG)
        rbgs_tile_kernel<RB_PROLONG><<<grid, RB_THREADS, 0, s>>>(L, ein, eout, ec, ncx, ncy, h2);
    else
        rbgs_tile_kernel<RB_PLAIN><<<grid, RB_THREADS, 0, s>>>(L, ein, eout, ec, ncx, ncy, h2);
}
