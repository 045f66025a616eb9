// Autotuner for the smoother and tile settings of the projection solves
// (a GPU tuning step; the paper's solver has no counterpart).
//
// mx_autotune times whole solves of the caller's inputs on scratch copies of
// U and phi, changing one setting at a time from the base options: the sweep
// counts (nu1, nu2), then the z-depth of the stencil tiles (tile_z), then (MAC,
// mixed precision) the single-pass sweep.  A change is kept when the solve
// converges and its CUDA-event time (second of two calls: the first one builds
// the plan and the loop graph) beats the best so far.  The winner is stored in
// the context's tune cache, which calls with nu1 = nu2 = 0 read.
#include <algorithm>
#include <cstring>
#include <vector>

#include "mx_internal.cuh"

namespace {

bool same_key(const mx_ctx::Tune &t, int op, int prec, const mx_geom *g) {
    if (t.op != op || t.prec != prec) return false;
    for (int d = 0; d < 3; d++)
        if (t.n[d] != g->n[d] || t.lo[d] != g->lo[d] || t.hi[d] != g->hi[d]) return false;
    return true;
}

const mx_ctx::Tune *find(const mx_ctx *c, int op, int prec, const mx_geom *g) {
    for (const auto &t : c->tune)
        if (same_key(t, op, prec, g)) return &t;
    return nullptr;
}

}  // namespace

void tune_apply(const mx_ctx *c, int op, const mx_geom *g, mx_opts &o) {
    if (o.nu1 != 0 || o.nu2 != 0) return;
    if (const mx_ctx::Tune *t = find(c, op, o.prec, g)) {
        o.nu1 = t->nu1;
        o.nu2 = t->nu2;
        o.fused = t->fused;
        o.tile_z = t->tile_z;
    } else {
        o.nu1 = 2;
        o.nu2 = 2;
    }
}

extern "C" int mx_tune_lookup(const mx_ctx *c, int op, int prec, const mx_geom *g, mx_opts *out) {
    if (!c || !g || !out) return 0;
    const mx_ctx::Tune *t = find(c, op, prec, g);
    if (!t) return 0;
    out->prec = prec;
    out->nu1 = t->nu1;
    out->nu2 = t->nu2;
    out->fused = t->fused;
    out->tile_z = t->tile_z;
    return 1;
}

extern "C" mx_status mx_autotune(mx_ctx *c, int op, const mx_geom *geom, const double *ux, const double *uy,
                                 const double *uz, const double *rho, const double *beta0, const double *sbar,
                                 const mx_opts *base, mx_opts *best, double *ms_best) {
    if (!c) return MX_ERR_ARG;
    if (!geom || !ux || !uy || !uz || !rho || !beta0 || !sbar) return set_err(c, MX_ERR_ARG, "autotune: null argument");
    if (op != MX_OP_MAC && op != MX_OP_NODAL) return set_err(c, MX_ERR_ARG, "autotune: op must be MX_OP_MAC or MX_OP_NODAL");
    for (int d = 0; d < 3; d++)
        if (geom->n[d] < 1) return set_err(c, MX_ERR_ARG, "autotune: empty box");
    mx_opts o;
    if (base) o = *base;
    else mx_default_opts(&o);
    if (o.nu1 == 0 && o.nu2 == 0) {
        o.nu1 = 2;
        o.nu2 = 2;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");

    // scratch copies of the velocity (in/out of a solve) and phi
    const long long n0 = geom->n[0], n1 = geom->n[1], n2 = geom->n[2];
    long long len[3], nphi;
    if (op == MX_OP_MAC) {
        len[0] = (n0 + 1) * n1 * n2;
        len[1] = n0 * (n1 + 1) * n2;
        len[2] = n0 * n1 * (n2 + 1);
        nphi = n0 * n1 * n2;
    } else {
        len[0] = len[1] = len[2] = n0 * n1 * n2;
        const auto nodes = [&](int d) { return (long long)geom->n[d] + (geom->lo[d] == MX_BC_PERIODIC ? 0 : 1); };
        nphi = nodes(0) * nodes(1) * nodes(2);
    }
    const double *src[3] = {ux, uy, uz};
    double *u[3] = {nullptr, nullptr, nullptr}, *phi = nullptr;
    auto release = [&]() {
        for (int d = 0; d < 3; d++)
            if (u[d]) cudaFree(u[d]);
        if (phi) cudaFree(phi);
    };
    for (int d = 0; d < 3; d++)
        if (cudaMalloc(&u[d], sizeof(double) * len[d]) != cudaSuccess) {
            cudaGetLastError();
            release();
            return set_err(c, MX_ERR_OOM, "autotune: scratch allocation failed");
        }
    if (cudaMalloc(&phi, sizeof(double) * nphi) != cudaSuccess) {
        cudaGetLastError();
        release();
        return set_err(c, MX_ERR_OOM, "autotune: scratch allocation failed");
    }

    // one candidate: two calls on fresh copies of U, the second one timed
    auto run = [&](const mx_opts &cand, double &ms, int &vc) -> mx_status {
        mx_info info;
        for (int rep = 0; rep < 2; rep++) {
            for (int d = 0; d < 3; d++)
                if (cudaMemcpyAsync(u[d], src[d], sizeof(double) * len[d], cudaMemcpyDeviceToDevice, c->stream) !=
                    cudaSuccess)
                    return set_err(c, MX_ERR_CUDA, "autotune: copy failed");
            const mx_status st = op == MX_OP_MAC
                                     ? mx_mac_project(c, geom, u[0], u[1], u[2], rho, beta0, sbar, phi, &cand, &info)
                                     : mx_nodal_project(c, geom, u[0], u[1], u[2], rho, beta0, sbar, phi, &cand, &info);
            if (st != MX_OK) return st;
        }
        ms = info.ms;
        vc = info.vcycles;
        return MX_OK;
    };

    mx_opts cur = o;
    double cur_ms = 0.0;
    int cur_vc = 0;
    bool have = false;
    auto consider = [&](mx_opts cand) -> mx_status {
        if (have) cand.max_outer = cand.max_vcycles = std::min(o.max_vcycles, 3 * cur_vc + 4);
        double ms;
        int vc;
        const mx_status st = run(cand, ms, vc);
        if (st == MX_ERR_NOCONV) return MX_OK;  // too slow to converge: not a candidate
        if (st != MX_OK) return st;
        if (!have || ms < cur_ms) {
            cand.max_outer = o.max_outer;
            cand.max_vcycles = o.max_vcycles;
            cur = cand;
            cur_ms = ms;
            cur_vc = vc;
            have = true;
        }
        return MX_OK;
    };

    mx_status st = MX_OK;
    // 1. sweep counts
    static const int NU[][2] = {{2, 2}, {1, 1}, {2, 1}, {1, 2}, {3, 2}, {2, 3}, {3, 3}, {4, 4}};
    for (const auto &nu : NU) {
        mx_opts cand = o;
        cand.nu1 = nu[0];
        cand.nu2 = nu[1];
        if ((st = consider(cand))) break;
    }
    // 2. tile depth along z of the stencil kernels
    if (!st && have) {
        const int tz[] = {0, 4, 8, 16};
        const int dflt = op == MX_OP_MAC ? 8 : 16;  // tile_z = 0
        const auto eff = [&](int z) { return z ? z : dflt; };
        const mx_opts at = cur;
        for (int z : tz) {
            if (eff(z) == eff(at.tile_z)) continue;
            mx_opts cand = at;
            cand.tile_z = z;
            if ((st = consider(cand))) break;
        }
    }
    // 3. single-pass sweeps (MAC, FP32 V-cycles only)
    if (!st && have && op == MX_OP_MAC && o.prec == MX_PREC_MIXED) {
        mx_opts cand = cur;
        cand.fused = cur.fused ? 0 : 1;
        st = consider(cand);
    }
    cudaStreamSynchronize(c->stream);
    release();
    if (st) return st;
    if (!have) return set_err(c, MX_ERR_NOCONV, "autotune: no candidate setting converged");

    mx_ctx::Tune t;
    t.op = op;
    t.prec = o.prec;
    for (int d = 0; d < 3; d++) {
        t.n[d] = geom->n[d];
        t.lo[d] = geom->lo[d];
        t.hi[d] = geom->hi[d];
    }
    t.nu1 = cur.nu1;
    t.nu2 = cur.nu2;
    t.fused = cur.fused;
    t.tile_z = cur.tile_z;
    t.ms = cur_ms;
    bool stored = false;
    for (auto &e : c->tune)
        if (same_key(e, op, o.prec, geom)) {
            e = t;
            stored = true;
        }
    if (!stored) c->tune.push_back(t);
    if (best) *best = cur;
    if (ms_best) *ms_best = cur_ms;
    return MX_OK;
}
