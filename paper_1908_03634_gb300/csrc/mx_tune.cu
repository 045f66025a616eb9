// Autotuner for the smoother and tile settings of the projection solves
// (a GPU tuning step; the paper's solver has no counterpart).
//
// mx_autotune times whole solves of the caller's inputs on scratch copies of
// U and phi, changing one setting at a time from the base options: the sweep
// counts (nu1, nu2), then the z-depth of the stencil tiles (tile_z), then (MAC,
// mixed precision) the single-pass sweep, or (nodal) the Chebyshev smoother
// with its own degree candidates.  A change is kept when the solve
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

// A batch is keyed by its box count and a hash of every box's geometry,
// stored in the entry's n[] (op = TUNE_BATCH).
constexpr int TUNE_BATCH = 100;

mx_geom batch_key(int nbox, const mx_geom *geoms) {
    unsigned long long h = 1469598103934665603ULL;  // FNV-1a
    auto mix = [&](long long v) {
        for (int b = 0; b < 8; b++) {
            h ^= (unsigned long long)((v >> (8 * b)) & 0xff);
            h *= 1099511628211ULL;
        }
    };
    for (int b = 0; b < nbox; b++)
        for (int d = 0; d < 3; d++) {
            mix(geoms[b].n[d]);
            mix(geoms[b].lo[d]);
            mix(geoms[b].hi[d]);
        }
    mx_geom k = {};
    k.n[0] = nbox;
    k.n[1] = int(h & 0x7fffffff);
    k.n[2] = int((h >> 32) & 0x7fffffff);
    return k;
}

void store(mx_ctx *c, int op, int prec, const mx_geom *g, const mx_opts &cur, double ms) {
    mx_ctx::Tune t;
    t.op = op;
    t.prec = prec;
    for (int d = 0; d < 3; d++) {
        t.n[d] = g->n[d];
        t.lo[d] = g->lo[d];
        t.hi[d] = g->hi[d];
    }
    t.nu1 = cur.nu1;
    t.nu2 = cur.nu2;
    t.fused = cur.fused;
    t.tile_z = cur.tile_z;
    t.smoother = cur.smoother;
    t.ms = ms;
    for (auto &e : c->tune)
        if (same_key(e, op, prec, g)) {
            e = t;
            return;
        }
    c->tune.push_back(t);
}

const int NU_CAND[][2] = {{2, 2}, {1, 1}, {2, 1}, {1, 2}, {3, 2}, {2, 3}, {3, 3}, {4, 4}};

}  // namespace

void tune_apply_batch(const mx_ctx *c, int nbox, const mx_geom *geoms, mx_opts &o) {
    if (o.nu1 != 0 || o.nu2 != 0) return;
    const mx_geom k = batch_key(nbox, geoms);
    if (const mx_ctx::Tune *t = find(c, TUNE_BATCH, o.prec, &k)) {
        o.nu1 = t->nu1;
        o.nu2 = t->nu2;
    } else {
        o.nu1 = 2;
        o.nu2 = 2;
    }
}

void tune_apply(const mx_ctx *c, int op, const mx_geom *g, mx_opts &o) {
    if (o.nu1 != 0 || o.nu2 != 0) return;
    if (const mx_ctx::Tune *t = find(c, op, o.prec, g)) {
        o.nu1 = t->nu1;
        o.nu2 = t->nu2;
        o.fused = t->fused;
        o.tile_z = t->tile_z;
        if (op == MX_OP_NODAL) o.smoother = t->smoother;
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
    out->smoother = t->smoother;
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
    for (const auto &nu : NU_CAND) {
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
    // 3'. the Chebyshev smoother (nodal) at the chosen tile depth: a step is one
    // pass over the nodes where a colour sweep is four, so its degrees run higher
    if (!st && have && op == MX_OP_NODAL && o.smoother == 0) {
        const int CH_CAND[][2] = {{1, 1}, {1, 2}, {2, 1}, {2, 2}, {1, 3}, {2, 3}, {3, 2}, {3, 3}};
        const mx_opts at = cur;
        for (const auto &nu : CH_CAND) {
            mx_opts cand = at;
            cand.smoother = 1;
            cand.nu1 = nu[0];
            cand.nu2 = nu[1];
            if ((st = consider(cand))) break;
        }
    }
    cudaStreamSynchronize(c->stream);
    release();
    if (st) return st;
    if (!have) return set_err(c, MX_ERR_NOCONV, "autotune: no candidate setting converged");

    store(c, op, o.prec, geom, cur, cur_ms);
    if (best) *best = cur;
    if (ms_best) *ms_best = cur_ms;
    return MX_OK;
}

extern "C" mx_status mx_autotune_batched(mx_ctx *c, int nbox, const mx_geom *geoms, const double *const *ux,
                                         const double *const *uy, const double *const *uz, const double *const *rho,
                                         const double *const *beta0, const double *const *sbar,
                                         const mx_opts *base, mx_opts *best, double *ms_best) {
    if (!c) return MX_ERR_ARG;
    if (nbox < 1 || !geoms || !ux || !uy || !uz || !rho || !beta0 || !sbar)
        return set_err(c, MX_ERR_ARG, "autotune_batched: nbox < 1 or a null array list");
    mx_opts o;
    if (base) o = *base;
    else mx_default_opts(&o);
    if (o.nu1 == 0 && o.nu2 == 0) o.nu1 = o.nu2 = 2;
    if (o.prec != MX_PREC_MIXED) return set_err(c, MX_ERR_ARG, "autotune_batched: batches run in mixed precision");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    // scratch copies of every box's velocity and phi
    std::vector<double *> u[3], phi(nbox, nullptr);
    std::vector<long long> len[3];
    for (int d = 0; d < 3; d++) {
        u[d].assign(nbox, nullptr);
        len[d].assign(nbox, 0);
    }
    auto release = [&]() {
        for (int b = 0; b < nbox; b++) {
            for (int d = 0; d < 3; d++)
                if (u[d][b]) cudaFree(u[d][b]);
            if (phi[b]) cudaFree(phi[b]);
        }
    };
    for (int b = 0; b < nbox; b++) {
        const long long n0 = geoms[b].n[0], n1 = geoms[b].n[1], n2 = geoms[b].n[2];
        if (n0 < 1 || n1 < 1 || n2 < 1 || !ux[b] || !uy[b] || !uz[b]) {
            release();
            return set_err(c, MX_ERR_ARG, "autotune_batched: bad box");
        }
        len[0][b] = (n0 + 1) * n1 * n2;
        len[1][b] = n0 * (n1 + 1) * n2;
        len[2][b] = n0 * n1 * (n2 + 1);
        bool ok = true;
        for (int d = 0; d < 3; d++) ok = ok && cudaMalloc(&u[d][b], sizeof(double) * len[d][b]) == cudaSuccess;
        ok = ok && cudaMalloc(&phi[b], sizeof(double) * n0 * n1 * n2) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            release();
            return set_err(c, MX_ERR_OOM, "autotune_batched: scratch allocation failed");
        }
    }
    const double *const *src[3] = {ux, uy, uz};
    std::vector<mx_info> infos(nbox);
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    auto run = [&](const mx_opts &cand, double &ms, int &vc) -> mx_status {
        for (int rep = 0; rep < 2; rep++) {
            for (int b = 0; b < nbox; b++)
                for (int d = 0; d < 3; d++)
                    if (cudaMemcpyAsync(u[d][b], src[d][b], sizeof(double) * len[d][b], cudaMemcpyDeviceToDevice,
                                        c->stream) != cudaSuccess)
                        return set_err(c, MX_ERR_CUDA, "autotune_batched: copy failed");
            cudaEventRecord(t0, c->stream);
            const mx_status st = mx_mac_project_batched(c, nbox, geoms, u[0].data(), u[1].data(), u[2].data(), rho,
                                                        beta0, sbar, phi.data(), &cand, infos.data());
            cudaEventRecord(t1, c->stream);
            if (st != MX_OK) return st;
            for (int b = 0; b < nbox; b++)
                if (infos[b].status != MX_OK) return MX_ERR_NOCONV;
        }
        cudaEventSynchronize(t1);
        float f = 0.f;
        cudaEventElapsedTime(&f, t0, t1);
        ms = f;
        vc = 0;
        for (int b = 0; b < nbox; b++) vc = std::max(vc, infos[b].vcycles);
        return MX_OK;
    };
    mx_opts cur = o;
    double cur_ms = 0.0;
    int cur_vc = 0;
    bool have = false;
    mx_status st = MX_OK;
    for (const auto &nu : NU_CAND) {
        mx_opts cand = o;
        cand.nu1 = nu[0];
        cand.nu2 = nu[1];
        if (have) cand.max_outer = cand.max_vcycles = std::min(o.max_vcycles, 3 * cur_vc + 4);
        double ms;
        int vc;
        const mx_status r = run(cand, ms, vc);
        if (r == MX_ERR_NOCONV) continue;
        if (r != MX_OK) {
            st = r;
            break;
        }
        if (!have || ms < cur_ms) {
            cand.max_outer = o.max_outer;
            cand.max_vcycles = o.max_vcycles;
            cur = cand;
            cur_ms = ms;
            cur_vc = vc;
            have = true;
        }
    }
    cudaStreamSynchronize(c->stream);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    release();
    if (st) return st;
    if (!have) return set_err(c, MX_ERR_NOCONV, "autotune_batched: no candidate setting converged");
    const mx_geom k = batch_key(nbox, geoms);
    store(c, TUNE_BATCH, o.prec, &k, cur, cur_ms);
    if (best) *best = cur;
    if (ms_best) *ms_best = cur_ms;
    return MX_OK;
}
