// C ABI of the projection library: context, argument checks, workspace plans,
// the multigrid hierarchy and the iterative-refinement driver of the MAC solve.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>

#include "mx_coarse.cuh"
#include "mx_stencil.cuh"
#include "mx_solver.cuh"

mx_status set_err(mx_ctx *ctx, mx_status s, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return s;
}

DGeom make_dgeom(const mx_geom *g) {
    DGeom d;
    for (int a = 0; a < 3; a++) {
        d.n[a] = g->n[a];
        d.lo[a] = g->lo[a];
        d.hi[a] = g->hi[a];
    }
    d.nxy = (long long)g->n[0] * g->n[1];
    d.N = d.nxy * g->n[2];
    d.h = g->dx;
    return d;
}

bool geom_singular(const DGeom &g) {
    for (int a = 0; a < 3; a++)
        if (g.lo[a] == MX_BC_DIRICHLET || g.hi[a] == MX_BC_DIRICHLET) return false;
    return true;
}

mx_status check_geom(mx_ctx *ctx, const mx_geom *g, bool nodal) {
    if (!g) return set_err(ctx, MX_ERR_ARG, "geom is NULL");
    long long N = 1;
    for (int a = 0; a < 3; a++) {
        if (g->n[a] < 1) return set_err(ctx, MX_ERR_ARG, "cell counts must be >= 1");
        if (g->lo[a] < 0 || g->lo[a] > 2 || g->hi[a] < 0 || g->hi[a] > 2)
            return set_err(ctx, MX_ERR_ARG, "unknown boundary type");
        if ((g->lo[a] == MX_BC_PERIODIC) != (g->hi[a] == MX_BC_PERIODIC))
            return set_err(ctx, MX_ERR_ARG, "a periodic axis must be periodic on both sides");
        if (g->lo[a] == MX_BC_PERIODIC && (g->n[a] % 2 != 0))
            return set_err(ctx, MX_ERR_ARG, "periodic axes need an even cell count");
        if (nodal && (g->lo[a] == MX_BC_DIRICHLET || g->hi[a] == MX_BC_DIRICHLET))
            return set_err(ctx, MX_ERR_ARG, "the nodal projection supports periodic and wall boundaries only");
        if (nodal && g->n[a] < 2) return set_err(ctx, MX_ERR_ARG, "nodal: cell counts must be >= 2");
        N *= g->n[a];
    }
    if (!(g->dx > 0.0) || !std::isfinite(g->dx)) return set_err(ctx, MX_ERR_ARG, "dx must be positive");
    if (N >= (1LL << 31)) return set_err(ctx, MX_ERR_ARG, "grid too large (>= 2^31 cells)");
    if (nodal) {
        long long M = 1;
        for (int a = 0; a < 3; a++) M *= g->n[a] + (g->lo[a] == MX_BC_PERIODIC ? 0 : 1);
        if (M >= (1LL << 31)) return set_err(ctx, MX_ERR_ARG, "grid too large (>= 2^31 nodes)");
    }
    return MX_OK;
}

int mac_levels(const DGeom &g0, DGeom *out) {
    int nl = 0;
    out[nl++] = g0;
    for (;;) {
        const DGeom &g = out[nl - 1];
        bool ok = nl < MX_MAXLEV;
        for (int a = 0; a < 3; a++) ok = ok && (g.n[a] % 2 == 0) && g.n[a] >= 4;
        if (!ok) break;
        DGeom c = g;
        for (int a = 0; a < 3; a++) c.n[a] = g.n[a] / 2;
        c.nxy = (long long)c.n[0] * c.n[1];
        c.N = c.nxy * c.n[2];
        c.h = 2.0 * g.h;
        out[nl++] = c;
    }
    return nl;
}

// ------------------------------------------------------------------------------
// tracing

static cudaEvent_t pool_event(mx_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(mx_ctx *c, cudaStream_t s, int phase) {
    if (!c || !c->prof) return;
    mx_ctx::Mark m{phase, pool_event(c), pool_event(c), 0};
    cudaEventRecord(m.a, s);
    c->marks.push_back(m);
}

void prof_end(mx_ctx *c, cudaStream_t s, int phase, int nlaunch) {
    if (!c || !c->prof || c->marks.empty()) return;
    mx_ctx::Mark &m = c->marks.back();
    if (m.phase != phase) return;
    m.n = nlaunch;
    cudaEventRecord(m.b, s);
}

void prof_flush(mx_ctx *c) {
    if (!c || c->marks.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto &m : c->marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            c->prof_ms[m.phase] += ms;
            c->prof_n[m.phase] += m.n;
        } else {
            cudaGetLastError();
        }
        c->ev_pool.push_back(m.a);
        c->ev_pool.push_back(m.b);
    }
    c->marks.clear();
}

// ------------------------------------------------------------------------------
// context

extern "C" {

mx_status mx_create(mx_ctx **out, int device, void *stream) {
    if (!out) return MX_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return MX_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return MX_ERR_CUDA;
    mx_ctx *c = new mx_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    c->max_partials = 1 << 17;
    if (cudaMalloc(&c->state, sizeof(SolveState) * 4) != cudaSuccess ||
        cudaMallocHost(&c->hstate, sizeof(SolveState) * 4) != cudaSuccess ||
        cudaMalloc(&c->partials, sizeof(double) * 3 * c->max_partials) != cudaSuccess ||
        cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
        coarse_init() != cudaSuccess) {
        cudaGetLastError();
        mx_destroy(c);
        return MX_ERR_CUDA;
    }
    *out = c;
    return MX_OK;
}

mx_status mx_destroy(mx_ctx *c) {
    if (!c) return MX_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    destroy_plans(c);
    prof_flush(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->state) cudaFree(c->state);
    if (c->hstate) cudaFreeHost(c->hstate);
    if (c->partials) cudaFree(c->partials);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
    return MX_OK;
}

mx_status mx_set_stream(mx_ctx *c, void *stream) {
    if (!c) return MX_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return MX_OK;
}

const char *mx_last_error(const mx_ctx *c) { return c ? c->err.c_str() : "null context"; }

mx_status mx_profile_enable(mx_ctx *c, int enable) {
    if (!c) return MX_ERR_ARG;
    prof_flush(c);
    c->prof = enable != 0;
    return MX_OK;
}

mx_status mx_profile_read(mx_ctx *c, double *ms, long long *launches) {
    if (!c || !ms || !launches) return MX_ERR_ARG;
    prof_flush(c);
    for (int p = 0; p < MX_PH_COUNT; p++) {
        ms[p] = c->prof_ms[p];
        launches[p] = c->prof_n[p];
        c->prof_ms[p] = 0.0;
        c->prof_n[p] = 0;
    }
    return MX_OK;
}

void mx_default_opts(mx_opts *o) {
    if (!o) return;
    o->rel_tol = 1e-10;
    o->max_outer = 100;
    o->max_vcycles = 100;
    o->prec = MX_PREC_MIXED;
    o->remove_mean = 1;
    o->use_initial_guess = 0;
    o->use_graph = 1;
    o->nu1 = 2;
    o->nu2 = 2;
    o->bottom_iters = 200;
    o->fused = 0;
    o->tile_z = 0;
    o->krylov = 0;
    o->smoother = 0;
}

int mx_device_supported(int device) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return p.major == 10 && p.minor == 3;
}

mx_status mx_fill_base_state(mx_ctx *c, const mx_geom *geom, int spherical, const double *prof, int nr, double dr,
                             const double center[3], double *out) {
    if (!c) return MX_ERR_ARG;
    mx_status st = check_geom(c, geom, false);
    if (st) return st;
    if (!prof || !out) return set_err(c, MX_ERR_ARG, "fill: null array");
    DGeom g = make_dgeom(geom);
    if (spherical) {
        if (nr < 2 || !(dr > 0.0) || !center) return set_err(c, MX_ERR_ARG, "fill: spherical needs nr >= 2, dr > 0, center");
        k_fill(c->stream, g, 1, prof, nr, dr, center[0], center[1], center[2], out);
    } else {
        if (nr < g.n[2]) return set_err(c, MX_ERR_ARG, "fill: planar profile shorter than n[2]");
        k_fill(c->stream, g, 0, prof, nr, 0.0, 0.0, 0.0, 0.0, out);
    }
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

}  // extern "C"
