// MAC projection driver: workspace plans, the V-cycle, the FP64
// iterative-refinement loop (FP32 V-cycles for the correction, FP64 residual
// and accumulation), optional CUDA-graph execution of that loop, and the
// mx_mac_project / mx_apply_op / mx_residual entry points.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mx_coarse.cuh"
#include "mx_krylov.cuh"
#include "mx_rbgs.cuh"
#include "mx_solver.cuh"
#include "mx_stencil.cuh"

// implemented with the nodal kernels
mx_status nodal_apply(mx_ctx *c, const mx_geom *geom, int prec, const double *rho, const double *beta0,
                      const double *phi, const double *f, double *out, double *rnorm);
void destroy_nodal_plans(mx_ctx *c);
void destroy_batch_plan(mx_ctx *c);
void destroy_radial_plans(mx_ctx *c);
void destroy_split_scratch(mx_ctx *c);
void destroy_comp_plan(mx_ctx *c);

// ------------------------------------------------------------------------------
// plans

template <typename T>
static void carve_level(Bump &b, Level<T> &L, const DGeom &g, bool coefs, bool fe) {
    L.g = g;
    if (coefs) {
        L.bx = b.take<T>(g.N);
        L.by = b.take<T>(g.N);
        L.bz = b.take<T>(g.N);
        L.hx = gper(g, 0) ? nullptr : b.take<T>((size_t)g.n[1] * g.n[2]);
        L.hy = gper(g, 1) ? nullptr : b.take<T>((size_t)g.n[0] * g.n[2]);
        L.hz = gper(g, 2) ? nullptr : b.take<T>((size_t)g.n[0] * g.n[1]);
    } else {
        L.bx = L.by = L.bz = L.hx = L.hy = L.hz = nullptr;
    }
    L.e2 = nullptr;
    if (fe) {
        L.f = b.take<T>(g.N);
        L.e = b.take<T>(g.N);
        L.e2 = b.take<T>(g.N);
    } else {
        L.f = L.e = L.e2 = nullptr;
    }
}

template <typename T>
static void carve_hier(Bump &b, Hier<T> &H, const DGeom *gs, int nl, bool level0_coefs) {
    H.nlev = nl;
    for (int l = 0; l < nl; l++) carve_level(b, H.lev[l], gs[l], l > 0 || level0_coefs, true);
    H.bot_scratch = b.take<T>(7 * (size_t)gs[nl - 1].N);
}

static void carve_plan(Bump &b, MacPlan &P) {
    DGeom gs[MX_MAXLEV];
    const int nl = mac_levels(P.g, gs);
    const DGeom &g = P.g;
    if (P.prec == MX_PREC_MIXED) {
        carve_hier(b, P.H32, gs, nl, true);
        DFArrays &D = P.D;
        D.bxl = b.take<float>(g.N);
        D.byl = b.take<float>(g.N);
        D.bzl = b.take<float>(g.N);
        D.hxl = gper(g, 0) ? nullptr : b.take<float>((size_t)g.n[1] * g.n[2]);
        D.hyl = gper(g, 1) ? nullptr : b.take<float>((size_t)g.n[0] * g.n[2]);
        D.hzl = gper(g, 2) ? nullptr : b.take<float>((size_t)g.n[0] * g.n[1]);
        D.fh = b.take<float>(g.N);
        D.fl = b.take<float>(g.N);
        D.ph = b.take<float>(g.N);
        D.pl = b.take<float>(g.N);
        D.ph2 = b.take<float>(g.N);
        D.pl2 = b.take<float>(g.N);
        D.b0h = b.take<float>(g.N);
        D.b0l = b.take<float>(g.N);
        P.tmp32 = b.take<float>(g.N);
        P.H64.nlev = 0;
        P.L64 = Level<double>{};
        P.L64.g = g;
    } else {
        carve_level(b, P.L64, g, true, true);
        carve_hier(b, P.H64, gs, nl, false);
        Level<double> &l0 = P.H64.lev[0];
        l0.bx = P.L64.bx; l0.by = P.L64.by; l0.bz = P.L64.bz;
        l0.hx = P.L64.hx; l0.hy = P.L64.hy; l0.hz = P.L64.hz;
        P.H32.nlev = 0;
    }
    P.Q.x = b.take<double>(g.N);
    P.Q.y = b.take<double>(g.N);
    P.Q.z = b.take<double>(g.N);
    P.Q.hx = gper(g, 0) ? nullptr : b.take<double>((size_t)g.n[1] * g.n[2]);
    P.Q.hy = gper(g, 1) ? nullptr : b.take<double>((size_t)g.n[0] * g.n[2]);
    P.Q.hz = gper(g, 2) ? nullptr : b.take<double>((size_t)g.n[0] * g.n[1]);
}

static bool same_geom(const DGeom &a, const DGeom &b) {
    for (int d = 0; d < 3; d++)
        if (a.n[d] != b.n[d] || a.lo[d] != b.lo[d] || a.hi[d] != b.hi[d]) return false;
    return a.h == b.h;
}

void free_mac_plan(MacPlan *p) {
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->mem) cudaFree(p->mem);
    if (p->kry_mem) cudaFree(p->kry_mem);
    delete p;
}

// A plan owned by the caller (not in the context's cache).
MacPlan *create_mac_plan(mx_ctx *c, const DGeom &g, int prec, mx_status *st) {
    *st = MX_OK;
    MacPlan *P = new MacPlan();
    P->g = g;
    P->prec = prec;
    Bump dry{nullptr, 0};
    carve_plan(dry, *P);
    P->bytes = dry.off + 256;
    if (cudaMalloc(&P->mem, P->bytes) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        *st = set_err(c, MX_ERR_OOM, "plan workspace cudaMalloc failed");
        return nullptr;
    }
    Bump real{(char *)P->mem, 0};
    carve_plan(real, *P);
    return P;
}

mx_status ensure_partials(mx_ctx *c, long long nblocks) {
    if (nblocks <= c->max_partials) return MX_OK;
    cudaStreamSynchronize(c->stream);
    cudaFree(c->partials);
    c->partials = nullptr;
    if (cudaMalloc(&c->partials, sizeof(double) * 3 * nblocks) != cudaSuccess) {
        cudaGetLastError();
        c->max_partials = 0;
        return set_err(c, MX_ERR_OOM, "reduction scratch cudaMalloc failed");
    }
    c->max_partials = int(nblocks);
    for (MacPlan *p : c->plans)  // graphs captured the old scratch pointer
        if (p->graph) {
            cudaGraphExecDestroy(p->graph);
            p->graph = nullptr;
        }
    return MX_OK;
}

MacPlan *get_mac_plan(mx_ctx *c, const DGeom &g, int prec, mx_status *st) {
    *st = ensure_partials(c, std::max<long long>(std::max(std::max(stencil_blocks(g), kry_dir_blocks(g)), red_blocks(g.N)),
                                                 std::max(df_resid_blocks(g), df_resid_parts(g))));
    if (*st) return nullptr;
    for (MacPlan *p : c->plans)
        if (p->prec == prec && same_geom(p->g, g)) {
            p->last_use = ++c->use_counter;
            return p;
        }
    // keep at most 4 plans: evict the least recently used
    if (c->plans.size() >= 4) {
        auto it = std::min_element(c->plans.begin(), c->plans.end(),
                                   [](MacPlan *a, MacPlan *b) { return a->last_use < b->last_use; });
        cudaStreamSynchronize(c->stream);
        free_mac_plan(*it);
        c->plans.erase(it);
    }
    MacPlan *P = create_mac_plan(c, g, prec, st);
    if (!P) return nullptr;
    P->last_use = ++c->use_counter;
    c->plans.push_back(P);
    return P;
}

void destroy_plans(mx_ctx *c) {
    for (MacPlan *p : c->plans) free_mac_plan(p);
    c->plans.clear();
    destroy_nodal_plans(c);
    destroy_batch_plan(c);
    destroy_radial_plans(c);
    destroy_split_scratch(c);
    destroy_comp_plan(c);
}

// ------------------------------------------------------------------------------
// V-cycle on the correction equation L e = r (level-0 f holds r, e is zeroed here)

// V-cycle on the correction equation L e = r (level-0 f holds r).
//  * levels of >= FUSED_MIN_CELLS cells (FP32, fused = 1): single-pass sweeps
//    ping-ponging between e and e2; the first pre-sweep starts from e = 0
//    without reading it and the first post-sweep applies the prolongation on
//    load; the first output buffer is chosen so that the result ends in e;
//  * other levels above the coarse end: two-pass colour kernels in place;
//  * the coarse end (levels of <= COARSE_MAX_CELLS cells, down to the bottom):
//    one single-CTA kernel; without such a level, a BiCGStab bottom kernel.
constexpr long long FUSED_MIN_CELLS = 1LL << 18;

template <typename T>
int coarse_start(const Hier<T> &H) {
    for (int l = 0; l < H.nlev; l++)
        if (H.lev[l].g.N <= COARSE_MAX_CELLS && coarse_fits(&H.lev[l], H.nlev - l)) return l;
    return H.nlev;
}

template <typename T>
void vcycle(cudaStream_t s, Hier<T> &H, int nu1, int nu2, int bot_iters, int singular, mx_ctx *pc, int fused,
            int zcap) {
    const int nl = H.nlev;
    const int lc = coarse_start(H);
    const int ldown = lc < nl ? lc : nl - 1;  // levels with their own kernels
    const bool can_fuse = sizeof(T) == sizeof(float) && fused && nu1 >= 1 && nu2 >= 1;
    auto is_fused = [&](int l) { return can_fuse && H.lev[l].g.N >= FUSED_MIN_CELLS && rbgs_fused_ok(H.lev[l].g); };
    T *cur[MX_MAXLEV];
    for (int l = 0; l < ldown; l++) {
        Level<T> &L = H.lev[l];
        if (l == 0) prof_begin(pc, s, MX_PH_SMOOTH_FINE);
        if (is_fused(l)) {
            float *bufs[2] = {(float *)L.e, (float *)L.e2};
            int w = ((nu1 + nu2) % 2 == 1) ? 0 : 1;
            const float *in = nullptr;
            for (int q = 0; q < nu1; q++) {
                k_rbgs_fused(s, *(Level<float> *)&L, in, bufs[w], q == 0 ? RB_ZERO : RB_PLAIN, nullptr);
                in = bufs[w];
                w ^= 1;
            }
            cur[l] = (T *)in;
        } else {
            // the first red pass starts from e = 0 without reading e
            if (nu1 == 0) cudaMemsetAsync(L.e, 0, sizeof(T) * L.g.N, s);
            for (int q = 0; q < nu1; q++) {
                k_rbgs(s, L, 0, q == 0, zcap);
                k_rbgs(s, L, 1, 0, zcap);
            }
            cur[l] = L.e;
        }
        if (l == 0) {
            prof_end(pc, s, MX_PH_SMOOTH_FINE, is_fused(0) ? nu1 : 2 * nu1);
            prof_begin(pc, s, MX_PH_RESTRICT_FINE);
        }
        Level<T> Lc = L;
        Lc.e = cur[l];
        k_resid_restrict(s, Lc, H.lev[l + 1], zcap);
        if (l == 0) {
            prof_end(pc, s, MX_PH_RESTRICT_FINE, 1);
            prof_begin(pc, s, MX_PH_COARSE);  // everything below the finest level
        }
    }
    if (ldown == 0) prof_begin(pc, s, MX_PH_COARSE);
    if (lc < nl) k_coarse_vcycle(s, &H.lev[lc], nl - lc, nu1, nu2, bot_iters, singular);
    else k_bottom(s, H.lev[nl - 1], H.bot_scratch, bot_iters, singular);
    if (ldown == 0) prof_end(pc, s, MX_PH_COARSE, 1);
    for (int l = ldown - 1; l >= 0; l--) {
        Level<T> &L = H.lev[l];
        if (l == 0) {
            prof_end(pc, s, MX_PH_COARSE, 0);
            prof_begin(pc, s, MX_PH_SMOOTH_FINE);
        }
        if (is_fused(l)) {
            const float *in = (const float *)cur[l];
            float *out = (float *)(cur[l] == L.e ? L.e2 : L.e);
            for (int q = 0; q < nu2; q++) {
                k_rbgs_fused(s, *(Level<float> *)&L, in, out, q == 0 ? RB_PROLONG : RB_PLAIN,
                             q == 0 ? (const Level<float> *)&H.lev[l + 1] : nullptr);
                in = out;
                out = (out == (float *)L.e) ? (float *)L.e2 : (float *)L.e;
            }
        } else {
            k_prolong(s, H.lev[l + 1], L, zcap);
            for (int q = 0; q < nu2; q++) {
                k_rbgs(s, L, 0, 0, zcap);
                k_rbgs(s, L, 1, 0, zcap);
            }
        }
        if (l == 0) prof_end(pc, s, MX_PH_SMOOTH_FINE, is_fused(0) ? nu2 : 1 + 2 * nu2);
    }
}
template int coarse_start<float>(const Hier<float> &);
template void vcycle<float>(cudaStream_t, Hier<float> &, int, int, int, int, mx_ctx *, int, int);
template void vcycle<double>(cudaStream_t, Hier<double> &, int, int, int, int, mx_ctx *, int, int);

template <typename T>
static void build_hierarchy(cudaStream_t s, Hier<T> &H) {
    for (int l = 0; l + 1 < H.nlev; l++) k_coarsen_coeffs(s, H.lev[l], H.lev[l + 1]);
}

// One refinement iteration after the residual: V-cycle, update, next residual.
// Mixed precision: FP32 V-cycle, double-float update and residual.
static void ir_body(cudaStream_t s, mx_ctx *c, MacPlan &P, Hier<float> &H, const mx_opts &o, int singular, int nb,
                    mx_ctx *pc) {
    vcycle(s, H, o.nu1, o.nu2, o.bottom_iters, singular, pc, o.fused, o.tile_z ? o.tile_z : 8);
    prof_begin(pc, s, MX_PH_RESID64);  // update phi += scale e fused with the next residual
    const int np = k_df_resid(s, H.lev[0], P.D, H.lev[0].e, c->state, c->partials);
    k_finalize_residual(s, c->partials, np, c->state, 1);
    prof_end(pc, s, MX_PH_RESID64, 2);
}
// One FCG(1) iteration after the residual (mx_krylov.cu): V-cycle, conjugate
// direction and line-search step, phi += t p fused with the next residual.
static void fcg_body(cudaStream_t s, mx_ctx *c, MacPlan &P, Hier<float> &H, const mx_opts &o, int singular,
                     mx_ctx *pc) {
    vcycle(s, H, o.nu1, o.nu2, o.bottom_iters, singular, pc, o.fused, o.tile_z ? o.tile_z : 8);
    Level<float> &L0 = H.lev[0];
    prof_begin(pc, s, MX_PH_UPDATE);
    k_kry_dot(s, P.g.N, L0.e, P.kq, c->state, c->partials);
    k_kry_dir(s, L0, L0.e, P.kp0, P.kp1, P.kq, c->state, c->partials);
    prof_end(pc, s, MX_PH_UPDATE, 4);
    prof_begin(pc, s, MX_PH_RESID64);
    const int np = k_df_resid(s, L0, P.D, P.kp0, c->state, c->partials, P.kp1);
    k_finalize_residual(s, c->partials, np, c->state, 1);
    prof_end(pc, s, MX_PH_RESID64, 2);
}
// Plain FP64: FP64 V-cycle, FP64 update and residual.
static void ir_body(cudaStream_t s, mx_ctx *c, MacPlan &P, Hier<double> &H, const mx_opts &o, int singular, int nb,
                    mx_ctx *pc, double *phi) {
    vcycle(s, H, o.nu1, o.nu2, o.bottom_iters, singular, pc, 0, o.tile_z ? o.tile_z : 8);
    prof_begin(pc, s, MX_PH_UPDATE);
    k_update<double>(s, P.g, phi, H.lev[0].e, c->state);
    prof_end(pc, s, MX_PH_UPDATE, 1);
    prof_begin(pc, s, MX_PH_RESID64);
    k_residual64<double>(s, P.L64, phi, P.L64.f, H.lev[0].f, c->state, c->partials, nb);
    k_finalize_residual(s, c->partials, nb, c->state);
    prof_end(pc, s, MX_PH_RESID64, 2);
}

template <typename T>
static void ir_first_residual(cudaStream_t s, mx_ctx *c, MacPlan &P, Hier<T> &H, double *phi, int nb, int zero_phi);
template <>
void ir_first_residual<float>(cudaStream_t s, mx_ctx *c, MacPlan &P, Hier<float> &H, double *, int nb, int zero_phi) {
    (void)nb;
    int np = df_resid_blocks(P.g);
    if (zero_phi) k_df_resid_zero(s, H.lev[0], P.D, c->state, c->partials);  // r = f
    else np = k_df_resid(s, H.lev[0], P.D, nullptr, c->state, c->partials);
    k_finalize_residual(s, c->partials, np, c->state, 1);
}
template <>
void ir_first_residual<double>(cudaStream_t s, mx_ctx *c, MacPlan &P, Hier<double> &H, double *phi, int nb, int) {
    k_residual64<double>(s, P.L64, phi, P.L64.f, H.lev[0].f, c->state, c->partials, nb);
    k_finalize_residual(s, c->partials, nb, c->state);
}

static void ir_step(cudaStream_t s, mx_ctx *c, MacPlan &P, Hier<float> &H, double *, const mx_opts &o, int singular,
                    int nb, mx_ctx *pc) {
    if (o.krylov) fcg_body(s, c, P, H, o, singular, pc);
    else ir_body(s, c, P, H, o, singular, nb, pc);
}
static void ir_step(cudaStream_t s, mx_ctx *c, MacPlan &P, Hier<double> &H, double *phi, const mx_opts &o,
                    int singular, int nb, mx_ctx *pc) {
    ir_body(s, c, P, H, o, singular, nb, pc, phi);
}

// Conditional-while graph of the refinement loop: the finalize kernel of each
// iteration sets the loop condition from the FP64 residual.
__global__ void set_cond_kernel(cudaGraphConditionalHandle h, const SolveState *st) {
    cudaGraphSetConditional(h, st->done ? 0u : 1u);
}

mx_status capture_while_graph(mx_ctx *c, cudaGraphExec_t *exec, const std::function<void(cudaStream_t)> &body) {
    cudaGraph_t graph;
    MX_CUDA(c, cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess) {
        cudaGraph_t inner = cp.conditional.phGraph_out[0];
        cudaStream_t cs;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            e = cudaStreamBeginCaptureToGraph(cs, inner, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                body(cs);
                set_cond_kernel<<<1, 1, 0, cs>>>(handle, c->state);
                cudaGraph_t captured;
                e = cudaStreamEndCapture(cs, &captured);
            }
            cudaStreamDestroy(cs);
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *exec = nullptr;
        return set_err(c, MX_ERR_CUDA, std::string("refinement-loop graph failed: ") + cudaGetErrorString(e));
    }
    return MX_OK;
}

template <typename T>
static mx_status run_loop_graph(mx_ctx *c, MacPlan &P, Hier<T> &H, double *phi, const mx_opts &o, int singular, int nb) {
    cudaStream_t s = c->stream;
    // the FP64 loop updates phi in place; the mixed loop never touches it
    const void *kphi = sizeof(T) == sizeof(double) ? (const void *)phi : nullptr;
    if (!P.graph || P.graph_phi != kphi || P.graph_nu1 != o.nu1 || P.graph_nu2 != o.nu2 ||
        P.graph_bot != o.bottom_iters || P.graph_fused != o.fused || P.graph_tilez != o.tile_z ||
        P.graph_krylov != o.krylov) {
        if (P.graph) {
            cudaGraphExecDestroy(P.graph);
            P.graph = nullptr;
        }
        mx_status st = capture_while_graph(
            c, &P.graph, [&](cudaStream_t cs) { ir_step(cs, c, P, H, phi, o, singular, nb, nullptr); });
        if (st) return st;
        P.graph_phi = kphi;
        P.graph_nu1 = o.nu1;
        P.graph_nu2 = o.nu2;
        P.graph_bot = o.bottom_iters;
        P.graph_fused = o.fused;
        P.graph_tilez = o.tile_z;
        P.graph_krylov = o.krylov;
    }
    // the while node runs its body while the condition is 1 (the host checked
    // that the first residual asked for a V-cycle)
    MX_CUDA(c, cudaGraphLaunch(P.graph, s));
    return MX_OK;
}

template <typename T>
static mx_status run_ir(mx_ctx *c, MacPlan &P, Hier<T> &H, double *phi, const mx_opts &o, int singular) {
    cudaStream_t s = c->stream;
    const int nb = stencil_blocks(P.g);
    prof_begin(c, s, MX_PH_RESID64);
    ir_first_residual<T>(s, c, P, H, phi, nb, !o.use_initial_guess);
    prof_end(c, s, MX_PH_RESID64, 2);
    if (o.use_graph && !c->prof) {
        // the loop is entered unconditionally by the while node; a first
        // residual that already meets the tolerance is handled on the host
        MX_CUDA(c, cudaMemcpyAsync(c->hstate, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        MX_CUDA(c, cudaStreamSynchronize(s));
        if (c->hstate->done) return MX_OK;
        return run_loop_graph<T>(c, P, H, phi, o, singular, nb);
    }
    for (;;) {
        MX_CUDA(c, cudaMemcpyAsync(c->hstate, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        MX_CUDA(c, cudaStreamSynchronize(s));
        if (c->hstate->done) break;
        ir_step(s, c, P, H, phi, o, singular, nb, c);
        prof_flush(c);
    }
    return MX_OK;
}

// ------------------------------------------------------------------------------

mx_status check_opts(mx_ctx *c, const mx_opts *in, mx_opts &o) {
    if (in) o = *in;
    else mx_default_opts(&o);
    if (!(o.rel_tol >= 0.0) || o.max_outer < 0 || o.max_vcycles < 0 || (o.prec != MX_PREC_FP64 && o.prec != MX_PREC_MIXED) ||
        o.nu1 < 0 || o.nu2 < 0 || o.nu1 > 16 || o.nu2 > 16 || o.bottom_iters < 1 || o.bottom_iters > 100000 ||
        !(o.tile_z == 0 || o.tile_z == 1 || o.tile_z == 2 || o.tile_z == 4 || o.tile_z == 8 || o.tile_z == 16) ||
        (o.krylov != 0 && o.krylov != 1) || (o.smoother != 0 && o.smoother != 1))
        return set_err(c, MX_ERR_ARG, "invalid options");
    if (o.krylov && o.prec != MX_PREC_MIXED) return set_err(c, MX_ERR_ARG, "krylov = 1 needs prec = MX_PREC_MIXED");
    return MX_OK;
}

// FCG buffers of a mixed plan: two directions and q, N floats each
static mx_status ensure_krylov(mx_ctx *c, MacPlan &P) {
    if (P.kry_mem) return MX_OK;
    const size_t per = ((size_t)P.g.N * sizeof(float) + 255) & ~size_t(255);
    if (cudaMalloc(&P.kry_mem, 3 * per) != cudaSuccess) {
        cudaGetLastError();
        P.kry_mem = nullptr;
        return set_err(c, MX_ERR_OOM, "krylov buffers: cudaMalloc failed");
    }
    P.kp0 = P.kry_mem;
    P.kp1 = (float *)((char *)P.kry_mem + per);
    P.kq = (float *)((char *)P.kry_mem + 2 * per);
    return MX_OK;
}

void setup_coefficients(mx_ctx *c, MacPlan &P, const double *rho, const double *beta0) {
    setup_coefficients_on(c->stream, P, rho, beta0);
}

void setup_coefficients_on(cudaStream_t s, MacPlan &P, const double *rho, const double *beta0) {
    if (P.prec == MX_PREC_MIXED) {
        k_mac_coeffs_df(s, P.H32.lev[0], P.D, rho, beta0, &P.Q);
        build_hierarchy(s, P.H32);
    } else {
        k_mac_coeffs64(s, P.L64, rho, beta0, &P.Q);
        build_hierarchy(s, P.H64);
    }
}

extern "C" mx_status mx_mac_project(mx_ctx *c, const mx_geom *geom, double *ux, double *uy, double *uz,
                                    const double *rho, const double *beta0, const double *sbar, double *phi,
                                    const mx_opts *opts, mx_info *info) {
    if (!c) return MX_ERR_ARG;
    mx_status st = check_geom(c, geom, false);
    if (st) return st;
    if (!ux || !uy || !uz || !rho || !beta0 || !sbar || !phi) return set_err(c, MX_ERR_ARG, "mac_project: null array");
    mx_opts o;
    if ((st = check_opts(c, opts, o))) return st;
    if (o.smoother) return set_err(c, MX_ERR_ARG, "smoother = 1 (Chebyshev) is for nodal solves");
    tune_apply(c, MX_OP_MAC, geom, o);
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    const DGeom g = make_dgeom(geom);
    const int singular = geom_singular(g);
    MacPlan *P = get_mac_plan(c, g, o.prec, &st);
    if (!P) return st;
    if (o.krylov && (st = ensure_krylov(c, *P))) return st;
    cudaStream_t s = c->stream;
    const int nb = stencil_blocks(g);
    const int nbr = red_blocks(g.N);
    MX_CUDA(c, cudaEventRecord(c->ev0, s));

    // device state: tolerance and caps
    SolveState init = {};
    init.tol = o.rel_tol;
    init.maxit = std::min(o.max_outer, o.max_vcycles);
    init.kry_restart = 1;
    *c->hstate = init;
    MX_CUDA(c, cudaMemcpyAsync(c->state, c->hstate, sizeof(SolveState), cudaMemcpyHostToDevice, s));

    prof_begin(c, s, MX_PH_SETUP);
    setup_coefficients(c, *P, rho, beta0);
    // right-hand side f = D(beta0 U) - beta0 Sbar, mean removal, norms
    // (mixed: double-float f into the plan's (fh, fl); FP64: f into L64.f)
    double *f64 = P->L64.f;
    if (o.prec == MX_PREC_MIXED) k_mac_rhs_df(s, g, ux, uy, uz, sbar, P->D, c->partials);
    else k_mac_rhs(s, g, ux, uy, uz, beta0, sbar, f64, c->partials, nb);
    k_finalize_rhs(s, c->partials, nb, c->state, g.N, singular && o.remove_mean, 0);
    if (singular && !o.remove_mean) {
        MX_CUDA(c, cudaMemcpyAsync(c->hstate, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        MX_CUDA(c, cudaStreamSynchronize(s));
        if (std::fabs(c->hstate->aux) > 1e-12 * c->hstate->fnorm) {
            if (info) {
                std::memset(info, 0, sizeof(*info));
                info->status = MX_ERR_INCOMPAT;
            }
            return set_err(c, MX_ERR_INCOMPAT, "singular problem: right-hand side has non-zero mean and remove_mean = 0");
        }
    }
    if (o.prec == MX_PREC_MIXED) {
        k_sub_mean_scale(s, g, c->state, P->D, c->partials, nbr);
        if (o.use_initial_guess) {
            k_df_from_double(s, g.N, phi, P->D);
        } else {
            MX_CUDA(c, cudaMemsetAsync(P->D.ph, 0, sizeof(float) * g.N, s));
            MX_CUDA(c, cudaMemsetAsync(P->D.pl, 0, sizeof(float) * g.N, s));
        }
    } else {
        k_sub_mean_norm(s, g, f64, c->state, c->partials, nbr);
        if (!o.use_initial_guess) MX_CUDA(c, cudaMemsetAsync(phi, 0, sizeof(double) * g.N, s));
    }
    k_finalize_rhs(s, c->partials, nbr, c->state, g.N, 0, 1);
    prof_end(c, s, MX_PH_SETUP, 0);

    if (o.prec == MX_PREC_MIXED) st = run_ir<float>(c, *P, P->H32, phi, o, singular);
    else st = run_ir<double>(c, *P, P->H64, phi, o, singular);
    if (st) return st;
    prof_begin(c, s, MX_PH_FINISH);
    // mixed: phi from its double-float form, with the partial sums of phi
    if (o.prec == MX_PREC_MIXED) k_df_final(s, g.N, P->D, c->state, phi, singular ? c->partials : nullptr);
    if (singular) {  // normalise mean(phi) = 0
        if (o.prec != MX_PREC_MIXED) k_sum_partials(s, g, phi, c->partials, nbr);
        k_finalize_sum(s, c->partials, nbr, &c->state->aux, 1.0 / double(g.N));
        k_sub_scalar(s, g.N, phi, &c->state->aux);
    }
    k_mac_correct(s, g, P->Q, phi, ux, uy, uz);
    if (o.prec == MX_PREC_MIXED) k_mac_divcheck_df(s, g, ux, uy, uz, sbar, P->D, c->state, c->partials);
    else k_mac_divcheck(s, g, ux, uy, uz, beta0, sbar, c->state, c->partials, nb);
    k_finalize_max(s, c->partials, nb, &c->state->div_err);
    prof_end(c, s, MX_PH_FINISH, (singular ? 3 : 0) + (o.prec == MX_PREC_MIXED ? 5 : 4));
    MX_CUDA(c, cudaEventRecord(c->ev1, s));
    MX_CUDA(c, cudaMemcpyAsync(c->hstate, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    MX_CUDA(c, cudaStreamSynchronize(s));
    MX_CUDA(c, cudaGetLastError());
    const SolveState &hs = *c->hstate;
    if (info) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        info->outer_iters = hs.iter;
        info->vcycles = hs.iter;
        info->rel_resid = hs.fnorm > 0 ? hs.rnorm / hs.fnorm : hs.rnorm;
        info->rel_resid_l2 = hs.fnorm2 > 0 ? hs.rnorm2 / hs.fnorm2 : hs.rnorm2;
        info->div_err_linf = hs.div_err;
        info->rhs_mean_removed = hs.mean;
        info->rhs_linf = hs.fnorm;
        info->ms = ms;
        info->status = hs.status;
    }
    if (hs.status != MX_OK) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "no convergence: relative residual %.3e after %d V-cycles", hs.rnorm / (hs.fnorm > 0 ? hs.fnorm : 1.0), hs.iter);
        return set_err(c, (mx_status)hs.status, buf);
    }
    return MX_OK;
}

// ------------------------------------------------------------------------------
// operator and residual entry points

__global__ void resid_combine_kernel(const double *f, const float *lphi, double *r, long long n, double *part) {
    double mx = 0.0, s2 = 0.0, s1 = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const float v = float(f[q]) - lphi[q];
        r[q] = double(v);
        mx = nmax(mx, fabs(double(v)));
        s2 += double(v) * double(v);
        s1 += double(v);
    }
    block_red3(mx, s2, s1);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = mx;
        part[3 * blockIdx.x + 1] = s2;
        part[3 * blockIdx.x + 2] = s1;
    }
}

static mx_status mac_apply_or_residual(mx_ctx *c, const mx_geom *geom, int prec, const double *rho, const double *beta0,
                                       const double *phi, const double *f, double *out, double *rnorm) {
    const DGeom g = make_dgeom(geom);
    mx_status st;
    MacPlan *P = get_mac_plan(c, g, prec, &st);
    if (!P) return st;
    cudaStream_t s = c->stream;
    if (prec == MX_PREC_FP64) k_mac_coeffs64(s, P->L64, rho, beta0);
    else k_mac_coeffs_df(s, P->H32.lev[0], P->D, rho, beta0);
    if (prec == MX_PREC_FP64) {
        if (f) {
            const int nb = stencil_blocks(g);
            k_residual_plain(s, P->L64, phi, f, out, c->partials, nb);
            if (rnorm) k_finalize_max(s, c->partials, nb, &c->state->rnorm);
        } else {
            k_apply<double>(s, P->L64, phi, out);
        }
    } else {
        Level<float> &l0 = P->H32.lev[0];
        k_cast<float>(s, g.N, phi, l0.e);
        k_apply<float>(s, l0, l0.e, P->tmp32);
        if (f) {
            const int nbr = red_blocks(g.N);
            resid_combine_kernel<<<nbr, 256, 0, s>>>(f, P->tmp32, out, g.N, c->partials);
            if (rnorm) k_finalize_max(s, c->partials, nbr, &c->state->rnorm);
        } else {
            k_uncast<float>(s, g.N, P->tmp32, out);
        }
    }
    if (rnorm) {
        MX_CUDA(c, cudaMemcpyAsync(c->hstate, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        MX_CUDA(c, cudaStreamSynchronize(s));
        *rnorm = c->hstate->rnorm;
    }
    MX_CUDA(c, cudaGetLastError());
    return MX_OK;
}

extern "C" mx_status mx_apply_op(mx_ctx *c, const mx_geom *geom, int op, int prec, const double *rho,
                                 const double *beta0, const double *phi, double *Lphi) {
    if (!c) return MX_ERR_ARG;
    const bool nodal = op == MX_OP_NODAL;
    if (op != MX_OP_MAC && !nodal) return set_err(c, MX_ERR_ARG, "unknown operator");
    if (prec != MX_PREC_FP64 && prec != MX_PREC_MIXED) return set_err(c, MX_ERR_ARG, "unknown precision");
    mx_status st = check_geom(c, geom, nodal);
    if (st) return st;
    if (!rho || !beta0 || !phi || !Lphi) return set_err(c, MX_ERR_ARG, "apply_op: null array");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    if (nodal) return nodal_apply(c, geom, prec, rho, beta0, phi, nullptr, Lphi, nullptr);
    return mac_apply_or_residual(c, geom, prec, rho, beta0, phi, nullptr, Lphi, nullptr);
}

extern "C" mx_status mx_residual(mx_ctx *c, const mx_geom *geom, int op, int prec, const double *rho,
                                 const double *beta0, const double *phi, const double *f, double *r, double *rnorm_linf) {
    if (!c) return MX_ERR_ARG;
    const bool nodal = op == MX_OP_NODAL;
    if (op != MX_OP_MAC && !nodal) return set_err(c, MX_ERR_ARG, "unknown operator");
    if (prec != MX_PREC_FP64 && prec != MX_PREC_MIXED) return set_err(c, MX_ERR_ARG, "unknown precision");
    mx_status st = check_geom(c, geom, nodal);
    if (st) return st;
    if (!rho || !beta0 || !phi || !f || !r) return set_err(c, MX_ERR_ARG, "residual: null array");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    if (nodal) return nodal_apply(c, geom, prec, rho, beta0, phi, f, r, rnorm_linf);
    return mac_apply_or_residual(c, geom, prec, rho, beta0, phi, f, r, rnorm_linf);
}
