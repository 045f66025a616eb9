// Batched MAC projections: many independent boxes of uneven sizes (AMR-style
// patches; the paper runs one 64^3 grid per MPI task, Sec. 4.1) solved
// together.  Each phase of the refinement loop -- every red or black pass and
// every restriction / prolongation of a level index, the double-float
// residual with its update, and the coarse end of all V-cycles -- is ONE
// launch over a work list of (box, tile) entries covering all boxes, so the
// loop costs the same number of launches for 96 boxes as for one.  Each box
// keeps its own convergence state; a converged box's tiles return at once.
// The loop runs as a CUDA graph with a conditional while node that continues
// while any box is unconverged.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mx_coarse.cuh"
#include "mx_solver.cuh"
#include "mx_stencil.cuh"

struct WorkRange {
    int off = 0, n = 0;
};

struct BatchPlan {
    int nbox = 0;
    std::vector<DGeom> geoms;
    std::vector<MacPlan *> box;
    std::vector<int> lc;       // first level of each box's coarse end
    int maxdown = 0;           // deepest per-level phase over all boxes
    int march = 0;             // the double-float residual's work list is of z-march blocks
    // device-side descriptors
    void *mem = nullptr;
    Level<float> *d_levs = nullptr;  // [nbox * MX_MAXLEV]
    DFBox *d_df = nullptr;           // [nbox]
    void *d_cargs = nullptr;         // coarse argument blocks
    SolveState *d_st = nullptr;      // [nbox]
    SolveState *h_st = nullptr;      // pinned mirror
    int *d_off = nullptr, *d_cnt = nullptr;
    int4 *d_work = nullptr;
    std::vector<WorkRange> rb, rr, pr;  // per level index
    std::vector<int> rr_zcf;            // per level index: fine planes per restriction tile (0: coarse tiles)
    WorkRange df;
    int nparts = 0;
    size_t coarse_smem = 0;
    // graph of the loop
    cudaGraphExec_t graph = nullptr;
    int g_nu1 = -1, g_nu2 = -1, g_bot = -1;
    // side streams for the per-box setup and finish (small kernels of different
    // boxes overlap), each with its own slice of the reduction scratch
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_done;
    cudaEvent_t fork = nullptr;
    long long part_stride = 0;  // doubles per side stream in the partials
};

static void free_batch(BatchPlan *B) {
    if (!B) return;
    for (cudaStream_t q : B->side) cudaStreamDestroy(q);
    for (cudaEvent_t e : B->side_done) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    for (MacPlan *p : B->box) free_mac_plan(p);
    if (B->mem) cudaFree(B->mem);
    if (B->h_st) cudaFreeHost(B->h_st);
    delete B;
}

void destroy_batch_plan(mx_ctx *c) {
    free_batch(c->batch);
    c->batch = nullptr;
}

static bool same_geoms(const BatchPlan *B, int nbox, const DGeom *g) {
    if (!B || B->nbox != nbox) return false;
    for (int b = 0; b < nbox; b++) {
        const DGeom &a = B->geoms[b];
        for (int d = 0; d < 3; d++)
            if (a.n[d] != g[b].n[d] || a.lo[d] != g[b].lo[d] || a.hi[d] != g[b].hi[d]) return false;
        if (a.h != g[b].h) return false;
    }
    return true;
}

static void add_grid(std::vector<int4> &w, int box, dim3 grid) {
    for (unsigned z = 0; z < grid.z; z++)
        for (unsigned y = 0; y < grid.y; y++)
            for (unsigned x = 0; x < grid.x; x++) w.push_back(make_int4(box, int(x), int(y), int(z)));
}

static BatchPlan *build_batch(mx_ctx *c, int nbox, const DGeom *g, const mx_opts &o, mx_status *st) {
    BatchPlan *B = new BatchPlan();
    B->nbox = nbox;
    B->geoms.assign(g, g + nbox);
    for (int b = 0; b < nbox; b++) {
        MacPlan *P = create_mac_plan(c, g[b], MX_PREC_MIXED, st);
        if (!P) {
            free_batch(B);
            return nullptr;
        }
        B->box.push_back(P);
        const int lc = coarse_start(P->H32);
        if (lc >= P->H32.nlev) {
            *st = set_err(c, MX_ERR_ARG, "batched: a box has no coarse level of <= 4096 cells (odd sizes too large)");
            free_batch(B);
            return nullptr;
        }
        B->lc.push_back(lc);
        B->maxdown = std::max(B->maxdown, lc);
    }
    // work lists
    std::vector<int4> work;
    B->rb.resize(B->maxdown);
    B->rr.resize(B->maxdown);
    B->pr.resize(B->maxdown);
    B->rr_zcf.assign(B->maxdown, 0);
    for (int l = 0; l < B->maxdown; l++) {
        B->rb[l].off = int(work.size());
        for (int b = 0; b < nbox; b++)
            if (l < B->lc[b]) add_grid(work, b, rbgs_grid(B->box[b]->H32.lev[l].g, ZC));
        B->rb[l].n = int(work.size()) - B->rb[l].off;
        // residual + restriction: the fine-cell form when every box's level has even
        // extents, its fine planes per tile halved while the tiles fill the GPU less than
        // four times at four blocks per SM (as for a single box)
        bool even = true;
        for (int b = 0; b < nbox; b++)
            if (l < B->lc[b]) {
                const DGeom &gf = B->box[b]->H32.lev[l].g;
                even = even && gf.n[0] % 2 == 0 && gf.n[1] % 2 == 0 && gf.n[2] % 2 == 0;
            }
        int zcf = 0;
        if (even) {
            auto tiles = [&](int z) {
                long long t = 0;
                for (int b = 0; b < nbox; b++)
                    if (l < B->lc[b]) {
                        const dim3 gr = resid_restrict_fine_grid(B->box[b]->H32.lev[l].g, z);
                        t += (long long)gr.x * gr.y * gr.z;
                    }
                return t;
            };
            zcf = 16;
            while (zcf > 2 && tiles(zcf) < 4 * 4 * 152) zcf >>= 1;
        }
        B->rr_zcf[l] = zcf;
        B->rr[l].off = int(work.size());
        for (int b = 0; b < nbox; b++)
            if (l < B->lc[b])
                add_grid(work, b, zcf ? resid_restrict_fine_grid(B->box[b]->H32.lev[l].g, zcf)
                                      : stencil_grid(B->box[b]->H32.lev[l + 1].g));
        B->rr[l].n = int(work.size()) - B->rr[l].off;
        B->pr[l].off = int(work.size());
        for (int b = 0; b < nbox; b++)
            if (l < B->lc[b]) add_grid(work, b, stencil_grid(B->box[b]->H32.lev[l].g));
        B->pr[l].n = int(work.size()) - B->pr[l].off;
    }
    B->df.off = int(work.size());
    std::vector<int> off(nbox), cnt(nbox), zcs(nbox);
    B->march = 2;  // the residual as a z-march (2: with row chunks) when every box allows it
    for (int b = 0; b < nbox; b++) B->march = std::min(B->march, df_march_usable(g[b]));
    int parts = 0;
    for (int b = 0; b < nbox; b++) {
        const dim3 gr = df_resid_batch_grid(g[b], B->march, &zcs[b]);
        add_grid(work, b, gr);
        off[b] = parts;
        cnt[b] = int(gr.x * gr.y * gr.z);
        parts += cnt[b];
    }
    B->df.n = int(work.size()) - B->df.off;
    B->nparts = parts;
    // side streams: NSIDE slices of the partials, each large enough for any box
    constexpr int NSIDE = 8;
    long long maxblk = 0;
    for (int b = 0; b < nbox; b++) maxblk = std::max<long long>(maxblk, std::max(stencil_blocks(g[b]), red_blocks(g[b].N)));
    B->part_stride = 3 * maxblk;
    if ((*st = ensure_partials(c, std::max<long long>(std::max(parts, 152 * 8), NSIDE * maxblk)))) {
        free_batch(B);
        return nullptr;
    }
    B->side.resize(NSIDE, nullptr);
    B->side_done.resize(NSIDE, nullptr);
    bool ok = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int q = 0; q < NSIDE && ok; q++)
        ok = cudaStreamCreateWithFlags(&B->side[q], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&B->side_done[q], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        *st = set_err(c, MX_ERR_CUDA, "batched: side stream creation failed");
        free_batch(B);
        return nullptr;
    }
    // host copies of the descriptors
    std::vector<Level<float>> levs((size_t)nbox * MX_MAXLEV);
    std::vector<DFBox> dfb(nbox);
    const size_t cab = coarse_args_bytes();
    std::vector<char> cargs(cab * nbox);
    for (int b = 0; b < nbox; b++) {
        Hier<float> &H = B->box[b]->H32;
        for (int l = 0; l < H.nlev; l++) levs[(size_t)b * MX_MAXLEV + l] = H.lev[l];
        dfb[b].L0 = H.lev[0];
        dfb[b].D = B->box[b]->D;
        dfb[b].part_off = off[b];
        dfb[b].zc = zcs[b];
        const int lc = B->lc[b];
        coarse_fill_args(cargs.data() + cab * b, &H.lev[lc], H.nlev - lc, o.nu1, o.nu2, o.bottom_iters,
                         geom_singular(g[b]));
        B->coarse_smem = std::max(B->coarse_smem, coarse_smem_bytes_f(&H.lev[lc], H.nlev - lc));
    }
    Bump dry{nullptr, 0};
    auto carve = [&](Bump &bm) {
        B->d_levs = bm.take<Level<float>>(levs.size());
        B->d_df = bm.take<DFBox>(nbox);
        B->d_cargs = bm.take<char>(cargs.size());
        B->d_st = bm.take<SolveState>(nbox);
        B->d_off = bm.take<int>(nbox);
        B->d_cnt = bm.take<int>(nbox);
        B->d_work = bm.take<int4>(work.size());
    };
    carve(dry);
    if (cudaMalloc(&B->mem, dry.off + 256) != cudaSuccess || cudaMallocHost(&B->h_st, sizeof(SolveState) * nbox) != cudaSuccess) {
        cudaGetLastError();
        *st = set_err(c, MX_ERR_OOM, "batched: descriptor allocation failed");
        free_batch(B);
        return nullptr;
    }
    Bump real{(char *)B->mem, 0};
    carve(real);
    cudaStream_t s = c->stream;
    cudaMemcpyAsync(B->d_levs, levs.data(), sizeof(Level<float>) * levs.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B->d_df, dfb.data(), sizeof(DFBox) * nbox, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B->d_cargs, cargs.data(), cargs.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B->d_off, off.data(), sizeof(int) * nbox, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B->d_cnt, cnt.data(), sizeof(int) * nbox, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B->d_work, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        *st = set_err(c, MX_ERR_CUDA, "batched: descriptor upload failed");
        free_batch(B);
        return nullptr;
    }
    B->g_nu1 = o.nu1;
    B->g_nu2 = o.nu2;
    B->g_bot = o.bottom_iters;
    *st = MX_OK;
    return B;
}

// one V-cycle of every active box, then the fused update + residual and the
// per-box convergence decision
static void batch_body(cudaStream_t s, mx_ctx *c, BatchPlan &B, const mx_opts &o) {
    for (int l = 0; l < B.maxdown; l++) {
        for (int q = 0; q < o.nu1; q++) {
            k_rbgs_batch(s, B.d_levs, B.d_work + B.rb[l].off, B.rb[l].n, B.d_st, l, 0, q == 0);
            k_rbgs_batch(s, B.d_levs, B.d_work + B.rb[l].off, B.rb[l].n, B.d_st, l, 1, 0);
        }
        k_resid_restrict_batch(s, B.d_levs, B.d_work + B.rr[l].off, B.rr[l].n, B.d_st, l, B.rr_zcf[l]);
    }
    k_coarse_vcycle_batch(s, B.d_cargs, B.d_st, B.nbox, B.coarse_smem);
    for (int l = B.maxdown - 1; l >= 0; l--) {
        k_prolong_batch(s, B.d_levs, B.d_work + B.pr[l].off, B.pr[l].n, B.d_st, l);
        for (int q = 0; q < o.nu2; q++) {
            k_rbgs_batch(s, B.d_levs, B.d_work + B.rb[l].off, B.rb[l].n, B.d_st, l, 0, 0);
            k_rbgs_batch(s, B.d_levs, B.d_work + B.rb[l].off, B.rb[l].n, B.d_st, l, 1, 0);
        }
    }
    k_df_resid_batch(s, B.d_df, B.d_work + B.df.off, B.df.n, B.d_st, c->partials, 1, B.march);
    k_finalize_residual_batch(s, c->partials, B.d_off, B.d_cnt, B.d_st, B.nbox);
}

__global__ void batch_any_active_kernel(cudaGraphConditionalHandle h, const SolveState *st, int nbox) {
    int any = 0;
    for (int b = 0; b < nbox; b++) any |= !st[b].done;
    cudaGraphSetConditional(h, any ? 1u : 0u);
}

static mx_status batch_graph(mx_ctx *c, BatchPlan &B, const mx_opts &o) {
    if (B.graph && B.g_nu1 == o.nu1 && B.g_nu2 == o.nu2 && B.g_bot == o.bottom_iters) return MX_OK;
    if (B.graph) {
        cudaGraphExecDestroy(B.graph);
        B.graph = nullptr;
    }
    cudaGraph_t graph;
    MX_CUDA(c, cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    MX_CUDA(c, cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    MX_CUDA(c, cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    MX_CUDA(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        batch_body(cs, c, B, o);
        batch_any_active_kernel<<<1, 1, 0, cs>>>(handle, B.d_st, B.nbox);
        cudaGraph_t captured;
        e = cudaStreamEndCapture(cs, &captured);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_err(c, MX_ERR_CUDA, std::string("batched graph capture failed: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&B.graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        B.graph = nullptr;
        return set_err(c, MX_ERR_CUDA, std::string("batched graph instantiate failed: ") + cudaGetErrorString(e));
    }
    B.g_nu1 = o.nu1;
    B.g_nu2 = o.nu2;
    B.g_bot = o.bottom_iters;
    return MX_OK;
}

extern "C" mx_status mx_mac_project_batched(mx_ctx *c, int nbox, const mx_geom *geoms, double *const *ux,
                                            double *const *uy, double *const *uz, const double *const *rho,
                                            const double *const *beta0, const double *const *sbar,
                                            double *const *phi, const mx_opts *opts, mx_info *infos) {
    if (!c) return MX_ERR_ARG;
    if (nbox < 1 || !geoms || !ux || !uy || !uz || !rho || !beta0 || !sbar || !phi)
        return set_err(c, MX_ERR_ARG, "batched: nbox < 1 or a null array list");
    mx_status st;
    mx_opts o;
    if ((st = check_opts(c, opts, o))) return st;
    if (o.krylov) return set_err(c, MX_ERR_ARG, "batched: krylov = 1 is for single MAC solves");
    if (o.smoother) return set_err(c, MX_ERR_ARG, "batched: smoother = 1 (Chebyshev) is for nodal solves");
    tune_apply_batch(c, nbox, geoms, o);
    std::vector<DGeom> g(nbox);
    for (int b = 0; b < nbox; b++) {
        if ((st = check_geom(c, &geoms[b], false))) return st;
        if (!ux[b] || !uy[b] || !uz[b] || !rho[b] || !beta0[b] || !sbar[b] || !phi[b])
            return set_err(c, MX_ERR_ARG, "batched: null array");
        g[b] = make_dgeom(&geoms[b]);
    }
    if (o.prec == MX_PREC_FP64 || o.nu1 < 1 || o.nu2 < 1) {
        // the plain FP64 reference: the boxes one after another
        for (int b = 0; b < nbox; b++) {
            mx_info info;
            st = mx_mac_project(c, &geoms[b], ux[b], uy[b], uz[b], rho[b], beta0[b], sbar[b], phi[b], &o, &info);
            if (infos) infos[b] = info;
            if (st != MX_OK && st != MX_ERR_NOCONV) return st;
        }
        return MX_OK;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, MX_ERR_CUDA, "cudaSetDevice failed");
    if (!same_geoms(c->batch, nbox, g.data()) || c->batch->g_nu1 != o.nu1 || c->batch->g_nu2 != o.nu2 ||
        c->batch->g_bot != o.bottom_iters) {
        destroy_batch_plan(c);
        c->batch = build_batch(c, nbox, g.data(), o, &st);
        if (!c->batch) return st;
    }
    BatchPlan &B = *c->batch;
    cudaStream_t s = c->stream;
    MX_CUDA(c, cudaEventRecord(c->ev0, s));
    for (int b = 0; b < nbox; b++) {
        SolveState init = {};
        init.tol = o.rel_tol;
        init.maxit = std::min(o.max_outer, o.max_vcycles);
        B.h_st[b] = init;
    }
    MX_CUDA(c, cudaMemcpyAsync(B.d_st, B.h_st, sizeof(SolveState) * nbox, cudaMemcpyHostToDevice, s));
    // the per-box setup and finish run on the side streams (box b on stream b mod
    // NSIDE, its partials in that stream's slice), joined back by events
    const int ns = int(B.side.size());
    auto fork = [&]() -> mx_status {
        MX_CUDA(c, cudaEventRecord(B.fork, s));
        for (int q = 0; q < ns; q++) MX_CUDA(c, cudaStreamWaitEvent(B.side[q], B.fork, 0));
        return MX_OK;
    };
    auto join = [&]() -> mx_status {
        for (int q = 0; q < ns; q++) {
            MX_CUDA(c, cudaEventRecord(B.side_done[q], B.side[q]));
            MX_CUDA(c, cudaStreamWaitEvent(s, B.side_done[q], 0));
        }
        return MX_OK;
    };
    // setup of every box: coefficients and hierarchy, RHS, mean, initial phi
    if ((st = fork())) return st;
    for (int b = 0; b < nbox; b++) {
        MacPlan &P = *B.box[b];
        const DGeom &gb = g[b];
        SolveState *sb = B.d_st + b;
        cudaStream_t ss = B.side[b % ns];
        double *part = c->partials + (b % ns) * B.part_stride;
        const int nb = stencil_blocks(gb), nbr = red_blocks(gb.N);
        const int singular = geom_singular(gb);
        setup_coefficients_on(ss, P, rho[b], beta0[b]);
        k_mac_rhs_df(ss, gb, ux[b], uy[b], uz[b], sbar[b], P.D, part);
        k_finalize_rhs(ss, part, nb, sb, gb.N, singular && o.remove_mean, 0);
        if (singular && !o.remove_mean) {
            MX_CUDA(c, cudaMemcpyAsync(B.h_st + b, sb, sizeof(SolveState), cudaMemcpyDeviceToHost, ss));
            MX_CUDA(c, cudaStreamSynchronize(ss));
            if (std::fabs(B.h_st[b].aux) > 1e-12 * B.h_st[b].fnorm) {
                join();
                return set_err(c, MX_ERR_INCOMPAT, "batched: a singular box has a right-hand side of non-zero mean");
            }
        }
        k_sub_mean_scale(ss, gb, sb, P.D, part, nbr);
        k_finalize_rhs(ss, part, nbr, sb, gb.N, 0, 1);
        if (o.use_initial_guess) k_df_from_double(ss, gb.N, phi[b], P.D);  // else zeroed by the first residual
    }
    if ((st = join())) return st;
    // refinement loop over all boxes (from phi = 0 the first residual is f, formed elementwise)
    if (o.use_initial_guess) k_df_resid_batch(s, B.d_df, B.d_work + B.df.off, B.df.n, B.d_st, c->partials, 0, B.march);
    else k_df_resid_zero_batch(s, B.d_df, B.d_work + B.df.off, B.df.n, B.d_cnt, B.d_st, c->partials);
    k_finalize_residual_batch(s, c->partials, B.d_off, B.d_cnt, B.d_st, nbox);
    MX_CUDA(c, cudaMemcpyAsync(B.h_st, B.d_st, sizeof(SolveState) * nbox, cudaMemcpyDeviceToHost, s));
    MX_CUDA(c, cudaStreamSynchronize(s));
    bool any = false;
    for (int b = 0; b < nbox; b++) any |= !B.h_st[b].done;
    if (any) {
        if (o.use_graph) {
            if ((st = batch_graph(c, B, o))) return st;
            MX_CUDA(c, cudaGraphLaunch(B.graph, s));
        } else {
            for (;;) {
                batch_body(s, c, B, o);
                MX_CUDA(c, cudaMemcpyAsync(B.h_st, B.d_st, sizeof(SolveState) * nbox, cudaMemcpyDeviceToHost, s));
                MX_CUDA(c, cudaStreamSynchronize(s));
                bool a = false;
                for (int b = 0; b < nbox; b++) a |= !B.h_st[b].done;
                if (!a) break;
            }
        }
    }
    // finish every box: phi, mean, correction, divergence check
    if ((st = fork())) return st;
    for (int b = 0; b < nbox; b++) {
        MacPlan &P = *B.box[b];
        const DGeom &gb = g[b];
        SolveState *sb = B.d_st + b;
        cudaStream_t ss = B.side[b % ns];
        double *part = c->partials + (b % ns) * B.part_stride;
        const int nb = stencil_blocks(gb), nbr = red_blocks(gb.N);
        k_df_final(ss, gb.N, P.D, sb, phi[b], geom_singular(gb) ? part : nullptr);
        if (geom_singular(gb)) {
            k_finalize_sum(ss, part, nbr, &sb->aux, 1.0 / double(gb.N));
            k_sub_scalar(ss, gb.N, phi[b], &sb->aux);
        }
        k_mac_correct(ss, gb, P.Q, phi[b], ux[b], uy[b], uz[b]);
        k_mac_divcheck_df(ss, gb, ux[b], uy[b], uz[b], sbar[b], P.D, sb, part);
        k_finalize_max(ss, part, nb, &sb->div_err);
    }
    if ((st = join())) return st;
    MX_CUDA(c, cudaEventRecord(c->ev1, s));
    MX_CUDA(c, cudaMemcpyAsync(B.h_st, B.d_st, sizeof(SolveState) * nbox, cudaMemcpyDeviceToHost, s));
    MX_CUDA(c, cudaStreamSynchronize(s));
    MX_CUDA(c, cudaGetLastError());
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    mx_status worst = MX_OK;
    for (int b = 0; b < nbox; b++) {
        const SolveState &hs = B.h_st[b];
        if (infos) {
            mx_info &in = infos[b];
            in.outer_iters = hs.iter;
            in.vcycles = hs.iter;
            in.rel_resid = hs.fnorm > 0 ? hs.rnorm / hs.fnorm : hs.rnorm;
            in.rel_resid_l2 = hs.fnorm2 > 0 ? hs.rnorm2 / hs.fnorm2 : hs.rnorm2;
            in.div_err_linf = hs.div_err;
            in.rhs_mean_removed = hs.mean;
            in.rhs_linf = hs.fnorm;
            in.ms = ms;
            in.status = hs.status;
        }
        if (hs.status != MX_OK) worst = (mx_status)hs.status;
    }
    if (worst != MX_OK) return set_err(c, worst, "batched: at least one box did not converge");
    return MX_OK;
}
