"""Benchmark: MAC projection solves/s to 1e-10 relative residual on the planar
256^3 workload (periodic x,y, walls in z, density contrast 1e5,
beta0 = rho0^(3/5), 16 Fourier modes, 3 hotspots; seeded synthetic inputs),
FP32 V-cycles inside FP64 iterative refinement, with the plain FP64 solve
beside it.

One step = one pass of the whole hot path: base-state Fill of beta0, face
coefficients and the multigrid hierarchy, right-hand side with mean removal,
the refinement loop (FP64 residual, FP32 V-cycle, FP64 update) to 1e-10, mean
normalisation, the velocity correction and the divergence check.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MAC projection solves/s to 1e-10 rel residual (planar 256^3, mixed FP32/FP64)"
UNIT = "solves/s"
WORKLOAD = "planar256"
N = 256


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mx", choices=["mx", "reference"])
    p.add_argument("--n", type=int, default=N, help="cube edge of the planar workload")
    p.add_argument("--star-n", type=int, default=512, help="cube edge of the average512 workload")
    p.add_argument("--comp-n", type=int, default=128, help="coarse cube edge of the composite workload")
    p.add_argument("--nodal-n", type=int, default=384,
                   help="cube edge of --workload nodal384 (smaller cases for profiling)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-fcg", action="store_true", help="skip the krylov = 1 comparison")
    p.add_argument("--krylov", action="store_true",
                   help="run the headline solves with krylov = 1 (FCG around the V-cycle; for profiling)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the nodal and batched workloads")
    p.add_argument("--workload", default="planar256",
                   choices=["planar256", "star512", "nodal-sweep", "nodal384", "batched96", "average512",
                            "composite"],
                   help="planar256: the headline line (+ nodal384 and batched96 extras); star512: the "
                        "full-star line; nodal-sweep: one line per nodal size 64^3..512^3; nodal384 / "
                        "batched96 / average512: that extra alone (for profiling)")
    p.add_argument("--fixed", default=None, metavar="NU1,NU2,TILE_Z[,SMOOTHER]",
                   help="skip the autotuner and use these smoother settings (for profiling a fixed "
                        "configuration, e.g. the tuned one); SMOOTHER (nodal384 only): 0 four-colour "
                        "Gauss-Seidel, 1 Chebyshev")
    p.add_argument("--no-graph", action="store_true",
                   help="run the refinement loop from the host (same kernels; for profilers that "
                        "cannot see inside conditional CUDA graphs)")
    return p.parse_args()


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------

def algorithmic_bytes_per_cell():
    """Compulsory DRAM bytes per finest-level cell of each traced phase
    (FP32 V-cycle arrays w = 4 B, FP64 arrays 8 B).
      smooth_fine   (one colour pass of red-black Gauss-Seidel, half a sweep):
                    a full sweep reads e, f, bx, by, bz and writes e = 6 x 4 B,
                    so one colour pass = 12 B/cell
      resid64       read phi, f, bx, by, bz (8 B each), write rhat (4 B) = 44 B
    """
    return {"smooth_fine": 12.0, "resid64": 44.0}


def mac_iteration_bytes_per_cell(nu1, nu2, w):
    """Algorithmic bytes per finest-level cell of one refinement iteration of the
    MAC solve (the fixed model of the measurement plan): a V-cycle(nu1, nu2) on
    all levels (N_total = 8/7 N) moves w (6 (nu1 + nu2) + 7.25) bytes per cell
    (a sweep reads phi, f, b_x, b_y, b_z and writes phi: 6w; residual +
    restriction 5.125w; prolongation + correction 2.125w), and the outer step
    adds the high-precision residual (5 reads x 8 B + 4 B written) and the
    update (20 B): 64 B/cell.  w = 4 (FP32 V-cycle) or 8 (plain FP64)."""
    return (8.0 / 7.0) * w * (6.0 * (nu1 + nu2) + 7.25) + 64.0


def mac_iteration_fp64_flops_per_cell(nu1, nu2):
    """FP64 flops per finest-level cell of one iteration of the plain FP64 solve:
    a Gauss-Seidel update 19 (6 products and sums of the neighbours, h^2 f, the
    5-term diagonal, one division counted as 1 flop), residual + restriction 22,
    prolongation 1 per level cell (8/7 N in all), and the outer FP64 residual
    with its norms and the update, 26."""
    return (8.0 / 7.0) * (19.0 * (nu1 + nu2) + 22.0 + 1.0) + 26.0


def roofline_per_vcycle(ncell, nu1, nu2, w, ms_solve, vcycles, hbm, loop_ms=None):
    """Fraction of the HBM roofline per refinement iteration: the model's bytes
    of one iteration over (solve time / iterations), against the measured copy
    peak.  The solve time includes the setup and finish passes, so this is the
    conservative figure; loop_ms (the traced time of the refinement loop alone)
    gives the loop-only one."""
    b = mac_iteration_bytes_per_cell(nu1, nu2, w) * ncell
    v = max(vcycles, 1)
    out = {"model_bytes_per_vcycle": b, "nu1": nu1, "nu2": nu2, "word_bytes": w,
           "ms_per_vcycle": ms_solve / v,
           "achieved_GBs": round(b / (ms_solve / v * 1e-3) / 1e9, 1),
           "frac": round(b / (ms_solve / v * 1e-3) / 1e9 / hbm, 4),
           "time": "whole solve / V-cycles (setup and finish included)"}
    if loop_ms:
        out["loop_only"] = {"ms_per_vcycle": loop_ms / v,
                            "frac": round(b / (loop_ms / v * 1e-3) / 1e9 / hbm, 4)}
    return out


def launches_per_solve(g, o, vcycles, graph, krylov=0):
    """Kernels the library launches for one mixed-precision MAC solve (fill
    included), from the solver's structure: setup 13 + first residual 2; per
    refinement iteration the V-cycle's launches on the levels above the coarse
    end (> 4096 cells: colour passes, residual+restriction, prolongation, or
    single-pass sweeps), the coarse-end CTA, update+residual and its finalize
    (+1 condition kernel inside the graph); finish 6 (4 without a mean to
    remove).  FCG (krylov = 1) adds 4 per iteration: the dot product, its
    finalize, the direction/stencil pass and the step finalize.  Checked against
    the ncu launch lists of the planar 256^3 solve."""
    dims = [list(g.n)]
    while all(d % 2 == 0 and d >= 4 for d in dims[-1]):
        dims.append([d // 2 for d in dims[-1]])
    nlev = len(dims)
    ncell = [d[0] * d[1] * d[2] for d in dims]
    ldown = next((l for l in range(nlev) if ncell[l] <= 4096), nlev - 1)
    per_iter = 1 + 2 + (1 if graph else 0) + (4 if krylov else 0)
    for l in range(ldown):
        fused = o.fused and ncell[l] >= (1 << 18) and dims[l][0] % 2 == 0
        per_iter += (o.nu1 + 1 + o.nu2) if fused else (2 * o.nu1 + 1 + 1 + 2 * o.nu2)
    setup = 1 + 1 + (nlev - 1) + 4 + 2
    singular = all(b != 2 for b in tuple(g.lo) + tuple(g.hi))  # no Dirichlet face
    finish = 6 if singular else 4   # phi (+ its sums), [mean, subtract], correct, check, max
    return setup + vcycles * per_iter + finish


def setup_inputs(mx, W, dev, n, copies):
    import torch
    w = W.planar256(device=dev, n=n)
    g = w.geom
    us = [[t.clone() for t in w.u] for _ in range(copies)]
    return w, g, us


def run_mx(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge
    from paper_1908_03634_gb300 import build as B
    B.build()
    import paper_1908_03634_gb300 as mx
    from paper_1908_03634_gb300 import sharding as S
    from paper_1908_03634_gb300 import workloads as W

    K, Wm = args.steps, args.warmup
    n = args.n
    copies = K + Wm
    w, g, us = setup_inputs(mx, W, dev, n, copies)
    rho, sbar, prof = w.rho.contiguous(), w.sbar.contiguous(), w.prof_beta0.contiguous()
    beta0 = torch.empty_like(rho)
    phi = torch.zeros_like(rho)
    stream = torch.cuda.current_stream()
    ctx = mx.mx_create(local, stream)
    graph = 0 if args.no_graph else 1
    # the library's autotuner picks sweep counts, tile depth and sweep kind on
    # these inputs (untimed); the timed solves then run with nu1 = nu2 = 0
    mx.mx_fill_base_state(ctx, g, 0, prof, g.dx, (0.5, 0.5, 0.5), beta0)
    t_tune = time.perf_counter()
    if args.fixed:
        a, b, z = (int(x) for x in args.fixed.split(","))
        tuned = mx.default_opts(prec=mx.MX_PREC_MIXED, use_graph=graph, nu1=a, nu2=b, tile_z=z)
        tuned64 = mx.default_opts(prec=mx.MX_PREC_FP64, use_graph=graph, nu1=a, nu2=b, tile_z=z)
    else:
        tuned, _ = mx.mx_autotune(ctx, mx.MX_OP_MAC, g, *w.u, rho, beta0, sbar,
                                  base=mx.default_opts(prec=mx.MX_PREC_MIXED, use_graph=graph))
        tuned64, _ = (None, None) if args.no_fp64 else mx.mx_autotune(
            ctx, mx.MX_OP_MAC, g, *w.u, rho, beta0, sbar,
            base=mx.default_opts(prec=mx.MX_PREC_FP64, use_graph=graph))
    t_tune = time.perf_counter() - t_tune
    kry = 1 if args.krylov else 0
    opts = (mx.default_opts(prec=mx.MX_PREC_MIXED, use_graph=graph, nu1=tuned.nu1, nu2=tuned.nu2,
                            tile_z=tuned.tile_z, krylov=kry) if args.fixed else
            mx.default_opts(prec=mx.MX_PREC_MIXED, use_graph=graph, nu1=0, nu2=0, krylov=kry))

    def step(u, o=opts):
        mx.mx_fill_base_state(ctx, g, 0, prof, g.dx, (0.5, 0.5, 0.5), beta0)
        return mx.mx_mac_project(ctx, g, u[0], u[1], u[2], rho, beta0, sbar, phi, o)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    infos = []
    for s in range(Wm):
        infos.append(step(us[s])[1])
    barrier()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(K):
        infos.append(step(us[Wm + s])[1])
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    # replicas: every rank solved K problems; the job's time is the slowest rank's
    value, ms_total = S.job_throughput(float(K), e0.elapsed_time(e1))
    last = infos[-1]
    assert all(i["status"] == 0 for i in infos), infos[-1]
    vcycles = statistics.mean(i["vcycles"] for i in infos[Wm:])
    launches = int(round(K * launches_per_solve(g, tuned, vcycles, graph, kry)))

    # ---- plain FP64 solve (the comparison) ----
    fp64 = None
    if not args.no_fp64:
        o64 = (mx.default_opts(prec=mx.MX_PREC_FP64, use_graph=graph, nu1=tuned64.nu1, nu2=tuned64.nu2,
                               tile_z=tuned64.tile_z) if args.fixed else
               mx.default_opts(prec=mx.MX_PREC_FP64, use_graph=graph, nu1=0, nu2=0))
        u64 = [t.clone() for t in w.u]
        step(u64, o64)  # warm-up (plan, graph)
        kk = max(2, min(5, K // 4))
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        i64 = []
        f0.record(stream)
        for s in range(kk):
            for d in range(3):
                u64[d].copy_(w.u[d])
            i64.append(step(u64, o64)[1])
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / kk
        fp64 = {"solves_per_s": 1e3 / ms64, "ms_per_solve": ms64, "vcycles": i64[-1]["vcycles"],
                "rel_resid": i64[-1]["rel_resid"],
                "div_err_rel": i64[-1]["div_err_linf"] / max(i64[-1]["rhs_linf"], 1e-300),
                "note": "includes a 3-array restore of U per solve"}

    # ---- FCG(1) (krylov = 1) against refinement, both timed in the same loop ----
    fcg = None
    if not args.no_fcg:
        def variant(o, kk):
            uv = [t.clone() for t in w.u]
            step(uv, o)  # warm-up (plan, graph)
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            iv = []
            v0.record(stream)
            for s in range(kk):
                for d in range(3):
                    uv[d].copy_(w.u[d])
                iv.append(step(uv, o)[1])
            v1.record(stream)
            torch.cuda.synchronize()
            assert all(i["status"] == 0 for i in iv), iv[-1]
            return v0.elapsed_time(v1) / kk, iv[-1]
        kk = max(3, min(8, K // 2))
        o_k = mx.default_opts(prec=mx.MX_PREC_MIXED, use_graph=graph, nu1=opts.nu1, nu2=opts.nu2,
                              tile_z=opts.tile_z, fused=opts.fused, krylov=1)
        ms_k, i_k = variant(o_k, kk)
        ms_r, i_r = variant(opts, kk)
        fcg = {"solves_per_s": 1e3 / ms_k, "ms_per_solve": ms_k, "vcycles": i_k["vcycles"],
               "rel_resid": i_k["rel_resid"],
               "refinement_same_loop": {"solves_per_s": 1e3 / ms_r, "ms_per_solve": ms_r, "vcycles": i_r["vcycles"]},
               "note": "both include a 3-array restore of U per solve"}

    # ---- traced pass: per-phase device time with CUDA events on the launching stream ----
    mx.mx_profile_enable(ctx, True)
    ut = [t.clone() for t in w.u]
    nt = 2
    for s in range(nt):
        for d in range(3):
            ut[d].copy_(w.u[d])
        step(ut)
    trace = mx.mx_profile_read(ctx)
    mx.mx_profile_enable(ctx, False)
    bpc = algorithmic_bytes_per_cell()
    ncell = g.ncell
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    phases = {}
    for name, (pms, pn) in trace.items():
        phases[name] = {"ms_per_step": pms / nt, "launches_per_step": pn / nt}
    sm_ms, sm_n = trace["smooth_fine"]
    per_launch_ms = sm_ms / max(sm_n, 1)
    # the tuned smoother: two colour passes (12 B/cell each) or single-pass sweeps (24 B/cell)
    fused0 = bool(tuned.fused) and ncell >= (1 << 18) and g.n[0] % 2 == 0
    sweep_bytes = 2 * bpc["smooth_fine"] if fused0 else bpc["smooth_fine"]
    achieved = sweep_bytes * ncell / (per_launch_ms * 1e-3) / 1e9
    r_ms, r_n = trace["resid64"]
    resid_per_launch = r_ms / max(r_n / 2, 1)   # resid64 phase = residual + its 1-block finalize
    traffic = None
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        traffic = tr.get("rbgs_fp32_per_launch_bytes_256")
    except (OSError, ValueError):
        pass
    if fused0:
        traffic = None  # the ncu figure is for the colour-pass kernel
    roofline = {"kernel": ("rbgs_march_kernel (finest level, one red+black sweep)" if fused0 else
                           "rbgs_kernel<float> (finest level, one colour)"), "bound": "hbm",
                "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "peak_source": peak_src, "traffic": traffic,
                "algorithmic_bytes_per_launch": sweep_bytes * ncell,
                "ms_per_launch": per_launch_ms,
                "resid64": {"ms_per_launch": resid_per_launch,
                            "achieved_GBs": round(bpc["resid64"] * ncell / (resid_per_launch * 1e-3) / 1e9, 1)}}

    # ---- per refinement iteration (the model's bytes per V-cycle over the time per
    # V-cycle), for the mixed solve and the plain FP64 one; for the FP64 solve also
    # the FP64-ALU bound from the measured FMA rate of the FP64 pipe ----
    loop_ms = sum(v["ms_per_step"] for k, v in phases.items() if k not in ("setup", "finish"))
    per_vc = {"mixed": roofline_per_vcycle(ncell, tuned.nu1, tuned.nu2, 4, ms_total / K, vcycles, hbm,
                                           loop_ms=loop_ms)}
    if fp64 is not None:
        n1, n2 = tuned64.nu1, tuned64.nu2
        per_vc["fp64"] = roofline_per_vcycle(ncell, n1, n2, 8, fp64["ms_per_solve"], fp64["vcycles"], hbm)
        try:
            p64 = mx.mx_probe_fma_peak(local, True)
            fl = mac_iteration_fp64_flops_per_cell(n1, n2) * ncell
            ach = fl / (fp64["ms_per_solve"] / max(fp64["vcycles"], 1) * 1e-3) / 1e12
            fp64["alu_bound"] = {"bound": "fp64_alu", "peak_tflops": round(p64, 3), "unit": "TFLOP/s",
                                 "peak_source": "measured FP64 FMA rate of this GPU (mx_probe_fma_peak)",
                                 "model_flops_per_vcycle": fl, "achieved_tflops": round(ach, 4),
                                 "frac": round(ach / p64, 4)}
        except Exception as e:  # noqa: BLE001 - the probe is a measurement extra
            fp64["alu_bound"] = {"error": str(e)}
        fp64["hbm_frac_per_vcycle"] = per_vc["fp64"]["frac"]
    roofline["per_vcycle"] = per_vc

    # ---- end to end through the C ABI with host buffers ----
    # Every step copies its inputs (rho, Sbar, the base-state profile, U) from
    # pinned host memory and reads its outputs (U, phi) back, all inside the
    # timed region.  Two device buffer sets and a copy stream overlap the
    # copies of steps i+1 (in) and i-1 (out) with the solve of step i.
    e2e = None
    if not args.no_e2e:
        pin = lambda t: t.cpu().pin_memory()
        h_in = [pin(rho), pin(sbar), pin(prof)] + [pin(t) for t in w.u]
        h_out = [torch.empty_like(t).pin_memory() for t in h_in[3:]] + [torch.empty_like(h_in[0]).pin_memory()]
        sets = [{"in": [torch.empty_like(t) for t in [rho, sbar, prof] + list(w.u)],
                 "beta0": torch.empty_like(beta0), "phi": torch.empty_like(phi)} for _ in range(2)]
        h2d = sum(t.numel() * 8 for t in h_in)
        d2h = sum(t.numel() * 8 for t in h_out)
        ke = max(3, min(10, K))
        cs = torch.cuda.Stream()
        ready = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]

        def copy_in(i):
            with torch.cuda.stream(cs):
                for src, dst in zip(h_in, sets[i % 2]["in"]):
                    dst.copy_(src, non_blocking=True)
                ready[i % 2].record(cs)

        def solve(i):
            st_ = sets[i % 2]
            d_rho, d_sbar, d_prof = st_["in"][:3]
            d_u = st_["in"][3:]
            stream.wait_event(ready[i % 2])
            mx.mx_fill_base_state(ctx, g, 0, d_prof, g.dx, (0.5, 0.5, 0.5), st_["beta0"])
            mx.mx_mac_project(ctx, g, d_u[0], d_u[1], d_u[2], d_rho, st_["beta0"], d_sbar, st_["phi"], opts)
            done[i % 2].record(stream)

        def copy_out_then_in(i, n):
            with torch.cuda.stream(cs):
                cs.wait_event(done[i % 2])
                for src, dst in zip(sets[i % 2]["in"][3:] + [sets[i % 2]["phi"]], h_out):
                    dst.copy_(src, non_blocking=True)
            if i + 2 < n:
                copy_in(i + 2)

        def run(n, start=None):
            copy_in(0)
            if n > 1:
                copy_in(1)
            for i in range(n):
                solve(i)
                copy_out_then_in(i, n)

        run(2)  # warm-up (plans, graphs, both buffer sets)
        torch.cuda.synchronize()
        barrier()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(cs)
        stream.wait_event(q0)
        run(ke)
        q1.record(cs)
        torch.cuda.synchronize()
        barrier()
        e2e_value, _ = S.job_throughput(float(ke), q0.elapsed_time(q1))
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "pipelined": "copies of steps i+1 (in) and i-1 (out) overlap the solve of step i"}

    # ---- the other workloads (nodal projection, batched patches) ----
    extras = {}
    if not args.no_extras:
        extras["nodal384"] = bench_nodal(mx, W, ctx, dev, stream, hbm=hbm)
        extras["batched96"] = bench_batched(mx, W, ctx, dev, stream, fp64=world == 1, rank=rank, world=world)
        extras["average512"] = bench_base(mx, W, ctx, dev, stream, hbm=hbm, cpu=rank == 0 and world == 1)
        torch.cuda.empty_cache()
        extras["star512"] = bench_star(mx, W, ctx, dev, stream, hbm=hbm)
        extras["planar32_fp64"] = bench_planar32_fp64(mx, W, ctx, dev, stream)
        extras["nodal_sweep"] = bench_nodal_sweep(mx, W, ctx, dev, stream, hbm)
        extras["composite"] = bench_composite(mx, W, ctx, dev, stream, hbm=hbm)

    # ---- CPU oracle baseline (rank 0, N = 1 only) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(n_sample=128, n_full=n)

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": ms_total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"planar{n}", "cells": g.ncell, "bc": "periodic x,y / wall z",
                   "density_contrast": 1e5, "beta0": "rho0^(3/5)", "rel_tol": 1e-10,
                   "precision": ("FP32 V-cycles as the FCG(1) preconditioner, double-float residual" if kry else
                                 "FP32 V-cycles in FP64 iterative refinement"),
                   "tuned": {"nu1": tuned.nu1, "nu2": tuned.nu2, "tile_z": tuned.tile_z, "fused": tuned.fused,
                             "fp64": None if tuned64 is None else {"nu1": tuned64.nu1, "nu2": tuned64.nu2,
                                                                   "tile_z": tuned64.tile_z},
                             "tuning_s": round(t_tune, 2), "source": "fixed" if args.fixed else "autotuner"},
                   "l2_policy": "inputs larger than L2 (fresh U copy per step, ~1.5 GB working set)",
                   "parallelism": f"replicas x{world}"},
        "vcycles_per_solve": vcycles, "rel_resid": last["rel_resid"], "div_err_linf": last["div_err_linf"],
        "rhs_linf": last["rhs_linf"], "div_err_rel": last["div_err_linf"] / max(last["rhs_linf"], 1e-300),
        "hbm_frac_per_vcycle": per_vc["mixed"]["frac"],
        "fp64": fp64, "fcg": fcg, "phases": phases, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk, **extras,
    }
    mx.mx_destroy(ctx)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def timed(fn, steps, stream):
    import torch
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    out = [fn(i) for i in range(steps)]
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b), out


def bench_nodal(mx, W, ctx, dev, stream, n=384, steps=3, warmup=2, fp64=True, hbm=6793.4, graph=True, fixed=None):
    """Nodal projection (Step 11) on the planar256 stratification at n^3 cells:
    mixed precision vs plain FP64, solves/s, time per V-cycle and the HBM
    fraction of one V-cycle against the model's algorithmic bytes."""
    import torch
    w = W.nodal384(device=dev, n=n)
    g = w.geom
    beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=dev)
    mx.mx_fill_base_state(ctx, g, 0, w.prof_beta0, g.dx, (0.5, 0.5, 0.5), beta0)
    phi = torch.zeros(mx.node_shape(g), dtype=torch.float64, device=dev)
    us = [[t.clone() for t in w.u] for _ in range(steps + warmup)]
    if fixed:
        a, b, z, *sm = (int(x) for x in fixed.split(","))
        tuned = mx.default_opts(use_graph=int(graph), nu1=a, nu2=b, tile_z=z, smoother=sm[0] if sm else 0)
        opts = tuned
    else:
        tuned, _ = mx.mx_autotune(ctx, mx.MX_OP_NODAL, g, *w.u, w.rho, beta0, w.sbar,
                                  base=mx.default_opts(use_graph=int(graph)))
        opts = mx.default_opts(use_graph=int(graph), nu1=0, nu2=0)
    run = lambda u, o: mx.mx_nodal_project(ctx, g, *u, w.rho, beta0, w.sbar, phi, o)[1]
    for i in range(warmup):
        run(us[i], opts)
    ms, infos = timed(lambda i: run(us[warmup + i], opts), steps, stream)
    vc = infos[-1]["vcycles"]
    nodes = phi.numel()
    # traced pass: per-phase device time (CUDA events on the stream)
    mx.mx_profile_enable(ctx, True)
    ut = [t.clone() for t in w.u]
    run(ut, opts)
    trace = {k: {"ms": v[0], "launches": v[1]} for k, v in mx.mx_profile_read(ctx).items()}
    mx.mx_profile_enable(ctx, False)
    # model bytes per V-cycle at the timed sweep counts (FP32): a sweep (four-colour
    # Gauss-Seidel) or a step (Chebyshev) reads phi, f, sigma and writes phi
    # (4w/node), residual+restriction 3.125w, prolongation 2.125w on every level
    # (N_total = 8/7 N), + the double-float residual and update of the refinement
    # loop (phi 8 read + 8 write, f 8, sigma 8, rhat 4)
    nu1, nu2 = tuned.nu1, tuned.nu2
    model = nodes * (8.0 / 7.0) * 4 * (4 * (nu1 + nu2) + 3.125 + 2.125) + nodes * 36
    ms_solve = ms / steps
    loop_ms = sum(v["ms"] for k, v in trace.items() if k not in ("setup", "finish"))
    last = infos[-1]
    out = {"workload": f"nodal{n}", "nodes": nodes, "solves_per_s": 1e3 / ms_solve, "ms_per_solve": ms_solve,
           "vcycles": vc, "rel_resid": last["rel_resid"], "div_err_linf": last["div_err_linf"],
           "rhs_linf": last["rhs_linf"], "div_err_rel": last["div_err_linf"] / max(last["rhs_linf"], 1e-300),
           "ms_per_vcycle_upper": ms_solve / max(vc, 1),
           "hbm_frac_per_vcycle": round(model / (ms_solve / max(vc, 1) * 1e-3) / 1e9 / hbm, 4),
           "hbm_frac_per_vcycle_loop_only": round(model / (loop_ms / max(vc, 1) * 1e-3) / 1e9 / hbm, 4),
           "model_bytes_per_vcycle": model, "model_nu": [nu1, nu2], "phases": trace,
           "tuned": {"nu1": tuned.nu1, "nu2": tuned.nu2, "tile_z": tuned.tile_z,
                     "smoother": "chebyshev" if tuned.smoother else "gauss-seidel-4colour"}}
    if fp64:
        o64 = mx.default_opts(prec=mx.MX_PREC_FP64, use_graph=int(graph), nu1=tuned.nu1, nu2=tuned.nu2,
                              tile_z=tuned.tile_z, smoother=tuned.smoother)
        u64 = [t.clone() for t in w.u]
        run(u64, o64)
        for d in range(3):
            u64[d].copy_(w.u[d])
        ms64, i64 = timed(lambda i: run(u64, o64), 1, stream)
        out["fp64"] = {"solves_per_s": 1e3 / ms64, "ms_per_solve": ms64, "vcycles": i64[-1]["vcycles"]}
    return out


def bench_batched(mx, W, ctx, dev, stream, npatch=96, steps=2, warmup=1, fp64=True, rank=0, world=1, graph=True,
                  fixed=None):
    """96 independent planar patches (sizes {32,48,64,96,128}^3) solved as one
    batch (one launch per phase over all patches), vs looping single FP64 solves.
    With several ranks each solves its shard of the patches (balanced by cells,
    no collective) and the line reports the whole job: all patches / the
    slowest rank's time."""
    import torch
    from paper_1908_03634_gb300 import sharding as S
    mine = S.shard_patches([a * b * c for a, b, c in W.batched_sizes(npatch)], world)[rank]
    ps = W.batched_patches(npatch, device=dev, only=mine)
    geoms = [p.geom for p in ps]
    cells = sum(g.ncell for g in geoms)
    b0 = []
    for p in ps:
        t = torch.empty(mx.cell_shape(p.geom), dtype=torch.float64, device=dev)
        mx.mx_fill_base_state(ctx, p.geom, 0, p.prof_beta0, p.geom.dx, (0.5, 0.5, 0.5), t)
        b0.append(t)
    phis = [torch.zeros(mx.cell_shape(g), dtype=torch.float64, device=dev) for g in geoms]
    sets = [[[t.clone() for t in p.u] for p in ps] for _ in range(steps + warmup)]

    def run(us, o):
        return mx.mx_mac_project_batched(ctx, geoms, [u[0] for u in us], [u[1] for u in us], [u[2] for u in us],
                                         [p.rho for p in ps], b0, [p.sbar for p in ps], phis, o)[1]
    # the batch's sweep counts from the library's autotuner (untimed), then nu1 = nu2 = 0
    if fixed:
        a, b, _ = (int(x) for x in fixed.split(","))
        tuned = mx.default_opts(nu1=a, nu2=b, use_graph=int(graph))
        opts = tuned
    else:
        tuned, _ = mx.mx_autotune_batched(ctx, geoms, [p.u[0] for p in ps], [p.u[1] for p in ps],
                                          [p.u[2] for p in ps], [p.rho for p in ps], b0, [p.sbar for p in ps],
                                          base=mx.default_opts(use_graph=int(graph)))
        opts = mx.default_opts(nu1=0, nu2=0, use_graph=int(graph))
    for i in range(warmup):
        run(sets[i], opts)
    if world > 1:
        torch.distributed.barrier()
    ms, infos = timed(lambda i: run(sets[warmup + i], opts), steps, stream)
    last = infos[-1]
    _, ms = S.job_throughput(0.0, ms)  # the slowest rank's time
    cells = int(S.sum_over_ranks(cells))
    ms_b = ms / steps
    out = {"workload": f"batched{npatch}", "patches": npatch, "cells": cells, "ms_per_batch": ms_b,
           "patch_solves_per_s": npatch * 1e3 / ms_b, "cells_per_s": cells * 1e3 / ms_b, "ranks": world,
           "tuned": {"nu1": tuned.nu1, "nu2": tuned.nu2},
           "vcycles_max": max(i["vcycles"] for i in last), "vcycles_mean": statistics.mean(i["vcycles"] for i in last),
           "rel_resid_max": max(i["rel_resid"] for i in last),
           "div_err_rel_max": max(i["div_err_linf"] / max(i["rhs_linf"], 1e-300) for i in last)}
    if fp64:
        o64 = mx.default_opts(prec=mx.MX_PREC_FP64)
        us = [[t.clone() for t in p.u] for p in ps]
        ms64, _ = timed(lambda i: run(us, o64), 1, stream)
        out["fp64_loop"] = {"ms_per_batch": ms64, "patch_solves_per_s": npatch * 1e3 / ms64}
    return out


def _avg_traffic(ncell):
    """DRAM bytes of one mx_average_radial call, scaled by the cell count from the
    ncu capture recorded in profiles/traffic.json (None if absent)."""
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        return round(tr["average_radial_call_per_cell_bytes"] * ncell)
    except (OSError, ValueError, KeyError):
        return None


def bench_base(mx, W, ctx, dev, stream, hbm=6793.4, steps=10, warmup=3, cpu=True, n=512):
    """Lateral Average and Fill (Sec. 3.1) on the 512^3 full star's density, centre
    on the corner (256, 256, 256): one step = Average onto the irregular base state
    (97,921 radial bins) + Fill back onto the cells.  Also times the planar Average
    (planar 256^3 density), the uniform-base-state interpolations and the oracle's
    radial average on a 256^3 sample.  The 1 GiB field is larger than L2."""
    import torch
    w = W.star512(device=dev, n=n)
    g = w.geom
    c = tuple(e // 2 for e in g.n)
    nb = mx.mx_radial_nbins(g, c)
    avg = torch.empty(nb, dtype=torch.float64, device=dev)
    out = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=dev)
    rho = w.rho

    def step(i):
        mx.mx_average_radial(ctx, g, c, rho, avg)
        mx.mx_fill_radial(ctx, g, c, avg, out)
    for i in range(warmup):
        step(i)
    ms, _ = timed(step, steps, stream)
    ms_avg, _ = timed(lambda i: mx.mx_average_radial(ctx, g, c, rho, avg), steps, stream)
    ms_fill, _ = timed(lambda i: mx.mx_fill_radial(ctx, g, c, avg, out), steps, stream)
    nr = 4 * g.n[0]
    dr = g.dx / 4
    prof = torch.empty(nr, dtype=torch.float64, device=dev)
    mx.mx_radial_to_uniform(ctx, g, c, avg, dr, prof)
    ms_uni, _ = timed(lambda i: mx.mx_radial_to_uniform(ctx, g, c, avg, dr, prof), steps, stream)
    mx.mx_fill_uniform(ctx, g, c, prof, dr, out)
    ms_fu, _ = timed(lambda i: mx.mx_fill_uniform(ctx, g, c, prof, dr, out), steps, stream)
    # velocity split (Appendix A) on the same star: the S - Sbar bracket, the Sbar profile
    # on the uniform base state (dr = dx/4), w0 from it, and w0 e_r on the MAC faces
    S = w.sbar
    bracket = torch.empty_like(S)
    mx.mx_subtract_lateral_average(ctx, g, 1, c, S, bracket)
    ms_sub, _ = timed(lambda i: mx.mx_subtract_lateral_average(ctx, g, 1, c, S, bracket), steps, stream)
    nru = 4 * g.n[0]
    dru = g.dx / 4
    r_edge = torch.arange(nru + 1, dtype=torch.float64, device=dev) * dru
    sbar_u = torch.empty(nru, dtype=torch.float64, device=dev)
    savg = torch.empty(nb, dtype=torch.float64, device=dev)
    mx.mx_average_radial(ctx, g, c, S, savg)
    mx.mx_radial_to_uniform(ctx, g, c, savg, dru, sbar_u)
    b0u = w.prof_beta0[:nru].contiguous()
    w0 = torch.empty(nru + 1, dtype=torch.float64, device=dev)
    mx.mx_w0_integrate(ctx, 1, r_edge, b0u, sbar_u, w0)
    ms_w0, _ = timed(lambda i: mx.mx_w0_integrate(ctx, 1, r_edge, b0u, sbar_u, w0), steps, stream)
    mx.mx_add_w0_faces(ctx, g, 1, c, r_edge, w0, *w.u)
    ms_faces, _ = timed(lambda i: mx.mx_add_w0_faces(ctx, g, 1, c, r_edge, w0, *w.u), steps, stream)
    nfaces = sum(t.numel() for t in w.u)
    del bracket
    N = g.ncell
    bytes_avg = 8.0 * N + 8.0 * nb
    bytes_fill = 8.0 * N
    a_avg = bytes_avg / (ms_avg / steps * 1e-3) / 1e9
    a_fill = bytes_fill / (ms_fill / steps * 1e-3) / 1e9
    del w, out
    torch.cuda.empty_cache()
    wp = W.planar256(device=dev)
    pp = torch.empty(wp.geom.n[2], dtype=torch.float64, device=dev)
    mx.mx_average_planar(ctx, wp.geom, wp.rho, pp)
    ms_pl, _ = timed(lambda i: mx.mx_average_planar(ctx, wp.geom, wp.rho, pp), steps, stream)
    a_pl = 8.0 * wp.geom.ncell / (ms_pl / steps * 1e-3) / 1e9
    r = {"workload": f"star{n} lateral average + fill", "metric": f"Average + Fill round trips/s (full star {n}^3, "
         "irregular base state)", "value": steps * 1e3 / ms, "unit": "round trips/s", "ms_per_step": ms / steps,
         "cells": N, "radial_bins": nb,
         "average_radial": {"ms": ms_avg / steps, "GB_s": a_avg, "launches": 2},
         "fill_radial": {"ms": ms_fill / steps, "GB_s": a_fill, "frac": a_fill / hbm, "launches": 1},
         "radial_to_uniform": {"ms": ms_uni / steps, "nr": nr, "launches": 1},
         "fill_uniform": {"ms": ms_fu / steps, "launches": 2},
         "average_planar_256": {"ms": ms_pl / steps, "GB_s": a_pl, "frac": a_pl / hbm, "launches": 2},
         "velocity_split": {
             "subtract_lateral_average": {"ms": ms_sub / steps, "launches": 3,
                                          "GB_s": 24.0 * N / (ms_sub / steps * 1e-3) / 1e9,
                                          "bytes": "8 B/cell read (average) + 8 read + 8 written (fill-subtract)"},
             "w0_integrate": {"ms": ms_w0 / steps, "nr": nru, "launches": 1},
             "add_w0_faces": {"ms": ms_faces / steps, "launches": 4,
                              "GB_s": 16.0 * nfaces / (ms_faces / steps * 1e-3) / 1e9,
                              "frac": 16.0 * nfaces / (ms_faces / steps * 1e-3) / 1e9 / hbm,
                              "bytes": "8 B read + 8 B written per face"}},
         "roofline": {"bound": "hbm", "achieved": round(a_avg, 1), "peak": hbm, "unit": "GB/s",
                      "frac": round(a_avg / hbm, 4), "traffic": _avg_traffic(N),
                      "kernel": "mx_average_radial (fold + bin kernels), 8 B/cell read + 8 B/bin written",
                      "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
         "gpu_launches_per_step": 3}
    if cpu:
        import numpy as np
        import oracle as O
        O.build()
        ns = min(n, 256)
        ws = W.star512(device="cpu", n=ns)
        f = ws.rho.numpy()
        t0 = time.perf_counter()
        O.average_radial(ws.geom, (ns // 2,) * 3, f)
        dt = time.perf_counter() - t0
        r["cpu_baseline"] = {"value": round((ns / n) ** 3 / dt, 4), "unit": f"averages/s of the {n}^3 field",
                             "cores": 1, "kind": "oracle",
                             "sample": f"oracle radial average of the star recipe at {ns}^3 ({dt:.2f} s), "
                                       f"scaled by ({ns}/{n})^3"}
    return r


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_solves(w, b0, nthreads, tol=1e-10):
    """nthreads independent oracle solves of the same inputs, run at the same time
    in host threads (the oracle's C code releases the GIL; each solve works on its
    own copies of U and phi).  Returns (wall seconds, infos)."""
    import concurrent.futures as cf

    import oracle as O

    def one(_):
        return O.mac_project(w.geom, w.u, w.rho, b0, w.sbar, tol=tol)[2]
    t0 = time.perf_counter()
    if nthreads == 1:
        infos = [one(0)]
    else:
        with cf.ThreadPoolExecutor(nthreads) as ex:
            infos = list(ex.map(one, range(nthreads)))
    return time.perf_counter() - t0, infos


def cpu_baseline_sample(n_sample, n_full):
    """The FP64 oracle (plain C) solving the same recipe at n_sample^3, scaled by
    (n_sample/n_full)^3 to the full workload (its cost per solve grows linearly
    with the cell count at a fixed iteration count): once on one core, and as
    throughput of one concurrent solve per host core (the reported value)."""
    import oracle as O
    from paper_1908_03634_gb300 import workloads as W
    O.build()
    w = W.planar256(device="cpu", n=n_sample)
    b0 = O.fill(w.geom, w.prof_beta0)
    scale = (n_sample / n_full) ** 3
    dt1, i1 = oracle_solves(w, b0, 1)
    nc = host_cores()
    dtn, _ = oracle_solves(w, b0, nc)
    return {"value": round(scale * nc / dtn, 6), "unit": UNIT, "cores": nc, "kind": "oracle",
            "sample": f"{nc} concurrent oracle solves (one per host core) of the planar{n_full} recipe at "
                      f"{n_sample}^3 in {dtn:.2f} s wall, each {i1[0]['iters']} MG-PCG iterations to 1e-10, "
                      f"scaled by ({n_sample}/{n_full})^3",
            "one_core": {"value": round(scale / dt1, 6), "cores": 1, "sample": f"one solve at {n_sample}^3 "
                         f"({dt1:.2f} s), scaled by ({n_sample}/{n_full})^3"}}


def run_reference(args):
    """The CPU oracle as the reference arm: each step solves the planar recipe at
    64^3 (a bounded sample) once per host core, concurrently; reported in solves/s
    of the full workload."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle as O
    from paper_1908_03634_gb300 import workloads as W
    O.build()
    ns = 64
    w = W.planar256(device="cpu", n=ns)
    b0 = O.fill(w.geom, w.prof_beta0)
    nc = host_cores()
    for _ in range(args.warmup):
        oracle_solves(w, b0, nc)
    t = 0.0
    for _ in range(args.steps):
        dt, infos = oracle_solves(w, b0, nc)
        t += dt
    dt = t / args.steps
    scale = (ns / args.n) ** 3
    v = scale * nc / dt
    sample = (f"{nc} concurrent oracle solves (one per host core) of the planar{args.n} recipe at {ns}^3 per "
              f"step ({dt:.3f} s wall, {infos[0]['iters']} MG-PCG iterations each), scaled by ({ns}/{args.n})^3")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"planar{args.n}", "rel_tol": 1e-10},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": nc, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def bench_star(mx, W, ctx, dev, stream, hbm=6793.4, steps=10, warmup=3, n=512):
    """Full-star MAC projection (Dirichlet walls, radial base state with the 1e-6
    floor beyond r = 0.45, 1e6 contrast) at n^3: mixed precision at the autotuned
    settings, the plain FP64 solve and FCG(1) beside it; solves/s, V-cycles and
    the HBM fraction per V-cycle (the same model as the planar line)."""
    import torch
    w = W.star512(device=dev, n=n)
    g = w.geom
    beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=dev)
    phi = torch.zeros_like(beta0)
    us = [[t.clone() for t in w.u] for _ in range(min(steps + warmup, 4))]

    def step(i, o):
        u = us[i % len(us)]
        for d in range(3):
            u[d].copy_(w.u[d])
        mx.mx_fill_base_state(ctx, g, 1, w.prof_beta0, w.prof_dr, w.center, beta0)
        return mx.mx_mac_project(ctx, g, *u, w.rho, beta0, w.sbar, phi, o)[1]
    mx.mx_fill_base_state(ctx, g, 1, w.prof_beta0, w.prof_dr, w.center, beta0)
    tuned, _ = mx.mx_autotune(ctx, mx.MX_OP_MAC, g, *w.u, w.rho, beta0, w.sbar)
    o = mx.default_opts(nu1=0, nu2=0)
    for i in range(warmup):
        step(i, o)
    ms, infos = timed(lambda i: step(i, o), steps, stream)
    o64 = mx.default_opts(prec=mx.MX_PREC_FP64, nu1=tuned.nu1, nu2=tuned.nu2, tile_z=tuned.tile_z)
    step(0, o64)
    k64 = 2
    ms64, i64 = timed(lambda i: step(i, o64), k64, stream)
    ok = mx.default_opts(nu1=0, nu2=0, krylov=1)
    step(0, ok)
    kk = max(2, steps // 2)
    msk, ik = timed(lambda i: step(i, ok), kk, stream)
    last = infos[-1]
    vc = last["vcycles"]
    ms_s = ms / steps
    out = {"workload": f"star{n}", "metric": f"MAC projection solves/s to 1e-10 (full star {n}^3, Dirichlet)",
           "value": 1e3 / ms_s, "unit": "solves/s", "ms_per_solve": ms_s, "vcycles": vc,
           "rel_resid": last["rel_resid"], "div_err_linf": last["div_err_linf"], "rhs_linf": last["rhs_linf"],
           "div_err_rel": last["div_err_linf"] / max(last["rhs_linf"], 1e-300),
           "per_vcycle": roofline_per_vcycle(g.ncell, tuned.nu1, tuned.nu2, 4, ms_s, vc, hbm),
           "fp64": {"solves_per_s": k64 * 1e3 / ms64, "ms_per_solve": ms64 / k64, "vcycles": i64[-1]["vcycles"],
                    "per_vcycle": roofline_per_vcycle(g.ncell, tuned.nu1, tuned.nu2, 8, ms64 / k64,
                                                      i64[-1]["vcycles"], hbm)},
           "fcg": {"solves_per_s": kk * 1e3 / msk, "ms_per_solve": msk / kk, "vcycles": ik[-1]["vcycles"],
                   "rel_resid": ik[-1]["rel_resid"]},
           "tuned": {"nu1": tuned.nu1, "nu2": tuned.nu2, "tile_z": tuned.tile_z, "fused": tuned.fused},
           "note": "each solve includes a 3-array restore of U and the Fill of beta0"}
    del w, us, beta0, phi
    torch.cuda.empty_cache()
    return out


def composite_iteration_bytes(nc, nf, nu1, nu2):
    """Algorithmic bytes of one refinement iteration of the composite projection
    (coarse level of nc cells, patch of nf cells): the FP64 composite residual
    (phi, rho, beta0, f read, r written: 40 B per cell; on the patch twice, before
    and after the coarse correction), the FP32 right-hand sides (r read, rhat
    written: 12 B per cell, and the fine residual read once more for the covered
    coarse cells: 8 B per fine cell), one V-cycle of each grid (the single-level
    model: 8/7 x 4 x (6 (nu1 + nu2) + 7.25) B per cell) and the FP64 updates (phi
    read and written, e read: 20 B per cell; the patch takes two)."""
    v = (8.0 / 7.0) * 4 * (6.0 * (nu1 + nu2) + 7.25)
    return nc * (40 + 12 + v + 20) + nf * (2 * 40 + 8 + 12 + v + 2 * 20)


def bench_composite(mx, W, ctx, dev, stream, hbm=6793.4, n=128, steps=5, warmup=2):
    """The two-level composite MAC projection on the planar workload with a
    ratio-2 patch over the middle half of the box (coarse n^3, patch n^3 fine
    cells): solves/s, refinement iterations and the HBM fraction per iteration."""
    import torch
    q = n // 4
    w = W.composite_planar(n, (q, q, q), (3 * q, 3 * q, 3 * q), W.H_1E5, 0.6, 16, 3, 1, device=dev)
    g = w.geom
    pc = torch.zeros_like(w.rho_c)
    pf = torch.zeros_like(w.rho_f)
    uc = [t.clone() for t in w.u_c]
    uf = [t.clone() for t in w.u_f]
    o = mx.default_opts()

    def step(i):
        for d in range(3):
            uc[d].copy_(w.u_c[d])
            uf[d].copy_(w.u_f[d])
        return mx.mx_mac_project_composite(ctx, g, w.plo, w.phi, uc, w.rho_c, w.beta0_c, w.sbar_c, pc, uf, w.rho_f,
                                           w.beta0_f, w.sbar_f, pf, o)[1]
    for i in range(warmup):
        step(i)
    ms, infos = timed(step, steps, stream)
    last = infos[-1]
    nc, nf = g.ncell, pf.numel()
    ms_s = ms / steps
    it = max(last["outer_iters"], 1)
    b = composite_iteration_bytes(nc, nf, 2, 2)
    out = {"workload": f"composite_planar{n}", "coarse_cells": nc, "fine_cells": nf, "patch": [w.plo, w.phi],
           "solves_per_s": 1e3 / ms_s, "ms_per_solve": ms_s, "iterations": last["outer_iters"],
           "vcycles": last["vcycles"], "rel_resid": last["rel_resid"],
           "div_err_rel": last["div_err_linf"] / max(last["rhs_linf"], 1e-300),
           "model_bytes_per_iteration": b, "ms_per_iteration": ms_s / it,
           "hbm_frac_per_iteration": round(b / (ms_s / it * 1e-3) / 1e9 / hbm, 4),
           "note": "each solve includes the restore of U on both levels; the refinement loop is one conditional CUDA graph"}
    del w, uc, uf, pc, pf
    torch.cuda.empty_cache()
    return out


def bench_planar32_fp64(mx, W, ctx, dev, stream, steps=20, warmup=3):
    """The 32^3 planar smoke configuration (H = 0.1, beta0 = rho0): plain FP64
    projection to 1e-10, solves/s (launch-latency bound at this size)."""
    import torch
    w = W.planar32(device=dev)
    g = w.geom
    beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=dev)
    mx.mx_fill_base_state(ctx, g, 0, w.prof_beta0, g.dx, (0.5, 0.5, 0.5), beta0)
    phi = torch.zeros_like(beta0)
    u = [t.clone() for t in w.u]
    o = mx.default_opts(prec=mx.MX_PREC_FP64)

    def step(i):
        for d in range(3):
            u[d].copy_(w.u[d])
        return mx.mx_mac_project(ctx, g, *u, w.rho, beta0, w.sbar, phi, o)[1]
    for i in range(warmup):
        step(i)
    ms, infos = timed(step, steps, stream)
    last = infos[-1]
    return {"workload": "planar32", "prec": "fp64", "solves_per_s": steps * 1e3 / ms, "ms_per_solve": ms / steps,
            "vcycles": last["vcycles"], "rel_resid": last["rel_resid"],
            "div_err_rel": last["div_err_linf"] / max(last["rhs_linf"], 1e-300)}


def bench_nodal_sweep(mx, W, ctx, dev, stream, hbm, sizes=(64, 128, 192, 256, 384, 512)):
    """The nodal projection's size sweep: per size the tuned mixed solve, its
    time per V-cycle and HBM fraction per V-cycle (FP64 beside it up to 256^3)."""
    import torch
    out = []
    for n in sizes:
        r = bench_nodal(mx, W, ctx, dev, stream, n=n, steps=2, warmup=1, fp64=(n <= 256), hbm=hbm)
        r.pop("phases", None)
        out.append(r)
        torch.cuda.empty_cache()
    return out


def run_other(args):
    """--workload star512 | nodal-sweep | nodal384 (single GPU) | batched96
    (patches sharded over the ranks under torchrun)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.workload != "batched96":
        if rank != 0:
            return
        world = 1
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    from paper_1908_03634_gb300 import build as B
    B.build()
    import paper_1908_03634_gb300 as mx
    from paper_1908_03634_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    ctx = mx.mx_create(local, stream)
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        peaks = {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    if args.workload == "average512":
        r = bench_base(mx, W, ctx, dev, stream, hbm=hbm, steps=args.steps, warmup=args.warmup,
                       cpu=not args.no_cpu_baseline, n=args.star_n)
        print(json.dumps(r), flush=True)
    elif args.workload == "nodal384":
        r = bench_nodal(mx, W, ctx, dev, stream, n=args.nodal_n, steps=args.steps, warmup=args.warmup,
                        fp64=not args.no_fp64, hbm=hbm, graph=not args.no_graph, fixed=args.fixed)
        print(json.dumps(r), flush=True)
    elif args.workload == "batched96":
        r = bench_batched(mx, W, ctx, dev, stream, steps=args.steps, warmup=args.warmup,
                          fp64=not args.no_fp64 and world == 1, rank=rank, world=world, graph=not args.no_graph,
                          fixed=args.fixed)
        if rank == 0:
            print(json.dumps(r), flush=True)
    elif args.workload == "composite":
        print(json.dumps(bench_composite(mx, W, ctx, dev, stream, hbm=hbm, n=args.comp_n, steps=args.steps,
                                         warmup=args.warmup)), flush=True)
    elif args.workload == "nodal-sweep":
        for r in bench_nodal_sweep(mx, W, ctx, dev, stream, hbm):
            print(json.dumps(r), flush=True)
    else:
        print(json.dumps(bench_star(mx, W, ctx, dev, stream, hbm=hbm, steps=args.steps, warmup=args.warmup)),
              flush=True)
    mx.mx_destroy(ctx)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload != "planar256":
        run_other(a)
    else:
        run_mx(a)
