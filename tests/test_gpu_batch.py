"""Batched MAC projections (many independent boxes, one launch per phase over a
work list of tiles of all boxes) through the C ABI.

Each box's phi must equal the single-box solve of the same box bit for bit
(the batched phases run the same per-tile arithmetic and take the same
convergence decisions), and match the FP64 oracle within 1e-8.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1908_03634_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def mx():
    from paper_1908_03634_gb300 import build as b
    b.build()
    O.build()
    import paper_1908_03634_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(mx):
    c = mx.mx_create(0)
    yield c
    mx.mx_destroy(c)


def cuda(a):
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(a)
    return a.to(DEV, torch.float64).contiguous()


def box_arrays(mx, ctx, w):
    g = w.geom
    beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_fill_base_state(ctx, g, 0, cuda(w.prof_beta0), w.prof_dr, w.center, beta0)
    return dict(u=[cuda(t) for t in w.u], rho=cuda(w.rho), beta0=beta0, sbar=cuda(w.sbar),
                phi=torch.zeros(mx.cell_shape(g), dtype=torch.float64, device=DEV))


def run_batch(mx, ctx, ws, **kw):
    arrs = [box_arrays(mx, ctx, w) for w in ws]
    st, infos = mx.mx_mac_project_batched(
        ctx, [w.geom for w in ws], [a["u"][0] for a in arrs], [a["u"][1] for a in arrs],
        [a["u"][2] for a in arrs], [a["rho"] for a in arrs], [a["beta0"] for a in arrs],
        [a["sbar"] for a in arrs], [a["phi"] for a in arrs], mx.default_opts(**kw),
        allow=(mx.MX_OK, mx.MX_ERR_NOCONV))
    torch.cuda.synchronize()
    return st, infos, arrs


def test_batched_matches_single_box_solves_and_oracle(mx, ctx):
    ws = W.batched_patches(npatch=7, sizes=(16, 24, 32, 48), seed=11)
    st, infos, arrs = run_batch(mx, ctx, ws)
    assert st == mx.MX_OK
    for w, info, a in zip(ws, infos, arrs):
        assert info["status"] == 0 and info["rel_resid"] <= 1e-10
        single = box_arrays(mx, ctx, w)
        s2, i2 = mx.mx_mac_project(ctx, w.geom, *single["u"], single["rho"], single["beta0"], single["sbar"],
                                   single["phi"], mx.default_opts())
        assert i2["vcycles"] == info["vcycles"]
        assert torch.equal(single["phi"], a["phi"])
        for d in range(3):
            assert torch.equal(single["u"][d], a["u"][d])
    # oracle parity for two boxes
    for w, a in list(zip(ws, arrs))[:2]:
        b0 = O.fill(w.geom, w.prof_beta0)
        _, phi_ref, oinfo = O.mac_project(w.geom, w.u, w.rho, b0, w.sbar, tol=1e-13, maxit=400)
        phi = a["phi"].cpu().numpy()
        assert np.abs(phi - phi_ref).max() <= 1e-8 * np.abs(phi_ref).max()


def test_batched_with_a_box_converged_at_start(mx, ctx):
    ws = W.batched_patches(npatch=3, sizes=(16, 32), seed=12)
    z = W.planar(16, 0.2, 0.6, 4, 1, 13)
    z.u = [torch.zeros_like(t) for t in z.u]
    z.sbar = torch.zeros_like(z.sbar)
    ws.insert(1, z)
    st, infos, arrs = run_batch(mx, ctx, ws)
    assert st == mx.MX_OK
    assert infos[1]["vcycles"] == 0 and torch.count_nonzero(arrs[1]["phi"]).item() == 0
    assert all(i["vcycles"] > 0 for j, i in enumerate(infos) if j != 1)


def test_batched_host_loop_equals_graph(mx, ctx):
    ws = W.batched_patches(npatch=4, sizes=(16, 32), seed=14)
    _, i1, a1 = run_batch(mx, ctx, ws, use_graph=1)
    _, i2, a2 = run_batch(mx, ctx, ws, use_graph=0)
    for x, y in zip(a1, a2):
        assert torch.equal(x["phi"], y["phi"])


def test_batched_fp64_loops_single_solves(mx, ctx):
    ws = W.batched_patches(npatch=3, sizes=(16, 24), seed=15)
    st, infos, arrs = run_batch(mx, ctx, ws, prec=0)
    assert st == mx.MX_OK and all(i["rel_resid"] <= 1e-10 for i in infos)
