"""The autotuner (mx_autotune) and the tile-depth option: the tuned setting is
one of the candidates and is cached per (operator, precision, geometry); the
caller's inputs are left untouched; a call with nu1 = nu2 = 0 reproduces the
explicit tuned call bit for bit; and the stencil tiles' z-depth never changes
a result (it only regroups the same per-cell arithmetic into blocks)."""
import numpy as np
import pytest
import torch

from paper_1908_03634_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
P, N = W.PERIODIC, W.NEUMANN


@pytest.fixture(scope="module")
def mx():
    from paper_1908_03634_gb300 import build as b
    b.build()
    import paper_1908_03634_gb300 as m
    return m


@pytest.fixture()
def ctx(mx):
    c = mx.mx_create(0)
    yield c
    mx.mx_destroy(c)


def mac_inputs(mx, ctx, w):
    g = w.geom
    beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_fill_base_state(ctx, g, 0, w.prof_beta0.to(DEV), w.prof_dr, w.center, beta0)
    return [t.to(DEV).contiguous() for t in w.u], w.rho.to(DEV), beta0, w.sbar.to(DEV)


def mac_solve(mx, ctx, w, inputs, **kw):
    u0, rho, beta0, sbar = inputs
    u = [t.clone() for t in u0]
    phi = torch.zeros(mx.cell_shape(w.geom), dtype=torch.float64, device=DEV)
    st, info = mx.mx_mac_project(ctx, w.geom, *u, rho, beta0, sbar, phi, mx.default_opts(**kw))
    torch.cuda.synchronize()
    return info, phi.cpu().numpy(), [x.cpu().numpy() for x in u]


def nodal_inputs(mx, ctx, w):
    g = w.geom
    beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_fill_base_state(ctx, g, 0, w.prof_beta0.to(DEV), w.prof_dr, w.center, beta0)
    return [t.to(DEV).contiguous() for t in w.u], w.rho.to(DEV), beta0, w.sbar.to(DEV)


def nodal_solve(mx, ctx, w, inputs, **kw):
    u0, rho, beta0, sbar = inputs
    u = [t.clone() for t in u0]
    phi = torch.zeros(mx.node_shape(w.geom), dtype=torch.float64, device=DEV)
    st, info = mx.mx_nodal_project(ctx, w.geom, *u, rho, beta0, sbar, phi, mx.default_opts(**kw))
    torch.cuda.synchronize()
    return info, phi.cpu().numpy(), [x.cpu().numpy() for x in u]


NU = {(2, 2), (1, 1), (2, 1), (1, 2), (3, 2), (2, 3), (3, 3), (4, 4)}
NU_CHEB = {(1, 1), (1, 2), (2, 1), (2, 2), (1, 3), (2, 3), (3, 2), (3, 3)}


@pytest.mark.parametrize("prec", [1, 0])
def test_mac_autotune_choice_cached_and_reproduced(mx, ctx, prec):
    w = W.planar(64, W.H_1E5, 0.6, 16, 3, 1)
    inputs = mac_inputs(mx, ctx, w)
    before = [t.clone() for t in inputs[0]]
    assert mx.mx_tune_lookup(ctx, mx.MX_OP_MAC, prec, w.geom) is None
    best, ms = mx.mx_autotune(ctx, mx.MX_OP_MAC, w.geom, *inputs[0], *inputs[1:],
                              base=mx.default_opts(prec=prec))
    assert ms > 0
    assert (best.nu1, best.nu2) in NU and best.tile_z in (0, 4, 8, 16) and best.fused in (0, 1)
    assert prec == 1 or best.fused == 0
    for a, b in zip(before, inputs[0]):
        assert torch.equal(a, b)
    hit = mx.mx_tune_lookup(ctx, mx.MX_OP_MAC, prec, w.geom)
    assert hit is not None and (hit.nu1, hit.nu2, hit.fused, hit.tile_z) == (best.nu1, best.nu2, best.fused,
                                                                            best.tile_z)
    assert mx.mx_tune_lookup(ctx, mx.MX_OP_MAC, 1 - prec, w.geom) is None
    auto = mac_solve(mx, ctx, w, inputs, prec=prec, nu1=0, nu2=0)
    expl = mac_solve(mx, ctx, w, inputs, prec=prec, nu1=best.nu1, nu2=best.nu2, fused=best.fused,
                     tile_z=best.tile_z)
    assert auto[0]["status"] == 0 and auto[0]["rel_resid"] <= 1e-10
    assert auto[0]["vcycles"] == expl[0]["vcycles"]
    assert np.array_equal(auto[1], expl[1])
    for d in range(3):
        assert np.array_equal(auto[2][d], expl[2][d])


def test_nodal_autotune_choice_cached_and_reproduced(mx, ctx):
    w = W.planar_nodal((40, 24, 32), 0.2, 0.6, 8, 2, 5)
    inputs = nodal_inputs(mx, ctx, w)
    before = [t.clone() for t in inputs[0]]
    best, ms = mx.mx_autotune(ctx, mx.MX_OP_NODAL, w.geom, *inputs[0], *inputs[1:])
    assert best.smoother in (0, 1)
    assert (best.nu1, best.nu2) in (NU if best.smoother == 0 else NU_CHEB)
    assert best.tile_z in (0, 4, 8, 16) and best.fused == 0
    assert mx.mx_tune_lookup(ctx, mx.MX_OP_NODAL, 1, w.geom).smoother == best.smoother
    for a, b in zip(before, inputs[0]):
        assert torch.equal(a, b)
    auto = nodal_solve(mx, ctx, w, inputs, nu1=0, nu2=0)
    expl = nodal_solve(mx, ctx, w, inputs, nu1=best.nu1, nu2=best.nu2, tile_z=best.tile_z, smoother=best.smoother)
    assert auto[0]["status"] == 0 and auto[0]["rel_resid"] <= 1e-10
    assert np.array_equal(auto[1], expl[1])


def test_untuned_auto_is_two_plus_two(mx, ctx):
    w = W.planar(32, 0.1, 1.0, 8, "center", 0)
    inputs = mac_inputs(mx, ctx, w)
    a = mac_solve(mx, ctx, w, inputs, nu1=0, nu2=0)
    b = mac_solve(mx, ctx, w, inputs, nu1=2, nu2=2)
    assert a[0]["vcycles"] == b[0]["vcycles"] and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("tz", [1, 2, 4, 16])
def test_tile_depth_does_not_change_results(mx, ctx, tz):
    w = W.planar((96, 64, 80), 0.3, 0.6, 8, 2, 11)
    inputs = mac_inputs(mx, ctx, w)
    ref = mac_solve(mx, ctx, w, inputs)
    got = mac_solve(mx, ctx, w, inputs, tile_z=tz)
    assert ref[0]["vcycles"] == got[0]["vcycles"] and np.array_equal(ref[1], got[1])
    wn = W.planar_nodal((40, 24, 32), 0.2, 0.6, 8, 2, 5)
    ni = nodal_inputs(mx, ctx, wn)
    nref = nodal_solve(mx, ctx, wn, ni)
    ngot = nodal_solve(mx, ctx, wn, ni, tile_z=tz)
    assert np.array_equal(nref[1], ngot[1])


@pytest.mark.parametrize("tz", [3, 32, -1])
def test_invalid_tile_depth_rejected(mx, ctx, tz):
    w = W.planar(32, 0.1, 1.0, 8, "center", 0)
    inputs = mac_inputs(mx, ctx, w)
    with pytest.raises(mx.MXError) as e:
        mac_solve(mx, ctx, w, inputs, tile_z=tz)
    assert e.value.status == mx.MX_ERR_ARG


def test_batched_autotune_choice_cached_and_reproduced(mx, ctx):
    ws = W.batched_patches(6, seed=5, sizes=(32, 48))
    arrs = []
    for w in ws:
        u, rho, beta0, sbar = mac_inputs(mx, ctx, w)
        arrs.append((u, rho, beta0, sbar))
    geoms = [w.geom for w in ws]
    cols = lambda k: [a[k] for a in arrs]
    us = cols(0)
    before = [[t.clone() for t in u] for u in us]
    best, ms = mx.mx_autotune_batched(ctx, geoms, [u[0] for u in us], [u[1] for u in us], [u[2] for u in us],
                                      cols(1), cols(2), cols(3))
    assert ms > 0 and (best.nu1, best.nu2) in NU
    for a, b in zip(before, us):
        for x, y in zip(a, b):
            assert torch.equal(x, y)

    def solve(**kw):
        uu = [[t.clone() for t in u] for u in us]
        phis = [torch.zeros(mx.cell_shape(g), dtype=torch.float64, device=DEV) for g in geoms]
        st, infos = mx.mx_mac_project_batched(ctx, geoms, [u[0] for u in uu], [u[1] for u in uu],
                                              [u[2] for u in uu], cols(1), cols(2), cols(3), phis,
                                              mx.default_opts(**kw))
        torch.cuda.synchronize()
        return infos, [p.cpu().numpy() for p in phis]

    auto = solve(nu1=0, nu2=0)
    expl = solve(nu1=best.nu1, nu2=best.nu2)
    assert all(i["status"] == 0 and i["rel_resid"] <= 1e-10 for i in auto[0])
    assert [i["vcycles"] for i in auto[0]] == [i["vcycles"] for i in expl[0]]
    for a, b in zip(auto[1], expl[1]):
        assert np.array_equal(a, b)
