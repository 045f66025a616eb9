"""GPU parity of the mixed MAC solve with flexible conjugate gradients
(mx_opts.krylov = 1: FCG(1) with the FP32 V-cycle as preconditioner) against the
FP64 oracle, through the C ABI.

FCG changes how the correction is applied, not the discrete system (Eq. div1,
div2; Appendix A), so the bars are those of the refinement loop: phi within
1e-8 relative max norm of the oracle solved to 1e-13, U element by element
within 1e-12 of the oracle's correction of the GPU phi, the residual at 1e-10
and the divergence of the projected U residual-sized.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1908_03634_gb300 import workloads as W

pytestmark = pytest.mark.gpu

P, N, D = W.PERIODIC, W.NEUMANN, W.DIRICHLET
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


def run(mx, ctx, w, **kw):
    g = w.geom
    beta0 = torch.empty(O.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_fill_base_state(ctx, g, int(w.spherical), cuda(w.prof_beta0), w.prof_dr, w.center, beta0)
    u = [cuda(t) for t in w.u]
    phi = torch.zeros(O.cell_shape(g), dtype=torch.float64, device=DEV)
    opts = mx.default_opts(**kw)
    st, info = mx.mx_mac_project(ctx, g, *u, cuda(w.rho), beta0, cuda(w.sbar), phi, opts,
                                 allow=(mx.MX_OK, mx.MX_ERR_NOCONV))
    torch.cuda.synchronize()
    return st, info, phi.cpu().numpy(), [x.cpu().numpy() for x in u]


WORKLOADS = {
    "planar32": lambda: W.planar32(),
    "planar256_at_48": lambda: W.planar(48, W.H_1E5, 0.6, 16, 3, 1),
    "star512_at_40": lambda: W.star(40, 32, 2),
    "ragged_neumann": lambda: W.planar((40, 24, 56), 0.2, 0.6, 8, 2, 7),
    "periodic_z": lambda: W.planar((64, 32, 48), 0.3, 0.6, 8, 2, 11, bc_z=W.PERIODIC),
    "dirichlet_z_ragged": lambda: W.planar((70, 18, 20), 0.3, 0.6, 8, 2, 12, bc_z=W.DIRICHLET),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_fcg_parity(mx, ctx, name):
    w = WORKLOADS[name]()
    st, info, phi, u = run(mx, ctx, w, prec=1, krylov=1)
    assert st == mx.MX_OK, info
    assert info["rel_resid"] <= 1e-10
    b0 = O.fill(w.geom, w.prof_beta0, spherical=w.spherical, dr=w.prof_dr, center=w.center)
    _, phi_ref, oinfo = O.mac_project(w.geom, w.u, w.rho, b0, w.sbar, tol=1e-13, maxit=400)
    assert oinfo["ok"]
    assert np.abs(phi - phi_ref).max() <= 1e-8 * np.abs(phi_ref).max()
    u_pred = O.mac_correct(w.geom, w.rho, phi, w.u)
    for d in range(3):
        scale = np.abs(w.u[d].numpy()).max() + np.abs(u_pred[d] - w.u[d].numpy()).max()
        assert np.abs(u[d] - u_pred[d]).max() <= 1e-12 * scale
    f, _ = O.mac_rhs(w.geom, w.u, b0, w.sbar)
    dv = O.mac_divergence(w.geom, u, b0) - b0 * w.sbar.numpy() - oinfo["mean"]
    assert np.abs(dv).max() <= 2e-10 * np.abs(f).max()
    assert info["div_err_linf"] <= 2e-10 * np.abs(f).max()


@pytest.mark.parametrize("name", ["planar256_at_48", "star512_at_40"])
def test_fcg_converges_with_single_sweeps(mx, ctx, name):
    """one red+black sweep before and after the coarse correction: FCG still
    reaches the oracle's phi (refinement with this cycle stalls or diverges on
    the 256^3 planar and star workloads)"""
    w = WORKLOADS[name]()
    st, info, phi, _ = run(mx, ctx, w, prec=1, krylov=1, nu1=1, nu2=1)
    assert st == mx.MX_OK and info["rel_resid"] <= 1e-10, info
    b0 = O.fill(w.geom, w.prof_beta0, spherical=w.spherical, dr=w.prof_dr, center=w.center)
    _, phi_ref, oinfo = O.mac_project(w.geom, w.u, w.rho, b0, w.sbar, tol=1e-13, maxit=400)
    assert oinfo["ok"] and np.abs(phi - phi_ref).max() <= 1e-8 * np.abs(phi_ref).max()


@pytest.mark.parametrize("name", ["planar256_at_48", "star512_at_40"])
def test_fcg_needs_no_more_vcycles_than_refinement(mx, ctx, name):
    """the conjugated direction with the exact line search contracts the error
    at least as fast as the plain refinement step (FCG(1) includes it)"""
    w = WORKLOADS[name]()
    a = run(mx, ctx, w, prec=1, krylov=1)
    b = run(mx, ctx, w, prec=1, krylov=0)
    assert a[1]["status"] == 0 and b[1]["status"] == 0
    assert a[1]["vcycles"] <= b[1]["vcycles"], (a[1]["vcycles"], b[1]["vcycles"])
    assert np.abs(a[2] - b[2]).max() <= 1e-8 * np.abs(b[2]).max()


def test_fcg_graph_and_host_loop_identical_and_deterministic(mx, ctx):
    w = W.planar(32, 0.1, 1.0, 8, "center", 0)
    r1 = run(mx, ctx, w, prec=1, krylov=1, use_graph=1)
    r2 = run(mx, ctx, w, prec=1, krylov=1, use_graph=0)
    r3 = run(mx, ctx, w, prec=1, krylov=1, use_graph=1)
    assert r1[1]["vcycles"] == r2[1]["vcycles"]
    assert np.array_equal(r1[2], r2[2]) and np.array_equal(r1[2], r3[2])


def test_fcg_after_refinement_on_the_same_plan(mx, ctx):
    """switching between the two loops on one cached plan re-captures the graph"""
    w = W.planar(32, 0.2, 0.6, 8, 2, 5)
    a = run(mx, ctx, w, prec=1, krylov=0)
    b = run(mx, ctx, w, prec=1, krylov=1)
    c = run(mx, ctx, w, prec=1, krylov=0)
    assert np.array_equal(a[2], c[2])
    assert b[1]["status"] == 0 and np.abs(a[2] - b[2]).max() <= 1e-8 * np.abs(a[2]).max()


def test_fcg_single_pass_sweeps_bit_identical(mx, ctx):
    w = W.planar(128, W.H_1E5, 0.6, 16, 3, 1)
    a = run(mx, ctx, w, prec=1, krylov=1, fused=1)
    b = run(mx, ctx, w, prec=1, krylov=1, fused=0)
    assert a[1]["vcycles"] == b[1]["vcycles"] and np.array_equal(a[2], b[2])


def test_fcg_zero_rhs_and_noconv(mx, ctx):
    g = W.Geom((16, 16, 16), 1.0 / 16, (P, P, N), (P, P, N))
    z = torch.zeros(O.cell_shape(g), dtype=torch.float64, device=DEV)
    u = [torch.zeros(g.face_shape(d), dtype=torch.float64, device=DEV) for d in range(3)]
    one = torch.ones_like(z)
    phi = torch.full_like(z, 3.0)
    st, info = mx.mx_mac_project(ctx, g, *u, one, one, z, phi, mx.default_opts(krylov=1))
    assert st == 0 and info["vcycles"] == 0 and torch.count_nonzero(phi).item() == 0
    w = W.planar(32, 0.1, 1.0, 8, "center", 0)
    st, info, *_ = run(mx, ctx, w, prec=1, krylov=1, max_outer=1)
    assert st == mx.MX_ERR_NOCONV and info["vcycles"] == 1 and 0 < info["rel_resid"] < 1


def test_krylov_option_errors(mx, ctx):
    g = W.Geom((8, 8, 8), 1.0 / 8, (P, P, N), (P, P, N))
    one = torch.ones(O.cell_shape(g), dtype=torch.float64, device=DEV)
    u = [torch.zeros(g.face_shape(d), dtype=torch.float64, device=DEV) for d in range(3)]
    for kw in ({"prec": 0, "krylov": 1}, {"krylov": 2}):
        with pytest.raises(mx.MXError) as e:
            mx.mx_mac_project(ctx, g, *u, one, one, one, one.clone(), mx.default_opts(**kw))
        assert e.value.status == mx.MX_ERR_ARG
    with pytest.raises(mx.MXError) as e:
        mx.mx_mac_project_batched(ctx, [g], *[[x] for x in u], [one], [one], [one], [one.clone()],
                                  mx.default_opts(krylov=1))
    assert e.value.status == mx.MX_ERR_ARG
    cu = [torch.zeros(O.cell_shape(g), dtype=torch.float64, device=DEV) for _ in range(3)]
    phin = torch.zeros((9, 8, 8), dtype=torch.float64, device=DEV)
    with pytest.raises(mx.MXError) as e:
        mx.mx_nodal_project(ctx, g, *cu, one, one, one, phin, mx.default_opts(krylov=1))
    assert e.value.status == mx.MX_ERR_ARG
