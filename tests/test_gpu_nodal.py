"""GPU parity of the nodal projection (Step 11; Eq. div3) against the FP64 CPU
oracle through the C ABI.

Tolerances: FP64 operator/residual 1e-12 of the terms' scale (rounding order
only); FP32 operator 3e-6 of the scale (20 FP32 terms); projection: phi within
1e-8 relative max norm of the oracle solved to 1e-13, U equal to the oracle's
correction of the GPU phi to 1e-12, GPU residual <= 1e-10.  The same bars hold
with either smoother (four-colour Gauss-Seidel or Chebyshev): the smoother
changes the iterates, not the converged answer.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1908_03634_gb300 import workloads as W

pytestmark = pytest.mark.gpu

P, N = W.PERIODIC, W.NEUMANN
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


def geom(n, bc):
    return W.Geom(tuple(n), 1.0 / n[0], tuple(bc), tuple(bc))


GEOMS = [((16, 16, 16), (P, P, N)), ((40, 12, 18), (P, P, N)), ((10, 6, 8), (N, N, N)),
         ((8, 8, 8), (P, P, P)), ((6, 4, 2), (N, P, N))]


@pytest.mark.parametrize("n,bc", GEOMS)
def test_nodal_apply_and_residual(mx, ctx, n, bc):
    g = geom(n, bc)
    rng = np.random.default_rng(8)
    cs, ns = O.cell_shape(g), O.node_shape(g)
    rho, beta0 = np.exp(rng.standard_normal(cs)), np.exp(rng.standard_normal(cs))
    phi, f = rng.standard_normal(ns), rng.standard_normal(ns)
    sigma = beta0 / rho
    ref = O.nd_apply(g, sigma, phi)
    scale = 32 * sigma.max() * np.abs(phi).max() / g.dx ** 2
    out = torch.empty(ns, dtype=torch.float64, device=DEV)
    mx.mx_apply_op(ctx, g, mx.MX_OP_NODAL, mx.MX_PREC_FP64, cuda(rho), cuda(beta0), cuda(phi), out)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * scale
    mx.mx_apply_op(ctx, g, mx.MX_OP_NODAL, mx.MX_PREC_MIXED, cuda(rho), cuda(beta0), cuda(phi), out)
    assert np.abs(out.cpu().numpy() - ref).max() <= 3e-6 * scale
    r = torch.empty_like(out)
    rn = mx.mx_residual(ctx, g, mx.MX_OP_NODAL, mx.MX_PREC_FP64, cuda(rho), cuda(beta0), cuda(phi), cuda(f), r)
    assert np.abs(r.cpu().numpy() - (f - ref)).max() <= 1e-12 * scale
    assert abs(rn - np.abs(f - ref).max()) <= 1e-12 * scale


NODAL_WORKLOADS = {
    "nodal384_at_24": lambda: W.planar_nodal(24, W.H_1E5, 0.6, 16, 3, 4),
    "ragged_40x24x32": lambda: W.planar_nodal((40, 24, 32), 0.2, 0.6, 8, 2, 5),
    "periodic_16": lambda: W.Workload(**{**W.planar_nodal(16, 0.3, 0.6, 8, 1, 6).__dict__,
                                         "geom": geom((16, 16, 16), (P, P, P))}),
}


def run_gpu_nodal(mx, ctx, w, prec, **kw):
    g = w.geom
    beta0 = torch.empty(O.cell_shape(g), dtype=torch.float64, device=DEV)
    if all(b == P for b in g.lo):
        beta0.copy_(torch.broadcast_to(cuda(w.prof_beta0)[:, None, None], beta0.shape))
    else:
        mx.mx_fill_base_state(ctx, g, 0, cuda(w.prof_beta0), w.prof_dr, w.center, beta0)
    u = [cuda(t) for t in w.u]
    phi = torch.zeros(O.node_shape(g), dtype=torch.float64, device=DEV)
    st, info = mx.mx_nodal_project(ctx, g, *u, cuda(w.rho), beta0, cuda(w.sbar), phi,
                                   mx.default_opts(prec=prec, **kw), allow=(mx.MX_OK, mx.MX_ERR_NOCONV))
    torch.cuda.synchronize()
    return st, info, phi.cpu().numpy(), [x.cpu().numpy() for x in u], beta0.cpu().numpy()


@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", list(NODAL_WORKLOADS))
def test_nodal_project_parity(mx, ctx, name, prec, smoother):
    w = NODAL_WORKLOADS[name]()
    g = w.geom
    st, info, phi, u, b0 = run_gpu_nodal(mx, ctx, w, prec, smoother=smoother)
    assert st == mx.MX_OK, info
    assert info["rel_resid"] <= 1e-10
    u_ref, phi_ref, oinfo = O.nd_project(g, w.u, w.rho, b0, w.sbar, tol=1e-13, maxit=400)
    assert oinfo["ok"]
    assert np.abs(phi - phi_ref).max() <= 1e-8 * np.abs(phi_ref).max()
    u_pred = O.nd_correct(g, w.rho, phi, w.u)
    for d in range(3):
        scale = np.abs(w.u[d].numpy()).max() + np.abs(u_pred[d] - w.u[d].numpy()).max()
        assert np.abs(u[d] - u_pred[d]).max() <= 1e-12 * scale
    assert abs(info["rhs_mean_removed"] - oinfo["mean"]) <= 1e-12 * max(1.0, abs(oinfo["mean"]))
    # the approximate projection's divergence error agrees with the oracle's measure of it
    f, _ = O.nd_rhs(g, u, b0, w.sbar, remove_mean=False)
    assert abs(info["div_err_linf"] - np.abs(f - oinfo["mean"]).max()) <= 1e-9 * np.abs(f).max()


def test_nodal_zero_rhs(mx, ctx):
    g = geom((8, 8, 8), (P, P, N))
    cs = O.cell_shape(g)
    one = torch.ones(cs, dtype=torch.float64, device=DEV)
    u = [torch.zeros(cs, dtype=torch.float64, device=DEV) for _ in range(3)]
    phi = torch.full(O.node_shape(g), 2.0, dtype=torch.float64, device=DEV)
    st, info = mx.mx_nodal_project(ctx, g, *u, one, one, torch.zeros_like(one), phi, mx.default_opts())
    assert st == 0 and info["vcycles"] == 0
    assert torch.count_nonzero(phi).item() == 0


def test_nodal_rejects_dirichlet(mx, ctx):
    g = geom((8, 8, 8), (W.DIRICHLET,) * 3)
    cs = O.cell_shape(g)
    one = torch.ones(cs, dtype=torch.float64, device=DEV)
    u = [one.clone() for _ in range(3)]
    phi = torch.zeros((9, 9, 9), dtype=torch.float64, device=DEV)
    with pytest.raises(mx.MXError) as e:
        mx.mx_nodal_project(ctx, g, *u, one, one, one, phi, mx.default_opts())
    assert e.value.status == mx.MX_ERR_ARG


@pytest.mark.parametrize("cheb", [None, (1, 2), (2, 3)])
@pytest.mark.parametrize("prec", [0, 1])
def test_nodal_graph_and_host_loop_identical(mx, ctx, prec, cheb):
    """The refinement loop captured as a conditional-while CUDA graph runs the
    same kernels as the host-driven loop: bit-identical phi and U, twice (with
    the Chebyshev smoother at odd step counts too, where the steps ping-pong
    between two correction buffers)."""
    w = NODAL_WORKLOADS["ragged_40x24x32"]()
    kw = {} if cheb is None else {"smoother": 1, "nu1": cheb[0], "nu2": cheb[1]}
    r1 = run_gpu_nodal(mx, ctx, w, prec, use_graph=1, **kw)
    r2 = run_gpu_nodal(mx, ctx, w, prec, use_graph=0, **kw)
    r3 = run_gpu_nodal(mx, ctx, w, prec, use_graph=1, **kw)
    assert r1[0] == mx.MX_OK and r1[1]["vcycles"] == r2[1]["vcycles"] > 0
    assert np.array_equal(r1[2], r2[2]) and np.array_equal(r1[2], r3[2])
    for d in range(3):
        assert np.array_equal(r1[3][d], r2[3][d])


@pytest.mark.parametrize("use_graph", [0, 1])
def test_nodal_iteration_cap_reports_noconv(mx, ctx, use_graph):
    w = NODAL_WORKLOADS["ragged_40x24x32"]()
    st, info, phi, _, _ = run_gpu_nodal(mx, ctx, w, 1, use_graph=use_graph, max_outer=2)
    assert st == mx.MX_ERR_NOCONV and info["status"] == mx.MX_ERR_NOCONV
    assert info["vcycles"] == 2 and info["rel_resid"] > 1e-10
    assert np.isfinite(phi).all()


@pytest.mark.parametrize("nu", [(1, 1), (2, 1), (1, 3), (3, 3), (4, 2)])
def test_nodal_chebyshev_degrees_converge_to_the_oracle(mx, ctx, nu):
    """Every split of the Chebyshev roots between pre- and post-smoothing
    converges to the oracle's phi."""
    w = NODAL_WORKLOADS["nodal384_at_24"]()
    st, info, phi, u, b0 = run_gpu_nodal(mx, ctx, w, 1, smoother=1, nu1=nu[0], nu2=nu[1])
    assert st == mx.MX_OK and info["rel_resid"] <= 1e-10, info
    _, phi_ref, oinfo = O.nd_project(w.geom, w.u, w.rho, b0, w.sbar, tol=1e-13, maxit=400)
    assert np.abs(phi - phi_ref).max() <= 1e-8 * np.abs(phi_ref).max()


def test_smoother_option_rejected_where_not_offered(mx, ctx):
    """smoother = 1 is a nodal option; the MAC and batched solves reject it, and
    every solve rejects an unknown smoother."""
    g = geom((8, 8, 8), (P, P, N))
    cs = O.cell_shape(g)
    one = torch.ones(cs, dtype=torch.float64, device=DEV)
    z = torch.zeros(cs, dtype=torch.float64, device=DEV)
    uf = [torch.zeros(tuple(reversed([g.n[e] + (1 if e == d else 0) for e in range(3)])), dtype=torch.float64,
                      device=DEV) for d in range(3)]
    with pytest.raises(mx.MXError) as e:
        mx.mx_mac_project(ctx, g, *uf, one, one, z, z.clone(), mx.default_opts(smoother=1))
    assert e.value.status == mx.MX_ERR_ARG
    with pytest.raises(mx.MXError) as e:
        mx.mx_mac_project_batched(ctx, [g], [uf[0]], [uf[1]], [uf[2]], [one], [one], [z], [z.clone()],
                                  mx.default_opts(smoother=1))
    assert e.value.status == mx.MX_ERR_ARG
    u = [z.clone() for _ in range(3)]
    phi = torch.zeros(O.node_shape(g), dtype=torch.float64, device=DEV)
    for bad in (2, -1):
        with pytest.raises(mx.MXError) as e:
            mx.mx_nodal_project(ctx, g, *u, one, one, z, phi, mx.default_opts(smoother=bad))
        assert e.value.status == mx.MX_ERR_ARG
