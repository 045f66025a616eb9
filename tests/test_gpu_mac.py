"""GPU parity of the MAC projection path (CUDA library through the C ABI)
against the FP64 CPU oracle, on the same seeded inputs.

Tolerances:
  * FP64 operator / residual / fill: 1e-12 of the terms' scale (rounding order
    differs between the two sides; nothing else may);
  * FP32 operator: 2e-6 of the terms' scale (FP32 unit roundoff 6e-8 times the
    7-term sum and the coefficient rounding);
  * projection: phi within 1e-8 relative max norm of the oracle solved to
    1e-13, U within 1e-8 of max|U|, GPU residual <= 1e-10 (the stated target).
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


def geom(n, lo, hi=None):
    return W.Geom(tuple(n), 1.0 / n[0], tuple(lo), tuple(hi if hi is not None else lo))


GEOMS = [
    ((32, 32, 32), (P, P, N)),
    ((70, 18, 20), (P, P, N)),      # several tiles + ragged tail in x, y, z
    ((37, 21, 9), (D, N, D)),       # odd sizes: the hierarchy stops at once
    ((48, 40, 24), (N, P, P)),
    ((16, 16, 16), (D, D, D)),
    ((2, 2, 2), (P, P, P)),
    ((1, 5, 3), (N, D, N)),
]


def rand_fields(g, seed):
    rng = np.random.default_rng(seed)
    cs = O.cell_shape(g)
    return np.exp(rng.standard_normal(cs)), np.exp(rng.standard_normal(cs)), rng.standard_normal(cs)


@pytest.mark.parametrize("n,bc", GEOMS)
def test_apply_fp64_and_fp32(mx, ctx, n, bc):
    g = geom(n, bc)
    rho, beta0, phi = rand_fields(g, 1)
    b = O.mac_coeffs(g, rho, beta0)
    ref = O.mac_apply(g, b, phi)
    scale = 12 * max(np.abs(x).max() for x in b) * np.abs(phi).max() / g.dx ** 2
    out = torch.empty(O.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_apply_op(ctx, g, mx.MX_OP_MAC, mx.MX_PREC_FP64, cuda(rho), cuda(beta0), cuda(phi), out)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * scale
    mx.mx_apply_op(ctx, g, mx.MX_OP_MAC, mx.MX_PREC_MIXED, cuda(rho), cuda(beta0), cuda(phi), out)
    assert np.abs(out.cpu().numpy() - ref).max() <= 2e-6 * scale


@pytest.mark.parametrize("n,bc", GEOMS[:4])
def test_residual_fp64(mx, ctx, n, bc):
    g = geom(n, bc)
    rho, beta0, phi = rand_fields(g, 2)
    f = np.random.default_rng(3).standard_normal(O.cell_shape(g))
    b = O.mac_coeffs(g, rho, beta0)
    ref = f - O.mac_apply(g, b, phi)
    scale = 12 * max(np.abs(x).max() for x in b) * np.abs(phi).max() / g.dx ** 2
    r = torch.empty_like(cuda(f))
    rn = mx.mx_residual(ctx, g, mx.MX_OP_MAC, mx.MX_PREC_FP64, cuda(rho), cuda(beta0), cuda(phi), cuda(f), r)
    assert np.abs(r.cpu().numpy() - ref).max() <= 1e-12 * scale
    assert abs(rn - np.abs(ref).max()) <= 1e-12 * scale


def test_fill_planar_and_spherical(mx, ctx):
    g = geom((24, 20, 28), (D, D, D))
    prof = np.linspace(1.0, 3.0, 40) ** 2
    out = torch.empty(O.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_fill_base_state(ctx, g, 0, cuda(prof), g.dx, (0.5, 0.5, 0.5), out)
    assert np.array_equal(out.cpu().numpy(), O.fill(g, prof))
    w = W.star(24, 4, 2)
    o2 = torch.empty((24, 24, 24), dtype=torch.float64, device=DEV)
    mx.mx_fill_base_state(ctx, w.geom, 1, cuda(w.prof_beta0), w.prof_dr, w.center, o2)
    ref = O.fill(w.geom, w.prof_beta0, spherical=True, dr=w.prof_dr, center=w.center)
    assert np.abs(o2.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max()   # FMA contraction differs


def run_gpu_project(mx, ctx, w, prec, **kw):
    g = w.geom
    beta0 = torch.empty(O.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_fill_base_state(ctx, g, int(w.spherical), cuda(w.prof_beta0), w.prof_dr, w.center, beta0)
    u = [cuda(t) for t in w.u]
    phi = torch.zeros(O.cell_shape(g), dtype=torch.float64, device=DEV)
    opts = mx.default_opts(prec=prec, **kw)
    st, info = mx.mx_mac_project(ctx, g, *u, cuda(w.rho), beta0, cuda(w.sbar), phi, opts,
                                 allow=(mx.MX_OK, mx.MX_ERR_NOCONV))
    torch.cuda.synchronize()
    return st, info, phi.cpu().numpy(), [x.cpu().numpy() for x in u], beta0.cpu().numpy()


def oracle_project(w):
    b0 = O.fill(w.geom, w.prof_beta0, spherical=w.spherical, dr=w.prof_dr, center=w.center)
    u, phi, info = O.mac_project(w.geom, w.u, w.rho, b0, w.sbar, tol=1e-13, maxit=400)
    assert info["ok"]
    return u, phi, info, b0


WORKLOADS = {
    "planar32": lambda: W.planar32(),
    "planar256_at_48": lambda: W.planar(48, W.H_1E5, 0.6, 16, 3, 1),
    "star512_at_40": lambda: W.star(40, 32, 2),
    "ragged_neumann": lambda: W.planar((40, 24, 56), 0.2, 0.6, 8, 2, 7),
}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_mac_project_parity(mx, ctx, name, prec):
    w = WORKLOADS[name]()
    st, info, phi, u, b0 = run_gpu_project(mx, ctx, w, prec)
    u_ref, phi_ref, oinfo, b0_ref = oracle_project(w)
    assert st == mx.MX_OK, info
    assert info["rel_resid"] <= 1e-10
    assert np.abs(b0 - b0_ref).max() <= 1e-14 * np.abs(b0_ref).max()
    assert np.abs(phi - phi_ref).max() <= 1e-8 * np.abs(phi_ref).max()
    # the velocity correction, element by element: the oracle's correction
    # applied to the GPU's phi (U differs from the oracle's U only through
    # grad(phi_gpu - phi_ref)/rho_f, which 1/rho amplifies in light layers)
    u_pred = O.mac_correct(w.geom, w.rho, phi, w.u)
    for d in range(3):
        scale = np.abs(w.u[d].numpy()).max() + np.abs(u_pred[d] - w.u[d].numpy()).max()
        assert np.abs(u[d] - u_pred[d]).max() <= 1e-12 * scale
    assert abs(info["rhs_mean_removed"] - oinfo["mean"]) <= 1e-12 * max(1.0, abs(oinfo["mean"]))
    # divergence of the projected U: residual-sized (Eq. div1 up to the solve tolerance)
    f, _ = O.mac_rhs(w.geom, w.u, b0_ref, w.sbar)
    fn = np.abs(f).max()
    dv = O.mac_divergence(w.geom, u, b0_ref) - b0_ref * w.sbar.numpy() - oinfo["mean"]
    assert np.abs(dv).max() <= 2e-10 * fn
    assert info["div_err_linf"] <= 2e-10 * fn


def test_graph_and_host_loop_identical_and_deterministic(mx, ctx):
    w = W.planar(32, 0.1, 1.0, 8, "center", 0)
    r1 = run_gpu_project(mx, ctx, w, 1, use_graph=1)
    r2 = run_gpu_project(mx, ctx, w, 1, use_graph=0)
    r3 = run_gpu_project(mx, ctx, w, 1, use_graph=1)
    assert r1[1]["vcycles"] == r2[1]["vcycles"]
    assert np.array_equal(r1[2], r2[2]) and np.array_equal(r1[2], r3[2])


def test_mixed_uses_fewer_fp64_cycles_than_fp64_cap(mx, ctx):
    w = W.planar(64, W.H_1E5, 0.6, 16, 3, 1)
    _, i32, p32, _, _ = run_gpu_project(mx, ctx, w, 1)
    _, i64, p64, _, _ = run_gpu_project(mx, ctx, w, 0)
    assert i32["status"] == 0 and i64["status"] == 0
    assert np.abs(p32 - p64).max() <= 1e-8 * np.abs(p64).max()
    assert i32["vcycles"] <= 2 * i64["vcycles"] + 2


def test_zero_rhs_gives_zero_phi(mx, ctx):
    g = geom((16, 16, 16), (P, P, N))
    z = torch.zeros(O.cell_shape(g), dtype=torch.float64, device=DEV)
    u = [torch.zeros(g.face_shape(d), dtype=torch.float64, device=DEV) for d in range(3)]
    one = torch.ones_like(z)
    phi = torch.full_like(z, 3.0)
    st, info = mx.mx_mac_project(ctx, g, *u, one, one, z, phi, mx.default_opts())
    assert st == 0 and info["vcycles"] == 0
    assert torch.count_nonzero(phi).item() == 0


def test_noconv_reports_info(mx, ctx):
    w = W.planar(32, 0.1, 1.0, 8, "center", 0)
    st, info, *_ = run_gpu_project(mx, ctx, w, 1, max_outer=1)
    assert st == mx.MX_ERR_NOCONV and info["status"] == mx.MX_ERR_NOCONV
    assert info["vcycles"] == 1 and 0 < info["rel_resid"] < 1


def test_incompatible_rhs_rejected(mx, ctx):
    g = geom((8, 8, 8), (P, P, N))
    one = torch.ones(O.cell_shape(g), dtype=torch.float64, device=DEV)
    u = [torch.zeros(g.face_shape(d), dtype=torch.float64, device=DEV) for d in range(3)]
    phi = torch.zeros_like(one)
    st, info = mx.mx_mac_project(ctx, g, *u, one, one, one, phi, mx.default_opts(remove_mean=0),
                                 allow=(mx.MX_ERR_INCOMPAT,))
    assert st == mx.MX_ERR_INCOMPAT


def test_argument_errors(mx, ctx):
    g = geom((7, 8, 8), (P, P, N))   # odd periodic axis
    one = torch.ones((8, 8, 7), dtype=torch.float64, device=DEV)
    u = [torch.zeros(g.face_shape(d), dtype=torch.float64, device=DEV) for d in range(3)]
    with pytest.raises(mx.MXError) as e:
        mx.mx_mac_project(ctx, g, *u, one, one, one, one.clone(), mx.default_opts())
    assert e.value.status == mx.MX_ERR_ARG
    g2 = geom((8, 8, 8), (P, N, N), (N, N, N))   # periodic on one side only
    one2 = torch.ones((8, 8, 8), dtype=torch.float64, device=DEV)
    u2 = [torch.zeros(g2.face_shape(d), dtype=torch.float64, device=DEV) for d in range(3)]
    with pytest.raises(mx.MXError) as e:
        mx.mx_mac_project(ctx, g2, *u2, one2, one2, one2, one2.clone(), mx.default_opts())
    assert e.value.status == mx.MX_ERR_ARG


FUSED_CASES = {
    # levels of >= 2^18 cells with even n_x run the single-pass kernel
    "planar128": lambda: W.planar(128, W.H_1E5, 0.6, 16, 3, 1),
    "ragged_136x104x96": lambda: W.planar((136, 104, 96), 0.2, 0.6, 8, 2, 7),
    "star_104": lambda: W.star(104, 32, 2),
    "planar32": lambda: W.planar32(),
    "periodic_z_128x64x96": lambda: W.planar((128, 64, 96), 0.3, 0.6, 8, 2, 11, bc_z=W.PERIODIC),
    "dirichlet_z_192x128x64": lambda: W.planar((192, 128, 64), 0.3, 0.6, 8, 2, 12, bc_z=W.DIRICHLET),
}


@pytest.mark.parametrize("nu", [(2, 2), (1, 1), (3, 2), (1, 2)])
@pytest.mark.parametrize("name", list(FUSED_CASES))
def test_single_pass_sweeps_bit_identical_to_two_pass(mx, ctx, name, nu):
    """The fused red+black sweep (with the prolongation applied on load) does
    per cell exactly the arithmetic of the two colour kernels."""
    if name != "planar128" and nu != (2, 2):
        pytest.skip("sweep-count variants on one workload")
    w = FUSED_CASES[name]()
    a = run_gpu_project(mx, ctx, w, 1, fused=1, nu1=nu[0], nu2=nu[1])
    b = run_gpu_project(mx, ctx, w, 1, fused=0, nu1=nu[0], nu2=nu[1])
    assert a[1]["vcycles"] == b[1]["vcycles"]
    assert np.array_equal(a[2], b[2])
    if nu == (2, 2):
        assert a[1]["status"] == 0 and a[1]["rel_resid"] <= 1e-10
