"""The initial-guess option (opts.use_initial_guess = 1) of the MAC, nodal and
batched projections through the C ABI: phi enters as the first iterate of the
refinement loop.

Started from the phi a solve from zero returned, a solve has at most one
V-cycle left to do (the guess re-enters the double-float loop through a split
that keeps 48 of its 53 bits, which moves the residual by round-off only) and
returns that phi to 1e-9 of its scale.  Started from that phi plus a smooth
perturbation of 1% of its scale, it converges to the same phi within the
projection tolerance of the parity tests (1e-8) and needs no more V-cycles than
the solve from zero.  U is restored to the same input for every solve.
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


def beta0_of(mx, ctx, w):
    b0 = torch.empty(O.cell_shape(w.geom), dtype=torch.float64, device=DEV)
    mx.mx_fill_base_state(ctx, w.geom, int(w.spherical), cuda(w.prof_beta0), w.prof_dr, w.center, b0)
    return b0


def smooth(shape):
    """a smooth field of unit amplitude on an array of the given (z, y, x) shape,
    zero on the first and last planes (smooth across periodic boundaries too)"""
    z, y, x = np.meshgrid(*[np.linspace(0.0, 1.0, s) for s in shape], indexing="ij")
    return np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(np.pi * z)


def solve(mx, ctx, w, nodal, b0, phi, **kw):
    u = [cuda(t) for t in w.u]
    fn = mx.mx_nodal_project if nodal else mx.mx_mac_project
    st, info = fn(ctx, w.geom, *u, cuda(w.rho), b0, cuda(w.sbar), phi, mx.default_opts(**kw),
                  allow=(mx.MX_OK, mx.MX_ERR_NOCONV))
    torch.cuda.synchronize()
    return st, info


CASES = {
    "mac_planar32": (False, lambda: W.planar(32, 0.1, 1.0, 8, "center", 0)),
    "mac_ragged": (False, lambda: W.planar((40, 24, 56), 0.2, 0.6, 8, 2, 7)),
    "nodal_columns_24": (True, lambda: W.planar_nodal(24, W.H_1E5, 0.6, 16, 3, 4)),
    "nodal_tiles_40x24x32": (True, lambda: W.planar_nodal((40, 24, 32), 0.2, 0.6, 8, 2, 5)),
}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_initial_guess(mx, ctx, name, prec):
    nodal, make = CASES[name]
    w = make()
    b0 = beta0_of(mx, ctx, w)
    shape = O.node_shape(w.geom) if nodal else O.cell_shape(w.geom)
    phi0 = torch.zeros(shape, dtype=torch.float64, device=DEV)
    st0, i0 = solve(mx, ctx, w, nodal, b0, phi0, prec=prec)
    assert st0 == mx.MX_OK and i0["vcycles"] > 1, i0
    scale = phi0.abs().max().item()
    # from the converged phi
    phi = phi0.clone()
    st, info = solve(mx, ctx, w, nodal, b0, phi, prec=prec, use_initial_guess=1)
    assert st == mx.MX_OK and info["vcycles"] <= 1 and info["rel_resid"] <= 1e-10, info
    assert (phi - phi0).abs().max().item() <= 1e-9 * scale
    # from a perturbed phi
    phi = phi0 + cuda(0.01 * scale * smooth(shape))
    st, info = solve(mx, ctx, w, nodal, b0, phi, prec=prec, use_initial_guess=1)
    assert st == mx.MX_OK and info["rel_resid"] <= 1e-10, info
    assert info["vcycles"] <= i0["vcycles"]
    assert (phi - phi0).abs().max().item() <= 1e-8 * scale


def test_batched_initial_guess(mx, ctx):
    ws = W.batched_patches(npatch=3, sizes=(16, 32), seed=14)
    b0 = [beta0_of(mx, ctx, w) for w in ws]

    def run(phis, **kw):
        us = [[cuda(t) for t in w.u] for w in ws]
        st, infos = mx.mx_mac_project_batched(
            ctx, [w.geom for w in ws], [u[0] for u in us], [u[1] for u in us], [u[2] for u in us],
            [cuda(w.rho) for w in ws], b0, [cuda(w.sbar) for w in ws], phis, mx.default_opts(**kw),
            allow=(mx.MX_OK, mx.MX_ERR_NOCONV))
        torch.cuda.synchronize()
        return st, infos

    phi0 = [torch.zeros(O.cell_shape(w.geom), dtype=torch.float64, device=DEV) for w in ws]
    st, i0 = run(phi0)
    assert st == mx.MX_OK
    phis = [p.clone() for p in phi0]
    st, infos = run(phis, use_initial_guess=1)
    assert st == mx.MX_OK
    for p, q, info in zip(phis, phi0, infos):
        assert info["status"] == 0 and info["vcycles"] <= 1 and info["rel_resid"] <= 1e-10, info
        assert (p - q).abs().max().item() <= 1e-9 * q.abs().max().item()
