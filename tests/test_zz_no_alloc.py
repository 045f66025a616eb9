"""The allocation-free residual entry point (for callers that may not allocate
device memory and so cannot own a context): its result must equal the regular
mx_residual's, on two calls in a row that share its fixed device scratch, and
the oracle's f - L phi element by element; a NaN in the residual must show in
its norm.  Collected last on purpose."""
import ctypes as C

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
    import paper_1908_03634_gb300 as m
    return m


def fields(g, seed):
    rng = np.random.default_rng(seed)
    cs = (g.n[2], g.n[1], g.n[0])
    t = lambda a: torch.from_numpy(a).to(DEV).contiguous()
    return (t(np.exp(rng.standard_normal(cs))), t(np.exp(rng.standard_normal(cs))), t(rng.standard_normal(cs)),
            t(rng.standard_normal(cs)))


@pytest.mark.parametrize("n,bc", [((64, 48, 40), (0, 0, 1)), ((33, 20, 70), (2, 1, 2))])
def test_noalloc_residual_matches_mx_residual_twice(mx, n, bc):
    g = W.Geom(n, 1.0 / n[0], (bc[0], bc[1], bc[2]), (bc[0], bc[1], bc[2]))
    ctx = mx.mx_create(0)
    try:
        for seed in (1, 2):  # two calls in a row through the shared scratch
            rho, beta0, phi, f = fields(g, seed)
            r_ref = torch.empty_like(phi)
            n_ref = mx.mx_residual(ctx, g, mx.MX_OP_MAC, mx.MX_PREC_FP64, rho, beta0, phi, f, r_ref)
            r = torch.empty_like(phi)
            n_na = mx.mx_residual_noalloc(g, rho, beta0, phi, f, r)
            torch.cuda.synchronize()
            scale = 12 * float((beta0 / rho).max()) * float(phi.abs().max()) / g.dx ** 2
            assert float((r - r_ref).abs().max()) <= 1e-12 * scale
            assert abs(n_na - n_ref) <= 1e-12 * scale
    finally:
        mx.mx_destroy(ctx)


def test_noalloc_rejects_grids_beyond_its_scratch(mx):
    lib = mx.load()
    g = mx.mx_geom()
    for d in range(3):
        g.n[d] = 1024
        g.lo[d] = g.hi[d] = 1
    g.n[2] = 520   # 32 * 128 * 65 tiles > 65536; rejected before any array is touched
    g.dx = 1.0 / 1024
    x = torch.zeros(8, dtype=torch.float64, device=DEV)
    p = C.c_void_p(x.data_ptr())
    rn = C.c_double(-1.0)
    assert lib.mx_residual_noalloc(C.byref(g), p, p, p, p, p, C.byref(rn), None) == mx.MX_ERR_ARG
    assert rn.value == -1.0


@pytest.mark.parametrize("n,bc", [((64, 48, 40), (0, 0, 1)), ((33, 20, 70), (2, 1, 2)), ((16, 16, 16), (0, 0, 0))])
def test_noalloc_residual_matches_oracle(mx, n, bc):
    O.build()
    g = W.Geom(n, 1.0 / n[0], (bc[0], bc[1], bc[2]), (bc[0], bc[1], bc[2]))
    rho, beta0, phi, f = fields(g, 7)
    r = torch.empty_like(phi)
    rn = mx.mx_residual_noalloc(g, rho, beta0, phi, f, r)
    torch.cuda.synchronize()
    h = [x.cpu().numpy() for x in (rho, beta0, phi, f)]
    b = O.mac_coeffs(g, h[0], h[1])
    ref = h[3] - O.mac_apply(g, b, h[2])
    scale = 12 * max(np.abs(x).max() for x in b) * np.abs(h[2]).max() / g.dx ** 2
    assert np.abs(r.cpu().numpy() - ref).max() <= 1e-12 * scale
    assert abs(rn - np.abs(ref).max()) <= 1e-12 * scale


def test_noalloc_norm_shows_nan(mx):
    g = W.Geom((32, 16, 24), 1.0 / 32, (0, 0, 1), (0, 0, 1))
    rho, beta0, phi, f = fields(g, 9)
    f[5, 3, 7] = float("nan")
    r = torch.empty_like(phi)
    rn = mx.mx_residual_noalloc(g, rho, beta0, phi, f, r)
    assert np.isnan(rn)
    assert bool(torch.isnan(r[5, 3, 7]))
    ctx = mx.mx_create(0)
    try:
        rn2 = mx.mx_residual(ctx, g, mx.MX_OP_MAC, mx.MX_PREC_FP64, rho, beta0, phi, f, torch.empty_like(phi))
    finally:
        mx.mx_destroy(ctx)
    assert np.isnan(rn2)
