"""GPU parity of the two-level composite MAC operator and divergence (refinement
ratio 2; the paper keeps its AMR as in its Paper V, end of Sec. 3.2) against
the composite oracle, element by element on the same seeded inputs.

Tolerance: both sides evaluate the same FP64 expressions in another order (and
the GPU contracts products into FMAs): 1e-12 of the largest output magnitude.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import composite as CP
from paper_1908_03634_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
P, N, D = CP.PERIODIC, CP.NEUMANN, CP.DIRICHLET


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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


CASES = [
    ((8, 8, 8), (N, N, N), (N, N, N), (2, 3, 2), (6, 6, 5)),
    ((8, 6, 10), (P, P, N), (P, P, N), (1, 1, 3), (4, 5, 9)),
    ((6, 6, 6), (P, P, P), (P, P, P), (2, 2, 2), (3, 3, 3)),
    ((10, 8, 8), (N, P, N), (N, P, N), (3, 1, 1), (9, 7, 7)),
    ((8, 8, 8), (P, P, D), (P, P, D), (2, 2, 2), (6, 5, 6)),
    ((40, 24, 36), (P, P, N), (P, P, N), (5, 3, 4), (37, 21, 30)),  # several blocks of threads per level
]


def setup(case, seed):
    n, lo, hi, plo, phi = case
    G = CP.Composite(n, 1.0 / n[0], lo, hi, plo, phi)
    g = W.Geom(n, 1.0 / n[0], lo, hi)
    rng = np.random.default_rng(seed)
    cs, fs = tuple(reversed(G.n)), tuple(reversed(G.nf))
    f = lambda s: np.exp(rng.standard_normal(s))
    return G, g, rng, f(cs), f(cs), f(fs), f(fs)


@pytest.mark.parametrize("case", CASES)
def test_composite_apply_parity(mx, ctx, case):
    G, g, rng, rc, bc, rf, bf = setup(case, 5)
    pc = rng.standard_normal(rc.shape)
    pf = rng.standard_normal(rf.shape)
    want_c, want_f = CP.apply(G, rc, bc, rf, bf, pc, pf)
    oc = torch.full(rc.shape, np.nan, dtype=torch.float64, device=DEV)
    of = torch.full(rf.shape, np.nan, dtype=torch.float64, device=DEV)
    mx.mx_composite_apply(ctx, g, G.plo, G.phi, dev(rc), dev(bc), dev(rf), dev(bf), dev(pc), dev(pf), oc, of)
    got_c, got_f = oc.cpu().numpy(), of.cpu().numpy()
    scale = max(np.abs(want_c[~G.covered]).max(), np.abs(want_f).max())
    assert np.abs(got_c[~G.covered] - want_c[~G.covered]).max() <= 1e-12 * scale
    assert np.all(got_c[G.covered] == 0.0)
    assert np.abs(got_f - want_f).max() <= 1e-12 * scale
    # conservation on the GPU's output (walls and periodic faces only)
    if G.singular:
        v = CP.volumes(G)
        y = CP.pack(G, got_c, got_f)
        assert abs(v @ y) <= 1e-12 * (v @ np.abs(y))


@pytest.mark.parametrize("case", CASES)
def test_composite_divergence_parity(mx, ctx, case):
    G, g, rng, rc, bc, rf, bf = setup(case, 6)
    uc = [rng.standard_normal(tuple(reversed([G.n[e] + (1 if e == d else 0) for e in range(3)]))) for d in range(3)]
    uf = [rng.standard_normal(tuple(reversed([G.nf[e] + (1 if e == d else 0) for e in range(3)]))) for d in range(3)]
    want = CP.divergence(G, uc, uf, bc, bf)
    want_c, want_f = CP.unpack(G, want)
    oc = torch.full(rc.shape, np.nan, dtype=torch.float64, device=DEV)
    of = torch.full(rf.shape, np.nan, dtype=torch.float64, device=DEV)
    mx.mx_composite_divergence(ctx, g, G.plo, G.phi, [dev(x) for x in uc], [dev(x) for x in uf], dev(bc), dev(bf),
                               oc, of)
    got_c, got_f = oc.cpu().numpy(), of.cpu().numpy()
    scale = max(np.abs(want_c[~G.covered]).max(), np.abs(want_f).max())
    assert np.abs(got_c[~G.covered] - want_c[~G.covered]).max() <= 1e-12 * scale
    assert np.abs(got_f - want_f).max() <= 1e-12 * scale


def test_composite_errors(mx, ctx):
    g = W.Geom((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3)
    z = torch.zeros((8, 8, 8), dtype=torch.float64, device=DEV)
    for plo, phi in (((0, 2, 2), (4, 6, 6)), ((2, 2, 2), (2, 6, 6)), ((2, 2, 2), (8, 6, 6))):
        nf = tuple(2 * (phi[d] - plo[d]) for d in (2, 1, 0))
        f = torch.zeros(nf, dtype=torch.float64, device=DEV)
        with pytest.raises(mx.MXError) as e:
            mx.mx_composite_apply(ctx, g, plo, phi, z, z, f, f, z, f, z, f)
        assert e.value.status == mx.MX_ERR_ARG
    lib = mx.load()
    import ctypes as C
    gg = mx.make_geom(g)
    b = (C.c_int * 3)(2, 2, 2)
    t = (C.c_int * 3)(6, 6, 6)
    p = C.c_void_p(z.data_ptr())
    assert lib.mx_composite_apply(ctx, C.byref(gg), b, t, None, p, p, p, p, p, p, p) == mx.MX_ERR_ARG
    assert lib.mx_composite_divergence(ctx, C.byref(gg), b, t, p, p, p, p, p, p, p, p, p, None) == mx.MX_ERR_ARG


@pytest.mark.parametrize("which", ["planar", "star"])
def test_composite_on_the_composite_workloads(mx, ctx, which):
    """the stratified box with a patch around its heating spot and the star with
    a patch over its core: operator (on the workload's phi-like field Sbar) and
    divergence of the workload's U, against the oracle"""
    if which == "planar":
        w = W.composite_planar(32, (8, 8, 8), (24, 24, 24), 0.2, 0.6, 8, "center", 7)
    else:
        w = W.composite_star(32, (12, 12, 12), (20, 20, 20), 8, 8)
    G = CP.Composite(w.geom.n, w.geom.dx, w.geom.lo, w.geom.hi, w.plo, w.phi)
    npy = lambda t: t.numpy()
    want_c, want_f = CP.apply(G, npy(w.rho_c), npy(w.beta0_c), npy(w.rho_f), npy(w.beta0_f), npy(w.sbar_c),
                              npy(w.sbar_f))
    oc = torch.full(tuple(w.rho_c.shape), np.nan, dtype=torch.float64, device=DEV)
    of = torch.full(tuple(w.rho_f.shape), np.nan, dtype=torch.float64, device=DEV)
    d = lambda t: t.to(DEV)
    mx.mx_composite_apply(ctx, w.geom, w.plo, w.phi, d(w.rho_c), d(w.beta0_c), d(w.rho_f), d(w.beta0_f),
                          d(w.sbar_c), d(w.sbar_f), oc, of)
    scale = max(np.abs(want_c[~G.covered]).max(), np.abs(want_f).max())
    assert np.abs(oc.cpu().numpy()[~G.covered] - want_c[~G.covered]).max() <= 1e-12 * scale
    assert np.abs(of.cpu().numpy() - want_f).max() <= 1e-12 * scale
    dv_c, dv_f = CP.unpack(G, CP.divergence(G, [npy(x) for x in w.u_c], [npy(x) for x in w.u_f], npy(w.beta0_c),
                                            npy(w.beta0_f)))
    mx.mx_composite_divergence(ctx, w.geom, w.plo, w.phi, [d(x) for x in w.u_c], [d(x) for x in w.u_f],
                               d(w.beta0_c), d(w.beta0_f), oc, of)
    scale = max(np.abs(dv_c[~G.covered]).max(), np.abs(dv_f).max())
    assert np.abs(oc.cpu().numpy()[~G.covered] - dv_c[~G.covered]).max() <= 1e-12 * scale
    assert np.abs(of.cpu().numpy() - dv_f).max() <= 1e-12 * scale
