"""GPU parity of the two-level composite MAC projection (coarse level plus one
ratio-2 fine patch; the paper's AMR, end of Sec. 3.2, with the projection of
Appendix A) against the composite oracle's sparse direct solve, element by
element on the same seeded inputs.

Bars: phi within 1e-8 relative max norm of the oracle's phi (the oracle solves
exactly, the GPU to a composite residual of 1e-10 of ||f||_inf); U on both
levels equal to the oracle's correction applied to the GPU's phi, to 1e-12 of
the velocity scale (FP64 on both sides, another evaluation order); the covered
coarse phi the mean of its fine cells; and the projection identity
D(beta0 U) - beta0 Sbar - c = f - L phi, residual-sized, on the GPU's output.
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


def face_shapes(n):
    return [tuple(reversed([n[e] + (1 if e == d else 0) for e in range(3)])) for d in range(3)]


def run_both(mx, ctx, G, g, rc, bc, sc, uc, rf, bf, sf, uf, **kw):
    """GPU projection and oracle solve of the same inputs; returns the GPU outputs,
    the oracle's phi and its info"""
    uc_g, uf_g = [dev(x) for x in uc], [dev(x) for x in uf]
    pc = torch.zeros(rc.shape, dtype=torch.float64, device=DEV)
    pf = torch.zeros(rf.shape, dtype=torch.float64, device=DEV)
    st, info = mx.mx_mac_project_composite(ctx, g, G.plo, G.phi, uc_g, dev(rc), dev(bc), dev(sc), pc, uf_g, dev(rf),
                                           dev(bf), dev(sf), pf, mx.default_opts(**kw))
    torch.cuda.synchronize()
    _, _, pc_ref, pf_ref, oinfo = CP.project(G, uc, uf, rc, bc, sc, rf, bf, sf)
    return info, pc.cpu().numpy(), pf.cpu().numpy(), [x.cpu().numpy() for x in uc_g], \
        [x.cpu().numpy() for x in uf_g], pc_ref, pf_ref, oinfo


def check(G, rc, bc, sc, uc, rf, bf, sf, uf, info, pc, pf, uc2, uf2, pc_ref, pf_ref, oinfo):
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10, info
    # phi on the unknowns (uncovered coarse, fine) and the covered coarse means
    ref = max(np.abs(pc_ref[~G.covered]).max(), np.abs(pf_ref).max())
    err = max(np.abs(pc[~G.covered] - pc_ref[~G.covered]).max(), np.abs(pf - pf_ref).max()) / ref
    assert err <= 1e-8, err
    fz, fy, fx = pf.shape
    means = pf.reshape(fz // 2, 2, fy // 2, 2, fx // 2, 2).mean(axis=(1, 3, 5))
    plo, phi = G.plo, G.phi
    assert np.abs(pc[plo[2]:phi[2], plo[1]:phi[1], plo[0]:phi[0]] - means).max() <= 1e-13 * ref
    # U: the oracle's correction of the GPU's phi, on both levels
    x = CP.pack(G, pc, pf)
    uc_p, uf_p = CP.correct(G, uc, uf, rc, rf, x)
    for d in range(3):
        sc_ = np.abs(uc[d]).max() + np.abs(uc_p[d] - uc[d]).max()
        assert np.abs(uc2[d] - uc_p[d]).max() <= 1e-12 * sc_, ("coarse", d)
        sf_ = np.abs(uf[d]).max() + np.abs(uf_p[d] - uf[d]).max()
        assert np.abs(uf2[d] - uf_p[d]).max() <= 1e-12 * sf_, ("fine", d)
    assert abs(info["rhs_mean_removed"] - oinfo["mean"]) <= 1e-12 * max(1.0, abs(oinfo["mean"]))
    # projection identity on the GPU's U: the divergence error is residual-sized
    fn = np.abs(oinfo["f"]).max()
    dv = CP.divergence(G, uc2, uf2, bc, bf) - CP.pack(G, bc * sc, bf * sf) - oinfo["mean"]
    assert np.abs(dv).max() <= 2e-10 * fn
    assert info["div_err_linf"] <= 2e-10 * fn


CASES = [
    ((8, 8, 8), (N, N, N), (2, 3, 2), (6, 6, 5)),
    ((8, 6, 10), (P, P, N), (1, 1, 3), (4, 5, 9)),
    ((6, 6, 6), (P, P, P), (2, 2, 2), (3, 3, 3)),
    ((10, 8, 8), (N, P, N), (3, 1, 1), (9, 7, 7)),
    ((8, 8, 8), (P, P, D), (2, 2, 2), (6, 5, 6)),
    ((12, 10, 8), (D, N, P), (3, 2, 2), (9, 8, 6)),
]


@pytest.mark.parametrize("case", CASES)
def test_composite_projection_parity(mx, ctx, case):
    n, bcs, plo, phi = case
    G = CP.Composite(n, 1.0 / n[0], bcs, bcs, plo, phi)
    g = W.Geom(n, 1.0 / n[0], bcs, bcs)
    rng = np.random.default_rng(11)
    cs, fs = tuple(reversed(G.n)), tuple(reversed(G.nf))
    rc, bc = np.exp(0.5 * rng.standard_normal(cs)), np.exp(0.5 * rng.standard_normal(cs))
    rf, bf = np.exp(0.5 * rng.standard_normal(fs)), np.exp(0.5 * rng.standard_normal(fs))
    sc, sf = rng.standard_normal(cs), rng.standard_normal(fs)
    uc = [rng.standard_normal(s) for s in face_shapes(G.n)]
    uf = [rng.standard_normal(s) for s in face_shapes(G.nf)]
    for d in range(3):  # periodic images equal, as the API asks
        if bcs[d] == P:
            idx = [slice(None)] * 3
            src, dst = list(idx), list(idx)
            src[2 - d], dst[2 - d] = 0, -1
            uc[d][tuple(dst)] = uc[d][tuple(src)]
    out = run_both(mx, ctx, G, g, rc, bc, sc, uc, rf, bf, sf, uf, max_outer=200, max_vcycles=200)
    check(G, rc, bc, sc, uc, rf, bf, sf, uf, *out)


@pytest.mark.parametrize("which", ["planar", "star"])
def test_composite_projection_on_the_composite_workloads(mx, ctx, which):
    """the stratified box with a patch around its heating spot and the star with
    a patch over its core"""
    if which == "planar":
        w = W.composite_planar(24, (6, 6, 6), (18, 18, 18), W.H_1E5, 0.6, 8, "center", 7)
    else:
        w = W.composite_star(24, (8, 8, 8), (16, 16, 16), 8, 8)
    G = CP.Composite(w.geom.n, w.geom.dx, w.geom.lo, w.geom.hi, w.plo, w.phi)
    npy = lambda t: t.numpy()
    args = (npy(w.rho_c), npy(w.beta0_c), npy(w.sbar_c), [npy(x) for x in w.u_c], npy(w.rho_f), npy(w.beta0_f),
            npy(w.sbar_f), [npy(x) for x in w.u_f])
    out = run_both(mx, ctx, G, w.geom, *args)
    check(G, *args, *out)


def test_composite_projection_errors(mx, ctx):
    g = W.Geom((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3)
    G = CP.Composite((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3, (2, 2, 2), (6, 6, 6))
    z = torch.zeros((8, 8, 8), dtype=torch.float64, device=DEV)
    f = torch.zeros((8, 8, 8), dtype=torch.float64, device=DEV)
    uc = [torch.zeros(s, dtype=torch.float64, device=DEV) for s in face_shapes(G.n)]
    uf = [torch.zeros(s, dtype=torch.float64, device=DEV) for s in face_shapes(G.nf)]
    for kw in ({"prec": mx.MX_PREC_FP64}, {"krylov": 1}, {"smoother": 1}):
        with pytest.raises(mx.MXError) as e:
            mx.mx_mac_project_composite(ctx, g, G.plo, G.phi, uc, z + 1, z + 1, z, z.clone(), uf, f + 1, f + 1, f,
                                        f.clone(), mx.default_opts(**kw))
        assert e.value.status == mx.MX_ERR_ARG
    # zero right-hand side: phi = 0 without an iteration
    pc, pf = z.clone() + 3.0, f.clone() + 3.0
    st, info = mx.mx_mac_project_composite(ctx, g, G.plo, G.phi, uc, z + 1, z + 1, z, pc, uf, f + 1, f + 1, f, pf,
                                           mx.default_opts())
    assert st == 0 and info["outer_iters"] == 0
    assert torch.count_nonzero(pc).item() == 0 and torch.count_nonzero(pf).item() == 0
