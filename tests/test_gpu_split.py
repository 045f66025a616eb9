"""GPU parity of the velocity split (Appendix A) against the FP64 oracle, through
the C ABI: the w0 integration (planar and spherical, uniform and irregular edges,
a cutoff), w0 e_r on the MAC faces, the S - Sbar bracket, and the split MAC
projection U = U~ + w0 e_r.

Tolerances: w0 sums the same terms in another order (a one-CTA scan against the
oracle's running sum): 1e-12 of max|w0|.  The face factors use the radius
(dx/2) sqrt(K) where the oracle takes the Euclidean norm, and one FMA: 1e-12 of
the velocity scale.  The bracket inherits the averages' double-float tolerance
(2^-40 of max|S| covers it).  The projection uses the MAC parity bars (phi 1e-8
of its max against the oracle solved to 1e-13; U element by element against the
oracle's correction of the GPU phi plus the oracle's w0 faces, 1e-12)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1908_03634_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
P, N, D = W.PERIODIC, W.NEUMANN, W.DIRICHLET


@pytest.fixture(scope="module")
def mx():
    from paper_1908_03634_gb300 import build as b
    b.build()
    O.build()
    import paper_1908_03634_gb300 as m
    return m


@pytest.fixture()
def ctx(mx):
    c = mx.mx_create(0)
    yield c
    mx.mx_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64))).to(DEV)


@pytest.mark.parametrize("sph", [0, 1])
@pytest.mark.parametrize("nr", [1, 5, 1023, 1025, 3000, 100000])
@pytest.mark.parametrize("irregular", [False, True])
def test_w0_parity(mx, ctx, sph, nr, irregular):
    rng = np.random.default_rng(nr + 7 * sph)
    dr = rng.uniform(0.5, 1.5, nr) if irregular else np.ones(nr)
    r = np.concatenate([[0.0], np.cumsum(dr)]) * (1.0 / nr)
    b = np.exp(-np.linspace(0, 4, nr)) + 0.1
    src = rng.standard_normal(nr)
    for cutoff in (-1, nr // 2):
        want = O.w0_integrate(sph, r, b, src, cutoff)
        out = torch.empty(nr + 1, dtype=torch.float64, device=DEV)
        mx.mx_w0_integrate(ctx, sph, dev(r), dev(b), dev(src), out, cutoff)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == 0.0
        assert np.abs(got - want).max() <= 1e-12 * max(np.abs(want).max(), 1e-300)


FACE_CASES = [((16, 16, 16), (8, 8, 8)), ((21, 12, 9), (7, 3, 9)), ((10, 9, 11), (-4, 5, 13)), ((7, 6, 5), (0, 0, 0))]


@pytest.mark.parametrize("n,c", FACE_CASES)
@pytest.mark.parametrize("nr", [60, 12])
def test_add_w0_faces_spherical_parity(mx, ctx, n, c, nr):
    """nr = 12: the edges end at 6 dx, so the outer faces take r^2 w0 held constant"""
    g = W.Geom(n, 1.0 / 16, (D, D, D), (D, D, D))
    r = np.arange(nr + 1) * (g.dx / 2)
    w0 = np.sin(9.0 * r) + 0.3 * r
    rng = np.random.default_rng(1)
    u = [rng.standard_normal(O.face_shape(g, d)) for d in range(3)]
    want = O.add_w0_faces(g, True, c, r, w0, u)
    ud = [dev(x) for x in u]
    mx.mx_add_w0_faces(ctx, g, 1, c, dev(r), dev(w0), *ud)
    torch.cuda.synchronize()
    scale = max(np.abs(x).max() for x in u) + np.abs(w0).max()
    for d in range(3):
        assert np.abs(ud[d].cpu().numpy() - want[d]).max() <= 1e-12 * scale


def test_add_w0_faces_planar_parity(mx, ctx):
    g = W.Geom((12, 10, 14), 1.0 / 14, (P, P, N), (P, P, D))
    w0 = np.linspace(0.0, 2.0, 15) ** 2
    rng = np.random.default_rng(2)
    u = [rng.standard_normal(O.face_shape(g, d)) for d in range(3)]
    want = O.add_w0_faces(g, False, None, np.arange(15) * g.dx, w0, u)
    ud = [dev(x) for x in u]
    mx.mx_add_w0_faces(ctx, g, 0, None, None, dev(w0), *ud)
    torch.cuda.synchronize()
    for d in range(3):
        assert np.array_equal(ud[d].cpu().numpy(), want[d])


@pytest.mark.parametrize("sph,n,c", [(1, (32, 32, 32), (16, 16, 16)), (1, (37, 23, 29), (18, 11, 15)),
                                     (0, (32, 24, 20), None), (0, (33, 7, 5), None)])
def test_subtract_lateral_average_parity(mx, ctx, sph, n, c):
    g = W.Geom(n, 1.0 / 32, (N, N, N), (N, N, N))
    rng = np.random.default_rng(3)
    S = rng.standard_normal(O.cell_shape(g)) + np.linspace(1, 3, n[0])
    want = O.subtract_lateral_average(g, sph, c, S)
    out = torch.empty(O.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_subtract_lateral_average(ctx, g, sph, c, dev(S), out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - want).max() <= 2.0**-40 * np.abs(S).max()


def split_case(kind):
    """(workload, spherical, corner, r_edge, base beta0, src) with the workload's
    S (its Sbar field) and base state"""
    if kind == "planar":
        w = W.planar(32, 0.2, 0.6, 8, 2, 5)
        g = w.geom
        w.geom = W.Geom(g.n, g.dx, (P, P, N), (P, P, D))  # wall bottom, outflow top
        nz = g.n[2]
        b = w.prof_beta0.numpy()[:nz]
        sbar = O.average_planar(w.geom, w.sbar.numpy())
        src = sbar - 0.05
        return w, 0, None, np.arange(nz + 1) * g.dx, b, src
    w = W.star(32, 8, 2)
    g = w.geom
    c = (16, 16, 16)
    nr = 4 * 28
    dr = g.dx / 4
    r = np.arange(nr + 1) * dr
    rc = (np.arange(nr) + 0.5) * dr
    b = np.interp(rc, (np.arange(w.prof_beta0.numel()) + 0.5) * w.prof_dr, w.prof_beta0.numpy())
    src = np.exp(-rc / 0.1) - 0.02
    return w, 1, c, r, b, src


@pytest.mark.parametrize("kind", ["planar", "spherical"])
def test_mac_project_split_parity(mx, ctx, kind):
    w, sph, c, r, b, src = split_case(kind)
    g = w.geom
    w0 = O.w0_integrate(sph, r, b, src)
    beta0 = O.fill(g, w.prof_beta0, spherical=bool(sph), dr=w.prof_dr, center=w.center)
    S = w.sbar.numpy()
    # GPU
    ud = [dev(x) for x in w.u]
    phi = torch.zeros(O.cell_shape(g), dtype=torch.float64, device=DEV)
    st, info = mx.mx_mac_project_split(ctx, g, sph, c, *ud, dev(w.rho), dev(beta0), dev(S), dev(r), dev(w0), phi,
                                       mx.default_opts())
    torch.cuda.synchronize()
    assert st == mx.MX_OK and info["rel_resid"] <= 1e-10
    # oracle: the bracket, the projection of U~, then w0 on the faces
    bracket = O.subtract_lateral_average(g, sph, c, S)
    u_ref, phi_ref, oinfo = O.mac_project(g, w.u, w.rho, beta0, bracket, tol=1e-13, maxit=400)
    assert oinfo["ok"]
    p = phi.cpu().numpy()
    assert np.abs(p - phi_ref).max() <= 1e-8 * np.abs(phi_ref).max()
    u_pred = O.add_w0_faces(g, sph, c, r, w0, O.mac_correct(g, w.rho, p, w.u))
    for d in range(3):
        scale = np.abs(w.u[d].numpy()).max() + np.abs(u_pred[d] - w.u[d].numpy()).max()
        assert np.abs(ud[d].cpu().numpy() - u_pred[d]).max() <= 1e-12 * scale
    if not sph:
        # planar: D(beta0 U) = beta0 (S - psi) up to the solve's residual (w0 is the
        # exact discrete inverse of the MAC divergence on laterally uniform beta0)
        f, _ = O.mac_rhs(g, w.u, beta0, bracket)
        dv = O.mac_divergence(g, [x.cpu().numpy() for x in ud], beta0) - beta0 * (S - 0.05)
        assert np.abs(dv).max() <= 2e-10 * np.abs(f).max() + 1e-12 * np.abs(beta0 * S).max()


def test_split_errors(mx, ctx):
    g = W.Geom((8, 8, 8), 1.0 / 8, (D, D, D), (D, D, D))
    out = torch.empty(9, dtype=torch.float64, device=DEV)
    z = torch.zeros(8, dtype=torch.float64, device=DEV)
    with pytest.raises(mx.MXError) as e:
        mx.mx_w0_integrate(ctx, 1, torch.zeros(9, dtype=torch.float64, device=DEV), z, z, out, cutoff=12)
    assert e.value.status == mx.MX_ERR_ARG
    u = [torch.zeros(O.face_shape(g, d), dtype=torch.float64, device=DEV) for d in range(3)]
    with pytest.raises(mx.MXError) as e:  # planar needs w0 on every z face
        mx.mx_add_w0_faces(ctx, g, 0, None, None, torch.zeros(5, dtype=torch.float64, device=DEV), *u)
    assert e.value.status == mx.MX_ERR_ARG
    with pytest.raises(mx.MXError) as e:  # radius table beyond 2^26 entries
        mx.mx_add_w0_faces(ctx, g, 1, (1 << 20, 0, 0), torch.zeros(9, dtype=torch.float64, device=DEV), out, *u)
    assert e.value.status == mx.MX_ERR_ARG
