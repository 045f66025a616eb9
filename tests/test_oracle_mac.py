"""Pins of the FP64 oracle's MAC projection against what the mathematics fixes.

Each test checks the oracle against something other than itself: closed-form
eigenpairs, an exact face-average identity, symmetry/definiteness, a dense
Gaussian-elimination solve, an FFT + Thomas direct solve, a manufactured
solution's second-order convergence and the projection's divergence identity
(Appendix A; Eq. div1).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from oracle import separable as S
from paper_1908_03634_gb300 import workloads as W

P, N, D = W.PERIODIC, W.NEUMANN, W.DIRICHLET


def geom(n, lo, hi=None):
    return W.Geom(tuple(n), 1.0 / n[0], tuple(lo), tuple(hi if hi is not None else lo))


def mode_1d(nn, k, bc, h):
    """closed-form eigenvector of the 1D 3-point operator with boundary bc."""
    i = np.arange(nn)
    if bc == P:
        return np.cos(2 * np.pi * k * i / nn + 0.3), -4 / h ** 2 * np.sin(np.pi * k / nn) ** 2
    if bc == N:   # even reflection about the wall face
        return np.cos(np.pi * k * (i + 0.5) / nn), -4 / h ** 2 * np.sin(np.pi * k / (2 * nn)) ** 2
    # odd reflection about the Dirichlet face
    return np.sin(np.pi * k * (i + 0.5) / nn), -4 / h ** 2 * np.sin(np.pi * k / (2 * nn)) ** 2


BCS = [P, N, D]


@pytest.mark.parametrize("bcx,bcy,bcz", list(itertools.product(BCS, BCS, BCS)))
def test_eigenpairs_constant_coefficient(oracle_lib, bcx, bcy, bcz):
    n = (8, 6, 10)
    g = geom(n, (bcx, bcy, bcz))
    h = g.dx
    coef = 2.5  # beta0 / rho
    rho = np.full(O.cell_shape(g), 2.0)
    beta0 = np.full(O.cell_shape(g), 5.0)
    b = O.mac_coeffs(g, rho, beta0)
    for ks in [(1, 1, 1), (3, 2, 5), (4, 3, 7)]:
        mx, lx = mode_1d(n[0], ks[0], bcx, h)
        my, ly = mode_1d(n[1], ks[1], bcy, h)
        mz, lz = mode_1d(n[2], ks[2], bcz, h)
        phi = mz[:, None, None] * my[None, :, None] * mx[None, None, :]
        Lp = O.mac_apply(g, b, phi)
        lam = coef * (lx + ly + lz)
        assert np.abs(Lp - lam * phi).max() <= 1e-13 * abs(lam) * np.abs(phi).max()


def test_face_average_is_arithmetic(oracle_lib):
    """(L x)_i = (b_{i+1/2} - b_{i-1/2})/h with b_f = (beta_L+beta_R)/(rho_L+rho_R)."""
    rng = np.random.default_rng(5)
    n = (12, 4, 4)
    g = geom(n, (N, P, P))
    h = g.dx
    bx = 1.0 + rng.random(n[0])
    rx = 1.0 + rng.random(n[0])
    beta0 = np.broadcast_to(bx[None, None, :], O.cell_shape(g)).copy()
    rho = np.broadcast_to(rx[None, None, :], O.cell_shape(g)).copy()
    b = O.mac_coeffs(g, rho, beta0)
    x = (np.arange(n[0]) + 0.5) * h
    phi = np.broadcast_to(x[None, None, :], O.cell_shape(g)).copy()
    Lp = O.mac_apply(g, b, phi)[0, 0, :]
    bf = (bx[:-1] + bx[1:]) / (rx[:-1] + rx[1:])     # faces 1..n-1
    expect = (bf[1:] - bf[:-1]) / h                   # cells 1..n-2
    assert np.allclose(Lp[1:-1], expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())
    # wall cells: only the interior face carries flux
    assert np.isclose(Lp[0], bf[0] / h, rtol=1e-12)
    assert np.isclose(Lp[-1], -bf[-1] / h, rtol=1e-12)


@pytest.mark.parametrize("bc", [(P, P, P), (P, P, N), (N, N, N), (D, D, D), (P, D, N), (N, P, D)])
def test_symmetry_and_definiteness(oracle_lib, bc):
    rng = np.random.default_rng(11)
    g = geom((6, 8, 10), bc)
    cs = O.cell_shape(g)
    rho = np.exp(rng.standard_normal(cs))
    beta0 = np.exp(rng.standard_normal(cs))
    b = O.mac_coeffs(g, rho, beta0)
    u, v = rng.standard_normal(cs), rng.standard_normal(cs)
    Lu, Lv = O.mac_apply(g, b, u), O.mac_apply(g, b, v)
    scale = np.abs(Lu).max() * np.abs(v).max() * u.size
    assert abs((Lu * v).sum() - (u * Lv).sum()) <= 1e-14 * scale
    assert (Lu * u).sum() < 0
    L1 = O.mac_apply(g, b, np.ones(cs))
    if O.singular(g):
        assert np.abs(L1).max() == 0.0
    else:
        assert np.abs(L1).max() > 0
        # -L positive definite: smallest eigenvalue of the dense matrix > 0
        A = np.stack([O.mac_apply(g, b, e.reshape(cs)).ravel() for e in np.eye(u.size)], axis=1)
        assert np.linalg.eigvalsh(-0.5 * (A + A.T)).min() > 0


@pytest.mark.parametrize("bc", [(P, P, N), (D, D, D), (P, D, N), (N, N, N), (P, P, P)])
def test_pcg_matches_dense_direct_8cubed(oracle_lib, bc):
    rng = np.random.default_rng(3)
    g = geom((8, 8, 8), bc)
    cs = O.cell_shape(g)
    rho = 1.0 + rng.random(cs)
    beta0 = 1.0 + rng.random(cs)
    b = O.mac_coeffs(g, rho, beta0)
    f = rng.standard_normal(cs)
    if O.singular(g):
        f -= f.mean()
    p_dense = O.mac_dense_solve(g, b, f)
    p_cg, it, rr = O.mac_solve(g, b, f, tol=1e-14)
    assert it > 0 and rr <= 1e-14
    assert np.abs(p_dense - p_cg).max() <= 1e-12 * np.abs(p_dense).max()


@pytest.mark.parametrize("n,bcz", [((32, 32, 32), N), ((32, 16, 48), D), ((64, 64, 64), N)])
def test_pcg_matches_separable_direct_solve(oracle_lib, n, bcz):
    """Noise-free planar stratification (the planar workload without noise):
    the operator separates and an FFT + tridiagonal solve is exact."""
    g = W.Geom(n, 1.0 / n[0], (P, P, bcz), (P, P, bcz))
    z = (np.arange(n[2]) + 0.5) * g.dx
    rz = np.exp(-z / W.H_1E5)
    bz = rz ** 0.6
    cs = O.cell_shape(g)
    rho = np.broadcast_to(rz[:, None, None], cs).copy()
    beta0 = np.broadcast_to(bz[:, None, None], cs).copy()
    f = np.random.default_rng(7).standard_normal(cs)
    if bcz == N:
        f -= f.mean()
    b = O.mac_coeffs(g, rho, beta0)
    p_direct = S.solve_layered(n, g.dx, bcz, rz, bz, f)
    p_cg, it, rr = O.mac_solve(g, b, f, tol=1e-13)
    assert rr <= 1e-13
    assert np.abs(p_direct - p_cg).max() <= 1e-10 * np.abs(p_direct).max()


def _mms(n, dirichlet):
    """manufactured solution: returns (geom, rho, beta0, f, phi_exact) at cell centres"""
    bc = (D, D, D) if dirichlet else (P, P, N)
    g = geom((n, n, n), bc)
    h = g.dx
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    Lz, eps = 0.3, 0.2
    s = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    rho = np.exp(-z / Lz) * (1 + eps * s)
    beta0 = np.exp(-0.6 * z / Lz)
    drho = [np.exp(-z / Lz) * eps * 2 * np.pi * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y),
            np.exp(-z / Lz) * eps * 2 * np.pi * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y),
            -rho / Lz]
    dbeta = [0 * z, 0 * z, -0.6 * beta0 / Lz]
    bfun = beta0 / rho
    db = [(dbeta[d] * rho - beta0 * drho[d]) / rho ** 2 for d in range(3)]
    if dirichlet:
        sx, sy, sz = np.sin(np.pi * x), np.sin(np.pi * y), np.sin(np.pi * z)
        cx, cy, cz = np.cos(np.pi * x), np.cos(np.pi * y), np.cos(np.pi * z)
        phi = sx * sy * sz
        grad = [np.pi * cx * sy * sz, np.pi * sx * cy * sz, np.pi * sx * sy * cz]
        lap = -3 * np.pi ** 2 * phi
    else:
        cx, cy, cz = np.cos(2 * np.pi * x), np.cos(2 * np.pi * y), np.cos(np.pi * z)
        sx, sy, sz = np.sin(2 * np.pi * x), np.sin(2 * np.pi * y), np.sin(np.pi * z)
        phi = cx * cy * cz
        grad = [-2 * np.pi * sx * cy * cz, -2 * np.pi * cx * sy * cz, -np.pi * cx * cy * sz]
        lap = -(4 + 4 + 1) * np.pi ** 2 * phi
    f = bfun * lap + sum(db[d] * grad[d] for d in range(3))
    if not dirichlet:
        f = f - f.mean()
    return g, rho, beta0, f, phi


@pytest.mark.parametrize("dirichlet", [False, True])
def test_manufactured_solution_second_order(oracle_lib, dirichlet):
    errs = []
    for n in (16, 32, 64):
        g, rho, beta0, f, phi_ex = _mms(n, dirichlet)
        b = O.mac_coeffs(g, rho, beta0)
        phi, it, rr = O.mac_solve(g, b, f, tol=1e-12)
        assert rr <= 1e-12
        if not dirichlet:
            phi_ex = phi_ex - phi_ex.mean()
        errs.append(np.abs(phi - phi_ex).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert min(ratios) >= 3.5, (errs, ratios)


@pytest.mark.parametrize("which", ["planar", "star"])
def test_projection_divergence_identity(oracle_lib, which):
    """After the correction, D(beta0 U) - beta0 Sbar - c equals the solve's
    residual f - L phi up to rounding (Appendix A; Eq. div1)."""
    if which == "planar":
        w = W.planar(24, 0.1, 1.0, 8, "center", 0)
        beta0 = O.fill(w.geom, w.prof_beta0)
    else:
        w = W.star(24, 8, 2)
        beta0 = O.fill(w.geom, w.prof_beta0, spherical=True, dr=w.prof_dr, center=w.center)
    g = w.geom
    b = O.mac_coeffs(g, w.rho, beta0)
    f, c = O.mac_rhs(g, w.u, beta0, w.sbar)
    phi, it, rr = O.mac_solve(g, b, f, tol=1e-6)   # loose on purpose: r is not small
    r = f - O.mac_apply(g, b, phi)
    u = O.mac_correct(g, w.rho, phi, w.u)
    d = O.mac_divergence(g, u, beta0) - beta0 * np.asarray(w.sbar) - c
    fn = np.abs(f).max()
    assert np.abs(r).max() > 1e-9 * fn
    assert np.abs(d - r).max() <= 1e-12 * fn
    if O.singular(g):
        assert abs(c) > 0
        assert abs(f.sum()) <= 1e-12 * fn * f.size
    # wall faces carry no velocity after the projection
    if g.lo[2] == N:
        assert np.all(u[2][0] == 0) and np.all(u[2][-1] == 0)


def test_fill_planar_injection(oracle_lib):
    g = geom((4, 5, 6), (P, P, N))
    prof = np.arange(10.0) ** 2
    out = O.fill(g, prof)
    assert np.array_equal(out, np.broadcast_to(prof[:6, None, None], O.cell_shape(g)))


def test_fill_spherical_linear_exact_and_radii(oracle_lib):
    n = 16
    g = geom((n, n, n), (D, D, D))
    dr = g.dx / 4
    rj = (np.arange(4096) + 0.5) * dr
    out = O.fill(g, 3.0 - 2.0 * rj, spherical=True, dr=dr)
    c = (np.arange(n) + 0.5) * g.dx - 0.5
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    assert np.abs(out - (3.0 - 2.0 * r)).max() <= 1e-13
    # every cell centre sits at r = dx sqrt(0.75 + 2m) for an integer m (Eq. radii)
    m = ((r / g.dx) ** 2 - 0.75) / 2
    assert np.abs(m - np.round(m)).max() < 1e-9
    # quadratic profile: linear interpolation error <= dr^2/8 * |p''|
    out2 = O.fill(g, rj ** 2, spherical=True, dr=dr)
    assert np.abs(out2 - r ** 2).max() <= dr ** 2 / 8 * 2 + 1e-14


def test_remove_mean_flag_and_dirichlet_keeps_mean(oracle_lib):
    w = W.planar(8, 0.1, 1.0, 4, "center", 0)
    beta0 = O.fill(w.geom, w.prof_beta0)
    f1, c1 = O.mac_rhs(w.geom, w.u, beta0, w.sbar, remove_mean=True)
    f0, c0 = O.mac_rhs(w.geom, w.u, beta0, w.sbar, remove_mean=False)
    assert c0 == 0.0 and abs(c1) > 0
    assert np.allclose(f0 - c1, f1, rtol=0, atol=1e-14 * np.abs(f0).max())
    ws = W.star(8, 4, 2)
    b0 = O.fill(ws.geom, ws.prof_beta0, spherical=True, dr=ws.prof_dr)
    _, cs = O.mac_rhs(ws.geom, ws.u, b0, ws.sbar, remove_mean=True)
    assert cs == 0.0


@pytest.mark.parametrize("bc", [(P, P, N), (D, D, D), (N, P, D)])
def test_sampled_residual_and_divergence_equal_full_arrays(oracle_lib, bc):
    """The one-cell-at-a-time functions used for full-size checks agree with
    the full-array definitions (coefficients from rho, beta0 directly)."""
    rng = np.random.default_rng(21)
    g = geom((10, 6, 8), bc)
    cs = O.cell_shape(g)
    rho, beta0, phi, f = np.exp(rng.standard_normal(cs)), np.exp(rng.standard_normal(cs)), \
        rng.standard_normal(cs), rng.standard_normal(cs)
    u = [rng.standard_normal(O.face_shape(g, d)) for d in range(3)]
    b = O.mac_coeffs(g, rho, beta0)
    r_full = (f - O.mac_apply(g, b, phi)).ravel()
    d_full = O.mac_divergence(g, u, beta0).ravel()
    idx = np.arange(r_full.size)
    assert np.array_equal(O.mac_residual_sample(g, rho, beta0, phi, f, idx), r_full)
    assert np.array_equal(O.mac_divergence_sample(g, u, beta0, idx), d_full)
