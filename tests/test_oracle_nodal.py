"""Pins of the FP64 oracle's nodal projection (Step 11, Eq. div3; Appendix A).

Checked against: the closed-form Fourier symbol of the trilinear stiffness
(1D stiffness x 1D consistent mass tensor products), symmetry in the
node-weighted inner product, the discrete adjoint relation between the nodal
divergence and the cell gradient, compatibility of the divergence, exactness
on linear fields, a dense direct solve and second-order convergence.
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_03634_gb300 import workloads as W

P, N = W.PERIODIC, W.NEUMANN


def geom(n, bc):
    return W.Geom(tuple(n), 1.0 / n[0], tuple(bc), tuple(bc))


def node_coords(g):
    ms = O.node_shape(g)[::-1]
    return [np.arange(ms[d]) * g.dx for d in range(3)]


@pytest.mark.parametrize("bc", [(P, P, P), (P, P, N), (N, N, N)])
def test_symbol_constant_sigma(oracle_lib, bc):
    n = (8, 6, 10)
    g = geom(n, bc)
    h = g.dx
    sigma = np.full(O.cell_shape(g), 1.7)
    x, y, z = node_coords(g)
    for ks in [(1, 1, 1), (2, 3, 4), (3, 1, 5)]:
        th, comps = [], []
        for d, (c, k) in enumerate(zip((x, y, z), ks)):
            if bc[d] == P:
                t = 2 * np.pi * k / n[d]
                comps.append(np.cos(t * np.arange(c.size) + 0.4))
            else:   # wall: even-reflection cosine on n+1 nodes
                t = np.pi * k / n[d]
                comps.append(np.cos(t * np.arange(c.size)))
            th.append(t)
        phi = comps[2][:, None, None] * comps[1][None, :, None] * comps[0][None, None, :]
        sym = 0.0
        for d in range(3):
            prod = 1.0
            for e in range(3):
                if e != d:
                    prod *= (2 + np.cos(th[e])) / 3
            sym += (2 - 2 * np.cos(th[d])) * prod
        lam = -1.7 / h ** 2 * sym
        Lp = O.nd_apply(g, sigma, phi)
        assert np.abs(Lp - lam * phi).max() <= 1e-12 * abs(lam)


@pytest.mark.parametrize("bc", [(P, P, P), (P, P, N), (N, N, N)])
def test_weighted_symmetry_definiteness_nullspace(oracle_lib, bc):
    rng = np.random.default_rng(1)
    g = geom((6, 4, 8), bc)
    sigma = np.exp(rng.standard_normal(O.cell_shape(g)))
    w = O.nd_weights(g)
    ns = O.node_shape(g)
    u, v = rng.standard_normal(ns), rng.standard_normal(ns)
    Lu, Lv = O.nd_apply(g, sigma, u), O.nd_apply(g, sigma, v)
    scale = np.abs(Lu).max() * u.size
    assert abs((w * Lu * v).sum() - (w * u * Lv).sum()) <= 1e-13 * scale
    assert (w * Lu * u).sum() < 0
    assert np.abs(O.nd_apply(g, sigma, np.ones(ns))).max() <= 1e-12 * np.abs(Lu).max()
    # weights: 1 inside, 1/2 on a wall face, 1/4 on a wall edge, 1/8 at a corner
    assert set(np.unique(w)).issubset({1.0, 0.5, 0.25, 0.125})
    assert np.isclose(w.sum(), np.prod(g.n))


@pytest.mark.parametrize("bc", [(P, P, P), (P, P, N), (N, N, N)])
def test_gradient_is_negative_adjoint_of_divergence(oracle_lib, bc):
    rng = np.random.default_rng(2)
    g = geom((6, 8, 4), bc)
    w = O.nd_weights(g)
    V = [rng.standard_normal(O.cell_shape(g)) for _ in range(3)]
    phi = rng.standard_normal(O.node_shape(g))
    DV = O.nd_divergence(g, V)
    G = O.nd_gradient(g, phi)
    lhs = (w * DV * phi).sum()
    rhs = -sum((V[d] * G[d]).sum() for d in range(3))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # compatibility: the weighted sum of any nodal divergence vanishes
    assert abs((w * DV).sum()) <= 1e-12 * np.abs(w * DV).sum()


def test_linear_fields_exact(oracle_lib):
    g = geom((6, 6, 6), (N, N, N))
    h = g.dx
    x, y, z = node_coords(g)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    phi = 2 * X - 3 * Y + 0.5 * Z
    G = O.nd_gradient(g, phi)
    assert np.allclose(G[0], 2) and np.allclose(G[1], -3) and np.allclose(G[2], 0.5)
    c = (np.arange(6) + 0.5) * h
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
    DV = O.nd_divergence(g, [cx, 2 * cy, -cz])
    assert np.allclose(DV[1:-1, 1:-1, 1:-1], 1 + 2 - 1, rtol=1e-12)
    # L of a linear function vanishes away from the walls
    Lp = O.nd_apply(g, np.ones(O.cell_shape(g)), phi)
    assert np.abs(Lp[1:-1, 1:-1, 1:-1]).max() <= 1e-10


@pytest.mark.parametrize("bc", [(P, P, N), (P, P, P), (N, N, N)])
def test_pcg_matches_dense_direct(oracle_lib, bc):
    rng = np.random.default_rng(4)
    g = geom((8, 8, 8), bc)
    sigma = 0.5 + rng.random(O.cell_shape(g))
    w = O.nd_weights(g)
    f = rng.standard_normal(O.node_shape(g))
    f -= (w * f).sum() / w.sum()
    p1 = O.nd_dense_solve(g, sigma, f)
    p2, it, rr = O.nd_solve(g, sigma, f, tol=1e-14)
    assert rr <= 1e-14
    assert np.abs(p1 - p2).max() <= 1e-12 * np.abs(p1).max()
    assert abs((w * p2).sum()) <= 1e-12 * np.abs(p2).sum()


def test_manufactured_solution_second_order(oracle_lib):
    errs = []
    for n in (16, 32, 64):
        g = geom((n, n, n), (P, P, N))
        h = g.dx
        x, y, z = node_coords(g)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        phi_ex = np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y) * np.cos(np.pi * Z)
        c = (np.arange(n) + 0.5) * h
        cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
        sigma = np.exp(-cz / 0.3) * (1 + 0.2 * np.sin(2 * np.pi * cx) * np.sin(2 * np.pi * cy))
        # f = div(sigma grad phi) evaluated analytically at nodes
        s_n = np.exp(-Z / 0.3) * (1 + 0.2 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y))
        ds = [np.exp(-Z / 0.3) * 0.2 * 2 * np.pi * np.cos(2 * np.pi * X) * np.sin(2 * np.pi * Y),
              np.exp(-Z / 0.3) * 0.2 * 2 * np.pi * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y),
              -s_n / 0.3]
        gr = [-2 * np.pi * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) * np.cos(np.pi * Z),
              -2 * np.pi * np.cos(2 * np.pi * X) * np.sin(2 * np.pi * Y) * np.cos(np.pi * Z),
              -np.pi * np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y) * np.sin(np.pi * Z)]
        f = s_n * (-9 * np.pi ** 2 * phi_ex) + sum(ds[d] * gr[d] for d in range(3))
        w = O.nd_weights(g)
        f -= (w * f).sum() / w.sum()
        phi, it, rr = O.nd_solve(g, sigma, f, tol=1e-12)
        assert rr <= 1e-12
        phi_ex = phi_ex - (w * phi_ex).sum() / w.sum()
        errs.append(np.abs(phi - phi_ex).max())
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert min(ratios) >= 3.5, (errs, ratios)


def test_approximate_projection_error_is_second_order(oracle_lib):
    """The nodal projection is approximate (D sigma G != L): its divergence
    error is not round-off but must shrink like h^2 for smooth data."""
    errs = []
    for n in (16, 32, 64):
        w = W.planar_nodal(n, 0.3, 0.6, 4, "center", 9)
        z = (np.arange(n) + 0.5) / n
        rho = np.broadcast_to(np.exp(-z / 0.3)[:, None, None], O.cell_shape(w.geom)).copy()
        beta0 = rho ** 0.6
        sbar = np.zeros(O.cell_shape(w.geom))
        u, phi, info = O.nd_project(w.geom, w.u, rho, beta0, sbar, tol=1e-12)
        assert info["ok"] and info["rel_resid"] <= 1e-12
        fn = np.abs(O.nd_rhs(w.geom, w.u, beta0, sbar)[0]).max()
        errs.append(info["div_err"] / fn)
    assert errs[0] / errs[1] >= 3.0 and errs[1] / errs[2] >= 3.0, errs


@pytest.mark.parametrize("bc", [(P, P, N), (N, N, N), (P, P, P)])
def test_sampled_nodal_residual_equals_full(oracle_lib, bc):
    rng = np.random.default_rng(22)
    g = geom((6, 4, 8), bc)
    sigma = np.exp(rng.standard_normal(O.cell_shape(g)))
    phi, f = rng.standard_normal(O.node_shape(g)), rng.standard_normal(O.node_shape(g))
    full = (f - O.nd_apply(g, sigma, phi)).ravel()
    got = O.nd_residual_sample(g, sigma, phi, f, np.arange(full.size))
    assert np.abs(got - full).max() <= 1e-12 * np.abs(full).max()


@pytest.mark.parametrize("bc", [(P, P, P), (P, P, N), (N, N, N)])
def test_jacobi_spectrum_within_one_and_a_half(oracle_lib, bc):
    """The spectrum of D^-1 L (D the diagonal of the nodal operator) lies in
    [-1.5, 0] for any positive coefficient field: each cell's trilinear
    stiffness matrix is at most 1.5 times its diagonal.  The Chebyshev smoother
    of the nodal solve takes 1.5 as the top of its interval.  Constant sigma
    on a grid that holds the mode (-1)^i reaches the bound."""
    import scipy.linalg as sl
    rng = np.random.default_rng(3)
    g = geom((6, 4, 8), bc)
    ns = O.node_shape(g)
    w = O.nd_weights(g).ravel()
    for sigma in (np.full(O.cell_shape(g), 2.3), np.exp(2.0 * rng.standard_normal(O.cell_shape(g)))):
        cols = []
        for k in range(int(np.prod(ns))):
            e = np.zeros(int(np.prod(ns)))
            e[k] = 1.0
            cols.append(O.nd_apply(g, sigma, e.reshape(ns)).ravel())
        M = np.stack(cols, axis=1)
        A = -(w[:, None] * M)                   # symmetric positive semidefinite
        assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
        lam = sl.eigh(A, np.diag(np.diag(A)), eigvals_only=True)
        assert lam.min() >= -1e-10 and lam.max() <= 1.5 * (1 + 1e-12), (lam.min(), lam.max())
        if np.ptp(sigma) == 0 and bc[0] == P:
            assert lam.max() >= 1.5 * (1 - 1e-12)
