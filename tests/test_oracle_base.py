"""Pins of the base-state mapping oracle (lateral average and fill, Sec. 3.1)
against facts fixed by geometry and algebra, not by the oracle itself:

- a cell centre at offsets (a + 1/2, b + 1/2, e + 1/2) dx from a corner lies at
  distance dx sqrt(0.75 + 2m) with m integer (Eq. radii): checked exactly on
  integers, (2a+1)^2 + (2b+1)^2 + (2e+1)^2 = 3 + 8m, and against the Euclidean
  distance of the cell centres;
- bin counts and sums against numpy's bincount over those brute-force radii;
- the average of a field that depends on the radius only is that function at
  r_m, and filling it back reproduces the field;
- the planar average of g(z) plus a zero-mean lateral wave is g(z);
- quadratic interpolation reproduces quadratics exactly and, on a cubic, equals
  numpy's degree-2 fit through the three points the stencil rule selects,
  written out independently here (nearest radial centre, shifted inward at the
  ends);
- the w0 integration of the velocity split (Appendix A): closed forms (w0 = s z
  for constant beta0 and source; a geometric beta0 profile; r^2 w0 = s r^3/3 in
  spherical geometry, on uniform and irregular edges; r^2 w0 held beyond a
  cutoff), and, in planar geometry, the MAC divergence of beta0 w0 e_z, computed
  by the projection oracle's own divergence, returning beta0 (Sbar - psi);
- w0 = a r on the faces gives the linear flow a (x - c) component by component;
- S - Sbar has zero lateral means and S - (S - Sbar) is constant on each
  plane / radius."""
import numpy as np
import pytest

import oracle as O
from paper_1908_03634_gb300 import workloads as W

N = W.NEUMANN


def geom(n, dx=1.0 / 32):
    return W.Geom(tuple(n), dx, (N, N, N), (N, N, N))


def centres(g):
    """cell-centre coordinates (z, y, x) grids, shape (nz, ny, nx)"""
    nx, ny, nz = g.n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (i + 0.5) * g.dx, (j + 0.5) * g.dx, (k + 0.5) * g.dx, (i, j, k)


CASES = [((16, 16, 16), (8, 8, 8)), ((20, 12, 9), (7, 3, 9)), ((11, 14, 17), (0, 14, 5)), ((8, 8, 8), (-3, 2, 11))]


@pytest.fixture(scope="module", autouse=True)
def _build():
    O.build()


@pytest.mark.parametrize("n,c", CASES)
def test_radius_identity_exact(n, c):
    g = geom(n)
    m = O.radial_index(g, c)
    _, _, _, (i, j, k) = centres(g)
    a, b, e = i - c[0], j - c[1], k - c[2]
    assert np.array_equal((2 * a + 1) ** 2 + (2 * b + 1) ** 2 + (2 * e + 1) ** 2, 3 + 8 * m)
    x, y, z, _ = centres(g)
    r = np.sqrt((x - c[0] * g.dx) ** 2 + (y - c[1] * g.dx) ** 2 + (z - c[2] * g.dx) ** 2)
    np.testing.assert_allclose(r, g.dx * np.sqrt(0.75 + 2 * m), rtol=1e-14)
    assert O.radial_nbins(g, c) == m.max() + 1


@pytest.mark.parametrize("n,c", CASES)
def test_radial_sums_and_counts_vs_bincount(n, c):
    g = geom(n)
    x, y, z, _ = centres(g)
    d2 = ((x - c[0] * g.dx) ** 2 + (y - c[1] * g.dx) ** 2 + (z - c[2] * g.dx) ** 2) / g.dx**2
    mb = np.rint((d2 - 0.75) / 2).astype(np.int64)  # brute force: m from the distance
    rng = np.random.default_rng(3)
    f = rng.standard_normal(g.n[::-1]) + 2.0
    nb = O.radial_nbins(g, c)
    avg, cnt = O.average_radial(g, c, f)
    assert cnt.sum() == f.size
    assert np.array_equal(cnt, np.bincount(mb.ravel(), minlength=nb))
    sums = np.bincount(mb.ravel(), weights=f.ravel(), minlength=nb)
    ok = cnt > 0
    np.testing.assert_allclose(avg[ok], sums[ok] / cnt[ok], rtol=1e-13, atol=1e-14)
    assert np.all(avg[~ok] == 0.0)


@pytest.mark.parametrize("n,c", CASES)
def test_radial_function_round_trip(n, c):
    g = geom(n)
    x, y, z, _ = centres(g)
    r = np.sqrt((x - c[0] * g.dx) ** 2 + (y - c[1] * g.dx) ** 2 + (z - c[2] * g.dx) ** 2)
    f = np.exp(-3.0 * r) + r**2
    avg, cnt = O.average_radial(g, c, f)
    m = np.arange(avg.size)
    rm = g.dx * np.sqrt(0.75 + 2 * m)
    ok = cnt > 0
    np.testing.assert_allclose(avg[ok], (np.exp(-3.0 * rm) + rm**2)[ok], rtol=1e-13)
    np.testing.assert_allclose(O.fill_irregular(g, c, avg), f, rtol=1e-13)
    base = np.arange(avg.size, dtype=np.float64) * 0.5 - 1.0
    assert np.array_equal(O.fill_irregular(g, c, base), base[O.radial_index(g, c)])


def test_planar_average():
    g = geom((12, 10, 7))
    x, y, z, (i, j, k) = centres(g)
    gz = 1.0 + z**2
    wave = np.cos(2 * np.pi * i / 12) * (1.0 + z) + np.sin(2 * np.pi * j / 10)  # mean 0 on every plane
    out = O.average_planar(g, gz + wave)
    np.testing.assert_allclose(out, 1.0 + ((np.arange(7) + 0.5) * g.dx) ** 2, rtol=1e-14, atol=1e-15)
    rng = np.random.default_rng(1)
    f = rng.standard_normal(g.n[::-1])
    np.testing.assert_allclose(O.average_planar(g, f), f.mean(axis=(1, 2)), rtol=1e-13, atol=1e-15)


def fit3(r, xs, ys):
    return np.polyval(np.polyfit(xs, ys, 2), r)


def stencil_mid(idx, n):
    return min(max(idx, 1), n - 2)


def test_fill_quadratic_exact_on_quadratics_and_stencil_on_cubic():
    g = geom((10, 9, 8), 0.1)
    ctr = np.array([0.43, 0.51, 0.38])
    dr = 0.037
    nr = 40
    rc = (np.arange(nr) + 0.5) * dr
    q = lambda r: 2.0 - 1.5 * r + 0.75 * r**2
    x, y, z, _ = centres(g)
    r = np.sqrt((x - ctr[0]) ** 2 + (y - ctr[1]) ** 2 + (z - ctr[2]) ** 2)
    np.testing.assert_allclose(O.fill_quadratic(g, q(rc), dr, ctr), q(r), rtol=1e-12)
    cub = lambda r: r**3 - 0.2 * r
    got = O.fill_quadratic(g, cub(rc), dr, ctr)
    want = np.empty_like(r)
    for p in np.ndindex(r.shape):
        jm = stencil_mid(int(r[p] // dr), nr)
        s = slice(jm - 1, jm + 2)
        want[p] = fit3(r[p], rc[s], cub(rc[s]))
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12)
    with pytest.raises(ValueError):
        O.fill_quadratic(g, np.ones(2), dr, ctr)


def test_average_to_uniform_exact_on_quadratics_and_stencil_on_cubic():
    g = geom((9, 9, 9), 0.1)
    c = (4, 4, 4)
    avg0, cnt = O.average_radial(g, c, np.zeros(g.n[::-1]))
    m = np.arange(cnt.size)
    rm = g.dx * np.sqrt(0.75 + 2 * m)
    dr = g.dx / 5
    nr = 40
    ru = (np.arange(nr) + 0.5) * dr
    q = lambda r: 1.0 + 2.0 * r - 3.0 * r**2
    np.testing.assert_allclose(O.average_to_uniform(q(rm), cnt, g.dx, nr, dr), q(ru), rtol=1e-12)
    cub = lambda r: 4 * r**3 + r
    got = O.average_to_uniform(cub(rm), cnt, g.dx, nr, dr)
    nz = np.flatnonzero(cnt)
    rn = rm[nz]
    for jj, r in enumerate(ru):
        best = int(np.argmin(np.abs(rn - r)))  # first minimum on a tie
        mid = stencil_mid(best, rn.size)
        s = slice(mid - 1, mid + 2)
        assert got[jj] == pytest.approx(fit3(r, rn[s], cub(rn[s])), rel=1e-9, abs=1e-12)
    with pytest.raises(ValueError):
        O.average_to_uniform(np.ones(3), np.array([1, 0, 1]), g.dx, 4, dr)


# ---- velocity split (Appendix A) -------------------------------------------------------

def test_w0_planar_closed_forms():
    nr, h = 24, 0.05
    r = np.arange(nr + 1) * h
    # constant beta0 and source: w0 = s z on every edge
    w = O.w0_integrate(False, r, np.full(nr, 2.5), np.full(nr, 0.3))
    np.testing.assert_allclose(w, 0.3 * r, rtol=1e-13, atol=1e-16)
    # geometric beta0_k = q^k: Q_{j+1} = h s (1 - q^(j+1)) / (1 - q), beta0 on an edge the mean
    q, s = 0.8, -1.7
    b = q ** np.arange(nr)
    w = O.w0_integrate(False, r, b, np.full(nr, s))
    j = np.arange(nr)
    Q = h * s * (1 - q ** (j + 1)) / (1 - q)
    be = np.where(j + 1 < nr, 0.5 * (q ** j + q ** np.minimum(j + 1, nr - 1)), q ** j)
    np.testing.assert_allclose(w[1:], Q / be, rtol=1e-12)
    assert w[0] == 0.0


def test_w0_spherical_closed_form_and_cutoff():
    nr, dr = 40, 0.01
    r = np.arange(nr + 1) * dr
    # constant beta0 and source: r^2 w0 = s r^3 / 3 exactly (the shell integrals telescope)
    w = O.w0_integrate(True, r, np.full(nr, 0.7), np.full(nr, 1.2))
    np.testing.assert_allclose(w[1:], 1.2 * r[1:] / 3.0, rtol=1e-12)
    # irregular edges (the rule does not assume uniform spacing)
    ri = np.concatenate([[0.0], np.cumsum(np.linspace(0.5, 1.5, nr)) * dr])
    wi = O.w0_integrate(True, ri, np.full(nr, 0.7), np.full(nr, 1.2))
    np.testing.assert_allclose(wi[1:], 1.2 * ri[1:] / 3.0, rtol=1e-11)
    # beyond the cutoff edge r^2 w0 stays at its cutoff value
    cut = 25
    wc = O.w0_integrate(True, r, np.linspace(1.0, 0.2, nr), np.linspace(0.5, -0.5, nr), cutoff=cut)
    wn = O.w0_integrate(True, r, np.linspace(1.0, 0.2, nr), np.linspace(0.5, -0.5, nr))
    assert np.array_equal(wc[:cut + 1], wn[:cut + 1])
    np.testing.assert_allclose(wc[cut + 1:] * r[cut + 1:] ** 2, wn[cut] * r[cut] ** 2, rtol=1e-14)


def test_w0_planar_matches_the_mac_divergence():
    """D(beta0_f w0 e_z) of the MAC discretisation returns beta0 (Sbar - psi) on every
    cell (wall bottom, outflow top): the 1D integration is the discrete inverse of the
    projection's divergence"""
    D, P = W.DIRICHLET, W.PERIODIC
    g = W.Geom((6, 5, 16), 1.0 / 16, (P, P, N), (P, P, D))
    rng = np.random.default_rng(4)
    b = np.exp(-np.arange(16) / 5.0)
    src = rng.standard_normal(16)
    w = O.w0_integrate(False, np.arange(17) * g.dx, b, src)
    u = [np.zeros(O.face_shape(g, d)) for d in range(3)]
    u = O.add_w0_faces(g, False, None, np.arange(17) * g.dx, w, u)
    beta0 = np.broadcast_to(b[:, None, None], O.cell_shape(g)).copy()
    div = O.mac_divergence(g, u, beta0)
    np.testing.assert_allclose(div, (b * src)[:, None, None] * np.ones(O.cell_shape(g)), rtol=1e-11, atol=1e-13)
    assert np.all(u[0] == 0) and np.all(u[1] == 0)


def test_add_w0_faces_spherical_linear_flow():
    """w0 = a r gives U += a (x - c) on every face, component by component"""
    g = geom((9, 8, 7), 0.1)
    c = (4, 5, 2)
    r = np.arange(0, 40) * 0.05
    a = 0.9
    u = O.add_w0_faces(g, True, c, r, a * r, [np.zeros(O.face_shape(g, d)) for d in range(3)])
    for d in range(3):
        sh = O.face_shape(g, d)
        idx = np.meshgrid(*[np.arange(n) for n in sh], indexing="ij")  # (z, y, x) order
        pos = [idx[2], idx[1], idx[0]]
        comp = pos[d] * g.dx - c[d] * g.dx  # a d-face sits at an integer position along d
        np.testing.assert_allclose(u[d], a * comp, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n,c", CASES[:3])
def test_subtract_lateral_average(n, c):
    g = geom(n)
    rng = np.random.default_rng(8)
    S = rng.standard_normal(g.n[::-1]) + 3.0
    out = O.subtract_lateral_average(g, True, c, S)
    avg, cnt = O.average_radial(g, c, out)
    assert np.all(np.abs(avg) < 1e-13)
    m = O.radial_index(g, c)
    sb = S - out  # constant on each bin: its bin mean
    np.testing.assert_allclose(sb, O.average_radial(g, c, S)[0][m], rtol=1e-14, atol=1e-14)
    outp = O.subtract_lateral_average(g, False, None, S)
    np.testing.assert_allclose(outp.mean(axis=(1, 2)), 0.0, atol=1e-13)
    np.testing.assert_allclose(S - outp, np.broadcast_to(S.mean(axis=(1, 2))[:, None, None], S.shape), rtol=1e-13)
