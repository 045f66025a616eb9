"""Pins of the two-level composite MAC oracle (refinement ratio 2; the paper
keeps its AMR as in its Paper V, end of Sec. 3.2).  Each pin is fixed by the
mathematics, not by the oracle itself:

  * conservation: with flux matching, the volume-weighted sum of L phi over the
    composite cells telescopes to the domain-boundary flux, 0 with walls and
    periodic faces, for any phi and any coefficients;
  * constants are in the null space (the ghost weights sum to 1);
  * a linear phi with constant coefficients gives L phi = 0 on every fine cell
    and every coarse cell off the domain faces (the ghost interpolation is
    exact for linear functions);
  * away from the patch, the composite rows are the single-level operator's
    (coarse grid, and the fine grid inside the patch);
  * the projection identity D(beta0 U_new) - beta0 Sbar - c = f - L phi;
  * second order: a manufactured solution's error falls by >= 3.5 when h halves;
  * planted mistakes in the ghost weights break the linear pin.
"""
import numpy as np
import pytest

import oracle as O
from oracle import composite as CP
from paper_1908_03634_gb300 import workloads as W

P, N, D = CP.PERIODIC, CP.NEUMANN, CP.DIRICHLET


def rand_case(G, seed):
    rng = np.random.default_rng(seed)
    cs = tuple(reversed(G.n))
    fs = tuple(reversed(G.nf))
    return (np.exp(rng.standard_normal(cs)), np.exp(rng.standard_normal(cs)), np.exp(rng.standard_normal(fs)),
            np.exp(rng.standard_normal(fs)), rng)


def centres(G):
    H = G.H
    fs = tuple(reversed(G.nf))
    zc, yc, xc = np.meshgrid(*[(np.arange(m) + 0.5) * H for m in reversed(G.n)], indexing="ij")
    zf, yf, xf = np.meshgrid(*[(G.plo[2 - q] + (np.arange(fs[q]) + 0.5) / 2) * H for q in range(3)], indexing="ij")
    return (xc, yc, zc), (xf, yf, zf)


CASES = [
    ((8, 8, 8), (N, N, N), (N, N, N), (2, 3, 2), (6, 6, 5)),
    ((8, 6, 10), (P, P, N), (P, P, N), (1, 1, 3), (4, 5, 9)),
    ((6, 6, 6), (P, P, P), (P, P, P), (2, 2, 2), (3, 3, 3)),  # one coarse cell: the thinnest patch
    ((9, 7, 8), (N, P, N), (N, P, N), (3, 1, 1), (8, 6, 7)),
]


@pytest.mark.parametrize("n,lo,hi,plo,phi", CASES)
def test_composite_conservation_and_constants(n, lo, hi, plo, phi):
    G = CP.Composite(n, 1.0 / n[0], lo, hi, plo, phi)
    rc, bc, rf, bf, rng = rand_case(G, 1)
    A = CP.operator_matrix(G, rc, bc, rf, bf)
    v = CP.volumes(G)
    for _ in range(3):
        y = A @ rng.standard_normal(G.nunk)
        assert abs(v @ y) <= 1e-12 * (v @ np.abs(y))
    assert np.abs(A @ np.ones(G.nunk)).max() <= 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("n,lo,hi,plo,phi", CASES)
def test_composite_linear_exact(n, lo, hi, plo, phi):
    G = CP.Composite(n, 1.0 / n[0], lo, hi, plo, phi)
    (xc, yc, zc), (xf, yf, zf) = centres(G)
    A = CP.operator_matrix(G, np.ones(xc.shape), np.ones(xc.shape), np.ones(xf.shape), np.ones(xf.shape))
    # off the non-periodic domain faces only (walls break a non-periodic linear field)
    inner = ~G.covered.copy()
    for d in range(3):
        if G.lo[d] != P:
            sl = [slice(None)] * 3
            sl[2 - d] = 0
            inner[tuple(sl)] = False
            sl[2 - d] = -1
            inner[tuple(sl)] = False
    for a in [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (0.3, -0.7, 1.1)]:
        # a periodic axis takes no linear component
        a = tuple(0.0 if G.lo[d] == P else a[d] for d in range(3))
        pc = a[0] * xc + a[1] * yc + a[2] * zc
        pf = a[0] * xf + a[1] * yf + a[2] * zf
        yc_, yf_ = CP.unpack(G, A @ CP.pack(G, pc, pf))
        scale = 1.0 / G.h ** 2
        assert np.abs(yf_).max() <= 1e-12 * scale
        assert np.abs(yc_[inner]).max() <= 1e-12 * scale


def test_composite_planted_ghost_weights_break_the_linear_pin(monkeypatch):
    G = CP.Composite((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3, (2, 3, 2), (6, 6, 5))
    (xc, yc, zc), (xf, yf, zf) = centres(G)
    ones = (np.ones(xc.shape), np.ones(xc.shape), np.ones(xf.shape), np.ones(xf.shape))
    # the ghost as the plain mean of C and F1 (as if C sat at the ghost's mirror
    # image): the weights sum to 1, so constants survive, but a linear field does
    # not (the linear interpolation 2/3 C + 1/3 F1 would, like the quadratic)
    monkeypatch.setattr(CP, "W_C", 0.5)
    monkeypatch.setattr(CP, "W_F1", 0.5)
    monkeypatch.setattr(CP, "W_F2", 0.0)
    A = CP.operator_matrix(G, *ones)
    assert np.abs(A @ np.ones(G.nunk)).max() <= 1e-9
    _, yf_ = CP.unpack(G, A @ CP.pack(G, xc, xf))
    assert np.abs(yf_).max() > 1.0


@pytest.mark.parametrize("n,lo,hi,plo,phi", CASES[:2])
def test_composite_rows_away_from_the_patch_are_single_level(n, lo, hi, plo, phi):
    G = CP.Composite(n, 1.0 / n[0], lo, hi, plo, phi)
    rc, bc, rf, bf, rng = rand_case(G, 2)
    pc = rng.standard_normal(rc.shape)
    pf = rng.standard_normal(rf.shape)
    yc_, yf_ = CP.apply(G, rc, bc, rf, bf, pc, pf)
    gc = W.Geom(G.n, G.H, G.lo, G.hi)
    ref_c = O.mac_apply(gc, O.mac_coeffs(gc, rc, bc), pc)
    far = np.ones(rc.shape, bool)  # coarse cells whose stencil misses the patch
    z0, z1 = max(plo[2] - 1, 0), phi[2] + 1
    y0, y1 = max(plo[1] - 1, 0), phi[1] + 1
    x0, x1 = max(plo[0] - 1, 0), phi[0] + 1
    far[z0:z1, y0:y1, x0:x1] = False
    assert far.sum() > 0
    assert np.abs(yc_[far] - ref_c[far]).max() <= 1e-12 * np.abs(ref_c).max()
    gf = W.Geom(G.nf, G.h, (N,) * 3, (N,) * 3)
    ref_f = O.mac_apply(gf, O.mac_coeffs(gf, rf, bf), pf)
    inner = np.zeros(rf.shape, bool)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.abs(yf_[inner] - ref_f[inner]).max() <= 1e-12 * np.abs(ref_f).max()


def face_fields(G, rng):
    cs = [tuple(reversed([G.n[e] + (1 if e == d else 0) for e in range(3)])) for d in range(3)]
    fs = [tuple(reversed([G.nf[e] + (1 if e == d else 0) for e in range(3)])) for d in range(3)]
    return [rng.standard_normal(s) for s in cs], [rng.standard_normal(s) for s in fs]


@pytest.mark.parametrize("n,lo,hi,plo,phi", CASES + [((8, 8, 8), (P, P, D), (P, P, D), (2, 2, 2), (6, 5, 6))])
def test_composite_projection_identity(n, lo, hi, plo, phi):
    G = CP.Composite(n, 1.0 / n[0], lo, hi, plo, phi)
    rc, bc, rf, bf, rng = rand_case(G, 3)
    uc, uf = face_fields(G, rng)
    sc = rng.standard_normal(rc.shape)
    sf = rng.standard_normal(rf.shape)
    uc2, uf2, pc, pf, info = CP.project(G, uc, uf, rc, bc, sc, rf, bf, sf)
    assert info["rel_resid"] <= 1e-12
    f = info["f"]
    dv = CP.divergence(G, uc2, uf2, bc, bf) - CP.pack(G, bc * sc, bf * sf) - info["mean"]
    assert np.abs(dv - info["resid"]).max() <= 1e-11 * np.abs(f).max()
    assert np.abs(dv).max() <= 1e-11 * np.abs(f).max()
    # walls carry no flow; coarse faces on the patch are the means of their fine faces
    for d in range(3):
        if G.lo[d] == N:
            sl = [slice(None)] * 3
            sl[2 - d] = 0
            assert np.all(uc2[d][tuple(sl)] == 0.0)
        t1, t2 = [t for t in range(3) if t != d]
        for p in (G.plo[d], G.phi[d]):
            face = [0, 0, 0]
            face[d], face[t1], face[t2] = p, G.plo[t1], G.plo[t2]
            ff = [0, 0, 0]
            ff[d] = 2 * (p - G.plo[d])
            want = 0.25 * sum(uf2[d][tuple(reversed([ff[0] + (e1 if t1 == 0 else 0) + (e2 if t2 == 0 else 0),
                                                      ff[1] + (e1 if t1 == 1 else 0) + (e2 if t2 == 1 else 0),
                                                      ff[2] + (e1 if t1 == 2 else 0) + (e2 if t2 == 2 else 0)]))]
                              for e1 in range(2) for e2 in range(2))
            assert uc2[d][face[2], face[1], face[0]] == pytest.approx(want, rel=1e-14, abs=1e-14)
    if G.singular:
        v = CP.volumes(G)
        x = CP.pack(G, pc, pf)
        assert abs(v @ x) <= 1e-12 * (v @ np.abs(x))


def test_composite_second_order():
    """walls all round, constant coefficients, phi* = cos(pi x) cos(pi y) cos(pi z)
    (zero normal derivative on the walls), f = -3 pi^2 phi* at the centres"""
    errs = []
    for n in (8, 16):
        G = CP.Composite((n,) * 3, 1.0 / n, (N,) * 3, (N,) * 3, (n // 4,) * 3, (3 * n // 4 - n // 8,) * 3)
        (xc, yc, zc), (xf, yf, zf) = centres(G)
        ex = lambda x, y, z: np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
        A = CP.operator_matrix(G, np.ones(xc.shape), np.ones(xc.shape), np.ones(xf.shape), np.ones(xf.shape))
        v = CP.volumes(G)
        f = CP.pack(G, -3 * np.pi ** 2 * ex(xc, yc, zc), -3 * np.pi ** 2 * ex(xf, yf, zf))
        f -= v @ f / v.sum()
        x = CP.solve(G, A, f)
        xs = CP.pack(G, ex(xc, yc, zc), ex(xf, yf, zf))
        xs -= v @ xs / v.sum()
        errs.append(np.abs(x - xs).max())
    assert errs[0] / errs[1] >= 3.5, errs


def test_composite_rejects_bad_patches():
    with pytest.raises(ValueError):
        CP.Composite((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3, (0, 2, 2), (4, 4, 4))  # touches a domain face
    with pytest.raises(ValueError):
        CP.Composite((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3, (2, 2, 2), (2, 4, 4))  # empty


# ---- several patches on the fine level (the batched layout with coarse-fine interfaces) ----

MULTI = [
    ((12, 10, 10), (N, N, N), (N, N, N), [((1, 1, 1), (4, 5, 4)), ((6, 2, 2), (11, 8, 9))]),
    # one coarse cell between the patches along x: its two x faces both match fine fluxes
    ((12, 8, 10), (P, P, N), (P, P, N), [((1, 1, 1), (5, 4, 4)), ((6, 1, 5), (10, 7, 9))]),
    ((10, 10, 10), (P, P, D), (P, P, D), [((2, 2, 2), (4, 4, 4)), ((6, 6, 6), (8, 8, 8)), ((2, 6, 2), (4, 8, 5))]),
]


def multi_case(case, seed):
    n, lo, hi, boxes = case
    G = CP.Composite(n, 1.0 / n[0], lo, hi, patches=boxes)
    rng = np.random.default_rng(seed)
    cs = tuple(reversed(G.n))
    fss = [tuple(reversed(nf)) for nf in G.nfs]
    e = lambda s: np.exp(rng.standard_normal(s))
    return G, rng, e(cs), e(cs), [e(s) for s in fss], [e(s) for s in fss]


def multi_centres(G):
    H = G.H
    zc, yc, xc = np.meshgrid(*[(np.arange(m) + 0.5) * H for m in reversed(G.n)], indexing="ij")
    fine = []
    for (plo, _), nf in zip(G.boxes, G.nfs):
        fine.append(np.meshgrid(*[(plo[2 - q] + (np.arange(nf[2 - q]) + 0.5) / 2) * H for q in range(3)],
                                indexing="ij")[::-1])
    return (xc, yc, zc), fine


@pytest.mark.parametrize("case", MULTI)
def test_multi_patch_conservation_null_space_and_linear(case):
    G, rng, rc, bc, rfs, bfs = multi_case(case, 7)
    A = CP.operator_matrix(G, rc, bc, rfs, bfs)
    v = CP.volumes(G)
    if G.singular:
        for _ in range(3):
            y = A @ rng.standard_normal(G.nunk)
            assert abs(v @ y) <= 1e-12 * (v @ np.abs(y))
        assert np.abs(A @ np.ones(G.nunk)).max() <= 1e-12 * np.abs(A).max()
    (xc, yc, zc), fine = multi_centres(G)
    ones_c = np.ones(xc.shape)
    ones_f = [np.ones(f[0].shape) for f in fine]
    A1 = CP.operator_matrix(G, ones_c, ones_c, ones_f, ones_f)
    inner = ~G.covered.copy()
    for d in range(3):
        if G.lo[d] != P:
            sl = [slice(None)] * 3
            sl[2 - d] = 0
            inner[tuple(sl)] = False
            sl[2 - d] = -1
            inner[tuple(sl)] = False
    for a in [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (0.3, -0.7, 1.1)]:
        a = tuple(0.0 if G.lo[d] == P else a[d] for d in range(3))
        pc = a[0] * xc + a[1] * yc + a[2] * zc
        pf = [a[0] * f[0] + a[1] * f[1] + a[2] * f[2] for f in fine]
        yc_, yf_ = CP.unpack(G, A1 @ CP.pack(G, pc, pf))
        for y in yf_:
            assert np.abs(y).max() <= 1e-12 / G.h ** 2
        assert np.abs(yc_[inner]).max() <= 1e-12 / G.h ** 2


@pytest.mark.parametrize("case", MULTI)
def test_multi_patch_rows_away_and_projection_identity(case):
    G, rng, rc, bc, rfs, bfs = multi_case(case, 8)
    pc = rng.standard_normal(rc.shape)
    pfs = [rng.standard_normal(r.shape) for r in rfs]
    yc_, _ = CP.apply(G, rc, bc, rfs, bfs, pc, pfs)
    gc = W.Geom(G.n, G.H, G.lo, G.hi)
    ref_c = O.mac_apply(gc, O.mac_coeffs(gc, rc, bc), pc)
    far = np.ones(rc.shape, bool)
    for plo, phi in G.boxes:
        far[max(plo[2] - 1, 0):phi[2] + 1, max(plo[1] - 1, 0):phi[1] + 1, max(plo[0] - 1, 0):phi[0] + 1] = False
    assert far.sum() > 0
    assert np.abs(yc_[far] - ref_c[far]).max() <= 1e-12 * np.abs(ref_c).max()
    # the projection identity with every patch's faces
    uc = [rng.standard_normal(tuple(reversed([G.n[e] + (1 if e == d else 0) for e in range(3)]))) for d in range(3)]
    ufs = [[rng.standard_normal(tuple(reversed([nf[e] + (1 if e == d else 0) for e in range(3)]))) for d in range(3)]
           for nf in G.nfs]
    sc = rng.standard_normal(rc.shape)
    sfs = [rng.standard_normal(r.shape) for r in rfs]
    uc2, uf2, _, _, info = CP.project(G, uc, ufs, rc, bc, sc, rfs, bfs, sfs)
    assert info["rel_resid"] <= 1e-12
    bsf = [b * s_ for b, s_ in zip(bfs, sfs)]
    dv = CP.divergence(G, uc2, uf2, bc, bfs) - CP.pack(G, bc * sc, bsf) - info["mean"]
    assert np.abs(dv).max() <= 1e-11 * np.abs(info["f"]).max()


def test_multi_patch_layout_rules():
    with pytest.raises(ValueError):  # touching patches (no coarse cell between)
        CP.Composite((12, 8, 8), 1.0 / 12, (N,) * 3, (N,) * 3, patches=[((1, 1, 1), (5, 4, 4)), ((5, 1, 1), (9, 4, 4))])
    with pytest.raises(ValueError):  # diagonal neighbours: the ghost stencils would read covered cells
        CP.Composite((12, 12, 8), 1.0 / 12, (N,) * 3, (N,) * 3,
                     patches=[((1, 1, 1), (5, 5, 4)), ((5, 5, 1), (9, 9, 4))])
    with pytest.raises(ValueError):
        CP.Composite((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3, patches=[])
    G = CP.Composite((12, 8, 8), 1.0 / 12, (N,) * 3, (N,) * 3, patches=[((1, 1, 1), (5, 4, 4)), ((6, 1, 1), (10, 4, 4))])
    assert G.npatch == 2 and G.nunk == G.nc + 2 * 8 * 6 * 6


def test_apply_at_rows_match_the_matrix():
    """sampled rows, one at a time, equal the assembled operator's (the form the
    full-size GPU checks will use)"""
    G, rng, rc, bc, rfs, bfs = multi_case(MULTI[1], 9)
    pc = rng.standard_normal(rc.shape)
    pfs = [rng.standard_normal(r.shape) for r in rfs]
    full = CP.operator_matrix(G, rc, bc, rfs, bfs) @ CP.pack(G, pc, pfs)
    cells, want = [], []
    for _ in range(60):
        if rng.random() < 0.5:
            while True:
                c = tuple(int(rng.integers(0, G.n[d])) for d in range(3))
                if not G.in_patch(c):
                    break
            cells.append(("c", c))
            want.append(full[int(G.cid[c[2], c[1], c[0]])])
        else:
            p = int(rng.integers(0, G.npatch))
            F = tuple(int(rng.integers(0, G.nfs[p][d])) for d in range(3))
            cells.append(("f", p, F))
            want.append(full[int(G.fids[p][F[2], F[1], F[0]])])
    got = CP.apply_at(G, rc, bc, rfs, bfs, pc, pfs, cells)
    assert np.abs(got - np.array(want)).max() <= 1e-13 * np.abs(full).max()


def test_apply_at_large_grid_far_rows_are_single_level():
    """a grid too large to assemble quickly here: coarse rows away from the patch
    equal the single-level oracle's at the same cells"""
    n = (64, 48, 40)
    G = CP.Composite(n, 1.0 / 64, (P, P, N), (P, P, N), (20, 12, 10), (44, 36, 30))
    rng = np.random.default_rng(10)
    cs, fs = tuple(reversed(G.n)), tuple(reversed(G.nf))
    rc, bc = np.exp(rng.standard_normal(cs)), np.exp(rng.standard_normal(cs))
    rf, bf = np.exp(rng.standard_normal(fs)), np.exp(rng.standard_normal(fs))
    pc, pf = rng.standard_normal(cs), rng.standard_normal(fs)
    gc = W.Geom(G.n, G.H, G.lo, G.hi)
    ref = O.mac_apply(gc, O.mac_coeffs(gc, rc, bc), pc)
    cells = []
    while len(cells) < 50:
        c = tuple(int(rng.integers(0, G.n[d])) for d in range(3))
        if all(c[d] < G.plo[d] - 1 or c[d] > G.phi[d] for d in range(3)):
            cells.append(("c", c))
    got = CP.apply_at(G, rc, bc, rf, bf, pc, pf, cells)
    want = np.array([ref[c[1][2], c[1][1], c[1][0]] for c in cells])
    assert np.abs(got - want).max() <= 1e-12 * np.abs(ref).max()
