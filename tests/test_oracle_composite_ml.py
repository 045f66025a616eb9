"""Pins of the multilevel composite MAC oracle (``oracle/composite_ml.py``;
ratio-2 levels, AMR as in the paper's Paper V, end of Sec. 3.2; the paper's
adaptive runs refine twice, Sec. 4):

  * with two levels it equals the one-level-of-patches oracle
    (``composite.py``), written separately, entry for entry;
  * conservation (volume sum of L phi = 0 on wall and periodic domains, any phi
    and coefficients) and constants in the null space on three levels;
  * a linear phi with constant coefficients gives L phi = 0 on every cell of
    the finer levels and on the level-0 cells off the domain faces;
  * second order: a manufactured solution's error falls by >= 3.5 when every
    level's h halves (three levels);
  * the layout rules (nesting, separation, thickness) are enforced: a box of
    level 2 or deeper keeps two parent cells inside its parent box, since the
    parent's ghost values read its first two layers.
"""
import numpy as np
import pytest

from oracle import composite as CP
from oracle import composite_ml as ML

P, N, D = ML.PERIODIC, ML.NEUMANN, ML.DIRICHLET


def per_level(H, f):
    return [f(tuple(reversed(H.n0)))] + [[f(tuple(reversed(b.n))) for b in H.boxes[l]] for l in range(1, H.nlev)]


def centres(H):
    """per-level (x, y, z) centre coordinates"""
    def grid(l, org, n):
        h = H.h(l)
        z, y, x = np.meshgrid(*[(org[q] + np.arange(n[q]) + 0.5) * h for q in (2, 1, 0)], indexing="ij")
        return x, y, z
    out = [grid(0, (0, 0, 0), H.n0)]
    for l in range(1, H.nlev):
        out.append([grid(l, b.glo, b.n) for b in H.boxes[l]])
    return out


TWO_LEVEL = [
    ((8, 8, 8), (N,) * 3, [((2, 3, 2), (6, 6, 5))]),
    ((12, 8, 10), (P, P, N), [((1, 1, 1), (5, 4, 4)), ((6, 1, 5), (10, 7, 9))]),
    ((10, 10, 10), (P, P, D), [((2, 2, 2), (4, 4, 4)), ((6, 6, 6), (8, 8, 8)), ((2, 6, 2), (4, 8, 5))]),
]


@pytest.mark.parametrize("n,lo,boxes", TWO_LEVEL)
def test_two_levels_equal_the_patch_oracle(n, lo, boxes):
    G = CP.Composite(n, 1.0 / n[0], lo, lo, patches=boxes)
    H = ML.Hierarchy(n, 1.0 / n[0], lo, lo, [boxes])
    assert G.nunk == H.nunk
    rng = np.random.default_rng(0)
    e = lambda s: np.exp(rng.standard_normal(s))
    rc, bc = e(tuple(reversed(n))), e(tuple(reversed(n)))
    rfs = [e(tuple(reversed(nf))) for nf in G.nfs]
    bfs = [e(tuple(reversed(nf))) for nf in G.nfs]
    A1 = CP.operator_matrix(G, rc, bc, rfs, bfs)
    A2 = ML.operator(H, [rc, rfs], [bc, bfs])
    assert abs(A1 - A2).max() <= 1e-14 * abs(A1).max()


THREE_LEVEL = [
    ((8, 8, 8), (N,) * 3, [[((2, 2, 2), (6, 6, 6))], [((6, 6, 6), (10, 10, 9))]]),
    ((10, 8, 8), (P, P, N), [[((1, 1, 1), (5, 7, 4)), ((6, 2, 4), (9, 6, 7))],
                             [((4, 4, 4), (7, 11, 6)), ((14, 6, 10), (16, 10, 12))]]),
    ((8, 8, 8), (D,) * 3, [[((2, 2, 2), (6, 6, 6))], [((6, 6, 6), (9, 10, 10))]]),
]


@pytest.mark.parametrize("n,lo,levels", THREE_LEVEL)
def test_three_levels_conservation_null_space_linear(n, lo, levels):
    H = ML.Hierarchy(n, 1.0 / n[0], lo, lo, levels)
    rng = np.random.default_rng(1)
    e = lambda s: np.exp(rng.standard_normal(s))
    A = ML.operator(H, per_level(H, e), per_level(H, e))
    v = ML.volumes(H)
    if H.singular:
        for _ in range(3):
            y = A @ rng.standard_normal(H.nunk)
            assert abs(v @ y) <= 1e-12 * (v @ np.abs(y))
        assert np.abs(A @ np.ones(H.nunk)).max() <= 1e-12 * np.abs(A).max()
    one = lambda s: np.ones(s)
    A1 = ML.operator(H, per_level(H, one), per_level(H, one))
    cen = centres(H)
    for a in [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (0.3, -0.7, 1.1)]:
        a = tuple(0.0 if H.bc_lo[d] == P else a[d] for d in range(3))
        lin = lambda xyz: a[0] * xyz[0] + a[1] * xyz[1] + a[2] * xyz[2]
        field = [lin(cen[0])] + [[lin(c) for c in cen[l]] for l in range(1, H.nlev)]
        y = A1 @ ML.join(H, field)
        scale = 1.0 / H.h(H.nlev - 1) ** 2
        for (l, k, loc, g) in H.cells():
            if l == 0 and any(H.bc_lo[d] != P and (g[d] == 0 or g[d] == H.n0[d] - 1) for d in range(3)):
                continue  # a wall or Dirichlet face breaks a linear field
            assert abs(y[H.uid(l, k, loc)]) <= 1e-12 * scale


def test_three_levels_second_order():
    """walls all round, constant coefficients, phi* = cos(pi x) cos(pi y) cos(pi z),
    f = -3 pi^2 phi* at the centres of every level; boxes scale with the grid"""
    errs = []
    for m in (1, 2):
        n = 8 * m
        levels = [[((2 * m, 2 * m, 2 * m), (6 * m, 6 * m, 6 * m))], [((6 * m, 6 * m, 6 * m), (10 * m, 10 * m, 10 * m))]]
        H = ML.Hierarchy((n,) * 3, 1.0 / n, (N,) * 3, (N,) * 3, levels)
        one = lambda s: np.ones(s)
        A = ML.operator(H, per_level(H, one), per_level(H, one))
        cen = centres(H)
        ex = lambda xyz: np.cos(np.pi * xyz[0]) * np.cos(np.pi * xyz[1]) * np.cos(np.pi * xyz[2])
        xs = ML.join(H, [ex(cen[0])] + [[ex(c) for c in cen[l]] for l in range(1, H.nlev)])
        v = ML.volumes(H)
        f = -3 * np.pi ** 2 * xs
        f -= v @ f / v.sum()
        x = ML.solve(H, A, f)
        xs -= v @ xs / v.sum()
        errs.append(np.abs(x - xs).max())
    assert errs[0] / errs[1] >= 3.5, errs


def test_split_join_round_trip():
    H = ML.Hierarchy((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3, THREE_LEVEL[0][2])
    x = np.random.default_rng(2).standard_normal(H.nunk)
    assert np.array_equal(ML.join(H, ML.split(H, x)), x)


def test_layout_rules():
    with pytest.raises(ValueError):  # level-2 box touching its parent box's faces
        ML.Hierarchy((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3, [[((2, 2, 2), (6, 6, 6))], [((4, 5, 5), (8, 9, 9))]])
    with pytest.raises(ValueError):  # one parent cell inside is not enough for a deeper level
        ML.Hierarchy((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3, [[((2, 2, 2), (6, 6, 6))], [((5, 6, 6), (10, 10, 10))]])
    with pytest.raises(ValueError):  # level-1 box at the domain face
        ML.Hierarchy((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3, [[((0, 2, 2), (4, 6, 6))]])
    with pytest.raises(ValueError):  # boxes of a level touching
        ML.Hierarchy((12, 8, 8), 1.0 / 12, (N,) * 3, (N,) * 3, [[((1, 1, 1), (5, 4, 4)), ((5, 1, 1), (9, 4, 4))]])
    with pytest.raises(ValueError):  # empty level
        ML.Hierarchy((8, 8, 8), 1.0 / 8, (N,) * 3, (N,) * 3, [[]])
