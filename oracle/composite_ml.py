"""Composite MAC operator (and its direct solve) on any number of ratio-2 levels.

TEST INFRASTRUCTURE (part of the oracle): only the tests, the smoke check and
the benchmark's CPU legs may use it.  The CUDA library shares nothing with it.

The paper keeps its AMR as in its Paper V (absent) with refinement ratio 2
between levels (end of Sec. 3.2), and its adaptive runs use two levels of
refinement (Sec. 4).  This module restates, for a hierarchy of levels, the
composite scheme of ``composite.py`` (one level of patches), written
independently of it: every level l >= 1 is a set of boxes given in the global
cell indices of level l - 1 ([lo, hi), refined by 2); a box keeps at least one
cell of level 0 from the domain faces (l = 1) or two cells of level l - 1 from
the faces of the level-(l-1) box it lies in (l >= 2: the ghosts of that box's
cells read its first two layers, which must stay unknowns), and one parent
cell from every other box of its level.  Unknowns: the cells of every level
not covered by the next finer level.  Between levels l - 1 and l: ghost values of level-l cells by linear
tangential interpolation of the level-(l-1) cell across and the normal
quadratic 8/15 C~ + 2/3 F1 - 1/5 F2; the level-(l-1) flux through a coarse-fine
face is the mean of the four level-l fluxes (flux matching); face coefficients
by arithmetic face means; the domain faces on level 0 as on one level.

Fields: level 0 as one array over the whole grid (x fastest); level l >= 1 as a
list with one array per box.  Functions return unknown-ordered vectors; use
``split`` / ``join`` to convert.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

PERIODIC, NEUMANN, DIRICHLET = 0, 1, 2
GHOST_C, GHOST_F1, GHOST_F2 = 8.0 / 15.0, 2.0 / 3.0, -1.0 / 5.0


class Box:
    def __init__(self, level, lo, hi):
        self.level = level
        self.lo = tuple(int(v) for v in lo)  # in level-(level-1) global indices
        self.hi = tuple(int(v) for v in hi)
        self.glo = tuple(2 * v for v in self.lo)  # own global indices
        self.ghi = tuple(2 * v for v in self.hi)
        self.n = tuple(self.ghi[d] - self.glo[d] for d in range(3))

    def contains_global(self, g):
        """g: a cell of this box's level in global indices"""
        return all(self.glo[d] <= g[d] < self.ghi[d] for d in range(3))

    def covers_parent(self, c):
        """c: a cell of the parent level in global indices"""
        return all(self.lo[d] <= c[d] < self.hi[d] for d in range(3))


class Hierarchy:
    def __init__(self, n, dx, lo, hi, levels):
        """levels: for l = 1, 2, ..., a list of (lo, hi) boxes in level-(l-1) global indices"""
        self.n0 = tuple(int(v) for v in n)
        self.dx0 = float(dx)
        self.bc_lo, self.bc_hi = tuple(lo), tuple(hi)
        for d in range(3):
            if (self.bc_lo[d] == PERIODIC) != (self.bc_hi[d] == PERIODIC):
                raise ValueError("periodic on one side only")
        self.nlev = 1 + len(levels)
        self.boxes = [[]] + [[Box(l + 1, a, b) for a, b in lv] for l, lv in enumerate(levels)]
        for l in range(1, self.nlev):
            if not self.boxes[l]:
                raise ValueError("a level without boxes")
            for bx in self.boxes[l]:
                if any(bx.hi[d] - bx.lo[d] < 1 for d in range(3)):
                    raise ValueError("a box must be one parent cell thick")
                # level 1: one cell from the domain faces (the ghosts' tangential
                # neighbours exist); deeper: two cells inside the parent box (the
                # parent's ghosts read its first two layers, which must stay unknowns)
                m = 1 if l == 1 else 2
                grown_lo = tuple(v - m for v in bx.lo)
                grown_hi = tuple(v + m for v in bx.hi)
                if l == 1:
                    ok = all(grown_lo[d] >= 0 and grown_hi[d] <= self.n0[d] for d in range(3))
                else:
                    ok = any(all(p.glo[d] <= grown_lo[d] and grown_hi[d] <= p.ghi[d] for d in range(3))
                             for p in self.boxes[l - 1])
                if not ok:
                    raise ValueError("a box must keep one parent cell from the domain faces (level 1) or two "
                                     "from its parent box's faces (deeper levels)")
            for i, a in enumerate(self.boxes[l]):
                for b in self.boxes[l][:i]:
                    if all(a.lo[d] - 1 < b.hi[d] and b.lo[d] < a.hi[d] + 1 for d in range(3)):
                        raise ValueError("boxes of a level must keep one parent cell apart")
        # unknown numbering: level 0 (x fastest), then each box of each level (x fastest)
        self.ids = []  # ids[l][k]: array over the box (level 0: the grid), -1 where covered
        nxt = 0
        for l in range(self.nlev):
            shapes = [self.n0] if l == 0 else [b.n for b in self.boxes[l]]
            origins = [(0, 0, 0)] if l == 0 else [b.glo for b in self.boxes[l]]
            lev_ids = []
            for shp, org in zip(shapes, origins):
                cov = np.zeros((shp[2], shp[1], shp[0]), dtype=bool)
                if l + 1 < self.nlev:
                    for fb in self.boxes[l + 1]:
                        a = [max(fb.lo[d] - org[d], 0) for d in range(3)]
                        b = [min(fb.hi[d] - org[d], shp[d]) for d in range(3)]
                        if all(a[d] < b[d] for d in range(3)):
                            cov[a[2]:b[2], a[1]:b[1], a[0]:b[0]] = True
                ids = -np.ones(cov.shape, dtype=np.int64)
                m = int((~cov).sum())
                ids[~cov] = nxt + np.arange(m)
                nxt += m
                lev_ids.append(ids)
            self.ids.append(lev_ids)
        self.nunk = nxt
        self.singular = all(b != DIRICHLET for b in self.bc_lo + self.bc_hi)

    def h(self, l):
        return self.dx0 / (2 ** l)

    def ngrid(self, l):
        return tuple(v * 2 ** l for v in self.n0)

    def locate(self, l, g):
        """(box index, local index) of the level-l cell with global index g, or
        None when level l has no cell there (outside its boxes); level 0 wraps
        periodic axes and returns None beyond a non-periodic domain face"""
        if l == 0:
            q = list(g)
            for d in range(3):
                if not 0 <= q[d] < self.n0[d]:
                    if self.bc_lo[d] != PERIODIC:
                        return None
                    q[d] %= self.n0[d]
            return 0, tuple(q)
        for k, b in enumerate(self.boxes[l]):
            if b.contains_global(g):
                return k, tuple(g[d] - b.glo[d] for d in range(3))
        return None

    def uid(self, l, k, loc):
        return int(self.ids[l][k][loc[2], loc[1], loc[0]])

    def fine_box_covering(self, l, g):
        """the level-(l+1) box covering the level-l cell g (global), or -1"""
        if l + 1 >= self.nlev:
            return -1
        for k, b in enumerate(self.boxes[l + 1]):
            if b.covers_parent(g):
                return k
        return -1

    def cells(self):
        """every unknown as (level, box, local index, global index)"""
        out = []
        for l in range(self.nlev):
            for k, ids in enumerate(self.ids[l]):
                org = (0, 0, 0) if l == 0 else self.boxes[l][k].glo
                nz, ny, nx = ids.shape
                for z in range(nz):
                    for y in range(ny):
                        for x in range(nx):
                            if ids[z, y, x] >= 0:
                                out.append((l, k, (x, y, z), (x + org[0], y + org[1], z + org[2])))
        return out


def _val(H, field, l, g):
    k, loc = H.locate(l, g)
    a = field[l] if l == 0 else field[l][k]
    return a[loc[2], loc[1], loc[0]]


def _face_b(beta_a, rho_a, beta_b, rho_b):
    return (0.5 * (beta_a + beta_b)) / (0.5 * (rho_a + rho_b))


def ghost(H, l, g, d, s):
    """the ghost of level-l cell g (global) across its box face along d, side s:
    (list of (unknown id, weight), the level-(l-1) global index of the cell across)"""
    C = [g[e] // 2 for e in range(3)]
    C[d] += s
    terms = []
    k, loc = H.locate(l - 1, tuple(C))
    terms.append((H.uid(l - 1, k, loc), GHOST_C))
    for t in range(3):
        if t == d:
            continue
        sig = 0.125 if g[t] % 2 else -0.125
        for step, w in ((1, sig), (-1, -sig)):
            q = list(C)
            q[t] += step
            k2, loc2 = H.locate(l - 1, tuple(q))
            terms.append((H.uid(l - 1, k2, loc2), GHOST_C * w))
    kf, locf = H.locate(l, g)
    terms.append((H.uid(l, kf, locf), GHOST_F1))
    g2 = list(g)
    g2[d] -= s
    kf2, locf2 = H.locate(l, tuple(g2))
    terms.append((H.uid(l, kf2, locf2), GHOST_F2))
    if any(col < 0 for col, _ in terms):
        raise AssertionError("a ghost value reads a covered cell: the layout rules were not enforced")
    return terms, tuple(C)


def _cf_fine_cells(c, d, s):
    """the four level-(l+1) global cells on the face of level-l cell c toward c + s e_d"""
    t1, t2 = [t for t in range(3) if t != d]
    Fd = 2 * (c[d] + s) + (0 if s > 0 else 1)
    out = []
    for a in range(2):
        for b in range(2):
            F = [0, 0, 0]
            F[d] = Fd
            F[t1] = 2 * c[t1] + a
            F[t2] = 2 * c[t2] + b
            out.append(tuple(F))
    return out


def operator(H, rho, beta0):
    """the composite operator as a sparse matrix; rho, beta0: per level (level 0
    an array, level l a list of per-box arrays)"""
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    for (l, k, loc, g) in H.cells():
        r = H.uid(l, k, loc)
        h = H.h(l)
        rg, bg = _val(H, rho, l, g), _val(H, beta0, l, g)
        for d in range(3):
            for s in (-1, 1):
                nb = list(g)
                nb[d] += s
                nb = tuple(nb)
                where = H.locate(l, nb)
                if where is None:
                    if l == 0:  # a non-periodic domain face
                        bc = H.bc_lo[d] if s < 0 else H.bc_hi[d]
                        if bc == DIRICHLET:
                            add(r, r, -2.0 * (bg / rg) / (h * h))
                        continue
                    # across this level's box boundary: the ghost from level l - 1
                    terms, C = ghost(H, l, g, d, s)
                    b = _face_b(bg, rg, _val(H, beta0, l - 1, C), _val(H, rho, l - 1, C))
                    for col, w in terms:
                        add(r, col, b * w / (h * h))
                    add(r, r, -b / (h * h))
                    continue
                kn, locn = where
                gn = nb if l > 0 else tuple(locn)  # level 0: the wrapped index
                if H.fine_box_covering(l, gn) < 0:
                    b = _face_b(bg, rg, _val(H, beta0, l, gn), _val(H, rho, l, gn))
                    add(r, H.uid(l, kn, locn), b / (h * h))
                    add(r, r, -b / (h * h))
                    continue
                # flux matching: the mean of the four level-(l+1) fluxes b (phi_F1 - phi_g)/h_f
                hf = H.h(l + 1)
                gc = g if l > 0 else tuple(gn[e] - s * (1 if e == d else 0) for e in range(3))
                for F in _cf_fine_cells(gc, d, s):
                    bf = _face_b(_val(H, beta0, l + 1, F), _val(H, rho, l + 1, F), bg, rg)
                    w = 0.25 * bf / (hf * h)
                    kf, locf = H.locate(l + 1, F)
                    add(r, H.uid(l + 1, kf, locf), w)
                    terms, _ = ghost(H, l + 1, F, d, -s)
                    for col, wt in terms:
                        add(r, col, -w * wt)
    return sp.csr_matrix((vals, (rows, cols)), shape=(H.nunk, H.nunk))


def volumes(H):
    v = np.empty(H.nunk)
    for (l, k, loc, g) in H.cells():
        v[H.uid(l, k, loc)] = H.h(l) ** 3
    return v


def join(H, field):
    """per-level field -> unknown-ordered vector"""
    x = np.empty(H.nunk)
    for (l, k, loc, g) in H.cells():
        a = field[l] if l == 0 else field[l][k]
        x[H.uid(l, k, loc)] = a[loc[2], loc[1], loc[0]]
    return x


def split(H, x):
    """unknown-ordered vector -> per-level field (covered cells: the mean of the
    eight finer cells, filled from the finest level down)"""
    out = [np.zeros(tuple(reversed(H.n0)))] + [[np.zeros(tuple(reversed(b.n))) for b in H.boxes[l]]
                                              for l in range(1, H.nlev)]
    for (l, k, loc, g) in H.cells():
        a = out[l] if l == 0 else out[l][k]
        a[loc[2], loc[1], loc[0]] = x[H.uid(l, k, loc)]
    for l in range(H.nlev - 1, 0, -1):
        for k, b in enumerate(H.boxes[l]):
            f = out[l][k]
            nz, ny, nx = f.shape
            avg = f.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5))
            for z in range(nz // 2):
                for y in range(ny // 2):
                    for xx in range(nx // 2):
                        gp = (b.lo[0] + xx, b.lo[1] + y, b.lo[2] + z)
                        kp, locp = H.locate(l - 1, gp)
                        tgt = out[l - 1] if l - 1 == 0 else out[l - 1][kp]
                        tgt[locp[2], locp[1], locp[0]] = avg[z, y, xx]
    return out


def solve(H, A, f):
    if not H.singular:
        return spla.spsolve(A.tocsc(), f)
    v = volumes(H)
    n = H.nunk
    B = sp.bmat([[A, sp.csr_matrix(np.ones((n, 1)))], [sp.csr_matrix(v.reshape(1, n)), None]]).tocsc()
    return spla.spsolve(B, np.concatenate([f, [0.0]]))[:n]
