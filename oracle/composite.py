"""Two-level composite MAC operator and projection, refinement ratio 2.

TEST INFRASTRUCTURE (part of the oracle): only the tests, the smoke check and
the benchmark's CPU legs may use it.  The CUDA library shares nothing with it.

The paper keeps its adaptive mesh refinement "algorithmically the same" as its
Paper V (Sec. 5 there, not available here) and states that levels refine by a
ratio of 2 (end of Sec. 3.2).  The composite discretisation below is therefore
a reading, chosen as the standard cell-centred ratio-2 scheme and consistent
with the single-level oracle (oracle.c):

  * Layout: a coarse level of n cells per axis (cell width H) with the domain's
    boundary conditions, and fine patches, each covering a coarse box
    [plo, phi) (cell width h = H/2, 2 (phi - plo) cells per axis).  A patch
    keeps at least one coarse cell from every face of the domain (so its
    boundary is a coarse-fine interface only), is at least one coarse cell
    thick, and keeps at least one coarse cell from every other patch (so no
    two fine cells of different patches touch and the coarse cells a ghost
    value reads are never covered).  Unknowns: phi on the coarse cells not
    covered by a patch, then on the fine cells patch by patch.
  * Face coefficients b = beta0_f / rho_f with arithmetic face means, as on one
    level; on a coarse-fine face, of the fine cell and the coarse cell across.
  * Fine ghost value across a coarse-fine face (normal direction d, fine cell F1
    on the interface, F2 the next one inward, C the coarse cell across): the
    coarse value is first interpolated linearly to the ghost's tangential
    position with the central differences of C's tangential neighbours
    (offsets of -H/4 or +H/4), then phi_g = 8/15 C~ + 2/3 F1 - 1/5 F2, the
    quadratic through the three centres evaluated at the ghost's (in the
    normal coordinate, measured from the ghost's centre: C at -h/2, F1 at +h,
    F2 at +2h).
  * Flux matching: a coarse cell's flux through a coarse-fine face is the mean
    of the four fine fluxes b (phi_F1 - phi_g)/h on it, so the composite
    divergence of any flux field telescopes (sum of volume x divergence = the
    domain-boundary flux).
  * Right-hand side f = D(beta0 U) - beta0 Sbar on both levels, the coarse
    cells' coarse-fine fluxes being the means of the fine beta0_f U_f; when no
    domain face is Dirichlet the volume-weighted mean is removed.
  * Correction U_f <- U_f - (dphi/dn) / rho_f on both levels (the fine
    coarse-fine faces with the ghost value); the coarse faces on and inside the
    patch then take the mean of the four fine faces on them, and the covered
    coarse phi the mean of its eight fine cells.

Arrays are numpy float64 in x-fastest order (shape (nz, ny, nx)); face arrays
carry n_d + 1 entries along their own direction, as elsewhere in the oracle.
Fine fields are one array per patch (a list), or a plain array with a single
patch.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

PERIODIC, NEUMANN, DIRICHLET = 0, 1, 2

# normal-direction ghost weights for (C~, F1, F2): the quadratic through the
# centres at normal coordinates -h/2 (C), h (F1) and 2h (F2) measured from the
# ghost's centre, evaluated at 0
W_C, W_F1, W_F2 = 8.0 / 15.0, 2.0 / 3.0, -1.0 / 5.0


class Composite:
    """Index maps of a coarse level with ratio-2 fine patches.

    n: coarse cells per axis (x, y, z); dx: coarse cell width; lo, hi: boundary
    type per axis; plo, phi: one patch as the coarse-index box [plo, phi), or
    patches: a list of such (plo, phi) boxes."""

    def __init__(self, n, dx, lo, hi, plo=None, phi=None, patches=None):
        self.n = tuple(int(v) for v in n)
        self.H = float(dx)
        self.h = self.H / 2.0
        self.lo = tuple(lo)
        self.hi = tuple(hi)
        if patches is None:
            patches = [(plo, phi)]
        self.boxes = [(tuple(int(v) for v in a), tuple(int(v) for v in b)) for a, b in patches]
        if not self.boxes:
            raise ValueError("no patch")
        for d in range(3):
            if self.lo[d] == PERIODIC and self.hi[d] != PERIODIC or self.hi[d] == PERIODIC and self.lo[d] != PERIODIC:
                raise ValueError("periodic on one side only")
        for a, b in self.boxes:
            for d in range(3):
                if not (1 <= a[d] and b[d] <= self.n[d] - 1 and b[d] - a[d] >= 1):
                    raise ValueError("a patch must keep one coarse cell from the domain faces and be one cell thick")
        for p in range(len(self.boxes)):
            for q in range(p):
                (a0, a1), (b0, b1) = self.boxes[p], self.boxes[q]
                if all(a0[d] - 1 < b1[d] and b0[d] < a1[d] + 1 for d in range(3)):
                    raise ValueError("patches must keep one coarse cell apart")
        nx, ny, nz = self.n
        self.owner = -np.ones((nz, ny, nx), dtype=np.int64)  # patch covering each coarse cell
        for p, (a, b) in enumerate(self.boxes):
            self.owner[a[2]:b[2], a[1]:b[1], a[0]:b[0]] = p
        cov = self.owner >= 0
        self.covered = cov
        self.cid = -np.ones((nz, ny, nx), dtype=np.int64)
        self.cid[~cov] = np.arange(int((~cov).sum()))
        self.nc = int((~cov).sum())
        self.nfs, self.fids = [], []
        off = self.nc
        for a, b in self.boxes:
            nf = tuple(2 * (b[d] - a[d]) for d in range(3))
            self.nfs.append(nf)
            self.fids.append(off + np.arange(nf[0] * nf[1] * nf[2], dtype=np.int64).reshape(nf[2], nf[1], nf[0]))
            off += nf[0] * nf[1] * nf[2]
        self.nunk = off
        self.singular = all(bc != DIRICHLET for bc in self.lo + self.hi)

    # the single-patch view
    @property
    def plo(self):
        return self.boxes[0][0]

    @property
    def phi(self):
        return self.boxes[0][1]

    @property
    def nf(self):
        return self.nfs[0]

    @property
    def fid(self):
        return self.fids[0]

    @property
    def npatch(self):
        return len(self.boxes)

    # ---- small helpers (index tuples are (x, y, z)) ----
    def coarse_nb(self, c, d, s):
        """coarse neighbour of cell c along d (s = -1 / +1), wrapped on a
        periodic axis; None beyond a non-periodic domain face"""
        q = list(c)
        q[d] += s
        if 0 <= q[d] < self.n[d]:
            return tuple(q)
        if self.lo[d] == PERIODIC:
            q[d] %= self.n[d]
            return tuple(q)
        return None

    def domain_bc(self, d, s):
        return self.lo[d] if s < 0 else self.hi[d]

    def patch_of(self, c):
        """the patch covering coarse cell c, or -1"""
        return int(self.owner[c[2], c[1], c[0]])

    def in_patch(self, c):
        return self.patch_of(c) >= 0

    def parent(self, F, p=0):
        """coarse cell containing fine cell F (patch-local index) of patch p"""
        return tuple(self.boxes[p][0][d] + F[d] // 2 for d in range(3))

    def fine_inside(self, F, p=0):
        return all(0 <= F[d] < self.nfs[p][d] for d in range(3))


def _fine_list(G, a):
    """a fine field as one array per patch"""
    if isinstance(a, (list, tuple)):
        if len(a) != G.npatch:
            raise ValueError("one fine array per patch")
        return [np.asarray(x) for x in a]
    if G.npatch != 1:
        raise ValueError("one fine array per patch")
    return [np.asarray(a)]


def _fine_faces(G, uf):
    """fine face fields as [patch][direction]"""
    if G.npatch == 1 and len(uf) == 3 and not isinstance(uf[0], (list, tuple)):
        return [list(uf)]
    if len(uf) != G.npatch:
        raise ValueError("one list of three face arrays per patch")
    return [list(x) for x in uf]


def _at(a, c):
    return a[c[2], c[1], c[0]]


def ghost_terms(G, F, d, s, p=0):
    """phi_g of fine cell F (patch-local, patch p) across its patch face along d
    on side s, as a list of (unknown index, weight); and the coarse cell across"""
    C = list(G.parent(F, p))
    C[d] += s
    C = tuple(C)
    terms = [(int(_at(G.cid, C)), W_C)]
    for t in range(3):
        if t == d:
            continue
        sig = -1.0 if F[t] % 2 == 0 else 1.0  # fine centre at -H/4 or +H/4 from its parent's
        cp = list(C)
        cm = list(C)
        cp[t] += 1
        cm[t] -= 1
        terms.append((int(_at(G.cid, tuple(cp))), W_C * sig / 8.0))
        terms.append((int(_at(G.cid, tuple(cm))), -W_C * sig / 8.0))
    F2 = list(F)
    F2[d] -= s
    terms.append((int(_at(G.fids[p], F)), W_F1))
    terms.append((int(_at(G.fids[p], tuple(F2))), W_F2))
    return C, terms


def _bmean(beta_a, rho_a, beta_b, rho_b):
    return (0.5 * (beta_a + beta_b)) / (0.5 * (rho_a + rho_b))


def _cf_cells(G, c, nb, d, s, q):
    """the four fine cells of patch q on the coarse-fine face between coarse cell c
    (outside) and coarse cell nb (covered by q), c + s e_d = nb"""
    plo = G.boxes[q][0]
    t1, t2 = [t for t in range(3) if t != d]
    Fd = 2 * (nb[d] - plo[d]) + (0 if s > 0 else 1)
    out = []
    for a in range(2):
        for bb in range(2):
            F = [0, 0, 0]
            F[d] = Fd
            F[t1] = 2 * (c[t1] - plo[t1]) + a
            F[t2] = 2 * (c[t2] - plo[t2]) + bb
            out.append(tuple(F))
    return out


def _coarse_row(G, c, rho_c, beta0_c, rho_f, beta0_f):
    """(column, value) entries of the row of uncovered coarse cell c"""
    H, h = G.H, G.h
    out = []
    r = int(_at(G.cid, c))
    rc, bc = _at(rho_c, c), _at(beta0_c, c)
    for d in range(3):
        for s in (-1, 1):
            nb = G.coarse_nb(c, d, s)
            if nb is None:
                if G.domain_bc(d, s) == DIRICHLET:  # phi = 0 at the face: (0 - phi)/(H/2)
                    out.append((r, -2.0 * (bc / rc) / (H * H)))
                continue
            q = G.patch_of(nb)
            if q < 0:
                b = _bmean(bc, rc, _at(beta0_c, nb), _at(rho_c, nb))
                out.append((int(_at(G.cid, nb)), b / (H * H)))
                out.append((r, -b / (H * H)))
                continue
            # coarse-fine face: the mean of the four fine fluxes b (phi_F1 - phi_g)/h
            for F in _cf_cells(G, c, nb, d, s, q):
                bf = _bmean(_at(beta0_f[q], F), _at(rho_f[q], F), bc, rc)
                w = 0.25 * bf / (h * H)
                out.append((int(_at(G.fids[q], F)), w))
                _, terms = ghost_terms(G, F, d, -s, q)
                for col, wt in terms:
                    out.append((col, -w * wt))
    return r, out


def _fine_row(G, p, F, rho_c, beta0_c, rho_f, beta0_f):
    """(column, value) entries of the row of fine cell F of patch p"""
    h = G.h
    out = []
    r = int(_at(G.fids[p], F))
    rf, bf_ = _at(rho_f[p], F), _at(beta0_f[p], F)
    for d in range(3):
        for s in (-1, 1):
            N = list(F)
            N[d] += s
            N = tuple(N)
            if G.fine_inside(N, p):
                b = _bmean(bf_, rf, _at(beta0_f[p], N), _at(rho_f[p], N))
                out.append((int(_at(G.fids[p], N)), b / (h * h)))
                out.append((r, -b / (h * h)))
            else:
                C, terms = ghost_terms(G, F, d, s, p)
                b = _bmean(bf_, rf, _at(beta0_c, C), _at(rho_c, C))
                for col, wt in terms:
                    out.append((col, b * wt / (h * h)))
                out.append((r, -b / (h * h)))
    return r, out


def operator_matrix(G, rho_c, beta0_c, rho_f, beta0_f):
    """The composite operator L as a sparse matrix on the unknown vector (coarse
    uncovered cells in x-fastest order, then the fine cells patch by patch)."""
    rho_f, beta0_f = _fine_list(G, rho_f), _fine_list(G, beta0_f)
    rows, cols, vals = [], [], []
    nx, ny, nz = G.n
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = (i, j, k)
                if G.in_patch(c):
                    continue
                r, ent = _coarse_row(G, c, rho_c, beta0_c, rho_f, beta0_f)
                for col, v in ent:
                    rows.append(r)
                    cols.append(col)
                    vals.append(v)
    for p in range(G.npatch):
        fx, fy, fz = G.nfs[p]
        for K in range(fz):
            for J in range(fy):
                for I in range(fx):
                    r, ent = _fine_row(G, p, (I, J, K), rho_c, beta0_c, rho_f, beta0_f)
                    for col, v in ent:
                        rows.append(r)
                        cols.append(col)
                        vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(G.nunk, G.nunk))


def apply_at(G, rho_c, beta0_c, rho_f, beta0_f, phi_c, phi_f, cells):
    """L phi at the listed cells only, one row at a time (for sampled checks of
    large composite grids): cells as ("c", (i, j, k)) for an uncovered coarse
    cell or ("f", p, (I, J, K)) for a fine cell of patch p."""
    rho_f, beta0_f = _fine_list(G, rho_f), _fine_list(G, beta0_f)
    x = pack(G, phi_c, phi_f)
    out = np.empty(len(cells))
    for q, cell in enumerate(cells):
        if cell[0] == "c":
            if G.in_patch(cell[1]):
                raise ValueError("a covered coarse cell has no row")
            _, ent = _coarse_row(G, tuple(cell[1]), rho_c, beta0_c, rho_f, beta0_f)
        else:
            _, ent = _fine_row(G, int(cell[1]), tuple(cell[2]), rho_c, beta0_c, rho_f, beta0_f)
        out[q] = sum(v * x[col] for col, v in ent)
    return out


def volumes(G):
    v = np.empty(G.nunk)
    v[:G.nc] = G.H ** 3
    v[G.nc:] = G.h ** 3
    return v


def pack(G, phi_c, phi_f):
    x = np.empty(G.nunk)
    x[:G.nc] = np.asarray(phi_c)[~G.covered]
    off = G.nc
    for a in _fine_list(G, phi_f):
        x[off:off + a.size] = a.ravel()
        off += a.size
    return x


def unpack(G, x):
    """(coarse array with covered cells = mean of their 8 fine cells, fine array
    (one patch) or list of fine arrays)"""
    nx, ny, nz = G.n
    pc = np.zeros((nz, ny, nx))
    pc[~G.covered] = x[:G.nc]
    pfs = []
    off = G.nc
    for (a, b), (fx, fy, fz) in zip(G.boxes, G.nfs):
        pf = np.asarray(x[off:off + fx * fy * fz]).reshape(fz, fy, fx)
        off += fx * fy * fz
        avg = pf.reshape(fz // 2, 2, fy // 2, 2, fx // 2, 2).mean(axis=(1, 3, 5))
        pc[a[2]:b[2], a[1]:b[1], a[0]:b[0]] = avg
        pfs.append(pf)
    return pc, (pfs[0] if G.npatch == 1 else pfs)


def apply(G, rho_c, beta0_c, rho_f, beta0_f, phi_c, phi_f):
    A = operator_matrix(G, rho_c, beta0_c, rho_f, beta0_f)
    return unpack(G, A @ pack(G, phi_c, phi_f))


def _fface(F, d, side):
    """index (x, y, z) of the fine face of cell F along d on side (0 low, 1 high)"""
    q = list(F)
    q[d] += side
    return tuple(q)


def divergence(G, uc, uf, beta0_c, beta0_f):
    """Composite D(beta0 U) as an unknown-ordered vector: coarse faces with the
    single-level rules (U taken as 0 on walls, beta0 of the interior cell on a
    Dirichlet face) except the coarse-fine faces, whose flux is the mean of the
    four fine beta0_f U_f; fine faces with beta0_f the mean of the fine cell and,
    on the patch boundary, the coarse cell across.  uf: three face arrays (one
    patch) or one such list per patch."""
    uf = _fine_faces(G, uf)
    beta0_f = _fine_list(G, beta0_f)
    out = np.zeros(G.nunk)
    H, h = G.H, G.h
    nx, ny, nz = G.n
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = (i, j, k)
                if G.in_patch(c):
                    continue
                r = int(_at(G.cid, c))
                bc = _at(beta0_c, c)
                acc = 0.0
                for d in range(3):
                    for s in (-1, 1):
                        face = list(c)
                        if s > 0:
                            face[d] += 1
                        face = tuple(face)
                        nb = G.coarse_nb(c, d, s)
                        if nb is None:
                            if G.domain_bc(d, s) == DIRICHLET:
                                acc += s * bc * _at(uc[d], face)
                            continue
                        q = G.patch_of(nb)
                        if q < 0:
                            acc += s * 0.5 * (bc + _at(beta0_c, nb)) * _at(uc[d], face)
                            continue
                        m = 0.0
                        for F in _cf_cells(G, c, nb, d, s, q):
                            ff = _fface(F, d, 0 if s > 0 else 1)
                            m += 0.25 * 0.5 * (_at(beta0_f[q], F) + bc) * _at(uf[q][d], ff)
                        acc += s * m
                out[r] = acc / H
    for p in range(G.npatch):
        fx, fy, fz = G.nfs[p]
        for K in range(fz):
            for J in range(fy):
                for I in range(fx):
                    F = (I, J, K)
                    r = int(_at(G.fids[p], F))
                    bf_ = _at(beta0_f[p], F)
                    acc = 0.0
                    for d in range(3):
                        for s in (-1, 1):
                            N = list(F)
                            N[d] += s
                            N = tuple(N)
                            ff = _fface(F, d, 1 if s > 0 else 0)
                            if G.fine_inside(N, p):
                                bn = _at(beta0_f[p], N)
                            else:
                                C = list(G.parent(F, p))
                                C[d] += s
                                bn = _at(beta0_c, tuple(C))
                            acc += s * 0.5 * (bf_ + bn) * _at(uf[p][d], ff)
                    out[r] = acc / h
    return out


def rhs(G, uc, uf, beta0_c, beta0_f, sbar_c, sbar_f, remove_mean=True):
    """f = D(beta0 U) - beta0 Sbar (unknown-ordered) and the removed mean c"""
    f = divergence(G, uc, uf, beta0_c, beta0_f)
    bsf = [np.asarray(b) * np.asarray(s_) for b, s_ in zip(_fine_list(G, beta0_f), _fine_list(G, sbar_f))]
    f -= pack(G, np.asarray(beta0_c) * np.asarray(sbar_c), bsf)
    c = 0.0
    if G.singular and remove_mean:
        v = volumes(G)
        c = float(v @ f / v.sum())
        f -= c
    return f, c


def solve(G, A, f):
    """L phi = f by a sparse direct solve; a singular problem (no Dirichlet face)
    is bordered with the volume-weighted mean: [L 1; V^T 0] [phi; l] = [f; 0]"""
    if not G.singular:
        return spla.spsolve(A.tocsc(), f)
    v = volumes(G)
    n = G.nunk
    B = sp.bmat([[A, sp.csr_matrix(np.ones((n, 1)))], [sp.csr_matrix(v.reshape(1, n)), None]]).tocsc()
    x = spla.spsolve(B, np.concatenate([f, [0.0]]))
    return x[:n]


def correct(G, uc, uf, rho_c, rho_f, x):
    """U <- U - (dphi/dn)/rho_f on both levels (x: unknown-ordered phi); the
    coarse faces on and inside the patches then take the mean of their four
    fine faces.  Returns new (uc, uf): uf as three arrays (one patch) or one
    such list per patch."""
    single = G.npatch == 1 and len(uf) == 3 and not isinstance(uf[0], (list, tuple))
    uc = [np.array(a, dtype=np.float64, copy=True) for a in uc]
    uf = [[np.array(a, dtype=np.float64, copy=True) for a in u3] for u3 in _fine_faces(G, uf)]
    rho_f = _fine_list(G, rho_f)
    H, h = G.H, G.h
    pc, pfs = unpack(G, x)
    if G.npatch == 1:
        pfs = [pfs]
    # coarse faces off the patches: single-level rules
    for d in range(3):
        shp = uc[d].shape  # (z, y, x)
        for k in range(shp[0]):
            for j in range(shp[1]):
                for i in range(shp[2]):
                    face = [i, j, k]
                    p = face[d]
                    lo_c = list(face)
                    lo_c[d] = p - 1
                    hi_c = list(face)
                    if p == 0 or p == G.n[d]:
                        if G.lo[d] == PERIODIC:
                            lo_c[d] %= G.n[d]
                            hi_c[d] %= G.n[d]
                        else:
                            bc = G.lo[d] if p == 0 else G.hi[d]
                            inner = tuple(hi_c) if p == 0 else tuple(lo_c)
                            if bc == DIRICHLET:
                                g = (_at(pc, inner) - 0.0) / (0.5 * H) if p == 0 else (0.0 - _at(pc, inner)) / (0.5 * H)
                                uc[d][k, j, i] -= g / _at(rho_c, inner)
                            else:
                                uc[d][k, j, i] = 0.0
                            continue
                    L, R = tuple(lo_c), tuple(hi_c)
                    if G.in_patch(L) or G.in_patch(R):
                        continue  # set from the fine faces below
                    g = (_at(pc, R) - _at(pc, L)) / H
                    uc[d][k, j, i] -= g / (0.5 * (_at(rho_c, L) + _at(rho_c, R)))
    for q in range(G.npatch):
        pf, nf = pfs[q], G.nfs[q]
        # fine faces
        for d in range(3):
            shp = uf[q][d].shape
            for K in range(shp[0]):
                for J in range(shp[1]):
                    for I in range(shp[2]):
                        face = [I, J, K]
                        p = face[d]
                        L = list(face)
                        L[d] = p - 1
                        R = list(face)
                        L, R = tuple(L), tuple(R)
                        if 0 < p < nf[d]:
                            g = (_at(pf, R) - _at(pf, L)) / h
                            rf = 0.5 * (_at(rho_f[q], L) + _at(rho_f[q], R))
                        else:
                            F = R if p == 0 else L
                            s = -1 if p == 0 else 1
                            C, terms = ghost_terms(G, F, d, s, q)
                            pg = sum(w * x[col] for col, w in terms)
                            g = (_at(pf, F) - pg) / h if p == 0 else (pg - _at(pf, F)) / h
                            rf = 0.5 * (_at(rho_f[q], F) + _at(rho_c, C))
                        uf[q][d][K, J, I] -= g / rf
        # coarse faces on and inside the patch: mean of the four fine faces
        plo, phi = G.boxes[q]
        for d in range(3):
            t1, t2 = [t for t in range(3) if t != d]
            for p in range(plo[d], phi[d] + 1):
                for a in range(plo[t1], phi[t1]):
                    for b in range(plo[t2], phi[t2]):
                        face = [0, 0, 0]
                        face[d], face[t1], face[t2] = p, a, b
                        m = 0.0
                        for e1 in range(2):
                            for e2 in range(2):
                                ff = [0, 0, 0]
                                ff[d] = 2 * (p - plo[d])
                                ff[t1] = 2 * (a - plo[t1]) + e1
                                ff[t2] = 2 * (b - plo[t2]) + e2
                                m += 0.25 * uf[q][d][ff[2], ff[1], ff[0]]
                        uc[d][face[2], face[1], face[0]] = m
    return uc, (uf[0] if single else uf)


def project(G, uc, uf, rho_c, beta0_c, sbar_c, rho_f, beta0_f, sbar_f, remove_mean=True):
    """The composite MAC projection: (uc_new, uf_new, phi_c, phi_f, info)"""
    A = operator_matrix(G, rho_c, beta0_c, rho_f, beta0_f)
    f, c = rhs(G, uc, uf, beta0_c, beta0_f, sbar_c, sbar_f, remove_mean)
    x = solve(G, A, f)
    r = f - A @ x
    uc2, uf2 = correct(G, uc, uf, rho_c, rho_f, x)
    pc, pf = unpack(G, x)
    fn = np.abs(f).max()
    info = {"mean": c, "rel_resid": float(np.abs(r).max() / fn) if fn > 0 else 0.0, "resid": r, "f": f, "x": x}
    return uc2, uf2, pc, pf, info
