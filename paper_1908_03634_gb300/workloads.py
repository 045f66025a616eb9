"""Seeded synthetic inputs for the MAC and nodal projection workloads.

This module only draws random numbers and evaluates closed-form input fields
(stratified density, the base-state profile, Fourier-mode velocities and
Gaussian heating hotspots).  It holds none of the projection's arithmetic: the
base-state Fill, the face coefficients, the divergence, the solve and the
correction live in the CUDA library and, independently, in the CPU oracle.
Both sides read the arrays produced here.

The workloads stand in for the paper's white-dwarf runs (Sec. 4.1 full-star
convection, Sec. 4.3 planar hot bubble), whose initial models and
microphysics are not available; the recipe is:

* planar: rho0(z) = exp(-z/H), beta0 = rho0**p, sampled at cell-centre heights
  (the planar base state is aligned with the Cartesian cells, Sec. 3.1);
* spherical: rho0(r) = (1 + (r/0.05)**2)**-2.5 for r <= 0.45, 1e-6 beyond
  (a density floor held outside a radius, the paper's cutoff-density idea),
  beta0 = rho0**0.6, tabulated at radial cell centres (j+1/2)*dr;
* cell density rho = rho0(x_cell) * (1 + 0.01*xi), xi ~ U[-1, 1];
* U^ADV,dagger = sum_m e_m sin(2 pi k_m.x + theta_m), k_m in {-4..4}^3 \\ {0},
  theta_m ~ U[0, 2pi), e_m a random unit vector, evaluated on face centres
  (MAC) or cell centres (nodal);
* Sbar = sum_c exp(-|x - x_c|^2 / w^2), w = 0.05.

All fields are float64 torch tensors in x-fastest order (index i + nx*(j + ny*k),
i.e. torch shape (nz, ny, nx)); face arrays have n_d + 1 entries along their
own direction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

PERIODIC, NEUMANN, DIRICHLET = 0, 1, 2


@dataclass
class Geom:
    """Cell counts, cell width and boundary type per face (lo/hi per axis)."""

    n: tuple
    dx: float
    lo: tuple = (PERIODIC, PERIODIC, NEUMANN)
    hi: tuple = (PERIODIC, PERIODIC, NEUMANN)

    @property
    def ncell(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def face_shape(self, d: int):
        """torch shape (z, y, x) of the d-face array."""
        nx, ny, nz = self.n
        return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][d]

    def node_shape(self):
        """torch shape of the nodal array: n nodes on a periodic axis, n+1 otherwise."""
        m = [self.n[d] + (0 if self.lo[d] == PERIODIC else 1) for d in range(3)]
        return (m[2], m[1], m[0])


@dataclass
class Workload:
    """One projection problem: geometry, base-state profile and cell/face fields."""

    name: str
    geom: Geom
    spherical: bool
    prof_beta0: torch.Tensor      # 1D base-state beta0 at radial cell centres
    prof_dr: float
    center: tuple
    rho: torch.Tensor             # cells
    sbar: torch.Tensor            # cells (the full constraint bracket)
    u: list                       # MAC: 3 face arrays; nodal: 3 cell arrays
    meta: dict = field(default_factory=dict)


def _streams(seed):
    ss = np.random.SeedSequence(seed)
    noise, modes, spots = ss.spawn(3)
    return (np.random.default_rng(noise), np.random.default_rng(modes),
            np.random.default_rng(spots))


def draw_modes(rng, m):
    """m Fourier modes: integer wavevectors in {-4..4}^3 minus 0, phases, unit polarisations."""
    ks, th, es = [], [], []
    while len(ks) < m:
        k = rng.integers(-4, 5, size=3)
        if not k.any():
            continue
        ks.append(k)
        th.append(rng.uniform(0.0, 2.0 * math.pi))
        g = rng.standard_normal(3)
        es.append(g / np.linalg.norm(g))
    return np.array(ks), np.array(th), np.array(es)


def _axis_points(n, h, staggered, device):
    i = torch.arange(n + (1 if staggered else 0), dtype=torch.float64, device=device)
    return i * h if staggered else (i + 0.5) * h


def _points(geom: Geom, d, device):
    """1D coordinates along x, y, z of the d-face centres (d=None: cell centres)."""
    return [_axis_points(geom.n[a], geom.dx, d == a, device) for a in range(3)]


def eval_modes(modes, comp, pts):
    """sum_m e_m[comp] sin(2 pi k_m.x + theta_m) on the tensor grid pts=(x, y, z)."""
    ks, th, es = modes
    x, y, z = pts
    out = torch.zeros((z.numel(), y.numel(), x.numel()), dtype=torch.float64, device=x.device)
    for k, t, e in zip(ks, th, es):
        if e[comp] == 0.0:
            continue
        ex = torch.exp(1j * (2 * math.pi * float(k[0])) * x.to(torch.complex128))
        ey = torch.exp(1j * (2 * math.pi * float(k[1])) * y.to(torch.complex128))
        ez = torch.exp(1j * (2 * math.pi * float(k[2])) * z.to(torch.complex128) + 1j * float(t))
        out += float(e[comp]) * (ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).imag
    return out


def eval_hotspots(centres, w, pts):
    x, y, z = pts
    out = torch.zeros((z.numel(), y.numel(), x.numel()), dtype=torch.float64, device=x.device)
    for c in centres:
        gx = torch.exp(-((x - c[0]) ** 2) / w ** 2)
        gy = torch.exp(-((y - c[1]) ** 2) / w ** 2)
        gz = torch.exp(-((z - c[2]) ** 2) / w ** 2)
        out += gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return out


def _periodic_faces(geom: Geom, u):
    """On periodic axes face n is the image of face 0: store the same value in both."""
    for d in range(3):
        if geom.lo[d] == PERIODIC:
            a = u[d]
            if d == 0:
                a[:, :, -1] = a[:, :, 0]
            elif d == 1:
                a[:, -1, :] = a[:, 0, :]
            else:
                a[-1, :, :] = a[0, :, :]
    return u


def _noise(rng, geom: Geom, device):
    xi = rng.uniform(-1.0, 1.0, size=geom.ncell)
    return torch.from_numpy(xi).reshape(geom.n[2], geom.n[1], geom.n[0]).to(device)


def planar(n, H, beta_exp, nmodes, spots, seed, device="cpu", name="planar",
           bc_z=NEUMANN):
    """Planar stratified box, periodic in x and y, walls in z.

    spots: "center" for one hotspot at (0.5, 0.5, 0.5), or an int count of
    hotspots with centres drawn from U[0.2, 0.8]^3.
    """
    if isinstance(n, int):
        n = (n, n, n)
    g = Geom(tuple(n), 1.0 / n[0], (PERIODIC, PERIODIC, bc_z), (PERIODIC, PERIODIC, bc_z))
    r_noise, r_modes, r_spots = _streams(seed)
    h = g.dx
    zc = (torch.arange(n[2], dtype=torch.float64, device=device) + 0.5) * h
    rho0 = torch.exp(-zc / H)
    prof_beta0 = rho0 ** beta_exp if beta_exp != 1.0 else rho0.clone()
    rho = rho0[:, None, None] * (1.0 + 0.01 * _noise(r_noise, g, device))
    modes = draw_modes(r_modes, nmodes)
    u = _periodic_faces(g, [eval_modes(modes, d, _points(g, d, device)) for d in range(3)])
    centres = [(0.5, 0.5, 0.5)] if spots == "center" else list(r_spots.uniform(0.2, 0.8, size=(spots, 3)))
    sbar = eval_hotspots(centres, 0.05, _points(g, None, device))
    return Workload(name, g, False, prof_beta0, h, (0.5, 0.5, 0.5), rho.contiguous(), sbar, u,
                    dict(H=H, beta_exp=beta_exp, modes=nmodes, seed=seed, centres=centres))


def star_rho0(r, r_core=0.05, r_floor=0.45, floor=1e-6):
    """Radial density of the full-star workload: a softened polytrope-like core,
    held at the floor value outside r_floor."""
    prof = (1.0 + (r / r_core) ** 2) ** -2.5
    return torch.where(r <= r_floor, prof, torch.full_like(prof, floor))


def star(n, nmodes, seed, device="cpu", name="star", nr=4096):
    """Full-star cube with homogeneous Dirichlet phi = 0 on all faces."""
    if isinstance(n, int):
        n = (n, n, n)
    D = DIRICHLET
    g = Geom(tuple(n), 1.0 / n[0], (D, D, D), (D, D, D))
    r_noise, r_modes, r_spots = _streams(seed)
    dr = g.dx / 4.0
    rj = (torch.arange(nr, dtype=torch.float64, device=device) + 0.5) * dr
    prof_beta0 = star_rho0(rj) ** 0.6
    x, y, z = _points(g, None, device)
    rc = torch.sqrt((z[:, None, None] - 0.5) ** 2 + (y[None, :, None] - 0.5) ** 2
                    + (x[None, None, :] - 0.5) ** 2)
    rho = star_rho0(rc) * (1.0 + 0.01 * _noise(r_noise, g, device))
    modes = draw_modes(r_modes, nmodes)
    u = [eval_modes(modes, d, _points(g, d, device)) for d in range(3)]
    sbar = eval_hotspots([(0.5, 0.5, 0.5)], 0.05, (x, y, z))
    return Workload(name, g, True, prof_beta0, dr, (0.5, 0.5, 0.5), rho.contiguous(), sbar, u,
                    dict(modes=nmodes, seed=seed, nr=nr))


def planar_nodal(n, H, beta_exp, nmodes, spots, seed, device="cpu", name="nodal"):
    """Planar box for the nodal projection: cell-centred velocity components."""
    w = planar(n, H, beta_exp, 0, spots, seed, device=device, name=name)
    _, r_modes, _ = _streams(seed)
    modes = draw_modes(r_modes, nmodes)
    pts = _points(w.geom, None, device)
    w.u = [eval_modes(modes, d, pts) for d in range(3)]
    w.meta["modes"] = nmodes
    return w


# --- the named workloads -------------------------------------------------------

H_1E5 = 1.0 / math.log(1e5)   # top/bottom density contrast 1e5 over the unit height


def planar32(device="cpu"):
    """32^3 planar box, rho0 = exp(-z/0.1), beta0 = rho0, 8 modes, central hotspot, seed 0."""
    return planar(32, 0.1, 1.0, 8, "center", 0, device, "planar32")


def planar256(device="cpu", n=256):
    """256^3 planar box, contrast 1e5, beta0 = rho0^(3/5), 16 modes, 3 hotspots, seed 1."""
    return planar(n, H_1E5, 0.6, 16, 3, 1, device, f"planar{n}")


def star512(device="cpu", n=512):
    """512^3 full star, Dirichlet walls, 32 modes, central hotspot, seed 2."""
    return star(n, 32, 2, device, f"star{n}")


def nodal384(device="cpu", n=384):
    """384^3-cell nodal projection with the planar256 stratification, 16 modes, seed 4."""
    return planar_nodal(n, H_1E5, 0.6, 16, 3, 4, device, f"nodal{n}")


PATCH_SIZES = (32, 48, 64, 96, 128)


def _batched_draws(npatch, seed, sizes):
    ss = np.random.SeedSequence(seed)
    top = np.random.default_rng(ss.spawn(1)[0])
    edges = top.choice(np.array(sizes), size=npatch)
    contrast = 10.0 ** top.uniform(2.0, 5.0, size=npatch)
    return edges, contrast


def batched_sizes(npatch=96, seed=3, sizes=PATCH_SIZES):
    """The (nx, ny, nz) cell counts of batched_patches(npatch, seed, sizes),
    without building the fields."""
    edges, _ = _batched_draws(npatch, seed, sizes)
    return [(int(e), int(e), int(e)) for e in edges]


def batched_patches(npatch=96, seed=3, device="cpu", sizes=PATCH_SIZES, nmodes=8, only=None):
    """Independent planar patches: cube edge uniform from sizes, density contrast
    log-uniform in [1e2, 1e5], each patch with its own seed stream.  only: build
    just these patch indices (a rank's shard), in order."""
    edges, contrast = _batched_draws(npatch, seed, sizes)
    out = []
    for p in (range(npatch) if only is None else only):
        H = 1.0 / math.log(contrast[p])
        out.append(planar(int(edges[p]), H, 0.6, nmodes, 1, (seed, p), device, f"patch{p}"))
    return out


# ---- two-level composite (AMR) inputs -------------------------------------------------

@dataclass
class CompositeWorkload:
    """A coarse level and one ratio-2 fine patch over the coarse box [plo, phi):
    the same closed-form fields evaluated at each level's cell and face centres
    (each level with its own density noise).  beta0 is given per cell on both
    levels (closed form at the cell centres)."""

    name: str
    geom: Geom
    plo: tuple
    phi: tuple
    rho_c: torch.Tensor
    beta0_c: torch.Tensor
    sbar_c: torch.Tensor
    u_c: list
    rho_f: torch.Tensor
    beta0_f: torch.Tensor
    sbar_f: torch.Tensor
    u_f: list
    meta: dict = field(default_factory=dict)


def _patch_points(geom: Geom, plo, phi, d, device):
    """1D coordinates of the fine patch's d-face centres (d=None: cell centres)"""
    h = geom.dx / 2.0
    out = []
    for a in range(3):
        m = 2 * (phi[a] - plo[a])
        i = torch.arange(m + (1 if d == a else 0), dtype=torch.float64, device=device)
        out.append(plo[a] * geom.dx + (i * h if d == a else (i + 0.5) * h))
    return out


def composite_planar(n, plo, phi, H, beta_exp, nmodes, spots, seed, device="cpu", name="composite_planar"):
    """The planar box of planar() (periodic x, y; walls in z) with a fine patch
    over the coarse box [plo, phi): rho0(z) = exp(-z/H), beta0 = rho0**p,
    rho = rho0 (1 + 0.01 xi) per level, the same Fourier-mode U and hotspot Sbar
    on both levels.  The patch keeps one coarse cell from the domain faces."""
    if isinstance(n, int):
        n = (n, n, n)
    g = Geom(tuple(n), 1.0 / n[0], (PERIODIC, PERIODIC, NEUMANN), (PERIODIC, PERIODIC, NEUMANN))
    ss = np.random.SeedSequence(seed)
    r_noise_c, r_noise_f, r_modes, r_spots = [np.random.default_rng(s) for s in ss.spawn(4)]
    modes = draw_modes(r_modes, nmodes)
    centres = [(0.5, 0.5, 0.5)] if spots == "center" else list(r_spots.uniform(0.2, 0.8, size=(spots, 3)))

    def level(pts_c, pts_f, rng, shape):
        z = pts_c[2]
        rho0 = torch.exp(-z / H)
        xi = torch.from_numpy(rng.uniform(-1.0, 1.0, size=int(np.prod(shape)))).reshape(shape).to(device)
        rho = (rho0[:, None, None] * (1.0 + 0.01 * xi)).contiguous()
        beta0 = (rho0 ** beta_exp)[:, None, None].expand(shape).contiguous()
        sbar = eval_hotspots(centres, 0.05, pts_c)
        u = [eval_modes(modes, d, pts_f[d]) for d in range(3)]
        return rho, beta0, sbar, u

    cshape = (n[2], n[1], n[0])
    rc, bc, sc, uc = level(_points(g, None, device), [_points(g, d, device) for d in range(3)], r_noise_c, cshape)
    uc = _periodic_faces(g, uc)
    nf = [2 * (phi[a] - plo[a]) for a in range(3)]
    fshape = (nf[2], nf[1], nf[0])
    rf, bf, sf, uf = level(_patch_points(g, plo, phi, None, device),
                           [_patch_points(g, plo, phi, d, device) for d in range(3)], r_noise_f, fshape)
    return CompositeWorkload(name, g, tuple(plo), tuple(phi), rc, bc, sc, uc, rf, bf, sf, uf,
                             dict(H=H, beta_exp=beta_exp, modes=nmodes, seed=seed, centres=centres))


def composite_star(n, plo, phi, nmodes, seed, device="cpu", name="composite_star"):
    """The full star of star() (Dirichlet faces) with a fine patch over the
    coarse box [plo, phi) (the core): rho0(r) as star_rho0, beta0 = rho0**0.6
    at the cell centres of each level, rho = rho0 (1 + 0.01 xi) per level, the
    same Fourier-mode U and central hotspot on both levels."""
    if isinstance(n, int):
        n = (n, n, n)
    Dd = DIRICHLET
    g = Geom(tuple(n), 1.0 / n[0], (Dd, Dd, Dd), (Dd, Dd, Dd))
    ss = np.random.SeedSequence(seed)
    r_noise_c, r_noise_f, r_modes = [np.random.default_rng(s) for s in ss.spawn(3)]
    modes = draw_modes(r_modes, nmodes)

    def level(pts_c, pts_f, rng, shape):
        x, y, z = pts_c
        r = torch.sqrt((z[:, None, None] - 0.5) ** 2 + (y[None, :, None] - 0.5) ** 2 + (x[None, None, :] - 0.5) ** 2)
        rho0 = star_rho0(r)
        xi = torch.from_numpy(rng.uniform(-1.0, 1.0, size=int(np.prod(shape)))).reshape(shape).to(device)
        rho = (rho0 * (1.0 + 0.01 * xi)).contiguous()
        beta0 = (rho0 ** 0.6).contiguous()
        sbar = eval_hotspots([(0.5, 0.5, 0.5)], 0.05, pts_c)
        u = [eval_modes(modes, d, pts_f[d]) for d in range(3)]
        return rho, beta0, sbar, u

    cshape = (n[2], n[1], n[0])
    rc, bc, sc, uc = level(_points(g, None, device), [_points(g, d, device) for d in range(3)], r_noise_c, cshape)
    nf = [2 * (phi[a] - plo[a]) for a in range(3)]
    fshape = (nf[2], nf[1], nf[0])
    rf, bf, sf, uf = level(_patch_points(g, plo, phi, None, device),
                           [_patch_points(g, plo, phi, d, device) for d in range(3)], r_noise_f, fshape)
    return CompositeWorkload(name, g, tuple(plo), tuple(phi), rc, bc, sc, uc, rf, bf, sf, uf,
                             dict(modes=nmodes, seed=seed))
