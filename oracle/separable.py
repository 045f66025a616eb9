"""Exact direct solve of the MAC system for horizontally uniform coefficients.

TEST INFRASTRUCTURE (part of the oracle).  When rho and beta0 depend on z only
(the planar workloads without their density noise) the face coefficient on x-
and y-faces is a per-layer constant B_k and the operator separates: a discrete
Fourier transform in x and y (periodic) diagonalises the horizontal part with
eigenvalues -4/h^2 sin^2(pi p/n), and each horizontal mode leaves a tridiagonal
system in z, solved by the Thomas algorithm.  This is an independent, exact
(up to rounding) solution of the same discrete system that the multigrid
solvers approximate; it uses no multigrid, no Gauss-Seidel and no code shared
with the C oracle.  Discretisation as in the oracle's header (Appendix A;
Eq. div1).
"""
from __future__ import annotations

import numpy as np

PERIODIC, NEUMANN, DIRICHLET = 0, 1, 2


def solve_layered(n, h, bcz, rho_z, beta_z, f):
    """Solve L phi = f for rho(z), beta0(z) on an (nx, ny, nz) grid, periodic in x, y.

    bcz: NEUMANN (walls) or DIRICHLET (phi = 0) at both z ends.
    f: numpy array of shape (nz, ny, nx).  For walls, f must have zero mean; the
    returned phi then has zero mean.
    """
    nx, ny, nz = n
    rho_z = np.asarray(rho_z, dtype=np.float64)
    beta_z = np.asarray(beta_z, dtype=np.float64)
    # horizontal faces join two cells of one layer: beta_f/rho_f = beta_k/rho_k
    B = (0.5 * (beta_z + beta_z)) / (0.5 * (rho_z + rho_z))
    # vertical faces k+1/2, k = 0..nz-2
    C = (0.5 * (beta_z[:-1] + beta_z[1:])) / (0.5 * (rho_z[:-1] + rho_z[1:]))
    ih2 = 1.0 / (h * h)
    lam_x = -4.0 * ih2 * np.sin(np.pi * np.arange(nx) / nx) ** 2
    lam_y = -4.0 * ih2 * np.sin(np.pi * np.arange(ny) / ny) ** 2
    lam = lam_y[:, None] + lam_x[None, :]                     # (ny, nx)
    fh = np.fft.fft2(f, axes=(1, 2))                           # (nz, ny, nx)
    # tridiagonal rows: sub[k] phi_{k-1} + diag[k] phi_k + sup[k] phi_{k+1} = fh_k
    sub = np.zeros(nz)
    sup = np.zeros(nz)
    sub[1:] = C * ih2
    sup[:-1] = C * ih2
    dvert = -(sub + sup)
    if bcz == DIRICHLET:
        # phi = 0 beyond the wall: one-sided flux with the interior cell's coefficient
        dvert[0] -= 2.0 * (beta_z[0] / rho_z[0]) * ih2
        dvert[-1] -= 2.0 * (beta_z[-1] / rho_z[-1]) * ih2
    diag = dvert[:, None, None] + B[:, None, None] * lam[None, :, :]
    rhs = fh.copy()
    singular = bcz != DIRICHLET
    if singular:
        # the (0,0) horizontal mode is singular: pin phi_0 = 0 in that mode
        diag = diag.copy()
        diag[0, 0, 0] = 1.0
        rhs[0, 0, 0] = 0.0
    # Thomas algorithm, vectorised over horizontal modes
    cp = np.zeros((nz, ny, nx), dtype=np.complex128)
    dp = np.zeros((nz, ny, nx), dtype=np.complex128)
    supm = np.broadcast_to(sup[:, None, None], (nz, ny, nx)).copy()
    subm = np.broadcast_to(sub[:, None, None], (nz, ny, nx)).copy()
    if singular:
        supm[0, 0, 0] = 0.0
    cp[0] = supm[0] / diag[0]
    dp[0] = rhs[0] / diag[0]
    for k in range(1, nz):
        den = diag[k] - subm[k] * cp[k - 1]
        cp[k] = supm[k] / den
        dp[k] = (rhs[k] - subm[k] * dp[k - 1]) / den
    ph = np.zeros_like(dp)
    ph[-1] = dp[-1]
    for k in range(nz - 2, -1, -1):
        ph[k] = dp[k] - cp[k] * ph[k + 1]
    phi = np.fft.ifft2(ph, axes=(1, 2)).real
    if singular:
        phi -= phi.mean()
    return phi
