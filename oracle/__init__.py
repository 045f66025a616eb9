"""FP64 CPU oracle for the MAC and nodal projections (plain C, loaded with ctypes).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs may import this package.  The CUDA
library never calls it and shares no code, header or table with it.

Arrays are float64 numpy arrays in x-fastest order (numpy shape (nz, ny, nx));
MAC face arrays carry n_d + 1 entries along their own direction, nodal arrays
have n nodes on a periodic axis and n + 1 on a wall axis.

``composite.py`` (numpy / scipy.sparse) holds the two-level composite MAC
operator and projection (refinement ratio 2, any number of fine patches) with a
sparse direct solve; ``composite_ml.py`` the composite operator on any number
of levels, written separately and equal to it on two.

Functions without a pin in the CPU tests: none.  Readings of the paper are
listed in the C sources' headers and in ``composite.py``'s.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["oracle.c", "oracle_nodal.c", "oracle_base.c"]

PERIODIC, NEUMANN, DIRICHLET = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (portable C, -O2, no FMA
    contraction, so that x86 and Arm builds round every operation alike)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double), ("lo", C.c_int * 3), ("hi", C.c_int * 3)]


_lib = None
_P = C.POINTER(C.c_double)


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        G = C.POINTER(_Geom)
        sig = {
            "or_fill_planar": (C.c_int, [G, _P, C.c_int, _P]),
            "or_fill_spherical": (C.c_int, [G, _P, C.c_int, C.c_double, _P, _P]),
            "or_mac_coeffs": (None, [G, _P, _P, _P, _P, _P]),
            "or_mac_apply": (None, [G, _P, _P, _P, _P, _P]),
            "or_mac_divergence": (None, [G, _P, _P, _P, _P, _P]),
            "or_mac_rhs": (None, [G, _P, _P, _P, _P, _P, C.c_int, _P, _P]),
            "or_mac_correct": (None, [G, _P, _P, _P, _P, _P]),
            "or_mac_solve": (C.c_int, [G, _P, _P, _P, _P, _P, C.c_double, C.c_int, _P]),
            "or_mac_dense_solve": (C.c_int, [G, _P, _P, _P, _P, _P]),
            "or_mac_project": (C.c_int, [G, _P, _P, _P, _P, _P, _P, _P, C.c_double, C.c_int, C.c_int, _P]),
            "or_mac_residual_sample": (None, [G, _P, _P, _P, _P, C.POINTER(C.c_long), C.c_long, _P]),
            "or_mac_divergence_sample": (None, [G, _P, _P, _P, _P, C.POINTER(C.c_long), C.c_long, _P]),
            "or_nd_residual_sample": (None, [G, _P, _P, _P, C.POINTER(C.c_long), C.c_long, _P]),
            "or_nd_nnode": (C.c_long, [G]),
            "or_nd_weights": (None, [G, _P]),
            "or_nd_apply": (None, [G, _P, _P, _P]),
            "or_nd_divergence": (None, [G, _P, _P, _P, _P]),
            "or_nd_gradient": (None, [G, _P, _P, _P, _P]),
            "or_nd_rhs": (None, [G, _P, _P, _P, _P, _P, C.c_int, _P, _P]),
            "or_nd_correct": (None, [G, _P, _P, _P, _P, _P]),
            "or_nd_solve": (C.c_int, [G, _P, _P, _P, C.c_double, C.c_int, _P]),
            "or_nd_dense_solve": (C.c_int, [G, _P, _P, _P]),
            "or_nd_project": (C.c_int, [G, _P, _P, _P, _P, _P, _P, _P, C.c_double, C.c_int, _P]),
            "or_average_planar": (None, [G, _P, _P]),
            "or_radial_nbins": (C.c_long, [G, _IP]),
            "or_radial_index": (None, [G, _IP, _LP]),
            "or_average_radial": (None, [G, _IP, _P, C.c_long, _P, _LP]),
            "or_fill_irregular": (None, [G, _IP, _P, _P]),
            "or_fill_quadratic": (C.c_int, [G, _P, C.c_int, C.c_double, _P, _P]),
            "or_average_to_uniform": (C.c_int, [C.c_long, _P, _LP, C.c_double, C.c_int, C.c_double, _P]),
            "or_w0_integrate": (C.c_int, [C.c_int, C.c_int, _P, _P, _P, C.c_int, _P]),
            "or_add_w0_faces": (None, [G, C.c_int, _IP, C.c_int, _P, _P, _P, _P, _P]),
            "or_subtract_lateral_average": (None, [G, C.c_int, _IP, _P, _P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _g(geom):
    g = _Geom()
    for d in range(3):
        g.n[d] = int(geom.n[d])
        g.lo[d] = int(geom.lo[d])
        g.hi[d] = int(geom.hi[d])
    g.h = float(geom.dx)
    return C.byref(g)


def _arr(a):
    """float64, C-contiguous numpy copy/view of a numpy array or CPU torch tensor."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_P)


_IP = C.POINTER(C.c_int)
_LP = C.POINTER(C.c_long)


def _corner(c):
    return (C.c_int * 3)(*[int(x) for x in c])


# ---- base-state mapping (Sec. 3.1: lateral average and fill) ---------------------------

def average_planar(geom, field):
    """Mean of the cells at each height: (nz,)."""
    out = np.empty(geom.n[2])
    _load().or_average_planar(_g(geom), _p(_arr(field)), _p(out))
    return out


def radial_nbins(geom, corner):
    return int(_load().or_radial_nbins(_g(geom), _corner(corner)))


def radial_index(geom, corner):
    """m of every cell (radius dx sqrt(0.75 + 2m)), shape (nz, ny, nx), int64."""
    out = np.empty(cell_shape(geom), dtype=np.int64)
    _load().or_radial_index(_g(geom), _corner(corner), out.ctypes.data_as(_LP))
    return out


def average_radial(geom, corner, field, nbins=None):
    """(mean per radius m, cell count per m) of the irregular base state."""
    nb = radial_nbins(geom, corner) if nbins is None else int(nbins)
    out = np.empty(nb)
    cnt = np.empty(nb, dtype=np.int64)
    _load().or_average_radial(_g(geom), _corner(corner), _p(_arr(field)), nb, _p(out), cnt.ctypes.data_as(_LP))
    return out, cnt


def fill_irregular(geom, corner, base):
    out = np.empty(cell_shape(geom))
    _load().or_fill_irregular(_g(geom), _corner(corner), _p(_arr(base)), _p(out))
    return out


def fill_quadratic(geom, prof, dr, center):
    prof = _arr(prof)
    out = np.empty(cell_shape(geom))
    c = np.ascontiguousarray(center, dtype=np.float64)
    rc = _load().or_fill_quadratic(_g(geom), _p(prof), prof.size, float(dr), _p(c), _p(out))
    if rc:
        raise ValueError("fill_quadratic needs at least 3 radial cells")
    return out


def w0_integrate(spherical, r_edge, beta0, src, cutoff=-1):
    """w0 on the nr + 1 base-state edges (Appendix A velocity split)."""
    r_edge, beta0, src = _arr(r_edge), _arr(beta0), _arr(src)
    nr = beta0.size
    assert r_edge.size == nr + 1 and src.size == nr
    out = np.empty(nr + 1)
    if _load().or_w0_integrate(int(spherical), nr, _p(r_edge), _p(beta0), _p(src), int(cutoff), _p(out)):
        raise ValueError("w0_integrate needs nr >= 1")
    return out


def add_w0_faces(geom, spherical, corner, r_edge, w0, u):
    """returns copies of the three face arrays with w0 e_r added"""
    r_edge, w0 = _arr(r_edge), _arr(w0)
    out = [np.array(x, dtype=np.float64, copy=True, order="C") for x in u]
    c = _corner(corner if corner is not None else (0, 0, 0))
    _load().or_add_w0_faces(_g(geom), int(spherical), c, w0.size - 1, _p(r_edge), _p(w0), _p(out[0]), _p(out[1]),
                            _p(out[2]))
    return out


def subtract_lateral_average(geom, spherical, corner, S):
    out = np.empty(cell_shape(geom))
    c = _corner(corner if corner is not None else (0, 0, 0))
    _load().or_subtract_lateral_average(_g(geom), int(spherical), c, _p(_arr(S)), _p(out))
    return out


def average_to_uniform(avg, count, dx, nr, dr):
    avg = _arr(avg)
    cnt = np.ascontiguousarray(count, dtype=np.int64)
    out = np.empty(int(nr))
    rc = _load().or_average_to_uniform(avg.size, _p(avg), cnt.ctypes.data_as(_LP), float(dx), int(nr), float(dr),
                                       _p(out))
    if rc:
        raise ValueError("average_to_uniform needs at least 3 non-empty radii")
    return out


def face_shape(geom, d):
    nx, ny, nz = geom.n
    return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][d]


def cell_shape(geom):
    return (geom.n[2], geom.n[1], geom.n[0])


def node_shape(geom):
    m = [geom.n[d] + (0 if geom.lo[d] == PERIODIC else 1) for d in range(3)]
    return (m[2], m[1], m[0])


def singular(geom):
    return all(geom.lo[d] != DIRICHLET and geom.hi[d] != DIRICHLET for d in range(3))


# --- Fill -------------------------------------------------------------------------

def fill(geom, prof, spherical=False, dr=None, center=(0.5, 0.5, 0.5)):
    lib = _load()
    prof = _arr(prof)
    out = np.empty(cell_shape(geom))
    if spherical:
        c = np.ascontiguousarray(center, dtype=np.float64)
        rc = lib.or_fill_spherical(_g(geom), _p(prof), prof.size, float(dr), _p(c), _p(out))
    else:
        rc = lib.or_fill_planar(_g(geom), _p(prof), prof.size, _p(out))
    if rc:
        raise ValueError("oracle fill: profile too short")
    return out


# --- MAC ----------------------------------------------------------------------------

def mac_coeffs(geom, rho, beta0):
    lib = _load()
    b = [np.empty(face_shape(geom, d)) for d in range(3)]
    lib.or_mac_coeffs(_g(geom), _p(_arr(rho)), _p(_arr(beta0)), _p(b[0]), _p(b[1]), _p(b[2]))
    return b


def mac_apply(geom, b, phi):
    lib = _load()
    b = [_arr(x) for x in b]
    out = np.empty(cell_shape(geom))
    lib.or_mac_apply(_g(geom), _p(b[0]), _p(b[1]), _p(b[2]), _p(_arr(phi)), _p(out))
    return out


def mac_divergence(geom, u, beta0):
    lib = _load()
    u = [_arr(x) for x in u]
    out = np.empty(cell_shape(geom))
    lib.or_mac_divergence(_g(geom), _p(u[0]), _p(u[1]), _p(u[2]), _p(_arr(beta0)), _p(out))
    return out


def mac_rhs(geom, u, beta0, sbar, remove_mean=True):
    lib = _load()
    u = [_arr(x) for x in u]
    f = np.empty(cell_shape(geom))
    m = C.c_double(0.0)
    lib.or_mac_rhs(_g(geom), _p(u[0]), _p(u[1]), _p(u[2]), _p(_arr(beta0)), _p(_arr(sbar)),
                   int(bool(remove_mean)), _p(f), C.byref(m))
    return f, m.value


def mac_correct(geom, rho, phi, u):
    lib = _load()
    u = [_arr(x).copy() for x in u]
    lib.or_mac_correct(_g(geom), _p(_arr(rho)), _p(_arr(phi)), _p(u[0]), _p(u[1]), _p(u[2]))
    return u


def mac_solve(geom, b, f, phi0=None, tol=1e-13, maxit=200):
    """MG-preconditioned CG; returns (phi, iterations, relative residual)."""
    lib = _load()
    b = [_arr(x) for x in b]
    phi = np.zeros(cell_shape(geom)) if phi0 is None else _arr(phi0).copy()
    rr = C.c_double(0.0)
    it = lib.or_mac_solve(_g(geom), _p(b[0]), _p(b[1]), _p(b[2]), _p(_arr(f)), _p(phi),
                          float(tol), int(maxit), C.byref(rr))
    if it == -2:
        raise RuntimeError("oracle mac_solve: coarse factorisation failed")
    return phi, it, rr.value


def mac_dense_solve(geom, b, f):
    lib = _load()
    b = [_arr(x) for x in b]
    phi = np.zeros(cell_shape(geom))
    rc = lib.or_mac_dense_solve(_g(geom), _p(b[0]), _p(b[1]), _p(b[2]), _p(_arr(f)), _p(phi))
    if rc:
        raise RuntimeError(f"oracle dense solve failed ({rc})")
    return phi


def mac_project(geom, u, rho, beta0, sbar, tol=1e-13, maxit=200, remove_mean=True, phi0=None):
    """Full MAC projection.  Returns (u_new, phi, info dict)."""
    lib = _load()
    u = [_arr(x).copy() for x in u]
    phi = np.zeros(cell_shape(geom)) if phi0 is None else _arr(phi0).copy()
    out = np.zeros(4)
    rc = lib.or_mac_project(_g(geom), _p(u[0]), _p(u[1]), _p(u[2]), _p(_arr(rho)), _p(_arr(beta0)),
                            _p(_arr(sbar)), _p(phi), float(tol), int(maxit), int(bool(remove_mean)), _p(out))
    info = dict(mean=out[0], rel_resid=out[1], div_err=out[2], iters=int(out[3]), ok=(rc == 0))
    return u, phi, info


def _idx(idx):
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    return idx, idx.ctypes.data_as(C.POINTER(C.c_long))


def mac_residual_sample(geom, rho, beta0, phi, f, idx):
    """f - L phi at the flat cell indices idx, one cell at a time from rho, beta0."""
    lib = _load()
    idx, ip = _idx(idx)
    out = np.empty(idx.size)
    lib.or_mac_residual_sample(_g(geom), _p(_arr(rho)), _p(_arr(beta0)), _p(_arr(phi)), _p(_arr(f)), ip, idx.size,
                               _p(out))
    return out


def mac_divergence_sample(geom, u, beta0, idx):
    lib = _load()
    u = [_arr(x) for x in u]
    idx, ip = _idx(idx)
    out = np.empty(idx.size)
    lib.or_mac_divergence_sample(_g(geom), _p(u[0]), _p(u[1]), _p(u[2]), _p(_arr(beta0)), ip, idx.size, _p(out))
    return out


def nd_residual_sample(geom, sigma, phi, f, idx):
    lib = _load()
    idx, ip = _idx(idx)
    out = np.empty(idx.size)
    lib.or_nd_residual_sample(_g(geom), _p(_arr(sigma)), _p(_arr(phi)), _p(_arr(f)), ip, idx.size, _p(out))
    return out


# --- nodal -------------------------------------------------------------------------

def nd_weights(geom):
    lib = _load()
    w = np.empty(node_shape(geom))
    lib.or_nd_weights(_g(geom), _p(w))
    return w


def nd_apply(geom, sigma, phi):
    lib = _load()
    out = np.empty(node_shape(geom))
    lib.or_nd_apply(_g(geom), _p(_arr(sigma)), _p(_arr(phi)), _p(out))
    return out


def nd_divergence(geom, v):
    lib = _load()
    v = [_arr(x) for x in v]
    out = np.empty(node_shape(geom))
    lib.or_nd_divergence(_g(geom), _p(v[0]), _p(v[1]), _p(v[2]), _p(out))
    return out


def nd_gradient(geom, phi):
    lib = _load()
    G = [np.empty(cell_shape(geom)) for _ in range(3)]
    lib.or_nd_gradient(_g(geom), _p(_arr(phi)), _p(G[0]), _p(G[1]), _p(G[2]))
    return G


def nd_rhs(geom, u, beta0, sbar, remove_mean=True):
    lib = _load()
    u = [_arr(x) for x in u]
    f = np.empty(node_shape(geom))
    m = C.c_double(0.0)
    lib.or_nd_rhs(_g(geom), _p(u[0]), _p(u[1]), _p(u[2]), _p(_arr(beta0)), _p(_arr(sbar)),
                  int(bool(remove_mean)), _p(f), C.byref(m))
    return f, m.value


def nd_correct(geom, rho, phi, u):
    lib = _load()
    u = [_arr(x).copy() for x in u]
    lib.or_nd_correct(_g(geom), _p(_arr(rho)), _p(_arr(phi)), _p(u[0]), _p(u[1]), _p(u[2]))
    return u


def nd_solve(geom, sigma, f, phi0=None, tol=1e-13, maxit=300):
    lib = _load()
    phi = np.zeros(node_shape(geom)) if phi0 is None else _arr(phi0).copy()
    rr = C.c_double(0.0)
    it = lib.or_nd_solve(_g(geom), _p(_arr(sigma)), _p(_arr(f)), _p(phi), float(tol), int(maxit), C.byref(rr))
    if it == -2:
        raise RuntimeError("oracle nd_solve: coarse factorisation failed")
    return phi, it, rr.value


def nd_dense_solve(geom, sigma, f):
    lib = _load()
    phi = np.zeros(node_shape(geom))
    rc = lib.or_nd_dense_solve(_g(geom), _p(_arr(sigma)), _p(_arr(f)), _p(phi))
    if rc:
        raise RuntimeError(f"oracle nodal dense solve failed ({rc})")
    return phi


def nd_project(geom, u, rho, beta0, sbar, tol=1e-13, maxit=300, phi0=None):
    lib = _load()
    u = [_arr(x).copy() for x in u]
    phi = np.zeros(node_shape(geom)) if phi0 is None else _arr(phi0).copy()
    out = np.zeros(4)
    rc = lib.or_nd_project(_g(geom), _p(u[0]), _p(u[1]), _p(u[2]), _p(_arr(rho)), _p(_arr(beta0)),
                           _p(_arr(sbar)), _p(phi), float(tol), int(maxit), _p(out))
    info = dict(mean=out[0], rel_resid=out[1], div_err=out[2], iters=int(out[3]), ok=(rc == 0))
    return u, phi, info
