"""Python binding of libmx (include/mx.h): the GB300 projection solver for the
MAESTROeX low Mach number time step (MAC and nodal projections, Appendix A).

Argument marshalling only: every step of a projection runs in the CUDA
library.  Arrays are torch CUDA float64 tensors (contiguous, x fastest, torch
shape (nz, ny, nx)); the binding passes ``data_ptr()`` and the current torch
stream.  There is no CPU fallback: if libmx.so is missing or fails to load,
every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmx.so")

MX_OK, MX_ERR_ARG, MX_ERR_CUDA, MX_ERR_OOM, MX_ERR_NOCONV, MX_ERR_INCOMPAT, MX_ERR_TIMEOUT = range(7)
MX_BC_PERIODIC, MX_BC_NEUMANN, MX_BC_DIRICHLET = 0, 1, 2
MX_PREC_FP64, MX_PREC_MIXED = 0, 1
MX_OP_MAC, MX_OP_NODAL = 0, 1
PHASES = ["setup", "resid64", "smooth_fine", "restrict_fine", "prolong_fine", "coarse", "update", "finish"]
STATUS_NAMES = {0: "MX_OK", 1: "MX_ERR_ARG", 2: "MX_ERR_CUDA", 3: "MX_ERR_OOM", 4: "MX_ERR_NOCONV",
                5: "MX_ERR_INCOMPAT", 6: "MX_ERR_TIMEOUT"}


class mx_geom(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("dx", C.c_double), ("lo", C.c_int * 3), ("hi", C.c_int * 3)]


class mx_opts(C.Structure):
    _fields_ = [("rel_tol", C.c_double), ("max_outer", C.c_int), ("max_vcycles", C.c_int), ("prec", C.c_int),
                ("remove_mean", C.c_int), ("use_initial_guess", C.c_int), ("use_graph", C.c_int),
                ("nu1", C.c_int), ("nu2", C.c_int), ("bottom_iters", C.c_int), ("fused", C.c_int),
                ("tile_z", C.c_int), ("krylov", C.c_int), ("smoother", C.c_int)]


class mx_info(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("vcycles", C.c_int), ("rel_resid", C.c_double),
                ("rel_resid_l2", C.c_double), ("div_err_linf", C.c_double), ("rhs_mean_removed", C.c_double),
                ("rhs_linf", C.c_double), ("ms", C.c_double), ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MXError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_VP = C.c_void_p
_DP = C.c_void_p
_IP3 = C.c_int * 3


def load():
    """Load the in-tree libmx.so (build it first with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library (paper_1908_03634_gb300.build.build())")
    lib = C.CDLL(LIB_PATH)
    G, O, I = C.POINTER(mx_geom), C.POINTER(mx_opts), C.POINTER(mx_info)
    sig = {
        "mx_create": (C.c_int, [C.POINTER(_VP), C.c_int, _VP]),
        "mx_destroy": (C.c_int, [_VP]),
        "mx_set_stream": (C.c_int, [_VP, _VP]),
        "mx_last_error": (C.c_char_p, [_VP]),
        "mx_default_opts": (None, [O]),
        "mx_device_supported": (C.c_int, [C.c_int]),
        "mx_fill_base_state": (C.c_int, [_VP, G, C.c_int, _DP, C.c_int, C.c_double, C.POINTER(C.c_double), _DP]),
        "mx_mac_project": (C.c_int, [_VP, G, _DP, _DP, _DP, _DP, _DP, _DP, _DP, O, I]),
        "mx_nodal_project": (C.c_int, [_VP, G, _DP, _DP, _DP, _DP, _DP, _DP, _DP, O, I]),
        "mx_apply_op": (C.c_int, [_VP, G, C.c_int, C.c_int, _DP, _DP, _DP, _DP]),
        "mx_residual": (C.c_int, [_VP, G, C.c_int, C.c_int, _DP, _DP, _DP, _DP, _DP, C.POINTER(C.c_double)]),
        "mx_residual_noalloc": (C.c_int, [G, _DP, _DP, _DP, _DP, _DP, C.POINTER(C.c_double), _VP]),
        "mx_profile_enable": (C.c_int, [_VP, C.c_int]),
        "mx_profile_read": (C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
        "mx_autotune": (C.c_int, [_VP, C.c_int, G, _DP, _DP, _DP, _DP, _DP, _DP, O, O, C.POINTER(C.c_double)]),
        "mx_tune_lookup": (C.c_int, [_VP, C.c_int, C.c_int, G, O]),
        "mx_autotune_batched": (C.c_int, [_VP, C.c_int, G, C.POINTER(_DP), C.POINTER(_DP), C.POINTER(_DP),
                                          C.POINTER(_DP), C.POINTER(_DP), C.POINTER(_DP), O, O,
                                          C.POINTER(C.c_double)]),
        "mx_mac_project_batched": (C.c_int, [_VP, C.c_int, G, C.POINTER(_DP), C.POINTER(_DP), C.POINTER(_DP),
                                             C.POINTER(_DP), C.POINTER(_DP), C.POINTER(_DP), C.POINTER(_DP), O, I]),
        "mx_radial_nbins": (C.c_longlong, [G, _IP3]),
        "mx_average_planar": (C.c_int, [_VP, G, _DP, _DP]),
        "mx_average_radial": (C.c_int, [_VP, G, _IP3, _DP, C.c_longlong, _DP, _VP]),
        "mx_fill_radial": (C.c_int, [_VP, G, _IP3, _DP, C.c_longlong, _DP]),
        "mx_radial_to_uniform": (C.c_int, [_VP, G, _IP3, _DP, C.c_int, C.c_double, _DP]),
        "mx_fill_uniform": (C.c_int, [_VP, G, _IP3, _DP, C.c_int, C.c_double, _DP]),
        "mx_w0_integrate": (C.c_int, [_VP, C.c_int, C.c_int, _DP, _DP, _DP, C.c_int, _DP]),
        "mx_add_w0_faces": (C.c_int, [_VP, G, C.c_int, _IP3, C.c_int, _DP, _DP, _DP, _DP, _DP]),
        "mx_subtract_lateral_average": (C.c_int, [_VP, G, C.c_int, _IP3, _DP, _DP]),
        "mx_composite_apply": (C.c_int, [_VP, G, _IP3, _IP3] + [_DP] * 8),
        "mx_composite_divergence": (C.c_int, [_VP, G, _IP3, _IP3] + [_DP] * 10),
        "mx_mac_project_split": (C.c_int, [_VP, G, C.c_int, _IP3, _DP, _DP, _DP, _DP, _DP, _DP, C.c_int, _DP, _DP,
                                           _DP, O, I]),
        "mx_probe_fma_peak": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double)]),
        "mx_mac_project_composite": (C.c_int, [_VP, G, _IP3, _IP3] + [_DP] * 14 + [O, I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names declared in include/mx.h and exported by the library."""
    return ["mx_create", "mx_destroy", "mx_set_stream", "mx_last_error", "mx_default_opts", "mx_device_supported",
            "mx_fill_base_state", "mx_mac_project", "mx_nodal_project", "mx_apply_op", "mx_residual",
            "mx_mac_project_batched", "mx_profile_enable", "mx_profile_read", "mx_residual_noalloc",
            "mx_autotune", "mx_tune_lookup", "mx_autotune_batched", "mx_radial_nbins", "mx_average_planar",
            "mx_average_radial", "mx_fill_radial", "mx_radial_to_uniform", "mx_fill_uniform", "mx_w0_integrate",
            "mx_add_w0_faces", "mx_subtract_lateral_average", "mx_mac_project_split", "mx_composite_apply",
            "mx_composite_divergence", "mx_probe_fma_peak", "mx_mac_project_composite"]


# --- marshalling helpers ---------------------------------------------------------------

def make_geom(geom) -> mx_geom:
    g = mx_geom()
    for d in range(3):
        g.n[d] = int(geom.n[d])
        g.lo[d] = int(geom.lo[d])
        g.hi[d] = int(geom.hi[d])
    g.dx = float(geom.dx)
    return g


def _ptr(t, shape=None, name="array"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name}: expected float64")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")
    return _VP(t.data_ptr())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return _VP(stream.cuda_stream)


def default_opts(**kw) -> mx_opts:
    o = mx_opts()
    load().mx_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def cell_shape(geom):
    return (geom.n[2], geom.n[1], geom.n[0])


def face_shape(geom, d):
    nx, ny, nz = geom.n
    return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][d]


def node_shape(geom):
    m = [geom.n[d] + (0 if geom.lo[d] == MX_BC_PERIODIC else 1) for d in range(3)]
    return (m[2], m[1], m[0])


# --- the entry points -------------------------------------------------------------------

def mx_create(device: int = 0, stream=None):
    lib = load()
    h = _VP()
    st = lib.mx_create(C.byref(h), int(device), _stream_handle(stream))
    if st != MX_OK:
        raise MXError(st, "mx_create failed")
    return h


def mx_destroy(ctx):
    return load().mx_destroy(ctx)


def mx_set_stream(ctx, stream=None):
    return load().mx_set_stream(ctx, _stream_handle(stream))


def mx_last_error(ctx) -> str:
    return load().mx_last_error(ctx).decode()


def _check(ctx, st, allow=(MX_OK,)):
    if st not in allow:
        raise MXError(st, mx_last_error(ctx))
    return st


def mx_fill_base_state(ctx, geom, spherical, prof, dr, center, out):
    g = make_geom(geom)
    c = (C.c_double * 3)(*center)
    st = load().mx_fill_base_state(ctx, C.byref(g), int(spherical), _ptr(prof, None, "prof"), int(prof.numel()),
                                   float(dr), c, _ptr(out, cell_shape(geom), "out"))
    return _check(ctx, st)


# ---- lateral average and fill (Sec. 3.1) ------------------------------------------------

def _corner(corner):
    return _IP3(*[int(x) for x in corner])


def mx_radial_nbins(geom, corner):
    n = load().mx_radial_nbins(C.byref(make_geom(geom)), _corner(corner))
    if n < 0:
        raise ValueError("mx_radial_nbins: corner out of range")
    return int(n)


def mx_average_planar(ctx, geom, field, prof):
    st = load().mx_average_planar(ctx, C.byref(make_geom(geom)), _ptr(field, cell_shape(geom), "field"),
                                  _ptr(prof, (geom.n[2],), "prof"))
    return _check(ctx, st)


def mx_average_radial(ctx, geom, corner, field, avg, count=None):
    """avg: float64 (nbins,); count: int64 (nbins,) or None."""
    import torch
    nb = avg.numel()
    cp = None
    if count is not None:
        if not (isinstance(count, torch.Tensor) and count.is_cuda and count.dtype == torch.int64
                and count.is_contiguous() and count.numel() == nb):
            raise TypeError("count: expected a contiguous int64 CUDA tensor of nbins entries")
        cp = _VP(count.data_ptr())
    st = load().mx_average_radial(ctx, C.byref(make_geom(geom)), _corner(corner),
                                  _ptr(field, cell_shape(geom), "field"), nb, _ptr(avg, (nb,), "avg"), cp)
    return _check(ctx, st)


def mx_fill_radial(ctx, geom, corner, base, out):
    nb = base.numel()
    st = load().mx_fill_radial(ctx, C.byref(make_geom(geom)), _corner(corner), _ptr(base, (nb,), "base"), nb,
                               _ptr(out, cell_shape(geom), "out"))
    return _check(ctx, st)


def mx_radial_to_uniform(ctx, geom, corner, avg, dr, prof):
    st = load().mx_radial_to_uniform(ctx, C.byref(make_geom(geom)), _corner(corner), _ptr(avg, None, "avg"),
                                     int(prof.numel()), float(dr), _ptr(prof, (prof.numel(),), "prof"))
    return _check(ctx, st)


def mx_fill_uniform(ctx, geom, corner, prof, dr, out):
    st = load().mx_fill_uniform(ctx, C.byref(make_geom(geom)), _corner(corner), _ptr(prof, None, "prof"),
                                int(prof.numel()), float(dr), _ptr(out, cell_shape(geom), "out"))
    return _check(ctx, st)


# ---- velocity split (Appendix A) ---------------------------------------------------------

def mx_w0_integrate(ctx, spherical, r_edge, beta0, src, w0, cutoff=-1):
    """w0 (nr + 1 edges) from the base-state beta0 and src = Sbar - psi (nr cells)."""
    nr = beta0.numel()
    st = load().mx_w0_integrate(ctx, int(spherical), nr, _ptr(r_edge, (nr + 1,), "r_edge"), _ptr(beta0, (nr,), "beta0"),
                                _ptr(src, (nr,), "src"), int(cutoff), _ptr(w0, (nr + 1,), "w0"))
    return _check(ctx, st)


def mx_add_w0_faces(ctx, geom, spherical, corner, r_edge, w0, ux, uy, uz):
    nr = w0.numel() - 1
    st = load().mx_add_w0_faces(ctx, C.byref(make_geom(geom)), int(spherical), _corner(corner or (0, 0, 0)), nr,
                                _ptr(r_edge, (nr + 1,), "r_edge") if r_edge is not None else None, _ptr(w0, None, "w0"),
                                _ptr(ux, face_shape(geom, 0), "ux"), _ptr(uy, face_shape(geom, 1), "uy"),
                                _ptr(uz, face_shape(geom, 2), "uz"))
    return _check(ctx, st)


def mx_subtract_lateral_average(ctx, geom, spherical, corner, S, out):
    st = load().mx_subtract_lateral_average(ctx, C.byref(make_geom(geom)), int(spherical),
                                            _corner(corner or (0, 0, 0)), _ptr(S, cell_shape(geom), "S"),
                                            _ptr(out, cell_shape(geom), "out"))
    return _check(ctx, st)


def _fine_shapes(geom, plo, phi):
    nf = [2 * (int(phi[d]) - int(plo[d])) for d in range(3)]
    cells = (nf[2], nf[1], nf[0])
    faces = [tuple(reversed([nf[e] + (1 if e == d else 0) for e in range(3)])) for d in range(3)]
    return cells, faces


def mx_composite_apply(ctx, geom, plo, phi, rho_c, beta0_c, rho_f, beta0_f, phi_c, phi_f, out_c, out_f):
    """L phi of the two-level composite operator (coarse geom + the fine patch [plo, phi))."""
    cs = cell_shape(geom)
    fs, _ = _fine_shapes(geom, plo, phi)
    st = load().mx_composite_apply(ctx, C.byref(make_geom(geom)), _corner(plo), _corner(phi),
                                   _ptr(rho_c, cs, "rho_c"), _ptr(beta0_c, cs, "beta0_c"), _ptr(rho_f, fs, "rho_f"),
                                   _ptr(beta0_f, fs, "beta0_f"), _ptr(phi_c, cs, "phi_c"), _ptr(phi_f, fs, "phi_f"),
                                   _ptr(out_c, cs, "out_c"), _ptr(out_f, fs, "out_f"))
    return _check(ctx, st)


def mx_composite_divergence(ctx, geom, plo, phi, uc, uf, beta0_c, beta0_f, out_c, out_f):
    """D(beta0 U) on the composite grid; uc, uf: lists of the three coarse / fine face arrays."""
    cs = cell_shape(geom)
    fs, ffs = _fine_shapes(geom, plo, phi)
    st = load().mx_composite_divergence(
        ctx, C.byref(make_geom(geom)), _corner(plo), _corner(phi),
        *[_ptr(uc[d], face_shape(geom, d), "uc") for d in range(3)], *[_ptr(uf[d], ffs[d], "uf") for d in range(3)],
        _ptr(beta0_c, cs, "beta0_c"), _ptr(beta0_f, fs, "beta0_f"), _ptr(out_c, cs, "out_c"), _ptr(out_f, fs, "out_f"))
    return _check(ctx, st)


def mx_mac_project_composite(ctx, geom, plo, phi, uc, rho_c, beta0_c, sbar_c, phi_c, uf, rho_f, beta0_f, sbar_f,
                             phi_f, opts=None, allow=(MX_OK,)):
    """Composite (coarse + one ratio-2 patch [plo, phi)) MAC projection; uc, uf:
    lists of the three coarse / fine face arrays (in/out).  Returns (status, info)."""
    cs = cell_shape(geom)
    fs, ffs = _fine_shapes(geom, plo, phi)
    info = mx_info()
    st = load().mx_mac_project_composite(
        ctx, C.byref(make_geom(geom)), _corner(plo), _corner(phi),
        *[_ptr(uc[d], face_shape(geom, d), "uc") for d in range(3)], _ptr(rho_c, cs, "rho_c"),
        _ptr(beta0_c, cs, "beta0_c"), _ptr(sbar_c, cs, "sbar_c"), _ptr(phi_c, cs, "phi_c"),
        *[_ptr(uf[d], ffs[d], "uf") for d in range(3)], _ptr(rho_f, fs, "rho_f"), _ptr(beta0_f, fs, "beta0_f"),
        _ptr(sbar_f, fs, "sbar_f"), _ptr(phi_f, fs, "phi_f"), C.byref(opts) if opts is not None else None,
        C.byref(info))
    _check(ctx, st, allow)
    return st, info.as_dict()


def mx_mac_project_split(ctx, geom, spherical, corner, ux, uy, uz, rho, beta0, S, r_edge, w0, phi, opts=None,
                         allow=(MX_OK,)):
    """U~ projected with the bracket S - Sbar, then w0 e_r added: (status, info)."""
    g = make_geom(geom)
    info = mx_info()
    cs = cell_shape(geom)
    nr = w0.numel() - 1
    st = load().mx_mac_project_split(ctx, C.byref(g), int(spherical), _corner(corner or (0, 0, 0)),
                                     _ptr(ux, face_shape(geom, 0), "ux"), _ptr(uy, face_shape(geom, 1), "uy"),
                                     _ptr(uz, face_shape(geom, 2), "uz"), _ptr(rho, cs, "rho"),
                                     _ptr(beta0, cs, "beta0"), _ptr(S, cs, "S"), nr,
                                     _ptr(r_edge, (nr + 1,), "r_edge") if r_edge is not None else None,
                                     _ptr(w0, None, "w0"), _ptr(phi, cs, "phi"),
                                     C.byref(opts) if opts is not None else None, C.byref(info))
    _check(ctx, st, allow)
    return st, info.as_dict()


def mx_mac_project(ctx, geom, ux, uy, uz, rho, beta0, sbar, phi, opts=None, allow=(MX_OK,)):
    """Returns (status, info dict).  Raises MXError unless the status is in allow."""
    g = make_geom(geom)
    info = mx_info()
    cs = cell_shape(geom)
    st = load().mx_mac_project(ctx, C.byref(g), _ptr(ux, face_shape(geom, 0), "ux"), _ptr(uy, face_shape(geom, 1), "uy"),
                               _ptr(uz, face_shape(geom, 2), "uz"), _ptr(rho, cs, "rho"), _ptr(beta0, cs, "beta0"),
                               _ptr(sbar, cs, "sbar"), _ptr(phi, cs, "phi"),
                               C.byref(opts) if opts is not None else None, C.byref(info))
    _check(ctx, st, allow)
    return st, info.as_dict()


def mx_nodal_project(ctx, geom, ux, uy, uz, rho, beta0, sbar, phi_nodes, opts=None, allow=(MX_OK,)):
    g = make_geom(geom)
    info = mx_info()
    cs = cell_shape(geom)
    st = load().mx_nodal_project(ctx, C.byref(g), _ptr(ux, cs, "ux"), _ptr(uy, cs, "uy"), _ptr(uz, cs, "uz"),
                                 _ptr(rho, cs, "rho"), _ptr(beta0, cs, "beta0"), _ptr(sbar, cs, "sbar"),
                                 _ptr(phi_nodes, node_shape(geom), "phi_nodes"),
                                 C.byref(opts) if opts is not None else None, C.byref(info))
    _check(ctx, st, allow)
    return st, info.as_dict()


def mx_autotune(ctx, op, geom, ux, uy, uz, rho, beta0, sbar, base=None):
    """Tune (nu1, nu2, tile_z, fused; nodal: smoother) on these inputs (left unmodified); returns
    (chosen mx_opts, ms of the tuned solve).  The choice is cached in ctx for
    calls with nu1 = nu2 = 0."""
    g = make_geom(geom)
    cs = cell_shape(geom)
    us = [face_shape(geom, d) for d in range(3)] if op == MX_OP_MAC else [cs] * 3
    best = mx_opts()
    ms = C.c_double(0.0)
    st = load().mx_autotune(ctx, int(op), C.byref(g), _ptr(ux, us[0], "ux"), _ptr(uy, us[1], "uy"),
                            _ptr(uz, us[2], "uz"), _ptr(rho, cs, "rho"), _ptr(beta0, cs, "beta0"),
                            _ptr(sbar, cs, "sbar"), C.byref(base) if base is not None else None, C.byref(best),
                            C.byref(ms))
    _check(ctx, st)
    return best, ms.value


def mx_autotune_batched(ctx, geoms, ux, uy, uz, rho, beta0, sbar, base=None):
    """Tune (nu1, nu2) for a batch (lists of per-box tensors, left unmodified);
    returns (chosen mx_opts, ms of the tuned batch); cached in ctx for batched
    calls with nu1 = nu2 = 0 on the same boxes."""
    n = len(geoms)
    G = (mx_geom * n)(*[make_geom(g) for g in geoms])

    def arr(ts, shapes, name):
        return (_VP * n)(*[_ptr(t, s, name) for t, s in zip(ts, shapes)])

    cs = [cell_shape(g) for g in geoms]
    best = mx_opts()
    ms = C.c_double(0.0)
    st = load().mx_autotune_batched(
        ctx, n, G, arr(ux, [face_shape(g, 0) for g in geoms], "ux"), arr(uy, [face_shape(g, 1) for g in geoms], "uy"),
        arr(uz, [face_shape(g, 2) for g in geoms], "uz"), arr(rho, cs, "rho"), arr(beta0, cs, "beta0"),
        arr(sbar, cs, "sbar"), C.byref(base) if base is not None else None, C.byref(best), C.byref(ms))
    _check(ctx, st)
    return best, ms.value


def mx_tune_lookup(ctx, op, prec, geom):
    """The cached tuned options for (op, prec, geom), or None."""
    g = make_geom(geom)
    o = default_opts()
    return o if load().mx_tune_lookup(ctx, int(op), int(prec), C.byref(g), C.byref(o)) else None


def mx_apply_op(ctx, geom, op, prec, rho, beta0, phi, out):
    g = make_geom(geom)
    cs = cell_shape(geom)
    vs = cs if op == MX_OP_MAC else node_shape(geom)
    st = load().mx_apply_op(ctx, C.byref(g), int(op), int(prec), _ptr(rho, cs, "rho"), _ptr(beta0, cs, "beta0"),
                            _ptr(phi, vs, "phi"), _ptr(out, vs, "Lphi"))
    return _check(ctx, st)


def mx_residual(ctx, geom, op, prec, rho, beta0, phi, f, r):
    """r = f - L phi; returns ||r||_inf."""
    g = make_geom(geom)
    cs = cell_shape(geom)
    vs = cs if op == MX_OP_MAC else node_shape(geom)
    rn = C.c_double(0.0)
    st = load().mx_residual(ctx, C.byref(g), int(op), int(prec), _ptr(rho, cs, "rho"), _ptr(beta0, cs, "beta0"),
                            _ptr(phi, vs, "phi"), _ptr(f, vs, "f"), _ptr(r, vs, "r"), C.byref(rn))
    _check(ctx, st)
    return rn.value


def mx_mac_project_batched(ctx, geoms, ux, uy, uz, rho, beta0, sbar, phi, opts=None, allow=(MX_OK,)):
    """Lists of per-box tensors.  Returns (status, list of info dicts)."""
    n = len(geoms)
    G = (mx_geom * n)(*[make_geom(g) for g in geoms])
    infos = (mx_info * n)()

    def arr(ts, shapes, name):
        return (_VP * n)(*[_ptr(t, s, name) for t, s in zip(ts, shapes)])

    cs = [cell_shape(g) for g in geoms]
    st = load().mx_mac_project_batched(
        ctx, n, G, arr(ux, [face_shape(g, 0) for g in geoms], "ux"), arr(uy, [face_shape(g, 1) for g in geoms], "uy"),
        arr(uz, [face_shape(g, 2) for g in geoms], "uz"), arr(rho, cs, "rho"), arr(beta0, cs, "beta0"),
        arr(sbar, cs, "sbar"), arr(phi, cs, "phi"), C.byref(opts) if opts is not None else None, infos)
    _check(ctx, st, allow)
    return st, [infos[i].as_dict() for i in range(n)]


def mx_profile_enable(ctx, enable=True):
    return _check(ctx, load().mx_profile_enable(ctx, int(bool(enable))))


def mx_profile_read(ctx):
    """{phase: (ms, launches)} accumulated since the last read."""
    n = len(PHASES)
    ms = (C.c_double * n)()
    ln = (C.c_longlong * n)()
    _check(ctx, load().mx_profile_read(ctx, ms, ln))
    return {PHASES[i]: (ms[i], ln[i]) for i in range(n)}


def mx_residual_noalloc(geom, rho, beta0, phi, f, r, stream=None):
    """FP64 MAC residual r = f - L phi without any device allocation (see
    include/mx.h); returns ||r||_inf.  Raises MXError on a non-zero status."""
    g = make_geom(geom)
    cs = cell_shape(geom)
    rn = C.c_double(0.0)
    st = load().mx_residual_noalloc(C.byref(g), _ptr(rho, cs, "rho"), _ptr(beta0, cs, "beta0"), _ptr(phi, cs, "phi"),
                                    _ptr(f, cs, "f"), _ptr(r, cs, "r"), C.byref(rn), _stream_handle(stream))
    if st != MX_OK:
        raise MXError(st, "mx_residual_noalloc failed")
    return rn.value


def mx_probe_fma_peak(device: int = 0, fp64: bool = True) -> float:
    """Measured FMA rate of the FP64 (or FP32) pipe in TFLOP/s (see include/mx.h)."""
    t = C.c_double(0.0)
    st = load().mx_probe_fma_peak(int(device), int(bool(fp64)), C.byref(t))
    if st != MX_OK:
        raise MXError(st, "mx_probe_fma_peak failed")
    return t.value
