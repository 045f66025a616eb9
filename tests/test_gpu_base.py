"""GPU parity of the lateral average and fill (Sec. 3.1, Eq. radii) against the
FP64 oracle, through the C ABI.

Tolerances.  The fills are gathers (bit-exact).  The uniform-base-state
interpolations evaluate the same 3-point Lagrange expression operation by
operation in FP64 on both sides (bit-exact when both start from the same bin
means; the fill of a uniform profile computes the cell radius as dx sqrt(0.75 +
2m) where the oracle takes the Euclidean norm, so it agrees to rounding, after
checking that no cell radius sits within 1e-9 of a radial cell boundary where
the two roundings could pick different stencils).  The averages sum in
double-float (operands kept to 48 bits, about 2^-47 relative rounding per
addition) in another order than the oracle's sequential FP64 sum: with n cells
per bin the rounding walk is about sqrt(n) 2^-47 of the mean magnitude, and the
tests allow 8 times that, tol = max(sqrt(n), 8) 2^-44 mean|f|."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1908_03634_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
N = W.NEUMANN


@pytest.fixture(scope="module")
def mx():
    from paper_1908_03634_gb300 import build as b
    b.build()
    O.build()
    import paper_1908_03634_gb300 as m
    return m


@pytest.fixture()
def ctx(mx):
    c = mx.mx_create(0)
    yield c
    mx.mx_destroy(c)


def geom(n, dx=1.0 / 64):
    return W.Geom(tuple(n), dx, (N, N, N), (N, N, N))


def field(g, seed, kind="star"):
    """a density-like radial profile with lateral structure plus noise"""
    rng = np.random.default_rng(seed)
    nz, ny, nx = g.n[2], g.n[1], g.n[0]
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx,
                          indexing="ij")
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
    f = np.exp(-8.0 * r) * (1.0 + 0.1 * np.sin(7 * x) * np.cos(5 * y)) + 1e-3 * rng.standard_normal(r.shape)
    if kind == "signed":
        f = f - f.mean()
    if kind == "wide":
        # magnitudes from 1e200 down to 1e-300 (below 2^-73 the sums take the scaled and
        # FP64 lanes of the accumulator), signs mixed on one side
        f = 10.0 ** (200.0 - 500.0 * r / max(r.max(), 1e-30)) * (1.0 + 0.5 * rng.standard_normal(r.shape) * (x < 0.3))
    return np.ascontiguousarray(f)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def tol_bins(f_abs_mean, n):
    return np.maximum(np.sqrt(n), 8.0) * 2.0**-44 * f_abs_mean + 1e-300


RADIAL = [
    ((32, 32, 32), (16, 16, 16)),      # centred star, several tiles and rows per group
    ((37, 23, 29), (18, 11, 15)),      # ragged, odd sizes
    ((300, 7, 5), (150, 3, 2)),        # rows longer than the fold CTA
    ((20, 12, 9), (7, 3, 9)),          # off-centre
    ((16, 9, 11), (-5, 4, 14)),        # corner outside the box
    ((1, 1, 1), (0, 0, 0)),            # one cell
    ((64, 48, 40), (32, 24, 20)),
    ((1030, 3, 4), (515, 1, 2)),       # even rows too long for the copy-engine fold
]


@pytest.mark.parametrize("n,c", RADIAL)
@pytest.mark.parametrize("kind", ["star", "signed", "wide"])
def test_average_radial_parity(mx, ctx, n, c, kind):
    g = geom(n)
    f = field(g, 7, kind)
    nb = mx.mx_radial_nbins(g, c)
    assert nb == O.radial_nbins(g, c)
    avg = torch.empty(nb, dtype=torch.float64, device=DEV)
    cnt = torch.empty(nb, dtype=torch.int64, device=DEV)
    mx.mx_average_radial(ctx, g, c, dev(f), avg, cnt)
    torch.cuda.synchronize()
    ref, rcnt = O.average_radial(g, c, f)
    assert np.array_equal(cnt.cpu().numpy(), rcnt)
    m = O.radial_index(g, c).ravel()
    absmean = np.bincount(m, weights=np.abs(f).ravel(), minlength=nb) / np.maximum(rcnt, 1)
    got = avg.cpu().numpy()
    assert np.all(np.abs(got - ref) <= tol_bins(absmean, rcnt))
    assert np.all(got[rcnt == 0] == 0.0)
    again = torch.empty_like(avg)
    mx.mx_average_radial(ctx, g, c, dev(f), again)
    assert torch.equal(avg, again)  # fixed summation order


def test_average_radial_unaligned_field(mx, ctx):
    """a field 8 bytes off a 16-byte boundary takes the scalar-load fold (same bits as
    the 16-byte-load fold); an output 8 bytes off takes the scalar-store fill"""
    g = geom((64, 40, 36))
    c = (32, 20, 18)
    f = field(g, 11)
    buf = torch.empty(f.size + 1, dtype=torch.float64, device=DEV)
    off = buf[1:].view(f.shape)
    off.copy_(dev(f))
    nb = mx.mx_radial_nbins(g, c)
    a = torch.empty(nb, dtype=torch.float64, device=DEV)
    b = torch.empty(nb, dtype=torch.float64, device=DEV)
    mx.mx_average_radial(ctx, g, c, off, a)
    mx.mx_average_radial(ctx, g, c, dev(f), b)
    torch.cuda.synchronize()
    ref, cnt = O.average_radial(g, c, f)
    absmean, _ = O.average_radial(g, c, np.abs(f))
    for x in (a, b):
        assert np.all(np.abs(x.cpu().numpy() - ref) <= tol_bins(absmean, cnt))
    assert torch.equal(a, b)
    obuf = torch.empty(f.size + 1, dtype=torch.float64, device=DEV)
    out = obuf[1:].view(f.shape)
    mx.mx_fill_radial(ctx, g, c, a, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), O.fill_irregular(g, c, a.cpu().numpy()))


@pytest.mark.parametrize("n,c", RADIAL)
def test_fill_radial_bit_exact(mx, ctx, n, c):
    g = geom(n)
    nb = mx.mx_radial_nbins(g, c)
    base = np.random.default_rng(2).standard_normal(nb)
    out = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_fill_radial(ctx, g, c, dev(base), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), O.fill_irregular(g, c, base))


def test_round_trip_radial_function(mx, ctx):
    """average then fill returns a purely radial field (to the averaging rounding)"""
    g = geom((48, 40, 44))
    c = (24, 20, 22)
    m = O.radial_index(g, c)
    f = np.exp(-0.01 * m.astype(np.float64)) + 0.5
    nb = mx.mx_radial_nbins(g, c)
    avg = torch.empty(nb, dtype=torch.float64, device=DEV)
    mx.mx_average_radial(ctx, g, c, dev(f), avg)
    out = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_fill_radial(ctx, g, c, avg, out)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), f, rtol=2.0**-40)


@pytest.mark.parametrize("shape", [(32, 32, 32), (37, 23, 11), (256, 3, 5), (1, 1, 1), (130, 70, 3)])
@pytest.mark.parametrize("kind", ["star", "signed", "offset", "wide"])
def test_average_planar_parity(mx, ctx, shape, kind):
    """kind offset: the field 8 bytes off a 16-byte boundary (scalar loads); wide:
    magnitudes from 1e200 to 1e-300"""
    g = geom(shape)
    f = field(g, 4, "star" if kind == "offset" else kind)
    out = torch.empty(g.n[2], dtype=torch.float64, device=DEV)
    fd = dev(f)
    if kind == "offset":
        buf = torch.empty(f.size + 1, dtype=torch.float64, device=DEV)
        fd = buf[1:].view(f.shape)
        fd.copy_(dev(f))
    mx.mx_average_planar(ctx, g, fd, out)
    torch.cuda.synchronize()
    ref = O.average_planar(g, f)
    nxy = g.n[0] * g.n[1]
    tol = tol_bins(np.abs(f).mean(axis=(1, 2)), nxy)
    assert np.all(np.abs(out.cpu().numpy() - ref) <= tol)


@pytest.mark.parametrize("n,c,nr,drf", [((32, 32, 32), (16, 16, 16), 140, 0.2), ((37, 23, 29), (18, 11, 15), 40, 0.7),
                                        ((20, 12, 9), (7, 3, 9), 30, 1.0), ((64, 48, 40), (32, 24, 20), 3, 30.0)])
def test_radial_to_uniform_bit_exact(mx, ctx, n, c, nr, drf):
    g = geom(n)
    f = field(g, 9)
    ref_avg, cnt = O.average_radial(g, c, f)
    dr = drf * g.dx
    want = O.average_to_uniform(ref_avg, cnt, g.dx, nr, dr)
    out = torch.empty(nr, dtype=torch.float64, device=DEV)
    mx.mx_radial_to_uniform(ctx, g, c, dev(ref_avg), dr, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)
    # composed with the GPU average: within the averaging tolerance, amplified by the
    # Lagrange weights (at most 1.25 in magnitude each inside the node span; wider
    # outside, so compare relative to the profile's scale)
    avg = torch.empty(ref_avg.size, dtype=torch.float64, device=DEV)
    mx.mx_average_radial(ctx, g, c, dev(f), avg)
    mx.mx_radial_to_uniform(ctx, g, c, avg, dr, out)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=0, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("n,c,nr,drf", [((32, 32, 32), (16, 16, 16), 140, 0.2), ((37, 23, 29), (18, 11, 15), 60, 0.5),
                                        ((16, 9, 11), (-5, 4, 14), 50, 0.9)])
def test_fill_uniform_parity(mx, ctx, n, c, nr, drf):
    g = geom(n)
    dr = drf * g.dx
    rc = (np.arange(nr) + 0.5) * dr
    prof = np.exp(-3.0 * rc) + np.sin(40.0 * rc)
    ctr = np.array(c, dtype=np.float64) * g.dx
    want = O.fill_quadratic(g, prof, dr, ctr)
    out = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
    mx.mx_fill_uniform(ctx, g, c, dev(prof), dr, out)
    torch.cuda.synchronize()
    m = O.radial_index(g, c)
    v = g.dx * np.sqrt(0.75 + 2.0 * m) / dr
    near = np.abs(v - np.rint(v)) < 1e-9
    assert near.mean() < 0.01
    got = out.cpu().numpy()
    np.testing.assert_allclose(got[~near], want[~near], rtol=0, atol=1e-12 * np.abs(prof).max())


def test_null_arrays_rejected(mx, ctx):
    """the C entry points check their pointers (the binding passes NULL for None)"""
    lib = mx.load()
    g = geom((8, 8, 8))
    gg = mx.make_geom(g)
    import ctypes as C
    c3 = (C.c_int * 3)(4, 4, 4)
    out = torch.zeros(mx.cell_shape(g), dtype=torch.float64, device=DEV)
    nb = mx.mx_radial_nbins(g, (4, 4, 4))
    assert lib.mx_average_radial(ctx, C.byref(gg), c3, None, nb, C.c_void_p(out.data_ptr()), None) == mx.MX_ERR_ARG
    assert lib.mx_fill_radial(ctx, C.byref(gg), c3, None, nb, C.c_void_p(out.data_ptr())) == mx.MX_ERR_ARG
    assert lib.mx_average_planar(ctx, C.byref(gg), None, C.c_void_p(out.data_ptr())) == mx.MX_ERR_ARG
    assert lib.mx_subtract_lateral_average(ctx, C.byref(gg), 1, c3, None, C.c_void_p(out.data_ptr())) == mx.MX_ERR_ARG
    assert lib.mx_w0_integrate(ctx, 1, 4, None, None, None, -1, None) == mx.MX_ERR_ARG
    assert "null" in mx.mx_last_error(ctx)


def test_errors(mx, ctx):
    g = geom((8, 8, 8))
    c = (4, 4, 4)
    nb = mx.mx_radial_nbins(g, c)
    f = torch.zeros(mx.cell_shape(g), dtype=torch.float64, device=DEV)
    with pytest.raises(mx.MXError) as e:
        mx.mx_average_radial(ctx, g, c, f, torch.empty(nb + 1, dtype=torch.float64, device=DEV))
    assert e.value.status == mx.MX_ERR_ARG
    with pytest.raises(ValueError):
        mx.mx_radial_nbins(g, (1 << 21, 0, 0))
    g1 = geom((1, 1, 1))
    a1 = torch.zeros(1, dtype=torch.float64, device=DEV)
    with pytest.raises(mx.MXError) as e:
        mx.mx_radial_to_uniform(ctx, g1, (0, 0, 0), a1, 0.1, torch.empty(4, dtype=torch.float64, device=DEV))
    assert e.value.status == mx.MX_ERR_ARG
    with pytest.raises(mx.MXError) as e:
        mx.mx_fill_uniform(ctx, g, c, torch.zeros(2, dtype=torch.float64, device=DEV), 0.1, f)
    assert e.value.status == mx.MX_ERR_ARG
