"""Parity at the full workload sizes, in the launch configuration the benchmark
times (default options: mixed precision, CUDA-graph loop), on outputs the
oracle computes one at a time: the residual f - L phi of the GPU's phi at
sampled cells/nodes (f from the oracle's own full-array RHS), the divergence
identity D(beta0 U) - beta0 Sbar - c = f - L phi of the GPU's projected U at
the same cells, and the normalisation of phi.

Element by element at the autotuned smoother settings (the benchmark's launch
configuration): phi of the planar 256^3 MAC solve and of the nodal solve at
192^3 cells (the hierarchy of the 384^3 workload from its 192^3 level down)
against the oracle solved to 1e-13, within 1e-8 relative max norm, and the
projected U against the oracle's correction of the GPU's phi to 1e-12.  The
oracle solves run in a host thread (its C code releases the GIL) while the GPU
tunes and solves.
"""
import threading

import numpy as np
import pytest
import torch

import oracle as O
from paper_1908_03634_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def mx():
    from paper_1908_03634_gb300 import build as b
    b.build()
    O.build()
    import paper_1908_03634_gb300 as m
    return m


def sample_cells(g, n, seed):
    rng = np.random.default_rng(seed)
    N = g.n[0] * g.n[1] * g.n[2]
    idx = rng.integers(0, N, size=n)
    # always include cells on the first and last planes (boundary closures)
    nxy = g.n[0] * g.n[1]
    edge = np.concatenate([rng.integers(0, nxy, size=n // 10), N - nxy + rng.integers(0, nxy, size=n // 10)])
    return np.unique(np.concatenate([idx, edge]))


def run_mac(mx, w):
    g = w.geom
    ctx = mx.mx_create(0)
    try:
        beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
        mx.mx_fill_base_state(ctx, g, int(w.spherical), w.prof_beta0.to(DEV), w.prof_dr, w.center, beta0)
        u = [t.clone() for t in w.u]
        phi = torch.zeros(mx.cell_shape(g), dtype=torch.float64, device=DEV)
        st, info = mx.mx_mac_project(ctx, g, *u, w.rho, beta0, w.sbar, phi, mx.default_opts())
        torch.cuda.synchronize()
    finally:
        mx.mx_destroy(ctx)
    return info, phi.cpu().numpy(), [x.cpu().numpy() for x in u]


@pytest.mark.parametrize("name", ["planar256", "star512"])
def test_mac_fullsize_sampled(mx, name):
    w = W.planar256(device=DEV) if name == "planar256" else W.star512(device=DEV)
    g = w.geom
    info, phi, u = run_mac(mx, w)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    rho, sbar, u0 = w.rho.cpu().numpy(), w.sbar.cpu().numpy(), [t.cpu().numpy() for t in w.u]
    prof, spherical, dr = w.prof_beta0.cpu().numpy(), w.spherical, w.prof_dr
    del w
    b0 = O.fill(g, prof, spherical=spherical, dr=dr, center=(0.5, 0.5, 0.5))
    f, c = O.mac_rhs(g, u0, b0, sbar)
    fn = np.abs(f).max()
    idx = sample_cells(g, 20000, 5)
    r = O.mac_residual_sample(g, rho, b0, phi, f, idx)
    assert np.abs(r).max() <= 1.05e-10 * fn
    d = O.mac_divergence_sample(g, u, b0, idx) - (b0 * sbar).ravel()[idx] - c
    assert np.abs(d - r).max() <= 1e-11 * fn
    assert abs(info["rhs_mean_removed"] - c) <= 1e-12 * max(1.0, abs(c))
    if O.singular(g):
        assert abs(phi.mean()) <= 1e-12 * np.abs(phi).max()


def test_nodal384_fullsize_sampled(mx):
    w = W.nodal384(device=DEV)
    g = w.geom
    ctx = mx.mx_create(0)
    try:
        beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
        mx.mx_fill_base_state(ctx, g, 0, w.prof_beta0.to(DEV), w.prof_dr, w.center, beta0)
        u = [t.clone() for t in w.u]
        phi = torch.zeros(mx.node_shape(g), dtype=torch.float64, device=DEV)
        st, info = mx.mx_nodal_project(ctx, g, *u, w.rho, beta0, w.sbar, phi, mx.default_opts())
        torch.cuda.synchronize()
    finally:
        mx.mx_destroy(ctx)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    b0 = beta0.cpu().numpy()
    rho, sbar = w.rho.cpu().numpy(), w.sbar.cpu().numpy()
    u0 = [t.cpu().numpy() for t in w.u]
    prof = w.prof_beta0.cpu().numpy()
    del w
    assert np.array_equal(b0, O.fill(g, prof))
    f, c = O.nd_rhs(g, u0, b0, sbar)
    fn = np.abs(f).max()
    phi = phi.cpu().numpy()
    M = phi.size
    idx = np.unique(np.random.default_rng(6).integers(0, M, size=20000))
    r = O.nd_residual_sample(g, b0 / rho, phi, f, idx)
    assert np.abs(r).max() <= 1.05e-10 * fn
    wts = O.nd_weights(g)
    assert abs((wts * phi).sum()) <= 1e-12 * np.abs(phi).max() * wts.sum()


def test_lateral_average_and_fill_fullsize(mx):
    """the 512^3 full star's density: radial average onto the irregular base state
    against the oracle on every bin, and the fill back bit for bit; the planar
    256^3 density's plane means."""
    w = W.star512(device=DEV)
    g = w.geom
    c = tuple(n // 2 for n in g.n)
    ctx = mx.mx_create(0)
    try:
        nb = mx.mx_radial_nbins(g, c)
        avg = torch.empty(nb, dtype=torch.float64, device=DEV)
        cnt = torch.empty(nb, dtype=torch.int64, device=DEV)
        mx.mx_average_radial(ctx, g, c, w.rho, avg, cnt)
        out = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
        mx.mx_fill_radial(ctx, g, c, avg, out)
        torch.cuda.synchronize()
        f = w.rho.cpu().numpy()
        ref, rcnt = O.average_radial(g, c, f)
        assert np.array_equal(cnt.cpu().numpy(), rcnt)
        absmean, _ = O.average_radial(g, c, np.abs(f))
        tol = np.maximum(np.sqrt(rcnt), 8.0) * 2.0**-44 * absmean + 1e-300
        a = avg.cpu().numpy()
        assert np.all(np.abs(a - ref) <= tol)
        assert np.array_equal(out.cpu().numpy(), O.fill_irregular(g, c, a))
        del out, f
        wp = W.planar256(device=DEV)
        prof = torch.empty(wp.geom.n[2], dtype=torch.float64, device=DEV)
        mx.mx_average_planar(ctx, wp.geom, wp.rho, prof)
        torch.cuda.synchronize()
        fp = wp.rho.cpu().numpy()
        refp = O.average_planar(wp.geom, fp)
        tolp = np.sqrt(fp[0].size) * 2.0**-44 * np.abs(fp).mean(axis=(1, 2))
        assert np.all(np.abs(prof.cpu().numpy() - refp) <= tolp)
    finally:
        mx.mx_destroy(ctx)


def in_thread(fn):
    """run fn() in a host thread; returns a join() giving its result"""
    box = {}

    def run():
        try:
            box["v"] = fn()
        except BaseException as e:  # noqa: BLE001 - re-raised in join
            box["e"] = e
    t = threading.Thread(target=run)
    t.start()

    def join():
        t.join()
        if "e" in box:
            raise box["e"]
        return box["v"]
    return join


def test_planar256_phi_parity_at_tuned_settings(mx):
    w = W.planar256(device=DEV)
    g = w.geom
    rho_h, sbar_h, u0 = w.rho.cpu().numpy(), w.sbar.cpu().numpy(), [t.cpu().numpy() for t in w.u]
    prof = w.prof_beta0.cpu().numpy()

    def oracle():
        b0 = O.fill(g, prof)
        u_ref, phi_ref, oinfo = O.mac_project(g, u0, rho_h, b0, sbar_h, tol=1e-13, maxit=400)
        assert oinfo["ok"]
        return phi_ref, oinfo
    ref = in_thread(oracle)
    ctx = mx.mx_create(0)
    try:
        beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
        mx.mx_fill_base_state(ctx, g, 0, w.prof_beta0, g.dx, (0.5, 0.5, 0.5), beta0)
        tuned, _ = mx.mx_autotune(ctx, mx.MX_OP_MAC, g, *w.u, w.rho, beta0, w.sbar)
        u = [t.clone() for t in w.u]
        phi = torch.zeros(mx.cell_shape(g), dtype=torch.float64, device=DEV)
        st, info = mx.mx_mac_project(ctx, g, *u, w.rho, beta0, w.sbar, phi, mx.default_opts(nu1=0, nu2=0))
        torch.cuda.synchronize()
    finally:
        mx.mx_destroy(ctx)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    phi, u = phi.cpu().numpy(), [x.cpu().numpy() for x in u]
    del w
    phi_ref, oinfo = ref()
    err = np.abs(phi - phi_ref).max() / np.abs(phi_ref).max()
    assert err <= 1e-8, (err, tuned.nu1, tuned.nu2, tuned.tile_z, tuned.fused)
    u_pred = O.mac_correct(g, rho_h, phi, u0)
    for d in range(3):
        scale = np.abs(u0[d]).max() + np.abs(u_pred[d] - u0[d]).max()
        assert np.abs(u[d] - u_pred[d]).max() <= 1e-12 * scale
    assert abs(info["rhs_mean_removed"] - oinfo["mean"]) <= 1e-12 * max(1.0, abs(oinfo["mean"]))


def test_nodal192_phi_parity_at_tuned_settings(mx):
    w = W.nodal384(device=DEV, n=192)
    g = w.geom
    rho_h, sbar_h, u0 = w.rho.cpu().numpy(), w.sbar.cpu().numpy(), [t.cpu().numpy() for t in w.u]
    prof = w.prof_beta0.cpu().numpy()

    def oracle():
        b0 = O.fill(g, prof)
        u_ref, phi_ref, oinfo = O.nd_project(g, u0, rho_h, b0, sbar_h, tol=1e-13, maxit=400)
        assert oinfo["ok"]
        return phi_ref
    ref = in_thread(oracle)
    ctx = mx.mx_create(0)
    try:
        beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
        mx.mx_fill_base_state(ctx, g, 0, w.prof_beta0, g.dx, (0.5, 0.5, 0.5), beta0)
        tuned, _ = mx.mx_autotune(ctx, mx.MX_OP_NODAL, g, *w.u, w.rho, beta0, w.sbar)
        u = [t.clone() for t in w.u]
        phi = torch.zeros(mx.node_shape(g), dtype=torch.float64, device=DEV)
        st, info = mx.mx_nodal_project(ctx, g, *u, w.rho, beta0, w.sbar, phi, mx.default_opts(nu1=0, nu2=0))
        torch.cuda.synchronize()
    finally:
        mx.mx_destroy(ctx)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    phi, u = phi.cpu().numpy(), [x.cpu().numpy() for x in u]
    del w
    phi_ref = ref()
    err = np.abs(phi - phi_ref).max() / np.abs(phi_ref).max()
    assert err <= 1e-8, (err, tuned.nu1, tuned.nu2, tuned.tile_z, tuned.smoother)
    u_pred = O.nd_correct(g, rho_h, phi, u0)
    for d in range(3):
        scale = np.abs(u0[d]).max() + np.abs(u_pred[d] - u0[d]).max()
        assert np.abs(u[d] - u_pred[d]).max() <= 1e-12 * scale


def test_planar256_two_pass_sweeps_bit_identical_to_single_pass(mx):
    """At full size the solve with the two colour passes per sweep equals, bit
    for bit, the one with the single-pass sweep kernel (red then black in one
    pass over memory, with the prolongation applied on load)."""
    w = W.planar256(device=DEV)
    g = w.geom
    ctx = mx.mx_create(0)
    try:
        beta0 = torch.empty(mx.cell_shape(g), dtype=torch.float64, device=DEV)
        mx.mx_fill_base_state(ctx, g, 0, w.prof_beta0, g.dx, (0.5, 0.5, 0.5), beta0)
        out = []
        for fused in (0, 1):
            u = [t.clone() for t in w.u]
            phi = torch.zeros(mx.cell_shape(g), dtype=torch.float64, device=DEV)
            st, info = mx.mx_mac_project(ctx, g, *u, w.rho, beta0, w.sbar, phi,
                                         mx.default_opts(nu1=2, nu2=3, fused=fused))
            out.append((info["vcycles"], phi))
        torch.cuda.synchronize()
    finally:
        mx.mx_destroy(ctx)
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1])
