"""The seeded input generators: determinism, shapes and the periodic-face convention."""
import numpy as np
import torch

from paper_1908_03634_gb300 import workloads as W


def test_deterministic_and_shapes():
    a, b = W.planar32(), W.planar32()
    g = a.geom
    assert a.rho.shape == (32, 32, 32) and a.sbar.shape == (32, 32, 32)
    for d in range(3):
        assert tuple(a.u[d].shape) == g.face_shape(d)
        assert torch.equal(a.u[d], b.u[d])
    assert torch.equal(a.rho, b.rho)
    assert a.prof_beta0.shape == (32,)


def test_periodic_image_faces_equal():
    w = W.planar(16, 0.2, 0.6, 8, 2, 5)
    assert torch.equal(w.u[0][:, :, 0], w.u[0][:, :, -1])
    assert torch.equal(w.u[1][:, 0, :], w.u[1][:, -1, :])
    assert not torch.equal(w.u[2][0], w.u[2][-1])


def test_recipe_values():
    w = W.planar32()
    z = (np.arange(32) + 0.5) / 32
    rho0 = np.exp(-z / 0.1)
    ratio = (w.rho.numpy() / rho0[:, None, None]) - 1.0
    assert np.abs(ratio).max() <= 0.01 + 1e-15 and np.abs(ratio).max() > 0.009
    s = W.star(16, 4, 2)
    assert s.prof_beta0.shape == (4096,)
    r = (torch.arange(4096, dtype=torch.float64) + 0.5) * s.prof_dr
    expect = torch.where(r <= 0.45, (1 + (r / 0.05) ** 2) ** -2.5, torch.full_like(r, 1e-6)) ** 0.6
    assert torch.allclose(s.prof_beta0, expect, rtol=1e-14)
    # H for the 1e5 contrast over the unit height
    assert abs(np.exp(1.0 / W.H_1E5) - 1e5) < 1e-6


def test_batched_patch_recipe():
    ps = W.batched_patches(npatch=6, sizes=(8, 12, 16))
    assert len(ps) == 6
    for p in ps:
        assert p.geom.n[0] in (8, 12, 16)


def test_composite_workloads_shapes_and_recipe():
    import numpy as np
    from oracle import composite as CP
    for make in (lambda: W.composite_planar(12, (3, 3, 3), (9, 9, 9), 0.2, 0.6, 4, "center", 5),
                 lambda: W.composite_star(12, (4, 4, 4), (8, 8, 8), 4, 6)):
        a, b = make(), make()
        assert torch.equal(a.rho_f, b.rho_f) and torch.equal(a.u_f[2], b.u_f[2])  # seeded
        nf = [2 * (a.phi[d] - a.plo[d]) for d in range(3)]
        assert tuple(a.rho_f.shape) == (nf[2], nf[1], nf[0]) == tuple(a.beta0_f.shape) == tuple(a.sbar_f.shape)
        for d in range(3):
            want = [nf[2], nf[1], nf[0]]
            want[2 - d] += 1
            assert tuple(a.u_f[d].shape) == tuple(want)
            assert tuple(a.u_c[d].shape) == a.geom.face_shape(d)
        # the hotspot at the domain centre lies in the patch, whose centres sample
        # its peak more closely than the coarse ones
        assert float(a.sbar_f.max()) > float(a.sbar_c.max())
        # a valid composite problem: the oracle's projection meets its identity
        G = CP.Composite(a.geom.n, a.geom.dx, a.geom.lo, a.geom.hi, a.plo, a.phi)
        npy = lambda t: t.numpy()
        uc2, uf2, _, _, info = CP.project(G, [npy(x) for x in a.u_c], [npy(x) for x in a.u_f], npy(a.rho_c),
                                          npy(a.beta0_c), npy(a.sbar_c), npy(a.rho_f), npy(a.beta0_f),
                                          npy(a.sbar_f))
        assert info["rel_resid"] <= 1e-12
        dv = (CP.divergence(G, uc2, uf2, npy(a.beta0_c), npy(a.beta0_f))
              - CP.pack(G, npy(a.beta0_c * a.sbar_c), npy(a.beta0_f * a.sbar_f)) - info["mean"])
        assert np.abs(dv).max() <= 1e-11 * np.abs(info["f"]).max()
