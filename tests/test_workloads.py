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
