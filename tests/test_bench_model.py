"""Host logic of bench.py: the byte model of one refinement iteration, the
per-V-cycle roofline fraction and the launch count the bench reports as
gpu_launches.  No GPU needed."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _G:
    def __init__(self, n, lo, hi):
        self.n, self.lo, self.hi = n, lo, hi


class _O:
    def __init__(self, nu1, nu2, fused=0):
        self.nu1, self.nu2, self.fused = nu1, nu2, fused


def test_iteration_bytes_of_the_tuned_planar256_vcycle():
    # (2,3) sweeps in FP32: 8/7 * 4 * (6 * 5 + 7.25) + 64 = 234.3 B per finest cell,
    # the figure an independent recomputation of the model gave for this solve
    assert bench.mac_iteration_bytes_per_cell(2, 3, 4) == pytest.approx(234.2857, abs=1e-3)
    # each extra sweep adds one read of phi, f, b_x, b_y, b_z and a write of phi on all levels
    d = bench.mac_iteration_bytes_per_cell(3, 3, 4) - bench.mac_iteration_bytes_per_cell(2, 3, 4)
    assert d == pytest.approx(8.0 / 7.0 * 6 * 4)
    # the plain FP64 V-cycle doubles the V-cycle words, not the outer 64 B
    assert bench.mac_iteration_bytes_per_cell(2, 3, 8) - 64 == pytest.approx(
        2 * (bench.mac_iteration_bytes_per_cell(2, 3, 4) - 64))


def test_roofline_per_vcycle_is_bytes_over_time_over_peak():
    n = 256 ** 3
    r = bench.roofline_per_vcycle(n, 2, 3, 4, ms_solve=10.25, vcycles=7, hbm=6777.0, loop_ms=8.6)
    b = bench.mac_iteration_bytes_per_cell(2, 3, 4) * n
    assert r["model_bytes_per_vcycle"] == pytest.approx(b)
    assert r["frac"] == pytest.approx(b / (10.25e-3 / 7) / 1e9 / 6777.0, abs=1e-4)
    assert r["loop_only"]["frac"] > r["frac"]


def test_launch_count_of_the_planar256_solve():
    # periodic x,y, walls in z: levels 256^3 .. 2^3, the coarse end from 16^3 (4096 cells);
    # per V-cycle 4 levels x (2*2 + 1 + 1 + 2*3) + update/residual + finalize (+ the
    # graph's condition kernel).  An ncu launch list of the solve from the host loop
    # counted 2647 launches of the library's kernels over 7 solves: 7 x 378 and one fill.
    g = _G((256, 256, 256), (0, 0, 1), (0, 0, 1))
    assert bench.launches_per_solve(g, _O(2, 3), 7, graph=False) == 378
    assert bench.launches_per_solve(g, _O(2, 3), 7, graph=True) == 385


def test_launch_count_without_a_mean_to_remove():
    # a Dirichlet face makes the operator non-singular: the finish has no mean pass
    per = _G((256, 256, 256), (0, 0, 1), (0, 0, 1))
    dir_ = _G((256, 256, 256), (0, 0, 2), (0, 0, 2))
    assert bench.launches_per_solve(per, _O(2, 3), 7, True) - bench.launches_per_solve(dir_, _O(2, 3), 7, True) == 2
