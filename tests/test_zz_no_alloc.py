"""The allocation-free entry point gives the same plans as gtmp_solve.

gtmp_solve_noalloc serves callers that may not allocate device memory while
planning (a real-time loop, a plugin whose host owns all device memory): it
takes every input and output from the caller and keeps its scratch in one
fixed device array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test; it must
pass alone in a fresh process as well as after the rest of the suite.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_2608_25830_b300 import binding, scenes

from parity import REL, scene_for

pytestmark = pytest.mark.gpu


def _noalloc(sc, Q, H):
    import torch
    L = Q.shape[0]
    path = torch.full((L,), -7, dtype=torch.int32, device="cuda")
    cost = torch.full((1,), -1.0, dtype=torch.float32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    binding.gtmp_solve_noalloc(sc.robot, sc.spheres, sc.boxes, sc.q_start, sc.q_goal, Q, H, path, cost, status)
    torch.cuda.synchronize()
    return path, cost, status


def _compare_two_calls(sc, M, L, H, seeds):
    p = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
    p.set_scene(sc)
    for seed in seeds:                      # two calls in a row share (and overwrite) the scratch
        p.sample_layers(seed, M)
        ref_path, ref_cost = p.solve()
        Q = p.get_layers()
        path, cost, status = _noalloc(sc, Q, H)
        assert int(status.cpu()[0]) == 0
        got_cost, want_cost = float(cost.cpu()[0]), float(ref_cost.cpu()[0])
        assert math.isinf(got_cost) == math.isinf(want_cost)
        if math.isfinite(want_cost):
            assert abs(got_cost - want_cost) <= REL * want_cost
        np.testing.assert_array_equal(path.cpu().numpy(), ref_path.cpu().numpy())
    p.close()


def _uneven_radii(sc):
    """The same arm with link-sphere radii 0.03 .. 0.05 m: the generic (non-uniform radius) kernel."""
    rob = sc.robot
    ls = rob.link_spheres.copy()
    n = ls.shape[0] * ls.shape[1]
    ls[:, :, 3] = np.linspace(0.03, 0.05, n, dtype=np.float32).reshape(ls.shape[:2])
    robot = dataclasses.replace(rob, link_spheres=np.ascontiguousarray(ls))
    base = dataclasses.replace(sc, robot=robot)
    return scenes.pick_endpoints(base, lambda q: oracle.config_free(base, q))


def test_noalloc_matches_gtmp_solve_arm():
    sc = scene_for("arm", 0, 7, 30)
    _compare_two_calls(sc, 256, 4, 32, seeds=(3, 4))


def test_noalloc_matches_gtmp_solve_point2d():
    sc = scenes.point2d_scene(0, 10)
    _compare_two_calls(sc, 32, 4, 16, seeds=(0, 9))


@pytest.mark.parametrize("dof", [7, 6])
def test_noalloc_odd_obstacle_counts(dof):
    sc = scene_for("arm", 5, dof, 20)                     # 13 spheres + 7 boxes: half-filled pairs
    assert sc.spheres.shape[0] % 2 == 1 and sc.boxes.shape[0] % 2 == 1
    _compare_two_calls(sc, 128, 4, 32, seeds=(1, 2))


def test_noalloc_generic_arm_kernels():
    _compare_two_calls(_uneven_radii(scene_for("arm", 3, 7, 23)), 96, 3, 24, seeds=(5, 6))
    _compare_two_calls(scene_for("arm", 4, 5, 21), 80, 3, 24, seeds=(7, 8))


def test_noalloc_allocates_no_device_memory():
    import torch
    sc = scene_for("arm", 0, 7, 30)
    M, L, H = 256, 4, 32
    p = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
    p.set_scene(sc)
    p.sample_layers(11, M)
    Q = p.get_layers()
    path = torch.empty(L, dtype=torch.int32, device="cuda")
    cost = torch.empty(1, dtype=torch.float32, device="cuda")
    status = torch.empty(1, dtype=torch.int32, device="cuda")
    binding.gtmp_solve_noalloc(sc.robot, sc.spheres, sc.boxes, sc.q_start, sc.q_goal, Q, H, path, cost, status)
    torch.cuda.synchronize()                               # warm-up: one-time set-up of this device
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        binding.gtmp_solve_noalloc(sc.robot, sc.spheres, sc.boxes, sc.q_start, sc.q_goal, Q, H, path, cost, status)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert int(status.cpu()[0]) == 0
    p.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    sc = scene_for("arm", 0, 7, 30)
    L, M = 8, 4096                         # needs about 1.7 MiB of scratch
    Q = torch.zeros((L, M, 7), dtype=torch.float32, device="cuda")
    path = torch.empty(L, dtype=torch.int32, device="cuda")
    cost = torch.empty(1, dtype=torch.float32, device="cuda")
    with pytest.raises(binding.GtmpError) as ei:
        binding.gtmp_solve_noalloc(sc.robot, sc.spheres, sc.boxes, sc.q_start, sc.q_goal, Q, 32, path, cost)
    assert ei.value.status == 1 and "scratch" in str(ei.value)
