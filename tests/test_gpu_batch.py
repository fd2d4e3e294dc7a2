"""Batched persistent solver: every problem equals its single-problem solve
(and the oracle on small cases), under every tiling, eagerly and replayed from
a captured CUDA graph."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2608_25830_b300 import binding, scenes

from parity import REL, check_values, scene_for

pytestmark = pytest.mark.gpu


def _mixed_problems():
    probs = []
    for k in range(4):
        probs.append((scenes.point2d_scene(10 + k, 5 + 9 * k), [32, 97, 64, 200][k], [3, 5, 4, 2][k], 100 + k))
    for k, (dof, M, L) in enumerate([(7, 64, 3), (7, 150, 4), (6, 96, 5), (5, 40, 3), (7, 33, 6), (6, 1, 1)]):
        probs.append((scene_for("arm", 20 + k, dof, 12 + 5 * k), M, L, 200 + k))
    return probs


def _single(sc, M, L, H, seed):
    p = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
    p.set_scene(sc)
    p.sample_layers(seed, M)
    path, cost = p.solve()
    p.synchronize()
    out = path.cpu().numpy(), float(cost.cpu()[0])
    p.close()
    return out


@pytest.fixture(scope="module")
def mixed():
    import torch
    probs = _mixed_problems()
    H = 32
    singles = [_single(sc, M, L, H, seed) for sc, M, L, seed in probs]
    return probs, H, singles


def _check_against_singles(b, probs, singles):
    paths = b.paths.cpu().numpy()
    costs = b.costs.cpu().numpy()
    for k, ((sc, M, L, seed), (p1, c1)) in enumerate(zip(probs, singles)):
        assert (costs[k] == c1) or (math.isinf(costs[k]) and math.isinf(c1)), (k, costs[k], c1)
        np.testing.assert_array_equal(paths[k, :L], p1, err_msg=f"problem {k}")
        assert np.all(paths[k, L:] == -1)


def test_batch_equals_single_solves(mixed):
    probs, H, singles = mixed
    b = binding.Batch(probs, H)
    b.solve()
    b.synchronize()
    _check_against_singles(b, probs, singles)
    assert b.L_max == max(L for _, _, L, _ in probs)
    assert b.nominal_checks == sum(H * (2 * M + (L - 1) * M * M) for _, M, L, _ in probs)
    b.close()


def test_stalled_dependency_times_out_and_the_batch_recovers(mixed):
    """Failure detection without a GPU fault: one dependency of the persistent
    solve is made unreachable on the host; the waiting items give up after
    their bounded wait (~2 s without progress), the others stop at once, the
    error word comes back as GTMP_ERR_TIMEOUT, and after restoring the targets
    the same batch object solves exactly again."""
    import time
    probs, H, singles = mixed
    b = binding.Batch(probs, H)
    L = binding.lib()
    assert L.gtmp_batch_inject_stall(b.handle, 4, 0) == 0       # a 7-DoF problem, L = 3
    t0 = time.time()
    b.solve()
    with pytest.raises(binding.GtmpError) as e:
        b.synchronize()
    assert e.value.status == 4
    assert time.time() - t0 < 60
    assert L.gtmp_batch_inject_stall(b.handle, 4, 3) == 1       # depth L has nothing waiting on it
    assert L.gtmp_batch_inject_stall(b.handle, len(probs), 0) == 1
    assert L.gtmp_batch_inject_stall(b.handle, -1, 0) == 0      # restore
    b.solve()
    b.synchronize()
    _check_against_singles(b, probs, singles)
    b.close()


@pytest.mark.parametrize("target,chunk", [(1, 1), (64, 3), (100, 8), (4096, 16), (1 << 20, 64)])
def test_every_tiling_gives_the_same_plans(mixed, target, chunk):
    probs, H, singles = mixed
    b = binding.Batch(probs, H)
    binding.gtmp_batch_set_tiling(b.handle, target, chunk)
    b.solve()
    b.synchronize()
    _check_against_singles(b, probs, singles)
    b.close()


@pytest.mark.parametrize("point,arm", [((1, 1), (1 << 20, 64)), ((1 << 20, 32), (100, 3))])
def test_per_kind_tilings_give_the_same_plans(mixed, point, arm):
    probs, H, singles = mixed
    b = binding.Batch(probs, H)
    binding.gtmp_batch_set_tiling(b.handle, *point, kind=binding.ROBOT_POINT)
    binding.gtmp_batch_set_tiling(b.handle, *arm, kind=binding.ROBOT_DH_ARM)
    assert binding.gtmp_batch_get_tilings(b.handle) == {binding.ROBOT_POINT: point, binding.ROBOT_DH_ARM: arm}
    b.solve()
    b.synchronize()
    _check_against_singles(b, probs, singles)
    assert binding.lib().gtmp_batch_set_kind_tiling(b.handle, 2, 4096, 8) == 1    # no such robot kind
    b.close()


@pytest.mark.parametrize("target", [1, 4096, 1 << 20])
def test_lazy_batch_gives_the_same_plans(mixed, target):
    probs, H, singles = mixed
    b = binding.Batch(probs, H, eval_mode=binding.EVAL_LAZY)
    binding.gtmp_batch_set_tiling(b.handle, target, 16)
    for _ in range(2):
        b.solve()
        b.synchronize()
        _check_against_singles(b, probs, singles)
    binding.gtmp_batch_set_eval_mode(b.handle, binding.EVAL_EARLY_EXIT)
    b.solve()
    b.synchronize()
    _check_against_singles(b, probs, singles)
    b.close()


def test_batch_rejects_tables_beyond_shared_memory():
    """Every item stages its problem's obstacle table and cost-to-go row (4 B per sample) in at most 200 KB of
    shared memory.  4096 boxes for a 7-joint arm (packed table: 2.5 float4 per box, 160 KB) at M = 16384
    (64 KB) exceed it and are refused at create, before any launch; the same boxes for a point robot (2 float4
    per box, 128 KB) fit and solve."""
    import dataclasses
    rng = np.random.default_rng(3)
    lo = rng.uniform(-1.0, 0.9, (4096, 3))
    boxes = np.concatenate([lo, lo + 0.01], 1).astype(np.float32)
    none = np.zeros((0, 4), np.float32)
    arm = dataclasses.replace(scene_for("arm", 1, 7, 4), spheres=none, boxes=boxes)
    with pytest.raises(binding.GtmpError) as e:
        binding.Batch([(arm, 16384, 1, 1)], 8)
    assert e.value.status == 5     # GTMP_ERR_UNSUPPORTED
    pt = dataclasses.replace(scenes.point2d_scene(1, 4), spheres=none, boxes=boxes)
    b = binding.Batch([(pt, 16384, 1, 1)], 8)
    b.solve()
    b.synchronize()
    b.close()


def test_batch_rejects_full_mode(mixed):
    probs, H, _ = mixed
    b = binding.Batch(probs[:2], H)
    assert binding.lib().gtmp_batch_set_eval_mode(b.handle, binding.EVAL_FULL) == 1
    assert binding.lib().gtmp_batch_set_eval_mode(b.handle, 9) == 1
    b.close()


def test_autotune_keeps_results(mixed):
    probs, H, singles = mixed
    b = binding.Batch(probs, H)
    ms = b.autotune(repeats=1)
    assert ms > 0
    t, c = binding.gtmp_batch_get_tiling(b.handle, binding.ROBOT_POINT)
    assert t in (4096, 16384, 65536, 262144) and c in (4, 8, 16, 32)
    t, c = binding.gtmp_batch_get_tiling(b.handle, binding.ROBOT_DH_ARM)
    assert t in (1024, 4096, 16384, 65536) and c in (4, 8, 16, 32)
    b.solve()
    b.synchronize()
    _check_against_singles(b, probs, singles)
    b.close()


def test_graph_capture_and_replay(mixed):
    import torch
    probs, H, singles = mixed
    b = binding.Batch(probs, H)
    s = torch.cuda.Stream()
    binding.gtmp_batch_set_stream(b.handle, ctypes.c_void_p(s.cuda_stream))
    with torch.cuda.stream(s):
        b.solve()                       # warm-up outside capture
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        binding.gtmp_batch_solve(b.handle, b.paths, b.costs)
    for _ in range(2):
        b.paths.fill_(-5)
        b.costs.fill_(-1.0)
        graph.replay()
        torch.cuda.synchronize()
        b.synchronize()
        _check_against_singles(b, probs, singles)
    b.close()


def test_small_batch_matches_oracle():
    probs = [(scenes.point2d_scene(3, 8), 24, 3, 5), (scene_for("arm", 8, 7, 20), 24, 2, 6),
             (scene_for("arm", 9, 6, 25), 16, 3, 7)]
    H = 16
    b = binding.Batch(probs, H)
    b.solve()
    b.synchronize()
    paths, costs = b.paths.cpu().numpy(), b.costs.cpu().numpy()
    for k, (sc, M, L, seed) in enumerate(probs):
        Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
        sol = oracle.solve(sc, Q, H)
        check_values([costs[k]], [sol.cost_lo], [sol.cost_hi], f"problem {k}")
        if math.isfinite(costs[k]):
            total, worst = oracle.path_cost(sc, Q, paths[k, :L], H)
            assert worst > -oracle.EPS_DEFAULT
            assert costs[k] == pytest.approx(total, rel=REL)
    b.close()
