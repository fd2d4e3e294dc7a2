"""Weighted-length edge costs (App. "General Costs") on the GPU against the
oracle: per-edge costs, every solve mode, restarts and informed expansion.

Tolerance: a weighted cost adds H float32 weights (each at most W = 1 + sum
a_b) in waypoint order and scales by |v - u| / (H - 1); its relative error
stays below H * 2^-24 * W / 1 ~ 1e-5 / 10 for the H <= 67 and W <= 12 used
here, so the REL = 1e-5 rule of the plain-length tests applies unchanged.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2608_25830_b300 import binding, scenes

from parity import REL, check_values, compare_solution, scene_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _planner(sc, M, L, H, R=1, mode=binding.EVAL_EARLY_EXIT, bumps=None):
    p = binding.Planner(sc.robot, M, L, H, R=R, max_obstacles=64, eval_mode=mode)
    p.set_scene(sc)
    p.set_cost_weight(bumps)
    return p


def _solution(p, unfused=False):
    path, cost = p.solve(unfused=unfused)
    V, S = p.values()
    p.synchronize()
    return V.cpu().numpy(), S.cpu().numpy(), path.cpu().numpy(), float(cost.cpu()[0])


CASES = [
    ("point2d", 2, 32, 4, 16, 0),
    ("point2d", 2, 37, 3, 16, 5),     # ragged M
    ("arm", 7, 48, 3, 32, 1),
    ("arm", 6, 40, 3, 32, 2),
    ("arm", 5, 23, 2, 12, 3),         # generic arm kernel
    ("arm", 7, 20, 2, 67, 7),         # H - 2 > 32: two waypoint rounds per warp
    ("arm", 7, 16, 2, 2, 6),          # H = 2: endpoints only
]


@pytest.mark.parametrize("kind,dof,M,L,H,seed", CASES[:5])
def test_weighted_edge_costs_match_oracle(torch_cuda, kind, dof, M, L, H, seed):
    sc = scene_for(kind, seed, dof, 30 if kind == "arm" else 10)
    b = scenes.weight_bumps(sc, seed)
    p = _planner(sc, M, L, H, bumps=b)
    p.sample_layers(seed, M)
    p.solve(unfused=True)
    Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    n_free = 0
    for l in range(L + 1):
        C = p.edge_costs(l).cpu().numpy()
        lab, cost = oracle.edge_block(sc, verts[l], verts[l + 1], H, bumps=b)
        clear = lab != oracle.AMBIGUOUS
        np.testing.assert_array_equal(np.isinf(C)[clear], (lab == oracle.COLLIDE)[clear], err_msg=f"layer {l}")
        free = lab == oracle.FREE
        np.testing.assert_allclose(C[free], cost[free], rtol=REL, err_msg=f"layer {l}")
        n_free += int(free.sum())
        _, length = oracle.edge_block(sc, verts[l], verts[l + 1], H)
        assert np.all(C[free] >= length[free] * (1 - REL))           # w >= 1
    assert n_free > 0


@pytest.mark.parametrize("kind,dof,M,L,H,seed", CASES)
@pytest.mark.parametrize("mode", [binding.EVAL_EARLY_EXIT, binding.EVAL_FULL, binding.EVAL_LAZY])
def test_weighted_solve_matches_oracle(torch_cuda, kind, dof, M, L, H, seed, mode):
    sc = scene_for(kind, seed, dof, 30 if kind == "arm" else 10)
    b = scenes.weight_bumps(sc, seed)
    p = _planner(sc, M, L, H, mode=mode, bumps=b)
    p.sample_layers(seed, M)
    V, S, path, cost = _solution(p)
    Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    sol = oracle.solve(sc, Q, H, bumps=b)
    compare_solution(sol, V, S, path, cost, f"weighted {kind} M={M} L={L} H={H} mode={mode}")
    if math.isfinite(cost):
        total, worst = oracle.path_cost(sc, Q, path, H, bumps=b)
        assert worst > -oracle.EPS_DEFAULT
        assert cost == pytest.approx(total, rel=REL)


@pytest.mark.parametrize("kind,dof,M,L,H,seed", CASES[:6])
def test_weighted_modes_and_unfused_agree_exactly(torch_cuda, kind, dof, M, L, H, seed):
    """Lane-per-waypoint (early exit, full, unfused) and lane-per-edge (lazy,
    point robot) forms of the weighted cost give the same bits."""
    sc = scene_for(kind, seed, dof, 30 if kind == "arm" else 10)
    b = scenes.weight_bumps(sc, seed)
    outs = []
    for mode in (binding.EVAL_EARLY_EXIT, binding.EVAL_FULL, binding.EVAL_LAZY):
        p = _planner(sc, M, L, H, mode=mode, bumps=b)
        p.sample_layers(seed, M)
        outs.append(_solution(p))
        outs.append(_solution(p, unfused=True))
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
        np.testing.assert_array_equal(o[2], outs[0][2])
        assert o[3] == outs[0][3]


@pytest.mark.parametrize("kind,dof", [("point2d", 2), ("arm", 7)])
def test_zero_weight_and_reset_give_the_plain_solve(torch_cuda, kind, dof):
    """Amplitude 0 makes every weight exactly 1 and the trapezoid sum exactly
    H - 1, so the cost is the length bit for bit; K = 0 restores the plain path."""
    sc = scene_for(kind, 2, dof, 30 if kind == "arm" else 10)
    M, L, H = 32, 3, 16
    plain = _planner(sc, M, L, H)
    plain.sample_layers(4, M)
    ref = _solution(plain)
    b = scenes.weight_bumps(sc, 2)
    b[:, -1] = 0.0
    for mode in (binding.EVAL_EARLY_EXIT, binding.EVAL_LAZY):
        p = _planner(sc, M, L, H, mode=mode, bumps=b)
        p.sample_layers(4, M)
        got = _solution(p)
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[2], ref[2])
        heavy = scenes.weight_bumps(sc, 2)
        p.set_cost_weight(heavy)
        w = _solution(p)
        if math.isfinite(ref[3]):
            assert w[3] > ref[3]                                   # every chain costs more
        p.set_cost_weight(None)
        back = _solution(p)
        np.testing.assert_array_equal(back[0], ref[0])
        np.testing.assert_array_equal(back[2], ref[2])


def test_weighted_anytime_restarts_match_oracle(torch_cuda):
    sc = scene_for("arm", 3, 6, 30)
    b = scenes.weight_bumps(sc, 3)
    R, M, L, H = 4, 24, 3, 16
    p = _planner(sc, M, L, H, R=R, bumps=b)
    paths, costs, best = p.anytime(21, R)
    p.synchronize()
    paths, costs, best = paths.cpu().numpy(), costs.cpu().numpy(), int(best.cpu()[0])
    sols = oracle.anytime(sc, 21, R, L, M, H, bumps=b)
    for r in range(R):
        V, S = p.values(r)
        compare_solution(sols[r], V.cpu().numpy(), S.cpu().numpy(), paths[r], costs[r], f"weighted restart {r}")


def test_weighted_ao_stages_match_oracle(torch_cuda):
    """Informed expansion keeps its ellipsoid under a weighted cost (w >= 1:
    a weighted cost bounds the length), so the stages stay bit-exact."""
    torch = torch_cuda
    sc = scene_for("arm", 4, 6, 30)
    b = scenes.weight_bumps(sc, 4)
    L, H, dof = 4, 16, 6
    sizes = [8, 16, 32]
    p = _planner(sc, sizes[-1], L, H, bumps=b)
    stage_path = torch.empty(L, dtype=torch.int32, device="cuda")
    stage_cost = torch.empty(1, dtype=torch.float32, device="cuda")
    best_path = torch.full((L,), -1, dtype=torch.int32, device="cuda")
    best_cost = torch.full((1,), math.inf, dtype=torch.float32, device="cuda")
    Q_ref = np.zeros((L, 0, dof), np.float32)
    for M in sizes:
        c_in = float(best_cost.cpu()[0])
        binding.aogtmp_expand(p.ctx, 99, M, stage_path, stage_cost, best_path, best_cost)
        p.synchronize()
        st, Q_ref = oracle.expand_layers(99, Q_ref, M, sc.q_start, sc.q_goal, sc.robot.q_lo, sc.robot.q_hi,
                                         np.float32(c_in))
        assert st == 0
        Q = p.get_layers().cpu().numpy()
        np.testing.assert_array_equal(Q.view(np.uint32), Q_ref.view(np.uint32), err_msg=f"stage M={M}")
        sol = oracle.solve(sc, Q_ref, H, bumps=b)
        V, S = p.values()
        compare_solution(sol, V.cpu().numpy(), S.cpu().numpy(), stage_path.cpu().numpy(),
                         float(stage_cost.cpu()[0]), f"weighted AO stage M={M}")


def test_cost_weight_rejects_bad_bumps(torch_cuda):
    sc = scenes.point2d_scene(0, 4)
    p = _planner(sc, 8, 2, 8)
    ok = np.array([[0.0, 0.0, 0.5, 1.0]], np.float32)
    L = binding.lib()
    f = binding._f32
    for bad, K in [(ok, -1), (np.repeat(ok, 17, axis=0), 17), (np.array([[0.0, 0.0, 0.0, 1.0]], np.float32), 1),
                   (np.array([[0.0, 0.0, 0.5, -1.0]], np.float32), 1),
                   (np.array([[np.nan, 0.0, 0.5, 1.0]], np.float32), 1),
                   (np.array([[0.0, 0.0, 1e-30, 1.0]], np.float32), 1),
                   (np.array([[0.0, 0.0, 0.5, 3e38], [0.0, 0.0, 0.5, 3e38]], np.float32), 2)]:
        b = f(bad)
        assert L.gtmp_set_cost_weight(p.ctx, binding._ptr(b), K) == 1, (bad, K)
    assert L.gtmp_set_cost_weight(p.ctx, None, 1) == 1
    assert L.gtmp_set_cost_weight(p.ctx, None, 0) == 0
    assert L.gtmp_set_cost_weight(p.ctx, binding._ptr(f(ok)), 1) == 0
