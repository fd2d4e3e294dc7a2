"""Parity of the CUDA planner (through the C ABI) with the CPU oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2608_25830_b300 import binding, scenes

from parity import REL, check_values, compare_solution, decisive, scene_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _planner(sc, M, L, H, R=1, mode=binding.EVAL_EARLY_EXIT, max_edge_len=math.inf, max_obstacles=64):
    p = binding.Planner(sc.robot, M, L, H, R=R, max_obstacles=max_obstacles, eval_mode=mode,
                        max_edge_len=max_edge_len)
    p.set_scene(sc)
    return p


def _gpu_solution(p, unfused=False):
    path, cost = p.solve(unfused=unfused)
    V, S = p.values()
    p.synchronize()
    return V.cpu().numpy(), S.cpu().numpy(), path.cpu().numpy(), float(cost.cpu()[0])


# ---------------------------------------------------------------------------
# samples: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,dof,M,L,seed", [("point2d", 2, 32, 4, 0), ("arm", 7, 100, 3, 5), ("arm", 6, 33, 2, 2**40 + 3)])
def test_uniform_samples_bit_exact(torch_cuda, kind, dof, M, L, seed):
    sc = scene_for(kind, 0, dof, 10)
    p = _planner(sc, M, L, 4)
    p.sample_layers(seed, M)
    Q = p.get_layers().cpu().numpy()
    ref = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    assert Q.dtype == np.float32
    np.testing.assert_array_equal(Q.view(np.uint32), ref.view(np.uint32))


# ---------------------------------------------------------------------------
# exact checker: configuration labels
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,dof,n_obs", [("point2d", 2, 10), ("arm", 7, 30), ("arm", 6, 40), ("arm", 5, 12)])
def test_config_labels_match_outside_band(torch_cuda, kind, dof, n_obs):
    torch = torch_cuda
    sc = scene_for(kind, 1, dof, n_obs)
    p = _planner(sc, 8, 1, 4)
    rng = np.random.default_rng(7)
    q = rng.uniform(sc.robot.q_lo, sc.robot.q_hi, (20000, dof)).astype(np.float32)
    gpu = p.label_configs(torch.from_numpy(q).cuda()).cpu().numpy()
    lab, margin = oracle.config_labels(sc, q)
    clear = lab != oracle.AMBIGUOUS
    np.testing.assert_array_equal(gpu[clear], (lab[clear] == oracle.COLLIDE).astype(np.uint8))
    assert 0.05 < gpu.mean() < 0.95  # the scene has both free and colliding configurations


def test_joint_sincos_against_fp64(torch_cuda):
    """The kinematics' own sine and cosine (Cody-Waite reduction by pi/2, Taylor series on |r| <= pi/4) stay
    within 1e-7 of FP64 over the whole argument range the joint bounds allow (|x| <= 6144), including the
    quadrant boundaries, zero and tiny arguments."""
    torch = torch_cuda
    rng = np.random.default_rng(5)
    k = np.arange(-3911, 3912)
    xs = np.concatenate([rng.uniform(-8, 8, 200000), rng.uniform(-6144, 6144, 200000),
                         k * (np.pi / 2), k * (np.pi / 2) + 1e-4, k * (np.pi / 4),
                         [0.0, -0.0, 1e-30, -1e-30, 1e-7, 6144.0, -6144.0]]).astype(np.float32)
    s, c = binding.gtmp_joint_sincos(torch.from_numpy(xs).cuda())
    s, c = s.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)
    x64 = xs.astype(np.float64)
    assert np.abs(s - np.sin(x64)).max() <= 1e-7
    assert np.abs(c - np.cos(x64)).max() <= 1e-7
    assert np.all(s[xs == 0.0] == 0.0) and np.all(c[xs == 0.0] == 1.0)
    assert binding.lib().gtmp_joint_sincos(None, -1, None, None, None) == 1


def test_arm_angle_bounds_are_enforced(torch_cuda):
    """Joint limits beyond +-4096 rad or a theta offset beyond +-2048 rad are refused at create; the label
    query marks a configuration with a coordinate beyond +-4096 rad (or NaN) as colliding."""
    import dataclasses
    torch = torch_cuda
    from paper_2608_25830_b300 import scenes
    base = scenes.dh_arm(3, 7)
    wide = dataclasses.replace(base, q_lo=np.full(7, -5000.0, np.float32), q_hi=np.full(7, 5000.0, np.float32))
    with pytest.raises(binding.GtmpError):
        binding.Planner(wide, 8, 1, 4)
    dh = base.dh.copy()
    dh[2, 3] = 3000.0
    with pytest.raises(binding.GtmpError):
        binding.Planner(dataclasses.replace(base, dh=dh), 8, 1, 4)
    edge = dataclasses.replace(base, q_lo=np.full(7, -4096.0, np.float32), q_hi=np.full(7, 4096.0, np.float32))
    q0 = np.zeros(7, np.float32)
    sc = scenes.Scene(edge, np.zeros((0, 4), np.float32), np.zeros((0, 6), np.float32), q0, q0)
    p = _planner(sc, 8, 1, 4)
    q = np.zeros((4, 7), np.float32)
    q[1, 3] = 4096.0
    q[2, 3] = 4097.0
    q[3, 5] = np.nan
    lab = p.label_configs(torch.from_numpy(q).cuda()).cpu().numpy()
    assert lab.tolist() == [0, 0, 1, 1]   # no obstacles: only the out-of-range rows are labelled colliding
    p.close()


@pytest.mark.parametrize("radius", [0.5, 0.99, 1.0, 1.5])
def test_config_labels_with_far_boxes_and_large_spheres(torch_cuda, radius):
    """The packed arm kernels clamp each box-axis gap at 1 (one saturating add), which decides the same as the
    plain gap only for robot spheres of radius below 1; larger radii take the generic kernel.  Boxes r + 0.5 to
    r + 2 m from the base make gaps above 1 common (about half the configurations collide), and the labels
    still equal the oracle's on both sides of r = 1."""
    import dataclasses
    torch = torch_cuda
    from paper_2608_25830_b300 import scenes
    rng = np.random.default_rng(11)
    robot = scenes.dh_arm(5, 7)
    sph = robot.link_spheres.copy()
    sph[:, :, 3] = radius
    robot = dataclasses.replace(robot, link_spheres=sph)
    d = rng.normal(size=(12, 3))
    c = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(radius + 0.5, radius + 2.0, (12, 1))
    h = rng.uniform(0.05, 0.3, (12, 3))
    boxes = np.concatenate([c - h, c + h], 1).astype(np.float32)
    q0 = np.zeros(7, np.float32)
    sc = scenes.Scene(robot, np.zeros((0, 4), np.float32), boxes, q0, q0)
    p = _planner(sc, 8, 1, 4)
    q = rng.uniform(robot.q_lo, robot.q_hi, (20000, 7)).astype(np.float32)
    gpu = p.label_configs(torch.from_numpy(q).cuda()).cpu().numpy()
    lab, margin = oracle.config_labels(sc, q)
    clear = lab != oracle.AMBIGUOUS
    np.testing.assert_array_equal(gpu[clear], (lab[clear] == oracle.COLLIDE).astype(np.uint8))
    assert 0.2 < gpu.mean() < 0.8
    p.close()


# ---------------------------------------------------------------------------
# unfused edge costs: labels and lengths per edge
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,dof,M,L,H", [("point2d", 2, 32, 4, 16), ("arm", 7, 40, 3, 32), ("arm", 6, 29, 2, 40)])
def test_edge_costs_match_oracle(torch_cuda, kind, dof, M, L, H):
    sc = scene_for(kind, 2, dof, 30 if kind == "arm" else 10)
    p = _planner(sc, M, L, H)
    p.sample_layers(11, M)
    p.solve(unfused=True)
    Q = oracle.sample_uniform(11, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    vl, _ = oracle.config_labels(sc, np.concatenate(verts))
    for l in range(L + 1):
        C = p.edge_costs(l).cpu().numpy()
        lab, cost = oracle.edge_block(sc, verts[l], verts[l + 1], H)
        clear = lab != oracle.AMBIGUOUS
        np.testing.assert_array_equal(np.isinf(C)[clear], (lab == oracle.COLLIDE)[clear], err_msg=f"layer {l}")
        free = lab == oracle.FREE
        np.testing.assert_allclose(C[free], cost[free], rtol=REL)


# ---------------------------------------------------------------------------
# fused solve: values, minimisers, path, cost
# ---------------------------------------------------------------------------

CASES = [
    ("point2d", 2, 32, 4, 16, 0),     # the 2D point-robot workload itself
    ("point2d", 2, 37, 3, 16, 5),     # ragged M
    ("arm", 7, 48, 3, 32, 1),
    ("arm", 6, 64, 4, 32, 2),
    ("arm", 5, 23, 2, 12, 3),         # generic (non-specialised) arm kernel
    ("arm", 7, 1, 1, 32, 4),          # M = 1, L = 1
    ("arm", 7, 40, 2, 2, 6),          # H = 2: endpoints only
    ("arm", 7, 20, 2, 67, 7),         # H - 2 > 32: two waypoint rounds per warp
]


@pytest.mark.parametrize("kind,dof,M,L,H,seed", CASES)
@pytest.mark.parametrize("mode", [binding.EVAL_EARLY_EXIT, binding.EVAL_FULL, binding.EVAL_LAZY])
def test_fused_solve_matches_oracle(torch_cuda, kind, dof, M, L, H, seed, mode):
    sc = scene_for(kind, seed, dof, 30 if kind == "arm" else 10)
    p = _planner(sc, M, L, H, mode=mode)
    p.sample_layers(seed, M)
    V, S, path, cost = _gpu_solution(p)
    Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    sol = oracle.solve(sc, Q, H)
    compare_solution(sol, V, S, path, cost, f"{kind} M={M} L={L} H={H} mode={mode}")
    if math.isfinite(cost):
        total, worst = oracle.path_cost(sc, Q, path, H)
        assert worst > -oracle.EPS_DEFAULT
        assert cost == pytest.approx(total, rel=REL)
        assert cost >= float(np.linalg.norm(sc.q_goal.astype(np.float64) - sc.q_start)) * (1 - REL)


@pytest.mark.parametrize("kind,dof,M,L,H,seed", CASES)
def test_lazy_path_solve_matches_plain_and_oracle(torch_cuda, kind, dof, M, L, H, seed):
    """Path-level lazy evaluation (optimistic min-plus sweeps, the winning chain checked exactly, its colliding
    edges left out, repeated): its cost equals gtmp_solve's bit for bit (optimistic costs bound the true ones
    from below and rounding is monotone, so the verified chain's float cost is the plain optimum), lies in the
    oracle's [V_lo, V_hi] band, and the chain it returns is free when the oracle re-checks it."""
    torch = torch_cuda
    sc = scene_for(kind, seed, dof, 30 if kind == "arm" else 10)
    p = _planner(sc, M, L, H)
    p.sample_layers(seed, M)
    _, plain_cost = p.solve()
    plain_cost = float(plain_cost.cpu()[0])
    path = torch.empty(L, dtype=torch.int32, device="cuda")
    cost = torch.empty(1, dtype=torch.float32, device="cuda")
    st = binding.gtmp_solve_lazy_path(p.ctx, path, cost)
    path, cost = path.cpu().numpy(), float(cost.cpu()[0])
    assert cost == plain_cost or (math.isinf(cost) and math.isinf(plain_cost))
    assert st["iterations"] >= 1 and st["colliding_edges"] >= st["iterations"] - 1
    Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    sol = oracle.solve(sc, Q, H)
    check_values([cost], [sol.cost_lo], [sol.cost_hi], f"{kind} M={M} L={L} lazy path")
    if math.isfinite(cost):
        total, worst = oracle.path_cost(sc, Q, path, H)
        assert worst > -oracle.EPS_DEFAULT, "returned chain collides"
        assert cost == pytest.approx(total, rel=REL)
    else:
        assert list(path) == [-1] * L
    p.close()


def test_lazy_path_weighted_goal_set_and_iteration_cap(torch_cuda):
    """Weighted-length costs and a goal set with terminal values go through the optimistic sweep as through
    gtmp_solve (equal costs); a cap of one iteration on a scene whose first optimistic chain collides ends
    with GTMP_ERR_TIMEOUT."""
    torch = torch_cuda
    from paper_2608_25830_b300 import scenes
    sc = scene_for("arm", 3, 7, 30)
    M, L, H = 96, 4, 32
    p = _planner(sc, M, L, H)
    p.set_cost_weight(scenes.weight_bumps(sc, 3))
    path = torch.empty(L, dtype=torch.int32, device="cuda")
    cost = torch.empty(1, dtype=torch.float32, device="cuda")
    capped = False
    for seed in (5, 6, 7):
        p.sample_layers(seed, M)
        _, plain_cost = p.solve()
        plain_cost = float(plain_cost.cpu()[0])
        st = binding.gtmp_solve_lazy_path(p.ctx, path, cost)
        assert float(cost.cpu()[0]) == plain_cost or math.isinf(plain_cost)
        if st["iterations"] > 1:
            with pytest.raises(binding.GtmpError) as e:
                binding.gtmp_solve_lazy_path(p.ctx, path, cost, max_iterations=1)
            assert e.value.status == 4   # GTMP_ERR_TIMEOUT
            capped = True
    assert capped, "no scene needed a second iteration: the cap is untested"
    rng = np.random.default_rng(9)
    goals = np.stack([sc.q_goal, sc.q_start * 0.5 + sc.q_goal * 0.5]).astype(np.float32)
    free = p.label_configs(torch.from_numpy(goals).cuda()).cpu().numpy() == 0
    goals = goals[free]
    if len(goals):
        binding.gtmp_set_goals(p.ctx, goals, rng.uniform(0.0, 0.5, len(goals)).astype(np.float32))
        p.sample_layers(11, M)
        _, plain_cost = p.solve()
        binding.gtmp_solve_lazy_path(p.ctx, path, cost)
        assert float(cost.cpu()[0]) == float(plain_cost.cpu()[0]) or math.isinf(float(plain_cost.cpu()[0]))
    assert binding.lib().gtmp_solve_lazy_path(p.ctx, 0, None, None, None) == 1
    p.close()


@pytest.mark.parametrize("kind,dof,M,L,H,seed", CASES[:5])
def test_fused_unfused_and_modes_agree_exactly(torch_cuda, kind, dof, M, L, H, seed):
    sc = scene_for(kind, seed, dof, 30 if kind == "arm" else 10)
    outs = []
    for mode in (binding.EVAL_EARLY_EXIT, binding.EVAL_FULL, binding.EVAL_LAZY):
        p = _planner(sc, M, L, H, mode=mode)
        p.sample_layers(seed, M)
        outs.append(_gpu_solution(p))
        outs.append(_gpu_solution(p, unfused=True))
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
        np.testing.assert_array_equal(o[2], outs[0][2])
        assert o[3] == outs[0][3] or (math.isnan(o[3]) and math.isnan(outs[0][3]))


def test_infeasible_and_edge_limit(torch_cuda):
    sc = scenes.point2d_scene(0, 10)
    wall = scenes.Scene(sc.robot, np.array([[0.0, 0.0, 0.0, 0.7]], np.float32), np.zeros((0, 6), np.float32),
                        sc.q_start, sc.q_goal)
    blocked = scenes.Scene(sc.robot, np.concatenate([wall.spheres, [[0.9, 0.9, 0.0, 0.05]]]).astype(np.float32),
                           wall.boxes, sc.q_start, sc.q_goal)   # the goal itself is covered
    p = _planner(blocked, 16, 2, 8)
    p.sample_layers(1, 16)
    V, S, path, cost = _gpu_solution(p)
    assert math.isinf(cost) and list(path) == [-1, -1]
    # an edge-length limit shorter than any possible hop
    p2 = _planner(sc, 16, 2, 8, max_edge_len=0.05)
    p2.sample_layers(1, 16)
    _, _, path2, cost2 = _gpu_solution(p2)
    assert math.isinf(cost2) and list(path2) == [-1, -1]


def test_no_obstacles_collinear_samples(torch_cuda):
    torch = torch_cuda
    sc = scenes.point2d_scene(0, 0)
    L, M = 3, 8
    rng = np.random.default_rng(0)
    Q = rng.uniform(-1, 1, (L, M, 2)).astype(np.float32)
    for l, t in enumerate([0.25, 0.5, 0.75]):
        Q[l, 5] = sc.q_start + np.float32(t) * (sc.q_goal - sc.q_start)
    p = _planner(sc, M, L, 8)
    p.set_layers(torch.from_numpy(Q).cuda())
    _, _, path, cost = _gpu_solution(p)
    assert list(path) == [5, 5, 5]
    assert cost == pytest.approx(float(np.linalg.norm(sc.q_goal.astype(np.float64) - sc.q_start)), rel=REL)


# ---------------------------------------------------------------------------
# anytime-gtmp: every restart is an independent gtmp
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [binding.EVAL_EARLY_EXIT, binding.EVAL_LAZY])
def test_anytime_restarts_match_oracle(torch_cuda, mode):
    sc = scene_for("arm", 3, 6, 30)
    R, M, L, H = 6, 24, 3, 16
    p = _planner(sc, M, L, H, R=R, mode=mode)
    paths, costs, best = p.anytime(21, R)
    p.synchronize()
    paths, costs, best = paths.cpu().numpy(), costs.cpu().numpy(), int(best.cpu()[0])
    sols = oracle.anytime(sc, 21, R, L, M, H)
    for r in range(R):
        check_values([costs[r]], [sols[r].cost_lo], [sols[r].cost_hi], f"restart {r}")
        V, S = p.values(r)
        compare_solution(sols[r], V.cpu().numpy(), S.cpu().numpy(), paths[r], costs[r], f"restart {r}")
    fin = np.isfinite(costs)
    if fin.any():
        assert costs[best] == costs[fin].min() and best == int(np.argmin(np.where(fin, costs, np.inf)))
    else:
        assert best == -1


# ---------------------------------------------------------------------------
# AO-GTMP: expand-samples bit-exact stage by stage, non-increasing best cost
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,dof,mode", [("arm", 6, binding.EVAL_EARLY_EXIT), ("point2d", 2, binding.EVAL_EARLY_EXIT),
                                           ("arm", 6, binding.EVAL_LAZY)])
def test_ao_stages_match_oracle(torch_cuda, kind, dof, mode):
    torch = torch_cuda
    sc = scene_for(kind, 4, dof, 30 if kind == "arm" else 12)
    L, H = 4, 16
    sizes = [8, 16, 32, 64]
    p = _planner(sc, sizes[-1], L, H, mode=mode)
    stage_path = torch.empty(L, dtype=torch.int32, device="cuda")
    stage_cost = torch.empty(1, dtype=torch.float32, device="cuda")
    best_path = torch.full((L,), -1, dtype=torch.int32, device="cuda")
    best_cost = torch.full((1,), math.inf, dtype=torch.float32, device="cuda")
    Q_ref = np.zeros((L, 0, dof), np.float32)
    prev_best = math.inf
    for M in sizes:
        c_in = float(best_cost.cpu()[0])
        binding.aogtmp_expand(p.ctx, 99, M, stage_path, stage_cost, best_path, best_cost)
        p.synchronize()
        st, Q_ref = oracle.expand_layers(99, Q_ref, M, sc.q_start, sc.q_goal, sc.robot.q_lo, sc.robot.q_hi,
                                         np.float32(c_in))
        assert st == 0
        Q = p.get_layers().cpu().numpy()
        np.testing.assert_array_equal(Q.view(np.uint32), Q_ref.view(np.uint32), err_msg=f"stage M={M}")
        sol = oracle.solve(sc, Q_ref, H)
        V, S = p.values()
        compare_solution(sol, V.cpu().numpy(), S.cpu().numpy(), stage_path.cpu().numpy(),
                         float(stage_cost.cpu()[0]), f"AO stage M={M}")
        b = float(best_cost.cpu()[0])
        assert b <= prev_best
        prev_best = b
        assert b == min(c_in, float(stage_cost.cpu()[0]))


# ---------------------------------------------------------------------------
# goal sets with terminal values (Alg. 1's G and V_g)
# ---------------------------------------------------------------------------

def _goal_set(sc, seed, G=3):
    """The scene's goal plus seeded configurations the oracle finds free."""
    rng = np.random.default_rng(seed + 100)
    cand = rng.uniform(sc.robot.q_lo, sc.robot.q_hi, (256, sc.robot.dof)).astype(np.float32)
    free = oracle.config_free(sc, cand)
    return np.array([sc.q_goal] + [c for c, f in zip(cand, free) if f][:G - 1], np.float32)


@pytest.mark.parametrize("kind,dof,M,L,H,seed", [("point2d", 2, 32, 3, 16, 1), ("arm", 7, 40, 3, 32, 2),
                                                 ("arm", 6, 24, 2, 16, 3)])
@pytest.mark.parametrize("mode", [binding.EVAL_EARLY_EXIT, binding.EVAL_FULL, binding.EVAL_LAZY])
@pytest.mark.parametrize("with_values", [False, True])
def test_goal_set_matches_oracle(torch_cuda, kind, dof, M, L, H, seed, mode, with_values):
    torch = torch_cuda
    sc = scene_for(kind, seed, dof, 30 if kind == "arm" else 10)
    goals = _goal_set(sc, seed)
    vals = np.array([0.6, 0.0, 0.3], np.float32)[:len(goals)] if with_values else None
    p = _planner(sc, M, L, H, mode=mode)
    binding.gtmp_set_goals(p.ctx, goals, vals)
    p.sample_layers(seed, M)
    V, S, path, cost = _gpu_solution(p)
    Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    sol = oracle.solve(sc, Q, H, goals=goals, goal_values=vals)
    compare_solution(sol, V, S, path, cost, f"{kind} goals mode={mode} values={with_values}")
    goal = torch.empty(1, dtype=torch.int32, device="cuda")
    binding.gtmp_get_goal_reached(p.ctx, 0, goal)
    p.synchronize()
    g = int(goal.cpu()[0])
    if not math.isfinite(cost):
        assert g == -1
        return
    assert 0 <= g < len(goals)
    last = int(path[-1])
    if decisive(sol, L)[last] and list(path) == list(sol.path):
        assert g == sol.sigma[L][last]
    # the chain through the reached goal costs what the planner returned
    verts = [sc.q_start] + [Q[l, path[l]] for l in range(L)] + [goals[g]]
    total = sum(oracle.lib().orc_edge_length(dof, oracle._ptr(oracle._c32(a), oracle._f32p),
                                             oracle._ptr(oracle._c32(b), oracle._f32p))
                for a, b in zip(verts[:-1], verts[1:]))
    total += 0.0 if vals is None else float(vals[g])
    assert cost == pytest.approx(total, rel=REL)


def test_single_goal_set_equals_endpoints(torch_cuda):
    sc = scene_for("arm", 5, 7, 30)
    M, L, H = 48, 3, 32
    outs = []
    for use_set in (False, True):
        p = _planner(sc, M, L, H)
        if use_set:
            binding.gtmp_set_goals(p.ctx, sc.q_goal[None, :], None)
        p.sample_layers(9, M)
        outs.append(_gpu_solution(p))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


def test_goal_set_restarts_and_ao_guard(torch_cuda):
    torch = torch_cuda
    sc = scene_for("arm", 3, 6, 30)
    R, M, L, H = 3, 20, 2, 16
    goals = _goal_set(sc, 3)
    vals = np.array([0.2, 0.0, 0.5], np.float32)
    p = _planner(sc, M, L, H, R=R)
    binding.gtmp_set_goals(p.ctx, goals, vals)
    paths, costs, best = p.anytime(21, R)
    p.synchronize()
    costs = costs.cpu().numpy()
    for r in range(R):
        Q = oracle.sample_uniform(21, r, L, M, sc.robot.q_lo, sc.robot.q_hi)
        sol = oracle.solve(sc, Q, H, goals=goals, goal_values=vals)
        check_values([costs[r]], [sol.cost_lo], [sol.cost_hi], f"restart {r}")
    # informed expansion is defined for one goal
    p2 = _planner(sc, 64, L, H)
    binding.gtmp_set_goals(p2.ctx, goals, None)
    t = lambda *s, d=torch.int32: torch.empty(*s, dtype=d, device="cuda")
    with pytest.raises(binding.GtmpError, match="UNSUPPORTED"):
        binding.aogtmp_expand(p2.ctx, 1, 16, t(L), t(1, d=torch.float32), t(L), t(1, d=torch.float32))


# ---------------------------------------------------------------------------
# layer sampling on C_free by rejection
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,dof,M,L,seed", [("point2d", 2, 64, 3, 3), ("arm", 7, 100, 3, 5), ("arm", 6, 50, 2, 9)])
def test_free_samples_bit_exact(torch_cuda, kind, dof, M, L, seed):
    torch = torch_cuda
    sc = scene_for(kind, 1, dof, 30 if kind == "arm" else 14)
    p = _planner(sc, M, L, 4)
    binding.gtmp_set_sampler(p.ctx, binding.SAMPLER_FREE, 128)
    p.sample_layers(seed, M)
    Q = p.get_layers().cpu().numpy()
    ref, used, und = oracle.sample_free(sc, seed, 0, L, M, max_attempts=128)
    decided = ~und
    assert decided.mean() > 0.99
    np.testing.assert_array_equal(Q[decided].view(np.uint32), ref[decided].view(np.uint32))
    lab = p.label_configs(torch.from_numpy(np.ascontiguousarray(Q.reshape(-1, dof))).cuda()).cpu().numpy()
    assert np.all(lab.reshape(L, M)[used >= 0] == 0)
    assert (used >= 1).any()       # some uniform samples collided and were redrawn


def test_free_sampler_restarts_match_oracle(torch_cuda):
    sc = scene_for("arm", 3, 6, 30)
    R, M, L, H = 3, 24, 3, 16
    p = _planner(sc, M, L, H, R=R)
    binding.gtmp_set_sampler(p.ctx, binding.SAMPLER_FREE, 64)
    paths, costs, best = p.anytime(33, R)
    p.synchronize()
    costs = costs.cpu().numpy()
    for r in range(R):
        Q, used, und = oracle.sample_free(sc, 33, r, L, M, max_attempts=64)
        if und.any():
            continue
        sol = oracle.solve(sc, Q, H)
        V, S = p.values(r)
        compare_solution(sol, V.cpu().numpy(), S.cpu().numpy(), paths[r].cpu().numpy(), costs[r], f"free restart {r}")


# ---------------------------------------------------------------------------
# obstacle counts around the checker's table limits: the link cull with its
# masked exact tests (<= 32 sphere pairs and <= 32 box pairs), the per-sphere
# prefilter it falls back to beyond that, and no cull table at all when the
# tables would not fit in shared memory
# ---------------------------------------------------------------------------

def _many_obstacles_scene(n_s, n_b, n_far, seed):
    """n_s spheres and n_b boxes around the arm (outside a 0.4 m ball about its base), plus n_far small
    spheres beyond its reach: they fill the tables without blocking every path."""
    base = scene_for("arm", 7, 7, 0)
    rng = np.random.default_rng(seed)
    cs = rng.uniform(-0.75, 0.75, (8 * n_s + 8, 3))
    cs = cs[np.linalg.norm(cs, axis=1) > 0.4][:n_s]
    spheres = np.concatenate([cs, rng.uniform(0.01, 0.025, (len(cs), 1))], 1)
    d = rng.normal(size=(n_far, 3))
    far = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(3.0, 4.0, (n_far, 1))
    spheres = np.concatenate([spheres, np.concatenate([far, np.full((n_far, 1), 0.01)], 1)]).astype(np.float32)
    cb = rng.uniform(-0.75, 0.75, (8 * n_b + 8, 3))
    cb = cb[np.linalg.norm(cb, axis=1) > 0.45][:n_b]
    h = rng.uniform(0.01, 0.03, (len(cb), 3))
    boxes = np.concatenate([cb - h, cb + h], 1).astype(np.float32)
    assert len(spheres) == n_s + n_far and len(boxes) == n_b
    sc = scenes.Scene(base.robot, spheres, boxes, base.q_start, base.q_goal, base.candidates)
    return scenes.pick_endpoints(sc, lambda q: oracle.config_free(sc, q))


@pytest.mark.parametrize("n_s,n_b,n_far,M,L,H", [
    (64, 60, 0, 48, 2, 16),         # 32 sphere pairs, 30 box pairs: the full 32-bit sphere mask
    (80, 30, 0, 48, 2, 16),         # 40 sphere pairs: per-sphere prefilter
    (40, 20, 1200, 12, 2, 8),       # cull table built, more than 64 pairs: prefilter
    (40, 20, 3800, 8, 2, 8),        # tables too large for a cull table
])
def test_obstacle_counts_around_table_limits(torch_cuda, n_s, n_b, n_far, M, L, H):
    sc = _many_obstacles_scene(n_s, n_b, n_far, n_s + n_b + n_far)
    n = len(sc.spheres) + len(sc.boxes)
    outs = []
    for mode in (binding.EVAL_EARLY_EXIT, binding.EVAL_FULL, binding.EVAL_LAZY):
        p = _planner(sc, M, L, H, mode=mode, max_obstacles=max(64, n))
        p.sample_layers(3, M)
        outs.append(_gpu_solution(p))
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[2], outs[0][2])
    Q = oracle.sample_uniform(3, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    sol = oracle.solve(sc, Q, H)
    V, S, path, cost = outs[0]
    compare_solution(sol, V, S, path, cost, f"{n} obstacles")


def test_fp32_fma_calibration_is_plausible(torch_cuda):
    """The measured FMA rate is positive and cannot exceed SMs x 128 lanes x 2 flops x the top clock."""
    torch = torch_cuda
    props = torch.cuda.get_device_properties(0)
    r = binding.gtmp_fp32_fma_peak()
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    assert 0.25 * ceiling < r < ceiling


def test_anytime_corridor_coverage_frequency(torch_cuda):
    """Sec. V's coverage probability on the appendix's layerwise-hitting
    instance (a walled strip |y| < w): a restart finds a chain iff every layer
    has a sample in the strip, Pr = (1 - (1 - w)^N)^L; 2048 restarts of the GPU
    anytime solver reproduce it, and the first 300 agree with the oracle."""
    w, N, L, H, R = 0.1, 12, 3, 16, 2048
    sc = scenes.corridor_scene(w, 0.3)
    p = _planner(sc, N, L, H, R=R)
    paths, costs, best = p.anytime(77, R)
    p.synchronize()
    costs = costs.cpu().numpy()
    freq = float(np.isfinite(costs).mean())
    expect = (1.0 - (1.0 - w) ** N) ** L
    assert abs(freq - expect) < 4.5 * math.sqrt(expect * (1 - expect) / R), (freq, expect)
    for r in range(300):
        Q = oracle.sample_uniform(77, r, L, N, sc.robot.q_lo, sc.robot.q_hi)
        sol = oracle.solve(sc, Q, H)
        assert math.isfinite(sol.cost_lo) == bool(np.isfinite(costs[r])), r


def test_anytime_single_class_coverage_lower_bound(torch_cuda):
    """Thm. 1 of Sec. V on the GPU anytime solver (2048 restarts of a wide strip, L = 2, N = 256): every
    restart whose samples hit every waypoint ball (found from the oracle's bit-identical samples) returns a
    chain no costlier than the chain through those samples, and the coverage frequency is at least
    1 - sum_m (1 - p_m)^N."""
    from test_oracle_pins import TUBE, ball_chain, tube_waypoint_balls
    cfg = TUBE
    sc = scenes.corridor_scene(cfg["w"], cfg["t"], cfg["x0"])
    centres, p_m = tube_waypoint_balls(cfg)
    L, N, H, R = cfg["L"], cfg["N"], cfg["H"], 2048
    p = _planner(sc, N, L, H, R=R)
    paths, costs, best = p.anytime(91, R)
    p.synchronize()
    costs = costs.cpu().numpy()
    all_hit = 0
    for r in range(R):
        Q = oracle.sample_uniform(91, r, L, N, sc.robot.q_lo, sc.robot.q_hi)
        chain = ball_chain(Q, centres, cfg["r"])
        if chain is None:
            continue
        all_hit += 1
        total, worst = oracle.path_cost(sc, Q, np.array(chain), H)
        assert worst > 0.0
        assert np.isfinite(costs[r]) and costs[r] <= total * (1 + REL), (r, costs[r], total)
    exact = (1.0 - (1.0 - p_m) ** N) ** L
    bound = 1.0 - L * (1.0 - p_m) ** N
    sigma = math.sqrt(exact * (1 - exact) / R)
    assert abs(all_hit / R - exact) < 4.5 * sigma, (all_hit / R, exact)
    assert float(np.isfinite(costs).mean()) >= bound - 4.5 * sigma


@pytest.mark.parametrize("mode", [binding.EVAL_EARLY_EXIT, binding.EVAL_LAZY])
def test_sample_and_solve_capture_in_a_cuda_graph(torch_cuda, mode):
    """Every step of a plan is enqueued on the context's stream with nothing
    synchronous in between, so sampling + solving captures into one CUDA
    graph; replays reproduce the direct calls bit for bit."""
    import ctypes
    torch = torch_cuda
    sc = scene_for("arm", 1, 7, 30)
    M, L, H = 48, 3, 32
    p = _planner(sc, M, L, H, mode=mode)
    s = torch.cuda.Stream()
    binding.gtmp_set_stream(p.ctx, ctypes.c_void_p(s.cuda_stream))
    path = torch.empty(L, dtype=torch.int32, device="cuda")
    cost = torch.empty(1, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        binding.gtmp_sample_layers(p.ctx, 5, M)
        binding.gtmp_solve(p.ctx, path, cost)
    s.synchronize()
    ref_path, ref_cost = path.clone(), cost.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        binding.gtmp_sample_layers(p.ctx, 5, M)
        binding.gtmp_solve(p.ctx, path, cost)
    for _ in range(3):
        path.fill_(-5)
        cost.fill_(-1.0)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(path, ref_path)
        assert torch.equal(cost, ref_cost)
    p.synchronize()


def test_ao_checkpoint_and_resume_is_bit_identical(torch_cuda):
    """AO-GTMP state is the samples, the best cost and the best path; Philox
    counters depend on (slot, layer, attempt), not on history, so a run that
    is checkpointed to the host after two stages, torn down and resumed in a
    fresh context ends exactly where an uninterrupted run ends."""
    torch = torch_cuda
    sc = scene_for("arm", 4, 6, 30)
    L, H, sizes = 4, 16, [8, 16, 32, 64]

    def fresh():
        p = _planner(sc, sizes[-1], L, H)
        st = (torch.empty(L, dtype=torch.int32, device="cuda"), torch.empty(1, dtype=torch.float32, device="cuda"))
        return p, st

    def stages(p, st, best, ms):
        for M in ms:
            binding.aogtmp_expand(p.ctx, 99, M, st[0], st[1], best[0], best[1])
        p.synchronize()

    p, st = fresh()
    best = (torch.full((L,), -1, dtype=torch.int32, device="cuda"),
            torch.full((1,), math.inf, dtype=torch.float32, device="cuda"))
    stages(p, st, best, sizes)
    ref = (p.get_layers().cpu().numpy(), best[0].cpu().numpy(), best[1].cpu().numpy(), st[1].cpu().numpy())
    p.close()

    p, st = fresh()
    best = (torch.full((L,), -1, dtype=torch.int32, device="cuda"),
            torch.full((1,), math.inf, dtype=torch.float32, device="cuda"))
    stages(p, st, best, sizes[:2])
    ckpt = (p.get_layers().cpu(), best[0].cpu(), best[1].cpu())   # host-side checkpoint
    p.close()

    p, st = fresh()
    p.set_layers(ckpt[0].cuda())
    best = (ckpt[1].cuda(), ckpt[2].cuda())
    stages(p, st, best, sizes[2:])
    got = (p.get_layers().cpu().numpy(), best[0].cpu().numpy(), best[1].cpu().numpy(), st[1].cpu().numpy())
    p.close()
    np.testing.assert_array_equal(got[0].view(np.uint32), ref[0].view(np.uint32))
    for a, b in zip(got[1:], ref[1:]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("mode", [binding.EVAL_EARLY_EXIT, binding.EVAL_FULL, binding.EVAL_LAZY])
def test_candidate_edge_count_of_a_solve(torch_cuda, mode):
    """Sec. IV-C: one solve covers 2M + (L - 1) M^2 candidate edges (start
    row, L - 1 interior transitions, goal column) in L + 1 fused launches,
    whatever the mode skips inside them."""
    sc = scene_for("arm", 2, 7, 30)
    M, L, H = 40, 3, 16
    p = _planner(sc, M, L, H, mode=mode)
    p.sample_layers(3, M)
    binding.gtmp_profile_read(p.ctx)                       # reset the counters
    binding.gtmp_profile_enable(p.ctx, True)
    p.solve()
    prof = binding.gtmp_profile_read(p.ctx)
    binding.gtmp_profile_enable(p.ctx, False)
    assert prof["fused_edges"] == 2 * M + (L - 1) * M * M
    assert prof["fused_launches"] == L + 1
    assert prof["fused_ms"] > 0.0
