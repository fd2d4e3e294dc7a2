"""Parity at the sizes of the anytime, AO, batched and surrogate workloads.

Each workload runs at its own size in the configuration bench.py times; the
oracle checks what it can compute in test time:

* Anytime-GTMP, 6-DoF arm, 30 obstacles, R = 64 restarts of M = 256, L = 6,
  H = 32 in one batch of launches: every restart's samples (bit-exact),
  values of every vertex, minimisers, path and cost against a full oracle
  solve of that restart, and the archive's best restart.
* AO-GTMP on the same scene, M = 64 -> 4096 doubling, L = 6: every stage's
  samples bit-exact against the oracle's expand-samples fed with the GPU's
  float32 best cost, the best cost non-increasing and equal to the minimum
  of the stage costs; at M = 4096 the whole goal column, sampled rows of every
  layer by Bellman's equation with oracle-realised edges, and the returned
  chain re-costed and re-checked.
* The batched workload: 512 problems (2D point robots with 5-40 disks and
  7-DoF arms with 5-40 obstacles, M log-uniform in [64, 2048], L in 3..12,
  H = 32) in one persistent launch with autotuned tiles: every problem equals
  its single-problem solve bit for bit, and 24 of them (the largest M, the
  largest L, the smallest and a seeded sample) are checked against the
  oracle: samples bit-exact, full oracle solves where M <= 160, else the goal
  column, Bellman rows of every layer and the returned chain.
* The surrogate workload: 7-DoF arm, 40 obstacles, M = 4096, L = 8, H = 32,
  surrogate trained on 2^21 configurations: the plain solve (samples, goal
  column, Bellman rows, chain) and the pruned solve at the workload's threshold
  and protection band, whose values must satisfy Bellman's equation over the
  edges its scoring kernel kept (read back with gtmp_surrogate_score), with
  oracle-realised edges, whose chain the oracle re-costs and finds free, and
  whose cost lies within 1 % of the plain one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2608_25830_b300 import binding, scenes

from parity import REL, check_values, compare_solution, scene_for

pytestmark = pytest.mark.gpu


def _bounds(labels, costs, Vn):
    lo = np.where((labels == oracle.FREE) | (labels == oracle.AMBIGUOUS), costs + Vn[None, :], np.inf).min(1)
    hi = np.where(labels == oracle.FREE, costs + Vn[None, :], np.inf).min(1)
    return lo, hi


def _bellman_rows(sc, verts, V, S, H, rows_per_layer, seed, keep=None, what=""):
    """Sampled rows of every layer: GPU value within the oracle's bounds of min_v c(u, v) + J_{l+1}(v) over
    oracle-realised edges (restricted to keep[l][row] where given), minimiser edge not colliding."""
    rng = np.random.default_rng(seed)
    L = len(verts) - 2
    for l in range(L + 1):
        n = len(verts[l])
        rows = np.arange(n) if n <= rows_per_layer else rng.choice(n, rows_per_layer, replace=False)
        fin = np.nonzero(np.isfinite(V[l, :n]))[0]
        if fin.size:
            rows = np.unique(np.concatenate([rows, rng.choice(fin, min(2, fin.size), replace=False)]))
        lab, cost = oracle.edge_block(sc, verts[l][rows], verts[l + 1], H)
        if keep is not None:
            lab = np.where(keep[l][rows], lab, oracle.COLLIDE)
        Vn = V[l + 1, :len(verts[l + 1])].astype(np.float64)
        lo, hi = _bounds(lab, cost, Vn)
        check_values(V[l, rows], lo, hi, f"{what} layer {l} rows {rows}")
        for k, i in enumerate(rows):
            if not math.isfinite(V[l, i]):
                assert S[l, i] == -1
                continue
            j = S[l, i]
            assert lab[k, j] != oracle.COLLIDE, f"{what} layer {l} row {i}: minimiser edge not available"
            assert cost[k, j] + Vn[j] == pytest.approx(float(V[l, i]), rel=REL)


def _check_chain(sc, Q, path, cost, H, what=""):
    if not math.isfinite(cost):
        assert list(path) == [-1] * len(path), what
        return
    total, worst = oracle.path_cost(sc, Q, path, H)
    assert worst > -oracle.EPS_DEFAULT, f"{what}: returned chain collides"
    assert cost == pytest.approx(total, rel=REL), what
    assert cost >= float(np.linalg.norm(sc.q_goal.astype(np.float64) - sc.q_start)) * (1 - REL)


# ---------------------------------------------------------------------------
# Anytime-GTMP, 64 restarts in one batch of launches
# ---------------------------------------------------------------------------

def test_anytime_64_restarts_at_size():
    wl = scenes.WORKLOADS["arm6_anytime_r64_m256_l6_h32"]
    R, M, L, H = wl["R"], wl["M"], wl["L"], wl["H"]
    sc = scene_for("arm", wl["seed"], wl["dof"], wl["n_obs"])
    seed = 1                                   # the bench's first timed seed
    p = binding.Planner(sc.robot, M, L, H, R=R, max_obstacles=64)
    p.set_scene(sc)
    paths, costs, best = p.anytime(seed, R)
    p.synchronize()
    paths, costs, best = paths.cpu().numpy(), costs.cpu().numpy(), int(best.cpu()[0])
    sols = oracle.anytime(sc, seed, R, L, M, H)
    for r in range(R):
        V, S = p.values(r)
        compare_solution(sols[r], V.cpu().numpy(), S.cpu().numpy(), paths[r], costs[r], f"restart {r}")
    fin = np.isfinite(costs)
    assert fin.sum() > R // 2
    assert costs[best] == costs[fin].min() and best == int(np.argmin(np.where(fin, costs, np.inf)))
    p.close()


# ---------------------------------------------------------------------------
# AO-GTMP, M = 64 -> 4096
# ---------------------------------------------------------------------------

def test_ao_schedule_at_size():
    import torch
    wl = scenes.WORKLOADS["arm6_ao_m64to4096_l6_h32"]
    L, H = wl["L"], wl["H"]
    sizes = []
    m = wl["M0"]
    while m <= wl["M1"]:
        sizes.append(m)
        m *= 2
    sc = scene_for("arm", wl["seed"], wl["dof"], wl["n_obs"])
    p = binding.Planner(sc.robot, sizes[-1], L, H, max_obstacles=64)
    p.set_scene(sc)
    sp = torch.empty(L, dtype=torch.int32, device="cuda")
    scost = torch.empty(1, dtype=torch.float32, device="cuda")
    bp = torch.full((L,), -1, dtype=torch.int32, device="cuda")
    bc = torch.full((1,), math.inf, dtype=torch.float32, device="cuda")
    Q_ref = np.zeros((L, 0, sc.robot.dof), np.float32)
    prev = math.inf
    for M in sizes:
        c_in = float(bc.cpu()[0])
        binding.aogtmp_expand(p.ctx, 1, M, sp, scost, bp, bc)
        p.synchronize()
        st, Q_ref = oracle.expand_layers(1, Q_ref, M, sc.q_start, sc.q_goal, sc.robot.q_lo, sc.robot.q_hi,
                                         np.float32(c_in))
        assert st == 0
        Q = p.get_layers().cpu().numpy()
        np.testing.assert_array_equal(Q.view(np.uint32), Q_ref.view(np.uint32), err_msg=f"stage M={M}")
        b, c_stage = float(bc.cpu()[0]), float(scost.cpu()[0])
        assert b <= prev and b == min(c_in, c_stage)
        prev = b
        _check_chain(sc, Q, sp.cpu().numpy(), c_stage, H, f"stage M={M}")
    # the last stage at M = 4096: goal column, Bellman rows, chain
    V, S = p.values()
    V, S = V.cpu().numpy(), S.cpu().numpy()
    verts = oracle.layer_vertices(Q_ref, sc.q_start, sc.q_goal)
    _bellman_rows(sc, verts, V, S, H, 3, 5, what="AO M=4096")
    lab, cost = oracle.edge_block(sc, verts[L], sc.q_goal[None, :], H)
    lo, hi = _bounds(lab, cost, np.zeros(1))
    check_values(V[L, :sizes[-1]], lo, hi, "AO M=4096 goal column")
    p.close()


# ---------------------------------------------------------------------------
# batched: 512 uneven problems in one persistent launch
# ---------------------------------------------------------------------------

def test_batch_512_at_size():
    wl = scenes.WORKLOADS["batched512_h32"]
    H = wl["H"]
    problems = []
    for bp in scenes.batch_problems(wl["seed"], wl["n"], H=H):
        sc = bp.scene
        if sc.candidates is not None:
            sc = scenes.pick_endpoints(sc, lambda q, s=sc: oracle.config_free(s, q))
        problems.append((sc, bp.M, bp.L, bp.seed))
    subset = problems[::max(1, len(problems) // 96)][:96]
    tune = binding.Batch(subset, H)
    tune.autotune(repeats=1)
    tiling = binding.gtmp_batch_get_tilings(tune.handle)
    tune.close()
    b = binding.Batch(problems, H)
    binding.gtmp_batch_set_tilings(b.handle, tiling)
    b.solve()
    b.synchronize()
    paths, costs = b.paths.cpu().numpy(), b.costs.cpu().numpy()
    b.close()
    Ms = np.array([M for _, M, _, _ in problems])
    Ls = np.array([L for _, _, L, _ in problems])
    arm = np.array([sc.robot.dof > 3 for sc, *_ in problems])
    rng = np.random.default_rng(3)
    order = list(np.argsort(-Ms * arm)[:4]) + list(np.argsort(-Ms * ~arm)[:2]) + list(np.argsort(-Ls)[:3])
    order += list(np.argsort(Ms)[:3]) + list(rng.choice(len(problems), 24, replace=False))
    pick = list(dict.fromkeys(int(k) for k in order))[:24]
    for k in sorted(pick):
        sc, M, L, seed = problems[k]
        p = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
        p.set_scene(sc)
        p.sample_layers(seed, M)
        path1, cost1 = p.solve()
        V, S = p.values()
        Q = p.get_layers().cpu().numpy()
        path1, cost1 = path1.cpu().numpy(), float(cost1.cpu()[0])
        V, S = V.cpu().numpy(), S.cpu().numpy()
        p.close()
        what = f"problem {k} (dof {sc.robot.dof}, M {M}, L {L})"
        # the batched result is the single-problem solve's, bit for bit
        assert costs[k] == cost1 or (math.isinf(costs[k]) and math.isinf(cost1)), what
        np.testing.assert_array_equal(paths[k, :L], path1, err_msg=what)
        Q_ref = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
        np.testing.assert_array_equal(Q.view(np.uint32), Q_ref.view(np.uint32), err_msg=what)
        if M <= 160:
            compare_solution(oracle.solve(sc, Q_ref, H), V, S, path1, cost1, what)
        else:
            verts = oracle.layer_vertices(Q_ref, sc.q_start, sc.q_goal)
            _bellman_rows(sc, verts, V, S, H, 2, k, what=what)
            lab, cost = oracle.edge_block(sc, verts[L], sc.q_goal[None, :], H)
            lo, hi = _bounds(lab, cost, np.zeros(1))
            check_values(V[L, :M], lo, hi, f"{what} goal column")
        _check_chain(sc, Q_ref, path1, cost1, H, what)


# ---------------------------------------------------------------------------
# surrogate: M = 4096, plain and pruned
# ---------------------------------------------------------------------------

def test_surrogate_workload_at_size():
    import torch
    wl = scenes.WORKLOADS["arm7_m4096_l8_h32_n40"]
    M, L, H = wl["M"], wl["L"], wl["H"]
    sc = scene_for("arm", wl["seed"], wl["dof"], wl["n_obs"])
    p = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
    p.set_scene(sc)
    binding.gtmp_surrogate_train(p.ctx, n_train=wl["n_train"], n_holdout=1 << 16, epochs=wl["epochs"], batch=1024,
                                 lr=1e-3, seed=1, fourier_sigma=wl["sigma"])
    seed = 1
    p.sample_layers(seed, M)
    Q_ref = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    np.testing.assert_array_equal(p.get_layers().cpu().numpy().view(np.uint32), Q_ref.view(np.uint32))
    verts = oracle.layer_vertices(Q_ref, sc.q_start, sc.q_goal)
    # plain solve
    path, cost = p.solve()
    V, S = p.values()
    V, S, path, cost = V.cpu().numpy(), S.cpu().numpy(), path.cpu().numpy(), float(cost.cpu()[0])
    lab, c = oracle.edge_block(sc, verts[L], sc.q_goal[None, :], H)
    lo, hi = _bounds(lab, c, np.zeros(1))
    check_values(V[L, :M], lo, hi, "plain goal column")
    _bellman_rows(sc, verts, V, S, H, 2, 11, what="plain")
    _check_chain(sc, Q_ref, path, cost, H, "plain")
    # pruned solve (the workload's threshold and protection band): Bellman over the kept edges
    thr = wl["threshold"]
    binding.gtmp_surrogate_set_protect(p.ctx, wl.get("protect", 0.0))
    pp = torch.empty(L, dtype=torch.int32, device="cuda")
    pc = torch.empty(1, dtype=torch.float32, device="cuda")
    st = binding.gtmp_solve_pruned(p.ctx, thr, pp, pc, score_waypoints=wl["score_waypoints"])
    Vp, Sp = p.values()
    Vp, Sp = Vp.cpu().numpy(), Sp.cpu().numpy()
    keep = []
    for l in range(L + 1):
        m = torch.empty((len(verts[l]), len(verts[l + 1])), dtype=torch.uint8, device="cuda")
        binding.gtmp_surrogate_score(p.ctx, l, thr, m, score_waypoints=wl["score_waypoints"])
        keep.append(m.cpu().numpy() != 1)
    assert 0.05 * st["edges"] < st["pruned"] == sum(int((~k).sum()) for k in keep)
    _bellman_rows(sc, verts, Vp, Sp, H, 2, 12, keep=keep, what="pruned")
    pc = float(pc.cpu()[0])
    _check_chain(sc, Q_ref, pp.cpu().numpy(), pc, H, "pruned")
    assert pc >= cost or (math.isinf(pc) and math.isinf(cost))
    assert pc <= cost * 1.01 or math.isinf(cost)   # the bar for the pruned solve: cost within 1 % of plain
    p.close()
