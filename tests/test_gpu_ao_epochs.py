"""AO-GTMP with epochs (Sec. IV-D) and the stage edge limit l_M(r) (Sec. V)
through the C ABI, against the oracle's replay of the same schedule.

The oracle is fed the GPU's float32 best cost after every stage (the informed
sampler and the rules read it), so both sides draw the same samples; then
every epoch/layer/sample decision and every edge limit must agree exactly and
every stage cost within the value tolerance of the plain tests."""
import math

import numpy as np
import pytest

import oracle
from paper_2608_25830_b300 import binding, scenes

from parity import REL, check_values, scene_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _chain_cost_and_margin(sc, chain, L, H):
    verts = [chain[k] for k in range(L + 2)]
    total, worst = 0.0, math.inf
    for a, b in zip(verts[:-1], verts[1:]):
        total += float(np.linalg.norm(b.astype(np.float64) - a))
        worst = min(worst, float(oracle.edge_margins(sc, a, b, H).min()))
    return total, worst


SCHEDULES = [
    # kind, dof, L_cap, schedule
    ("point2d", 2, 5, dict(L0=1, M0=4, M_max=16, stages=7, reach=1.2, r=0.05, varsigma=0.05, limit_edges=True)),
    ("point2d", 2, 4, dict(L0=2, M0=8, M_max=32, stages=6, reach=math.inf, r=0.0, varsigma=0.0, limit_edges=False)),
    ("arm", 6, 6, dict(L0=2, M0=8, M_max=32, stages=7, reach=3.0, r=0.1, varsigma=0.1, limit_edges=True)),
]


@pytest.mark.parametrize("kind,dof,L_cap,sched", SCHEDULES)
def test_ao_epochs_match_the_oracle_replay(torch_cuda, kind, dof, L_cap, sched):
    sc = scene_for(kind, 3, dof, 8 if kind == "point2d" else 30)
    H = 16
    p = binding.Planner(sc.robot, sched["M_max"], L_cap, H, max_obstacles=64)
    p.set_scene(sc)
    chain, cost, log, best_layers = p.ao_run(11, **sched)
    p.synchronize()
    assert len(log) == sched["stages"]
    ref = oracle.ao_run(sc, 11, H=H, L_cap=L_cap, best_feed=[r["best_cost"] for r in log], **sched)
    best = math.inf
    for k, (g, o) in enumerate(zip(log, ref)):
        assert (g["epoch"], g["L"], g["M"]) == (o["epoch"], o["L"], o["M"]), f"stage {k}"
        assert np.float32(g["edge_limit"]) == o["edge_limit"], f"stage {k} limit"
        assert o["status"] == 0
        check_values([g["stage_cost"]], [o["stage_cost"]], [o["stage_cost_hi"]], f"stage {k} cost")
        assert g["best_cost"] == min(best, g["stage_cost"]) or (math.isinf(best) and math.isinf(g["stage_cost"]))
        best = g["best_cost"]
    assert float(cost.cpu()[0]) == best
    ch = chain.cpu().numpy()
    if math.isfinite(best):
        assert 1 <= best_layers <= L_cap
        total, worst = _chain_cost_and_margin(sc, ch, best_layers, H)
        assert total == pytest.approx(best, rel=REL)
        assert worst > -oracle.EPS_DEFAULT
        np.testing.assert_array_equal(ch[0], sc.q_start)
        np.testing.assert_array_equal(ch[best_layers + 1], sc.q_goal)
        assert np.isnan(ch[best_layers + 2:]).all()
    else:
        assert best_layers == 0 and np.isnan(ch).all()
    assert len({r["epoch"] for r in log}) >= 2
    # the context stays at the last epoch's layers and samples
    assert p.L == log[-1]["L"]


def test_ao_run_layer_rule_fires_and_limits_edges(torch_cuda):
    sc = scene_for("point2d", 3, 2, 8)
    p = binding.Planner(sc.robot, 16, 5, 16, max_obstacles=64)
    p.set_scene(sc)
    _, _, log, _ = p.ao_run(11, L0=1, M0=4, M_max=16, stages=4, reach=1.2, r=0.05, varsigma=0.05, limit_edges=True)
    assert log[0]["L"] == 1 and math.isinf(log[0]["edge_limit"])
    c = log[0]["best_cost"]
    assert math.isfinite(c)
    need = math.ceil(c / (1.2 - 0.15)) - 1
    assert need > 1 and log[1]["L"] == min(need, 5) and log[1]["epoch"] == 1
    assert log[1]["edge_limit"] == pytest.approx(c / (log[1]["L"] + 1) + 0.15, rel=1e-6)


def test_ao_run_rejects_bad_schedules_and_goal_sets(torch_cuda):
    torch = torch_cuda
    sc = scenes.point2d_scene(0, 4)
    p = binding.Planner(sc.robot, 16, 3, 8, max_obstacles=8)
    p.set_scene(sc)
    chain = torch.empty((5, 2), dtype=torch.float32, device="cuda")
    cost = torch.empty(1, dtype=torch.float32, device="cuda")
    bad = [dict(L0=0), dict(L0=4), dict(M0=0), dict(M_max=2), dict(M_max=32), dict(stages=0),
           dict(reach=0.1, r=0.05, varsigma=0.0), dict(r=-1.0), dict(reach=float("nan"))]
    for b in bad:
        s = dict(L0=1, M0=4, M_max=16, stages=2, reach=math.inf, r=0.0, varsigma=0.0, limit_edges=0)
        s.update(b)
        sch = binding.GtmpAoSchedule(s["L0"], s["M0"], s["M_max"], s["stages"], s["reach"], s["r"], s["varsigma"],
                                     s["limit_edges"])
        with pytest.raises(binding.GtmpError) as e:
            binding.aogtmp_run(p.ctx, 1, sch, chain, cost)
        assert e.value.status == 1, b
    binding.gtmp_set_goals(p.ctx, np.stack([sc.q_goal, sc.q_goal * 0.5]))
    sch = binding.GtmpAoSchedule(1, 4, 16, 2, math.inf, 0.0, 0.0, 0)
    with pytest.raises(binding.GtmpError) as e:
        binding.aogtmp_run(p.ctx, 1, sch, chain, cost)
    assert e.value.status == 5


def test_num_layers_and_edge_limit_setters(torch_cuda):
    """After gtmp_set_num_layers the context solves the new layout exactly as a context created with it."""
    sc = scene_for("arm", 2, 7, 30)
    M, H = 32, 16
    big = binding.Planner(sc.robot, M, 6, H, max_obstacles=64)
    big.set_scene(sc)
    big.set_num_layers(3)
    small = binding.Planner(sc.robot, M, 3, H, max_obstacles=64)
    small.set_scene(sc)
    for p in (big, small):
        p.sample_layers(7, M)
    a, b = big.solve(), small.solve()
    big.synchronize()
    np.testing.assert_array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())
    assert float(a[1].cpu()[0]) == float(b[1].cpu()[0])
    binding.gtmp_set_max_edge_len(big.ctx, 1e-3)
    big.sample_layers(7, M)
    path, c = big.solve()
    big.synchronize()
    assert math.isinf(float(c.cpu()[0]))
    for bad in (0, 7):
        with pytest.raises(binding.GtmpError):
            big.set_num_layers(bad)
    with pytest.raises(binding.GtmpError):
        binding.gtmp_set_max_edge_len(big.ctx, 0.0)
