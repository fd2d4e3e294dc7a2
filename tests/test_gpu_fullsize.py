"""Parity at the benchmark's full size (7-DoF arm, 20 spheres + 10 boxes,
M = 1024, L = 8, H = 32), in the launch configuration bench.py times.

The oracle cannot realise all 7.3 M edges in test time, so it checks what it
can compute one by one: the whole sample set (bit-exact), the whole last layer
(1024 edges to the goal), whole rows of sampled vertices in every other layer
(Bellman's equation J_l(u) = min_v c(u,v) + J_{l+1}(v) of the GPU's values,
with every c(u,v) and its collision label computed by the oracle), the
minimisers of those rows, and the returned chain (re-costed, every waypoint
re-checked).  Full-evaluation mode must return the same values bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2608_25830_b300 import binding, scenes

from parity import REL, check_values, scene_for

pytestmark = pytest.mark.gpu

M, L, H = 1024, 8, 32
ROWS_PER_LAYER = 6


@pytest.fixture(scope="module")
def fullsize():
    import torch
    sc = scene_for("arm", 0, 7, 30)
    out = {}
    for mode in (binding.EVAL_EARLY_EXIT, binding.EVAL_FULL, binding.EVAL_LAZY):
        p = binding.Planner(sc.robot, M, L, H, max_obstacles=64, eval_mode=mode)
        p.set_scene(sc)
        p.sample_layers(7, M)
        path, cost = p.solve()
        V, S = p.values()
        Q = p.get_layers()
        p.synchronize()
        out[mode] = dict(Q=Q.cpu().numpy(), V=V.cpu().numpy().astype(np.float64), S=S.cpu().numpy(),
                         path=path.cpu().numpy(), cost=float(cost.cpu()[0]))
        p.close()
    return sc, out


def _bounds(labels, costs, Vnext_lo, Vnext_hi):
    lo = np.where((labels == oracle.FREE) | (labels == oracle.AMBIGUOUS), costs + Vnext_lo[None, :], np.inf).min(1)
    hi = np.where(labels == oracle.FREE, costs + Vnext_hi[None, :], np.inf).min(1)
    return lo, hi


def test_samples_bit_exact(fullsize):
    sc, out = fullsize
    ref = oracle.sample_uniform(7, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    np.testing.assert_array_equal(out[binding.EVAL_EARLY_EXIT]["Q"].view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("mode", [binding.EVAL_FULL, binding.EVAL_LAZY])
def test_other_modes_are_identical(fullsize, mode):
    _, out = fullsize
    a, b = out[binding.EVAL_EARLY_EXIT], out[mode]
    np.testing.assert_array_equal(a["V"], b["V"])
    np.testing.assert_array_equal(a["S"], b["S"])
    np.testing.assert_array_equal(a["path"], b["path"])


def test_last_layer_completely(fullsize):
    sc, out = fullsize
    o = out[binding.EVAL_EARLY_EXIT]
    Q = o["Q"]
    lab, cost = oracle.edge_block(sc, Q[L - 1], sc.q_goal[None, :], H)
    lo, hi = _bounds(lab, cost, np.zeros(1), np.zeros(1))
    check_values(o["V"][L, :M], lo, hi, "layer L")


def test_bellman_rows_in_every_layer(fullsize):
    """Sampled rows of layers 0..L-1: GPU value = min over oracle edges of c + GPU next-layer value."""
    sc, out = fullsize
    o = out[binding.EVAL_EARLY_EXIT]
    Q, V, S = o["Q"], o["V"], o["S"]
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    rng = np.random.default_rng(0)
    for l in range(0, L):
        n = len(verts[l])
        rows = np.arange(n) if n <= ROWS_PER_LAYER else rng.choice(n, ROWS_PER_LAYER, replace=False)
        # prefer rows that have a finite value so the minimiser is exercised too
        fin = np.nonzero(np.isfinite(V[l, :n]))[0]
        if fin.size:
            rows = np.unique(np.concatenate([rows, rng.choice(fin, min(3, fin.size), replace=False)]))
        lab, cost = oracle.edge_block(sc, verts[l][rows], verts[l + 1], H)
        Vn = V[l + 1, :len(verts[l + 1])]
        lo, hi = _bounds(lab, cost, Vn, Vn)
        check_values(V[l, rows], lo, hi, f"layer {l} rows {rows}")
        for k, i in enumerate(rows):
            if not math.isfinite(V[l, i]):
                assert S[l, i] == -1
                continue
            j = S[l, i]
            assert lab[k, j] != oracle.COLLIDE, f"layer {l} row {i}: minimiser edge collides"
            assert cost[k, j] + Vn[j] == pytest.approx(V[l, i], rel=REL)


def test_returned_chain(fullsize):
    sc, out = fullsize
    o = out[binding.EVAL_EARLY_EXIT]
    assert o["cost"] == pytest.approx(o["V"][0, 0], rel=0, abs=0)
    if not math.isfinite(o["cost"]):
        assert list(o["path"]) == [-1] * L
        return
    total, worst = oracle.path_cost(sc, o["Q"], o["path"], H)
    assert worst > -oracle.EPS_DEFAULT
    assert o["cost"] == pytest.approx(total, rel=REL)
    assert o["cost"] >= float(np.linalg.norm(sc.q_goal.astype(np.float64) - sc.q_start)) * (1 - REL)
    # the chain follows the minimisers
    i = 0
    for l in range(L):
        i_next = o["S"][l, i]
        assert o["path"][l] == i_next
        i = i_next
