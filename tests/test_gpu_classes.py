"""Class-augmented value iteration (Prop. 1) on the GPU against the oracle: the
same set of class labels, the minimum cost of every class, and chains that
carry their label and cost (re-labelled from subtended angles, re-costed and
re-checked by the oracle)."""
import math

import numpy as np
import pytest

import oracle
from paper_2608_25830_b300 import binding, scenes

from parity import REL, scene_for

pytestmark = pytest.mark.gpu


def _box_scene():
    base = scenes.point2d_scene(0, 0)
    disks = np.array([[0.35, -0.3, 0.0, 0.12], [-0.4, 0.25, 0.0, 0.1]], np.float32)
    boxes = np.array([[-0.15, -0.1, -1.0, 0.1, 0.2, 1.0]], np.float32)
    return scenes.Scene(base.robot, disks, boxes, base.q_start, base.q_goal)


CASES = [
    ("cfg1", lambda: scenes.point2d_scene(0, 10), 32, 4, 16, 0),   # the 2D point-robot workload itself
    ("ragged", lambda: scenes.point2d_scene(3, 6), 37, 3, 16, 5),
    ("boxes", _box_scene, 24, 3, 12, 2),
    ("deep", lambda: scenes.point2d_scene(5, 8), 16, 6, 16, 7),
]


def _oracle_classes(sc, Q, H):
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    edges = oracle.realize_edges(sc, verts, H)
    assert all(int((e[0] == oracle.AMBIGUOUS).sum()) == 0 for e in edges)
    tables = oracle.class_value_iteration(edges, verts, oracle.obstacle_centres_2d(sc))
    return tables, verts, edges


@pytest.mark.parametrize("name,make,M,L,H,seed", CASES)
def test_classes_match_oracle(name, make, M, L, H, seed):
    sc = make()
    p = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
    p.set_scene(sc)
    p.sample_layers(seed, M)
    got, n = p.solve_classes(max_labels=1024, max_classes=1024)
    assert n == len(got)
    Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    tables, verts, _ = _oracle_classes(sc, Q, H)
    want = {chi: c for chi, (c, _, _) in tables[0][0].items()}
    assert set(got) == set(want), (name, len(got), len(want))
    centres = oracle.obstacle_centres_2d(sc)
    for chi, (c, path) in got.items():
        assert c == pytest.approx(want[chi], rel=REL), (name, chi)
        pts = [verts[0][0]] + [verts[l + 1][path[l]] for l in range(L)] + [verts[-1][0]]
        assert tuple(oracle.polygon_winding(pts, q) for q in centres) == chi
        total, worst = oracle.path_cost(sc, Q, path, H)
        assert worst > -oracle.EPS_DEFAULT
        assert c == pytest.approx(total, rel=REL)
    # the best class is the plain optimum, bit for bit (float addition is monotone)
    path, cost = p.solve(unfused=True)
    p.synchronize()
    c0 = float(cost.cpu()[0])
    if got:
        assert min(c for c, _ in got.values()) == c0
    else:
        assert math.isinf(c0)
    p.close()


def test_table_overflow_is_reported_and_the_context_stays_usable():
    sc = scenes.point2d_scene(2, 16)
    M, L, H = 64, 4, 16
    p = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
    p.set_scene(sc)
    p.sample_layers(2, M)
    with pytest.raises(RuntimeError, match="OOM|max_labels"):
        p.solve_classes(max_labels=32, max_classes=32)
    got, n = p.solve_classes(max_labels=2048, max_classes=2048)
    assert n == len(got) > 32


def test_arm_robot_is_unsupported():
    sc = scene_for("arm", 0, 7, 10)
    p = binding.Planner(sc.robot, 8, 2, 4, max_obstacles=64)
    p.set_scene(sc)
    p.sample_layers(1, 8)
    with pytest.raises(RuntimeError, match="UNSUPPORTED|planar"):
        p.solve_classes()
    p.close()
