"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a published value, a closed form, an
invariant, brute force, or an independent library routine, chosen so that a
plausible slip (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import stats
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import dijkstra

import oracle
from paper_2608_25830_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_samples_are_uniform_in_box():
    lo = np.array([-math.pi, -1.0, 0.25], np.float32)
    hi = np.array([math.pi, 3.0, 0.5], np.float32)
    Q = oracle.sample_uniform(7, 3, 2, 4000, lo, hi)
    assert Q.dtype == np.float32 and Q.shape == (2, 4000, 3)
    for k in range(3):
        x = Q[..., k].ravel().astype(np.float64)
        assert x.min() >= lo[k] and x.max() < hi[k]
        p = stats.kstest((x - lo[k]) / (hi[k] - lo[k]), "uniform").pvalue
        assert p > 1e-4, (k, p)
    # layers, restarts and seeds give different streams; same arguments repeat exactly
    assert not np.array_equal(Q[0], Q[1])
    assert not np.array_equal(Q, oracle.sample_uniform(7, 4, 2, 4000, lo, hi))
    assert not np.array_equal(Q, oracle.sample_uniform(8, 3, 2, 4000, lo, hi))
    assert np.array_equal(Q, oracle.sample_uniform(7, 3, 2, 4000, lo, hi))
    # coordinates within one vertex are not copies of each other
    assert np.corrcoef(Q[0, :, 0], Q[0, :, 1])[0, 1] ** 2 < 0.01


# ---------------------------------------------------------------------------
# Forward kinematics: closed forms of simple chains
# ---------------------------------------------------------------------------

def _robot(dh, link_sph):
    dh = np.asarray(dh, np.float32)
    dof = dh.shape[0]
    return scenes.Robot(scenes.ROBOT_DH_ARM, dof, dh, np.asarray(link_sph, np.float32),
                        np.full(dof, -math.pi, np.float32), np.full(dof, math.pi, np.float32))


def _empty_scene(robot):
    return scenes.Scene(robot, np.zeros((0, 4), np.float32), np.zeros((0, 6), np.float32),
                        np.zeros(robot.dof, np.float32), np.zeros(robot.dof, np.float32))


def test_fk_planar_chain_closed_form():
    a = [0.3, 0.2, 0.1]
    dh = [[0.0, ai, 0.0, 0.0] for ai in a]
    origin_sph = np.zeros((3, 1, 4))
    origin_sph[:, 0, 3] = 0.01
    sc = _empty_scene(_robot(dh, origin_sph))
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rng.uniform(-math.pi, math.pi, 3)
        got = oracle.fk_spheres(sc, q)
        phi = np.cumsum(q)
        x = np.cumsum(np.array(a, np.float32).astype(np.float64) * np.cos(phi))
        y = np.cumsum(np.array(a, np.float32).astype(np.float64) * np.sin(phi))
        np.testing.assert_allclose(got[:, 0], x, atol=1e-12)
        np.testing.assert_allclose(got[:, 1], y, atol=1e-12)
        np.testing.assert_allclose(got[:, 2], 0.0, atol=1e-12)
        np.testing.assert_allclose(got[:, 3], 0.01, rtol=1e-6)


def test_fk_twisted_two_link_closed_form():
    # link 1 twisted by +pi/2: o1 = (a1 c1, a1 s1, d1),
    # o2 - o1 = (a2 c2 c1 + d2 s1, a2 c2 s1 - d2 c1, a2 s2)   (worked out by hand)
    a1, d1, a2, d2 = 0.25, 0.05, 0.2, 0.07
    dh = [[d1, a1, math.pi / 2, 0.0], [d2, a2, 0.0, 0.0]]
    sph = np.zeros((2, 1, 4))
    sph[:, 0, 3] = 0.02
    rob = _robot(dh, sph)
    a1, d1, a2, d2 = (float(np.float32(v)) for v in (a1, d1, a2, d2))
    sc = _empty_scene(rob)
    rng = np.random.default_rng(1)
    for _ in range(20):
        q1, q2 = rng.uniform(-math.pi, math.pi, 2)
        got = oracle.fk_spheres(sc, [q1, q2])
        c1, s1, c2, s2 = math.cos(q1), math.sin(q1), math.cos(q2), math.sin(q2)
        o1 = np.array([a1 * c1, a1 * s1, d1])
        o2 = o1 + np.array([a2 * c2 * c1 + d2 * s1, a2 * c2 * s1 - d2 * c1, a2 * s2])
        np.testing.assert_allclose(got[0, :3], o1, atol=1e-7)   # float32 pi/2 twist: 4e-8 off exact
        np.testing.assert_allclose(got[1, :3], o2, atol=1e-7)


def test_fk_generated_arm_spheres_lie_on_link_segments():
    """Generated link spheres sit at fixed fractions of the segment between frame origins."""
    rob = scenes.dh_arm(3, 7)
    origin = rob.link_spheres.copy()
    origin[:, :, :3] = 0.0                       # same robot with spheres at the frame origins
    frames = _empty_scene(scenes.Robot(rob.kind, rob.dof, rob.dh, origin[:, :1], rob.q_lo, rob.q_hi))
    sc = _empty_scene(rob)
    fr = (np.arange(4) + 0.5) / 4
    rng = np.random.default_rng(2)
    for _ in range(10):
        q = rng.uniform(-math.pi, math.pi, 7)
        o = np.vstack([np.zeros(3), oracle.fk_spheres(frames, q)[:, :3]])
        s = oracle.fk_spheres(sc, q)[:, :3].reshape(7, 4, 3)
        for i in range(7):
            expect = o[i][None, :] + fr[:, None] * (o[i + 1] - o[i])[None, :]
            np.testing.assert_allclose(s[i], expect, atol=2e-7)
            # rigid-motion invariant: |o_i - o_{i-1}| = sqrt(a^2 + d^2)
            d, a = float(rob.dh[i, 0]), float(rob.dh[i, 1])
            assert abs(np.linalg.norm(o[i + 1] - o[i]) - math.hypot(a, d)) < 1e-12


# ---------------------------------------------------------------------------
# Collision margins: hand cases with known distances
# ---------------------------------------------------------------------------

def _point_scene(spheres=(), boxes=(), radius=0.0, dof=3):
    rob = scenes.Robot(scenes.ROBOT_POINT, dof, np.zeros((dof, 4), np.float32), np.zeros((dof, 0, 4), np.float32),
                       np.full(dof, -2, np.float32), np.full(dof, 2, np.float32), radius)
    return scenes.Scene(rob, np.asarray(spheres, np.float32).reshape(-1, 4), np.asarray(boxes, np.float32).reshape(-1, 6),
                        np.zeros(dof, np.float32), np.zeros(dof, np.float32))


def test_margin_sphere_cases():
    sc = _point_scene(spheres=[(0.5, 0.0, 0.0, 0.25)], radius=0.125)
    assert oracle.config_margin(sc, [0.0, 0.0, 0.0]) == pytest.approx(0.5 - 0.25 - 0.125, abs=1e-15)
    assert oracle.config_margin(sc, [0.125, 0.0, 0.0]) == pytest.approx(0.0, abs=1e-15)       # tangent
    assert oracle.config_margin(sc, [0.5, 0.0, 0.0]) == pytest.approx(-0.375, abs=1e-15)      # centred
    assert oracle.config_margin(sc, [0.5, 3.0, 4.0]) == pytest.approx(5.0 - 0.375, abs=1e-12)  # 3-4-5


def test_margin_box_face_edge_corner_inside():
    box = (0.0, 0.0, 0.0, 1.0, 2.0, 3.0)
    sc = _point_scene(boxes=[box])
    m = lambda q: oracle.config_margin(sc, q)
    assert m([-0.5, 1.0, 1.0]) == pytest.approx(0.5)                      # face
    assert m([-0.3, -0.4, 1.0]) == pytest.approx(0.5)                     # edge (3-4-5)
    assert m([2.0, 4.0, 5.0]) == pytest.approx(3.0)                       # corner (1,2,2)
    assert m([0.5, 1.0, 1.0]) == pytest.approx(-0.5)                      # inside: nearest face x
    assert m([0.9, 1.0, 1.5]) == pytest.approx(-0.1)                      # inside: nearest face x=1
    assert m([0.5, 1.9, 1.5]) == pytest.approx(-0.1)                      # inside: nearest face y=2
    assert m([1.0, 1.0, 1.0]) == pytest.approx(0.0)                       # on the face
    sc_r = _point_scene(boxes=[box], radius=0.25)
    assert oracle.config_margin(sc_r, [-0.5, 1.0, 1.0]) == pytest.approx(0.25)


def test_margin_brute_force_over_pairs():
    rob = scenes.dh_arm(5, 6)
    rng = np.random.default_rng(3)
    sph, box = scenes.arm_obstacles(rng, 9)
    sc = scenes.Scene(rob, sph, box, np.zeros(6, np.float32), np.zeros(6, np.float32))
    for _ in range(5):
        q = rng.uniform(-math.pi, math.pi, 6)
        S = oracle.fk_spheres(sc, q)
        best = math.inf
        for c in S:
            for o in sph.astype(np.float64):
                best = min(best, np.linalg.norm(c[:3] - o[:3]) - o[3] - c[3])
            for b in box.astype(np.float64):
                # distance to the box by dense projection onto the box (outside) / faces (inside)
                clamp = np.minimum(np.maximum(c[:3], b[:3]), b[3:])
                if np.all(clamp == c[:3]):
                    dist = -min(np.min(c[:3] - b[:3]), np.min(b[3:] - c[:3]))
                else:
                    dist = np.linalg.norm(c[:3] - clamp)
                best = min(best, dist - c[3])
        assert oracle.config_margin(sc, q) == pytest.approx(best, abs=1e-12)


# ---------------------------------------------------------------------------
# Straight-line local planner: waypoint rule and tri-state labels
# ---------------------------------------------------------------------------

def test_edge_label_waypoints():
    # disk of radius 0.2 at x = 0.5 on the segment (0,0) -> (1,0), H = 3 checks x = 0, 0.5, 1
    sc = _point_scene(spheres=[(0.5, 0.0, 0.0, 0.2)], dof=2)
    lab, cost = oracle.edge_block(sc, [[0.0, 0.0]], [[1.0, 0.0]], 3)
    assert lab[0, 0] == oracle.COLLIDE and cost[0, 0] == 1.0
    # a disk between waypoints is missed: the checker is the paper's discretised SEV
    sc2 = _point_scene(spheres=[(0.25, 0.0, 0.0, 0.1)], dof=2)
    lab, _ = oracle.edge_block(sc2, [[0.0, 0.0]], [[1.0, 0.0]], 3)
    assert lab[0, 0] == oracle.FREE
    lab, _ = oracle.edge_block(sc2, [[0.0, 0.0]], [[1.0, 0.0]], 5)   # t = 0.25 hits it
    assert lab[0, 0] == oracle.COLLIDE
    # tangent waypoint (distance exactly the radius) is ambiguous
    sc3 = _point_scene(spheres=[(0.5, 0.25, 0.0, 0.25)], dof=2)
    lab, _ = oracle.edge_block(sc3, [[0.0, 0.0]], [[1.0, 0.0]], 3)
    assert lab[0, 0] == oracle.AMBIGUOUS
    # edge-length limit removes the edge
    lab, _ = oracle.edge_block(sc2, [[0.0, 0.0]], [[0.0, 1.0]], 3, max_len=0.5)
    assert lab[0, 0] == oracle.COLLIDE
    # endpoint in collision
    lab, _ = oracle.edge_block(sc, [[0.5, 0.0]], [[0.5, 1.0]], 2)
    assert lab[0, 0] == oracle.COLLIDE


def test_edge_margins_match_config_margins():
    a = scenes.arm_scene(1, 7, 12)
    rng = np.random.default_rng(4)
    u = rng.uniform(-3, 3, 7).astype(np.float32)
    v = rng.uniform(-3, 3, 7).astype(np.float32)
    H = 9
    m = oracle.edge_margins(a, u, v, H)
    assert m[0] == oracle.config_margin(a, u.astype(np.float64))
    assert m[-1] == oracle.config_margin(a, v.astype(np.float64))
    t = np.float32(4) / np.float32(8)           # t = 0.5 exactly: the midpoint waypoint
    mid = (np.float64(t) * (v - u).astype(np.float64) + u).astype(np.float32)
    assert m[4] == oracle.config_margin(a, mid.astype(np.float64))


# ---------------------------------------------------------------------------
# Graph search: brute force, Dijkstra, Alg. 1's Jacobi form, closed forms
# ---------------------------------------------------------------------------

def _small_problem(seed=0, M=4, L=3, n_obs=12):
    sc = scenes.point2d_scene(seed, n_obs)
    Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    return sc, Q


@pytest.mark.parametrize("seed", range(6))
def test_value_iteration_equals_brute_force(seed):
    sc, Q = _small_problem(seed, M=4, L=3, n_obs=6 + seed)
    H = 16
    sol = oracle.solve(sc, Q, H)
    verts = sol.verts
    best, best_chain = math.inf, None
    for chain in itertools.product(range(4), repeat=3):
        idx = (0,) + chain + (0,)
        total = 0.0
        for l in range(4):
            lab, cost = sol.edges[l]
            if lab[idx[l], idx[l + 1]] != oracle.FREE:
                total = math.inf
                break
            total += cost[idx[l], idx[l + 1]]
        if total < best:
            best, best_chain = total, chain
    assert sol.cost_lo == pytest.approx(best, rel=1e-12) if math.isfinite(best) else math.isinf(sol.cost_lo)
    if math.isfinite(best):
        assert tuple(sol.path) == best_chain
    else:
        assert list(sol.path) == [-1, -1, -1]


@pytest.mark.parametrize("seed", range(4))
def test_value_iteration_equals_dijkstra(seed):
    sc, Q = _small_problem(seed, M=12, L=4, n_obs=10)
    sol = oracle.solve(sc, Q, 16)
    sizes = [len(v) for v in sol.verts]
    off = np.concatenate([[0], np.cumsum(sizes)])
    rows, cols, w = [], [], []
    for l, (lab, cost) in enumerate(sol.edges):
        a, b = np.nonzero(lab == oracle.FREE)
        rows += list(off[l] + a)
        cols += list(off[l + 1] + b)
        w += list(cost[a, b])
    n = off[-1]
    G = csr_matrix((w, (rows, cols)), shape=(n, n))
    dist = dijkstra(G, directed=True, indices=0)
    assert dist[n - 1] == pytest.approx(sol.cost_lo, rel=1e-12) if math.isfinite(sol.cost_lo) else math.isinf(dist[n - 1])
    # every vertex's cost-to-go equals its Dijkstra distance to the goal (reverse graph)
    back = dijkstra(G.T.tocsr(), directed=True, indices=n - 1)
    for l in range(len(sizes)):
        np.testing.assert_allclose(sol.V_lo[l], back[off[l]:off[l + 1]], rtol=1e-12)


def test_jacobi_form_of_algorithm1_matches_backward_pass():
    """Alg. 1 initialises V_h to 0 and sweeps L+1 times; the result is the backward pass."""
    sc, Q = _small_problem(2, M=8, L=5, n_obs=8)
    sol = oracle.solve(sc, Q, 16)
    L = Q.shape[0]
    C = [np.where(lab == oracle.FREE, cost, np.inf) for lab, cost in sol.edges]
    Vh = [np.zeros(Q.shape[1]) for _ in range(L)]       # V_h <- 0
    Vg = np.zeros(1)
    Vs = 0.0
    for _ in range(L + 1):
        new = [None] * L
        new[L - 1] = np.min(C[L] + Vg[None, :], axis=1)
        for m in range(L - 1):
            new[m] = np.min(C[m + 1] + Vh[m + 1][None, :], axis=1)
        Vs = float(np.min(C[0][0] + Vh[0]))
        Vh = new
    for m in range(L):
        np.testing.assert_allclose(Vh[m], sol.V_lo[m + 1], rtol=1e-12)
    assert Vs == pytest.approx(sol.cost_lo, rel=1e-12)


def test_collinear_samples_give_straight_line_cost():
    sc = _point_scene(dof=2)
    sc.q_start = np.array([-0.5, -0.25], np.float32)
    sc.q_goal = np.array([0.5, 0.25], np.float32)
    L, M = 3, 5
    rng = np.random.default_rng(0)
    Q = rng.uniform(-1, 1, (L, M, 2)).astype(np.float32)
    # plant one exactly collinear point per layer (t = 1/4, 1/2, 3/4 are exact in binary)
    for l, t in enumerate([0.25, 0.5, 0.75]):
        Q[l, (l * 2 + 1) % M] = sc.q_start + np.float32(t) * (sc.q_goal - sc.q_start)
    sol = oracle.solve(sc, Q, 8)
    assert sol.cost_lo == pytest.approx(math.hypot(1.0, 0.5), rel=1e-14)
    assert list(sol.path) == [1, 3, 0]


def test_infeasible_graph_reports_infinity_and_minus_one():
    sc = _point_scene(spheres=[(0.0, 0.0, 0.0, 5.0)], dof=2)        # everything in collision
    Q = oracle.sample_uniform(0, 0, 3, 4, [-1, -1], [1, 1])
    sol = oracle.solve(sc, Q, 4)
    assert math.isinf(sol.cost_lo) and math.isinf(sol.cost_hi)
    assert list(sol.path) == [-1, -1, -1]


@pytest.mark.parametrize("seed", range(3))
def test_returned_chain_is_free_and_costs_what_it_claims(seed):
    a = scenes.arm_scene(seed, 6, 20)
    a = scenes.pick_endpoints(a, lambda q: oracle.config_free(a, q))
    Q = oracle.sample_uniform(seed, 0, 3, 24, a.robot.q_lo, a.robot.q_hi)
    sol = oracle.solve(a, Q, 16)
    straight = float(np.linalg.norm(a.q_goal.astype(np.float64) - a.q_start))
    if math.isfinite(sol.cost_lo):
        total, worst = oracle.path_cost(a, Q, sol.path, 16)
        assert total == pytest.approx(sol.cost_lo, rel=1e-12)
        assert worst > -oracle.EPS_DEFAULT
        assert sol.cost_lo >= straight * (1 - 1e-12)
    assert sol.cost_lo <= sol.cost_hi


# ---------------------------------------------------------------------------
# Informed sampling (X_f(c), Sec. IV-D) and expand-samples (Alg. 1)
# ---------------------------------------------------------------------------

def _informed_draws(d, c, n, lo=-50.0, hi=50.0, seed=11):
    q0 = np.linspace(-1, 1, d).astype(np.float32)
    qg = (q0[::-1] * 0.5 + 0.3).astype(np.float32)
    par = oracle.informed_params(q0, qg, c)
    xs = []
    i = 0
    while len(xs) < n:
        for a in range(1 << 12):
            ok, x = oracle.informed_attempt(seed, i, 0, a, par, np.full(d, lo), np.full(d, hi))
            if ok:
                xs.append(x)
                break
        i += 1
    return q0, qg, par, np.array(xs, np.float64)


@pytest.mark.parametrize("d", [2, 6])
def test_informed_samples_in_ellipsoid_and_uniform(d):
    q0 = np.linspace(-1, 1, d).astype(np.float32)
    qg = (q0[::-1] * 0.5 + 0.3).astype(np.float32)
    cmin = float(np.linalg.norm(qg.astype(np.float64) - q0))
    c = 1.7 * cmin
    q0, qg, par, X = _informed_draws(d, c, 1500)
    s = np.linalg.norm(X - q0, axis=1) + np.linalg.norm(X - qg, axis=1)
    assert np.all(s <= c * (1 + 1e-6))
    # r1, r2 are the semi-axes of the informed set: foci distance c_min
    assert par["r1"] == pytest.approx(c / 2, rel=1e-6)
    assert par["r2"] == pytest.approx(math.sqrt(c * c - cmin * cmin) / 2, rel=1e-5)
    # back to the unit ball: the radius of a uniform point of the d-ball has CDF rho^d
    a = par["axis"].astype(np.float64)
    Y = X - par["centre"].astype(np.float64)
    along = Y @ a
    perp = Y - along[:, None] * a[None, :]
    Z = perp / float(par["r2"]) + (along / float(par["r1"]))[:, None] * a[None, :]
    rho = np.linalg.norm(Z, axis=1)
    assert rho.max() <= 1 + 1e-5
    assert stats.kstest(rho ** d, "uniform").pvalue > 1e-4
    # the direction along the major axis is symmetric and spans the whole axis
    assert abs(np.mean(along)) < 0.1 * float(par["r1"])
    assert np.max(np.abs(along)) > 0.8 * float(par["r1"])


def test_informed_box_rejection_and_degenerate_bound():
    d = 3
    q0 = np.zeros(d, np.float32)
    qg = np.array([1, 0, 0], np.float32)
    par = oracle.informed_params(q0, qg, 3.0)
    lo, hi = np.full(d, -0.5, np.float32), np.full(d, 0.5, np.float32)
    hits = 0
    for a in range(2000):
        ok, x = oracle.informed_attempt(5, 0, 0, a, par, lo, hi)
        if ok:
            hits += 1
            assert np.all(x >= lo) and np.all(x <= hi)
    assert hits > 0
    # c = c_min: the informed set collapses onto the segment q0 -> qg
    par = oracle.informed_params(q0, qg, 1.0)
    assert float(par["r2"]) == 0.0
    for a in range(200):
        ok, x = oracle.informed_attempt(5, 1, 0, a, par, np.full(d, -5, np.float32), np.full(d, 5, np.float32))
        if ok:
            assert abs(x[1]) == 0 and abs(x[2]) == 0 and -1e-6 <= x[0] <= 1 + 1e-6


def test_expand_with_infinite_bound_is_the_uniform_stream():
    lo, hi = np.full(4, -1, np.float32), np.full(4, 1, np.float32)
    st, Q = oracle.expand_layers(9, np.zeros((3, 0, 4), np.float32), 16, np.zeros(4), np.ones(4) * 0.5, lo, hi, math.inf)
    assert st == 0
    np.testing.assert_array_equal(Q, oracle.sample_uniform(9, 0, 3, 16, lo, hi))


def test_expand_keeps_old_samples_and_mixes_heuristic_midpoints():
    d = 3
    lo, hi = np.full(d, -2, np.float32), np.full(d, 2, np.float32)
    q0 = np.array([-1, -1, 0], np.float32)
    qg = np.array([1, 1, 0], np.float32)
    _, Q0 = oracle.expand_layers(4, np.zeros((4, 0, d), np.float32), 32, q0, qg, lo, hi, math.inf)
    c = 4.0
    st, Q = oracle.expand_layers(4, Q0, 256, q0, qg, lo, hi, c)
    assert st == 0
    np.testing.assert_array_equal(Q[:, :32], Q0)
    L = Q.shape[0]
    n_mid = 0
    n_new = 0
    for l in range(L):
        prev = q0[None, :] if l == 0 else Q0[l - 1]
        nxt = qg[None, :] if l == L - 1 else Q0[l + 1]
        for x in Q[l, 32:]:
            n_new += 1
            # brute force: is x the midpoint of some u in the previous layer and its nearest next-layer vertex?
            is_mid = False
            for u in prev:
                j = int(np.argmin(((nxt.astype(np.float64) - u) ** 2).sum(1)))
                if np.array_equal(x, (np.float32(0.5) * (u + nxt[j])).astype(np.float32)):
                    is_mid = True
                    break
            if is_mid:
                n_mid += 1
            else:
                s = np.linalg.norm(x.astype(np.float64) - q0) + np.linalg.norm(x.astype(np.float64) - qg)
                assert s <= c * (1 + 1e-6)
    # fair coin: about half of the new samples are heuristic midpoints
    assert abs(n_mid / n_new - 0.5) < 0.08, n_mid / n_new


# ---------------------------------------------------------------------------
# class-augmented value iteration (Prop. 1) on planar scenes
# ---------------------------------------------------------------------------

def test_edge_labels_sum_to_the_winding_of_the_closed_chain():
    """Summing the triangle labels u -> v -> g over a chain gives the winding numbers of the loop (chain,
    then g -> start) computed independently from subtended angles."""
    rng = np.random.default_rng(11)
    for trial in range(200):
        centres = [tuple(c) for c in rng.uniform(-1, 1, (4, 2))]
        pts = rng.uniform(-1, 1, (rng.integers(3, 8), 2)).astype(np.float32)
        # keep points away from the centres (the winding number is undefined on the loop)
        if min(np.hypot(*(pts - np.array(c, np.float32)).T).min() for c in centres) < 1e-3:
            continue
        g = pts[-1]
        lab = np.zeros(len(centres), int)
        for a, b in zip(pts[:-1], pts[1:]):
            lab += np.array(oracle.edge_class_label(a, b, g, centres))
        want = [oracle.polygon_winding(list(pts), c) for c in centres]
        assert list(lab) == want, (trial, lab, want)


def test_triangle_winding_hand_cases():
    a, b, c = (0.0, 0.0), (1.0, 0.0), (0.0, 1.0)
    assert oracle.triangle_winding(a, b, c, (0.25, 0.25)) == 1          # counter-clockwise, inside
    assert oracle.triangle_winding(a, c, b, (0.25, 0.25)) == -1         # clockwise, inside
    assert oracle.triangle_winding(a, b, c, (1.0, 1.0)) == 0            # outside
    assert oracle.triangle_winding(a, b, c, (0.5, 0.0)) == 0            # on an edge: outside by convention
    assert oracle.triangle_winding(a, b, (2.0, 0.0), (0.5, 0.0)) == 0   # degenerate triangle


def _chain_labels_brute_force(sc, Q, H, centres):
    """Every chain q0 -> Q[0][i1] -> ... -> qg with all edges free: label from subtended angles, cost."""
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    edges = oracle.realize_edges(sc, verts, H)
    L, M = Q.shape[0], Q.shape[1]
    best = {}
    for chain in itertools.product(range(M), repeat=L):
        idx = [0] + list(chain) + [0]
        ok, cost = True, 0.0
        for l in range(L + 1):
            lab, c = edges[l][0][idx[l], idx[l + 1]], edges[l][1][idx[l], idx[l + 1]]
            assert lab != oracle.AMBIGUOUS
            if lab != oracle.FREE:
                ok = False
                break
            cost += float(c)
        if not ok:
            continue
        pts = [verts[l][idx[l]] for l in range(L + 2)]
        chi = tuple(oracle.polygon_winding(pts, p) for p in centres)
        if chi not in best or cost < best[chi]:
            best[chi] = cost
    return best, verts, edges


@pytest.mark.parametrize("seed,n_obs,M,L", [(3, 4, 5, 3), (7, 6, 4, 3), (12, 3, 6, 2)])
def test_class_value_iteration_equals_brute_force(seed, n_obs, M, L):
    sc = scenes.point2d_scene(seed, n_obs)
    H = 16
    Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    centres = oracle.obstacle_centres_2d(sc)
    best, verts, edges = _chain_labels_brute_force(sc, Q, H, centres)
    tables = oracle.class_value_iteration(edges, verts, centres)
    got = {chi: c for chi, (c, _, _) in tables[0][0].items()}
    assert set(got) == set(best)
    for chi in best:
        assert got[chi] == pytest.approx(best[chi], rel=1e-12)
    # the best over classes is the plain value iteration's optimum
    V, _, _ = oracle.value_iteration(edges, ambiguous_free=False)
    if best:
        assert min(best.values()) == pytest.approx(V[0][0], rel=1e-12)
    else:
        assert math.isinf(V[0][0])
    # every extracted chain carries its label and its cost
    for chi, (c, path) in oracle.class_paths(tables).items():
        pts = [verts[0][0]] + [verts[l + 1][path[l]] for l in range(L)] + [verts[-1][0]]
        assert tuple(oracle.polygon_winding(pts, p) for p in centres) == chi
        total, worst = oracle.path_cost(sc, Q, np.array(path), H)
        assert total == pytest.approx(c, rel=1e-12) and worst > oracle.EPS_DEFAULT


def test_class_value_iteration_single_disk_has_two_sides():
    """One disk on the straight line between the endpoints: chains pass it on either side, two labels
    (winding 0 and +-1 about its centre, depending on the side relative to the closing segment)."""
    base = scenes.point2d_scene(0, 0)
    disk = np.array([[0.05, -0.03, 0.0, 0.3]], np.float32)   # off the segment q0 -> qg
    sc = scenes.Scene(base.robot, disk, np.zeros((0, 6), np.float32), base.q_start, base.q_goal)
    L, M, H = 2, 24, 16
    Q = oracle.sample_uniform(5, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    edges = oracle.realize_edges(sc, verts, H)
    tables = oracle.class_value_iteration(edges, verts, oracle.obstacle_centres_2d(sc))
    labels = set(tables[0][0])
    # passing on the closing segment's side of the centre winds 0 times, the other side once
    assert labels in ({(0,), (1,)}, {(0,), (-1,)})


@pytest.mark.parametrize("seed", [0, 4])
def test_goal_set_value_iteration_equals_brute_force(seed):
    """Alg. 1's goal set G with terminal values V_g: the value of q0 is the minimum over every chain and every
    goal of the chain's cost plus that goal's value; the last layer's minimiser is that goal."""
    sc = scenes.point2d_scene(seed, 4)
    L, M, H = 2, 6, 16
    Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    goals = np.array([sc.q_goal, [0.85, -0.7], [-0.75, 0.8]], np.float32)
    vals = np.array([0.0, 0.4, 0.15])
    verts = oracle.layer_vertices(Q, sc.q_start, goals)
    assert verts[-1].shape == (3, 2)
    edges = oracle.realize_edges(sc, verts, H)
    best, best_goal = math.inf, -1
    for chain in itertools.product(range(M), repeat=L):
        for gi in range(3):
            idx = [0] + list(chain) + [gi]
            total = 0.0
            for l in range(L + 1):
                lab = edges[l][0][idx[l], idx[l + 1]]
                assert lab != oracle.AMBIGUOUS
                if lab != oracle.FREE:
                    total = math.inf
                    break
                total += float(edges[l][1][idx[l], idx[l + 1]])
            total += vals[gi]
            if total < best:
                best, best_goal = total, gi
    sol = oracle.solve(sc, Q, H, goals=goals, goal_values=vals)
    assert sol.cost_lo == pytest.approx(best, rel=1e-12)
    if math.isfinite(best):
        assert sol.sigma[L][sol.path[-1]] == best_goal
        np.testing.assert_array_equal(sol.V_lo[-1], vals)


# ---------------------------------------------------------------------------
# layer sampling on C_free (Sec. III: pi_m lives on C_m and C_free)
# ---------------------------------------------------------------------------

def test_free_sampler_without_obstacles_is_the_uniform_sampler():
    sc = scenes.point2d_scene(0, 0)
    Q, used, und = oracle.sample_free(sc, 7, 0, 3, 50)
    np.testing.assert_array_equal(Q.view(np.uint32),
                                  oracle.sample_uniform(7, 0, 3, 50, sc.robot.q_lo, sc.robot.q_hi).view(np.uint32))
    assert np.all(used == 0) and not und.any()


def _arm_scene_with_free_ends(seed):
    sc = scenes.arm_scene(seed, 7, 30)
    return scenes.pick_endpoints(sc, lambda q: oracle.config_free(sc, q))


@pytest.mark.parametrize("kind", ["point2d", "arm"])
def test_free_sampler_keeps_free_uniform_samples_and_rejects_colliding_ones(kind):
    sc = scenes.point2d_scene(2, 14) if kind == "point2d" else _arm_scene_with_free_ends(1)
    L, M = 3, 200
    Q, used, und = oracle.sample_free(sc, 11, 2, L, M, max_attempts=256)
    U = oracle.sample_uniform(11, 2, L, M, sc.robot.q_lo, sc.robot.q_hi)
    lab_u, _ = oracle.config_labels(sc, U.reshape(-1, sc.robot.dof))
    lab_q, _ = oracle.config_labels(sc, Q.reshape(-1, sc.robot.dof))
    free_u = (lab_u == oracle.FREE).reshape(L, M)
    # a uniform sample that is free is kept as is (attempt 0)
    np.testing.assert_array_equal(Q[free_u].view(np.uint32), U[free_u].view(np.uint32))
    assert np.all(used[free_u] == 0)
    # every accepted sample is free; colliding uniform samples were replaced
    acc = used >= 0
    assert np.all(lab_q.reshape(L, M)[acc] == oracle.FREE)
    replaced = ~free_u & acc
    assert replaced.any() and np.all(used[replaced] >= 1)
    assert acc.mean() > 0.99


def test_free_sampler_is_uniform_on_the_free_space():
    """Accepted samples against an independent uniform batch restricted to C_free (two-sample KS per
    coordinate), on a scene where a third of the box collides."""
    sc = scenes.point2d_scene(4, 25)
    Q, used, _ = oracle.sample_free(sc, 5, 0, 4, 1000, max_attempts=256)
    X = Q.reshape(-1, 2)[used.reshape(-1) >= 0]
    rng = np.random.default_rng(99)
    Y = rng.uniform(sc.robot.q_lo, sc.robot.q_hi, (20000, 2)).astype(np.float32)
    Y = Y[oracle.config_labels(sc, Y)[0] == oracle.FREE]
    frac_coll = 1 - len(Y) / 20000
    assert 0.1 < frac_coll < 0.7
    for k in range(2):
        assert stats.ks_2samp(X[:, k], Y[:, k]).pvalue > 1e-3, k


# ---------------------------------------------------------------------------
# Weighted length (App. "General Costs"): w(q) = 1 + sum_b a_b max(0, 1 -
# |q - c_b|^2 / s_b^2), edge cost = trapezoid rule of w on the H waypoints
# ---------------------------------------------------------------------------

def test_weight_field_hand_values():
    b = np.array([[0.0, 0.0, 2.0, 3.0],          # centre (0, 0), s = 2, a = 3
                  [1.0, 0.0, 1.0, 0.5]])         # centre (1, 0), s = 1, a = 0.5
    assert oracle.weight([0.0, 0.0], b[:1]) == 4.0                 # centre: 1 + a
    assert oracle.weight([1.0, 0.0], b[:1]) == 1.0 + 3.0 * 0.75    # |q - c| = s / 2
    assert oracle.weight([0.0, 2.0], b[:1]) == 1.0                 # on the support's boundary
    assert oracle.weight([0.0, -5.0], b[:1]) == 1.0                # outside: the clamp, not a negative bump
    assert oracle.weight([1.0, 0.0], b) == 1.0 + 3.0 * 0.75 + 0.5  # overlapping bumps add
    assert oracle.weight([0.0, 0.0], np.zeros((0, 4))) == 1.0


def test_weighted_length_without_weight_is_the_length():
    rng = np.random.default_rng(5)
    for _ in range(20):
        u, v = rng.uniform(-1, 1, (2, 7)).astype(np.float32)
        length = oracle.lib().orc_edge_length(7, oracle._ptr(u, oracle._f32p), oracle._ptr(v, oracle._f32p))
        assert oracle.weighted_length(u, v, 32, None) == length
        zero = np.concatenate([rng.uniform(-1, 1, 7), [0.7, 0.0]])[None, :]    # amplitude 0
        assert oracle.weighted_length(u, v, 32, zero) == pytest.approx(length, rel=1e-15)
        far = np.concatenate([np.full(7, 9.0), [0.5, 4.0]])[None, :]           # support away from the edge
        assert oracle.weighted_length(u, v, 32, far) == pytest.approx(length, rel=1e-15)


@pytest.mark.parametrize("H", [2, 3, 17])
def test_weighted_length_of_a_quadratic_weight_closed_form(H):
    """Inside one bump w(u + t e) = f(t) is a quadratic in t; the composite
    trapezoid rule with n = H - 1 intervals then errs by exactly
    (f'(1) - f'(0)) h^2 / 12 = f'' h^2 / 12, h = 1/n (Euler-Maclaurin ends at
    the first derivative term).  Dyadic endpoints make every waypoint exact."""
    u = np.array([-0.25, 0.125], np.float32)
    v = np.array([0.5, -0.375], np.float32)
    c, s, a = np.array([0.0625, 0.0]), 2.0, 3.0
    e, p = v.astype(np.float64) - u, u.astype(np.float64) - c
    integral = 1.0 + a * (1.0 - (p @ p + p @ e + (e @ e) / 3.0) / s ** 2)
    f2 = -2.0 * a * (e @ e) / s ** 2
    h = 1.0 / (H - 1)
    expect = math.sqrt(e @ e) * (integral + f2 * h * h / 12.0)
    got = oracle.weighted_length(u, v, H, np.concatenate([c, [s, a]])[None, :])
    assert got == pytest.approx(expect, rel=1e-13)


def test_weighted_length_converges_to_the_exact_integral():
    """An edge that crosses a bump's support: the exact integral is the
    closed form of the quadratic over the chord [t1, t2]; the trapezoid rule
    on the waypoints approaches it as H grows."""
    u = np.array([-0.8, 0.1], np.float32)
    v = np.array([0.7, 0.35], np.float32)
    c, s, a = np.array([0.05, 0.3]), 0.45, 2.5
    e, p = v.astype(np.float64) - u, u.astype(np.float64) - c
    A, B, C0 = e @ e, 2.0 * (p @ e), p @ p - s * s
    r = math.sqrt(B * B - 4.0 * A * C0)
    t1, t2 = max((-B - r) / (2 * A), 0.0), min((-B + r) / (2 * A), 1.0)
    bump = a * ((t2 - t1) * (1.0 - (p @ p) / s ** 2) - (p @ e) / s ** 2 * (t2 ** 2 - t1 ** 2)
                - A / (3.0 * s ** 2) * (t2 ** 3 - t1 ** 3))
    exact = math.sqrt(A) * (1.0 + bump)
    b = np.concatenate([c, [s, a]])[None, :]
    assert abs(oracle.weighted_length(u, v, 17, b) / exact - 1.0) < 1e-3
    assert abs(oracle.weighted_length(u, v, 16385, b) / exact - 1.0) < 1e-7


def test_weighted_length_is_between_length_and_w_max_times_length():
    rng = np.random.default_rng(11)
    b = np.concatenate([rng.uniform(-1, 1, (6, 3)), rng.uniform(0.2, 1.0, (6, 1)), rng.uniform(0, 2, (6, 1))], axis=1)
    w_max = 1.0 + b[:, 4].sum()
    for _ in range(50):
        u, v = rng.uniform(-1, 1, (2, 3)).astype(np.float32)
        length = float(np.linalg.norm(v.astype(np.float64) - u))
        wl = oracle.weighted_length(u, v, 24, b)
        assert length * (1 - 1e-15) <= wl <= w_max * length * (1 + 1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_weighted_value_iteration_equals_brute_force(seed):
    sc, Q = _small_problem(seed, M=4, L=3, n_obs=6 + seed)
    H = 16
    rng = np.random.default_rng(100 + seed)
    b = np.concatenate([rng.uniform(-1, 1, (3, 2)), rng.uniform(0.3, 0.8, (3, 1)), rng.uniform(0.5, 3, (3, 1))], axis=1)
    sol = oracle.solve(sc, Q, H, bumps=b)
    verts = sol.verts
    best, best_chain = math.inf, None
    for chain in itertools.product(range(4), repeat=3):
        idx = (0,) + chain + (0,)
        total = 0.0
        for l in range(4):
            lab, _ = sol.edges[l]
            if lab[idx[l], idx[l + 1]] != oracle.FREE:
                total = math.inf
                break
            total += oracle.weighted_length(verts[l][idx[l]], verts[l + 1][idx[l + 1]], H, b)
        if total < best:
            best, best_chain = total, chain
    assert sol.cost_lo == pytest.approx(best, rel=1e-12) if math.isfinite(best) else math.isinf(sol.cost_lo)
    if math.isfinite(best):
        assert tuple(sol.path) == best_chain
        total, _ = oracle.path_cost(sc, Q, sol.path, H, bumps=b)
        assert total == pytest.approx(best, rel=1e-12)


# ---------------------------------------------------------------------------
# AO-GTMP epochs (Sec. IV-D) and the edge limit l_M(r) (Sec. V): hand values
# ---------------------------------------------------------------------------

def test_ao_edge_limit_hand_values():
    # c = 6 over L + 1 = 3 edges, 2r + varsigma = 1: l = 2 + 1 = 3
    assert oracle.ao_edge_limit(6.0, 2, 0.25, 0.5) == np.float32(3.0)
    assert oracle.ao_edge_limit(6.0, 2, 0.25, 0.5, base=2.5) == np.float32(2.5)   # the context's own limit caps it
    assert oracle.ao_edge_limit(np.inf, 2, 0.25, 0.5, base=7.0) == np.float32(7.0)  # no chain yet
    assert oracle.ao_edge_limit(10.0, 4, 0.0, 0.0) == np.float32(2.0)              # r = varsigma = 0: c / (L + 1)


def test_ao_schedule_saturation_without_a_reach():
    """reach = +inf: epochs end only when the samples reach their cap, then one more layer."""
    seq, L, M = [], 2, 8
    for _ in range(7):
        seq.append((L, M))
        L, M, _ = oracle.ao_next(L, M, 3.0, 5, 8, 32, math.inf, 0.1, 0.1)
    assert seq == [(2, 8), (2, 16), (2, 32), (3, 8), (3, 16), (3, 32), (4, 8)]
    assert oracle.ao_next(5, 32, 3.0, 5, 8, 32, math.inf, 0.0, 0.0) == (5, 8, True)   # at capacity: fresh epoch


def test_ao_schedule_layer_rule_hand_values():
    # reach 3, 2r + varsigma = 1: a chain of cost c needs L + 1 >= c / 2 edges
    assert oracle.ao_next(2, 8, 9.0, 8, 8, 64, 3.0, 0.25, 0.5) == (4, 8, True)     # ceil(4.5) - 1 = 4 > 2
    assert oracle.ao_next(2, 8, 5.5, 8, 8, 64, 3.0, 0.25, 0.5) == (2, 16, False)   # ceil(2.75) - 1 = 2: holds
    assert oracle.ao_next(2, 8, 6.5, 8, 8, 64, 3.0, 0.25, 0.5) == (3, 8, True)     # ceil(3.25) - 1 = 3
    assert oracle.ao_next(2, 8, 40.0, 6, 8, 64, 3.0, 0.25, 0.5) == (6, 8, True)    # clamped to the capacity
    assert oracle.ao_next(6, 8, 40.0, 6, 8, 64, 3.0, 0.25, 0.5) == (6, 16, False)  # at capacity the rule rests
    assert oracle.ao_next(2, 8, math.inf, 8, 8, 64, 3.0, 0.25, 0.5) == (2, 16, False)  # no chain yet


def test_ao_run_epochs_on_a_planar_scene():
    """The oracle's own run: best cost non-increasing, epochs exactly where the rules put them, every edge of
    each stage's chain within that stage's limit, fresh samples at each epoch."""
    sc = scenes.point2d_scene(3, 8)
    sched = dict(L0=1, M0=4, M_max=16, stages=7, reach=1.2, r=0.05, varsigma=0.05, limit_edges=True)
    log = oracle.ao_run(sc, 5, H=16, L_cap=5, **sched)
    best = math.inf
    for k, rec in enumerate(log):
        assert rec["status"] == 0
        assert rec["best_cost"] <= best
        best = rec["best_cost"]
        if k + 1 < len(log):
            nxt = log[k + 1]
            L2, M2, new = oracle.ao_next(rec["L"], rec["M"], np.float32(best), 5, 4, 16, 1.2, 0.05, 0.05)
            assert (nxt["L"], nxt["M"], nxt["epoch"] == rec["epoch"] + 1) == (L2, M2, new)
            if not new:   # within an epoch the samples are kept (nested graphs)
                np.testing.assert_array_equal(nxt["Q"][:, :rec["M"]], rec["Q"])
        sol = rec["solution"]
        if math.isfinite(sol.cost_lo):
            verts = [sc.q_start] + [rec["Q"][l, sol.path[l]] for l in range(rec["L"])] + [sc.q_goal]
            for a, b in zip(verts[:-1], verts[1:]):
                assert np.linalg.norm(b.astype(np.float64) - a) <= float(rec["edge_limit"]) * (1 + 1e-7)
    assert len({r["epoch"] for r in log}) >= 2


# ---------------------------------------------------------------------------
# Coverage probability (Sec. V): the layerwise-hitting instance of the
# appendix's proposition, where the bound holds with equality
# ---------------------------------------------------------------------------

def corridor_cover_probability(w, N, L):
    """A free strip |y| < w of the box [-1, 1]^2 (uniform samples land in it with
    probability tau = w), convex, walled off from the rest: a chain exists iff
    every layer has a sample in the strip, so Pr[cover] = (1 - (1 - w)^N)^L."""
    return (1.0 - (1.0 - w) ** N) ** L


def test_corridor_coverage_frequency_matches_the_closed_form():
    w, N, L, H, K = 0.1, 12, 3, 16, 600
    sc = scenes.corridor_scene(w, 0.3)
    hits = 0
    for r in range(K):
        Q = oracle.sample_uniform(77, r, L, N, sc.robot.q_lo, sc.robot.q_hi)
        sol = oracle.solve(sc, Q, H)
        if math.isfinite(sol.cost_lo):
            hits += 1
            # every vertex of the returned chain lies in the strip
            assert all(abs(float(Q[l, sol.path[l], 1])) < w for l in range(L))
    p = corridor_cover_probability(w, N, L)
    sigma = math.sqrt(p * (1 - p) / K)
    assert abs(hits / K - p) < 4.5 * sigma, (hits / K, p)
    # the proposition's upper bound (1 - (1 - tau)^N)^M with tau = w is attained here; the theorem's lower
    # bound 1 - L (1 - p_m)^N with waypoint balls of radius w is below it
    p_m = math.pi * w * w / 4.0
    assert 1.0 - L * (1.0 - p_m) ** N <= p


# ---------------------------------------------------------------------------
# Coverage of one class (Thm. 1 of Sec. V with the straight-line case of its
# tube lemma): a lower bound from waypoint balls
# ---------------------------------------------------------------------------

TUBE = dict(w=0.45, t=0.3, x0=0.5, L=2, N=256, H=16, r=0.1)


def tube_waypoint_balls(cfg):
    """The reference path f = the segment q0 -> qg (length 1, clearance 0.45 in the strip and the box), its
    layer points f(t_m), t_m = m / (L + 1), and the ball mass p_m = pi r^2 / 4 under uniform sampling of
    [-1, 1]^2 (the balls lie inside the box and the free strip)."""
    L, x0 = cfg["L"], cfg["x0"]
    centres = [np.array([-x0 + 2 * x0 * m / (L + 1), 0.0]) for m in range(1, L + 1)]
    length, clearance = 2 * x0, min(cfg["w"], 1.0 - x0)
    # the straight-line case of the tube lemma needs length / (L + 1) + r < clearance
    assert length / (L + 1) + cfg["r"] < clearance
    return centres, math.pi * cfg["r"] ** 2 / 4.0


def ball_chain(Q, centres, r):
    """Indices of one sample per layer inside its waypoint ball (the first), or None if a layer misses."""
    out = []
    for l, c in enumerate(centres):
        d = np.linalg.norm(Q[l].astype(np.float64) - c[None, :], axis=1)
        hit = np.nonzero(d < r)[0]
        if hit.size == 0:
            return None
        out.append(int(hit[0]))
    return out


def test_single_class_coverage_lower_bound():
    """Thm. 1: Pr[cover] >= 1 - sum_m (1 - p_m)^N (straight-line planner: a free segment is always found, so
    the planner term vanishes).  The free strip is simply connected, so covering f's class is finding a chain.
    Per graph: whenever every layer has a sample in its waypoint ball, the chain through those samples is free
    at every waypoint (the tube lemma) and the optimum costs at most as much; over 300 graphs the frequency of
    'every layer hits' matches its exact value prod_m (1 - (1 - p_m)^N), and coverage is at least the bound."""
    cfg = TUBE
    sc = scenes.corridor_scene(cfg["w"], cfg["t"], cfg["x0"])
    centres, p_m = tube_waypoint_balls(cfg)
    L, N, H, K = cfg["L"], cfg["N"], cfg["H"], 300
    all_hit = covered = 0
    for k in range(K):
        Q = oracle.sample_uniform(91, k, L, N, sc.robot.q_lo, sc.robot.q_hi)
        sol = oracle.solve(sc, Q, H)
        covered += math.isfinite(sol.cost_lo)
        chain = ball_chain(Q, centres, cfg["r"])
        if chain is None:
            continue
        all_hit += 1
        total, worst = oracle.path_cost(sc, Q, np.array(chain), H)
        assert worst > 0.0, (k, worst)                         # the ball chain is free
        assert sol.cost_lo <= total * (1 + 1e-12), (k, sol.cost_lo, total)
    exact = (1.0 - (1.0 - p_m) ** N) ** L
    bound = 1.0 - L * (1.0 - p_m) ** N
    assert bound <= exact
    sigma = math.sqrt(exact * (1 - exact) / K)
    assert abs(all_hit / K - exact) < 4.5 * sigma, (all_hit / K, exact)
    assert covered / K >= bound - 4.5 * sigma, (covered / K, bound)
    assert covered >= all_hit
