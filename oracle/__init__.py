"""CPU oracle for the layered-graph planner (GTMP, straight-line local planner).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``, never by the library.  It shares no
code with the CUDA path: the per-edge work lives in ``gtmp_oracle.c`` (plain C,
FP64, OpenMP over edges), the graph search below is plain numpy in FP64.

What it computes (Sec. III-A/B, Sec. IV-B and Alg. 1 of the paper): for
layers V_0 = {q0}, V_1..V_L (the samples), V_{L+1} = {qg}, every edge between
adjacent layers gets a tri-state label from the straight-line checker and the
cost ||v - u||; the backward value iteration
    J_{L+1}(qg) = 0,  J_l(u) = min_v c(u, v) + J_{l+1}(v)
(absent edges cost +inf) gives the cost-to-go of every vertex and a minimiser
sigma_l(u) (first index among equal values); following sigma from q0 gives one
minimum-cost chain.  Edges whose label is "ambiguous" (a waypoint within
+-eps of contact) are resolved both ways: ambiguous -> free gives V_lo,
ambiguous -> collide gives V_hi; any correct checker's optimum lies between.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

FREE, COLLIDE, AMBIGUOUS = 0, 1, 2
TAG_UNIFORM, TAG_INFORMED, TAG_COIN = 1, 2, 3
EPS_DEFAULT = 1e-6

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        _declare(_lib)
    return _lib


class OrcScene(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("dof", ctypes.c_int32),
        ("dh", ctypes.POINTER(ctypes.c_double)),
        ("spl", ctypes.c_int32),
        ("link_sph", ctypes.POINTER(ctypes.c_double)),
        ("point_radius", ctypes.c_double),
        ("n_s", ctypes.c_int32), ("spheres", ctypes.POINTER(ctypes.c_double)),
        ("n_b", ctypes.c_int32), ("boxes", ctypes.POINTER(ctypes.c_double)),
    ]


class OrcEllipsoid(ctypes.Structure):
    _fields_ = [("centre", ctypes.c_float * 64), ("axis", ctypes.c_float * 64),
                ("r1", ctypes.c_float), ("r2", ctypes.c_float), ("cmin", ctypes.c_float)]


_P = ctypes.POINTER
_u32p, _f32p, _f64p, _i8p = _P(ctypes.c_uint32), _P(ctypes.c_float), _P(ctypes.c_double), _P(ctypes.c_int8)


def set_threads(n: int = 0) -> int:
    """OpenMP threads of the per-edge loops (n <= 0 leaves them); returns the count in effect."""
    return int(lib().orc_set_threads(int(n)))


def _declare(L):
    L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.orc_sample_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, _f32p, _f32p, _f32p]
    L.orc_num_robot_spheres.argtypes = [_P(OrcScene)]
    L.orc_num_robot_spheres.restype = ctypes.c_int
    L.orc_fk_spheres.argtypes = [_P(OrcScene), _f64p, _f64p]
    L.orc_config_margin.argtypes = [_P(OrcScene), _f64p]
    L.orc_config_margin.restype = ctypes.c_double
    L.orc_config_labels.argtypes = [_P(OrcScene), ctypes.c_int, _f32p, ctypes.c_double, _i8p, _f64p]
    L.orc_sample_free.argtypes = [_P(OrcScene), ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, _f32p,
                                  _f32p, ctypes.c_double, ctypes.c_int, _f32p, _P(ctypes.c_int32), _i8p]
    L.orc_edge_label.argtypes = [_P(OrcScene), _f32p, _f32p, ctypes.c_int, ctypes.c_double]
    L.orc_edge_label.restype = ctypes.c_int
    L.orc_edge_length.argtypes = [ctypes.c_int, _f32p, _f32p]
    L.orc_edge_length.restype = ctypes.c_double
    L.orc_edge_block.argtypes = [_P(OrcScene), _f32p, ctypes.c_int, _f32p, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_double, _f64p, ctypes.c_int, _i8p, _f64p]
    L.orc_weight.argtypes = [ctypes.c_int, _f64p, _f64p, ctypes.c_int]
    L.orc_weight.restype = ctypes.c_double
    L.orc_weighted_length.argtypes = [ctypes.c_int, _f32p, _f32p, ctypes.c_int, _f64p, ctypes.c_int]
    L.orc_weighted_length.restype = ctypes.c_double
    L.orc_edge_margins.argtypes = [_P(OrcScene), _f32p, _f32p, ctypes.c_int, _f64p]
    L.orc_informed_params.argtypes = [ctypes.c_int, _f32p, _f32p, ctypes.c_float, _P(OrcEllipsoid)]
    L.orc_informed_attempt.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_int, _P(OrcEllipsoid), _f32p, _f32p, _f32p]
    L.orc_informed_attempt.restype = ctypes.c_int
    L.orc_expand_layers.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    _f32p, _f32p, _f32p, _f32p, ctypes.c_float, ctypes.c_int, _f32p]
    L.orc_expand_layers.restype = ctypes.c_int
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_set_threads.restype = ctypes.c_int


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Philox and uniform layer sampling
# ---------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def sample_uniform(seed: int, restart: int, L: int, M: int, q_lo, q_hi) -> np.ndarray:
    """Alg. 1 uniform layer samples, float32 [L][M][dof]."""
    lo, hi = _c32(q_lo), _c32(q_hi)
    dof = lo.shape[0]
    Q = np.zeros((L, M, dof), np.float32)
    lib().orc_sample_uniform(seed, restart, L, M, dof, _ptr(lo, _f32p), _ptr(hi, _f32p), _ptr(Q, _f32p))
    return Q


# ---------------------------------------------------------------------------
# Scene marshalling and geometry
# ---------------------------------------------------------------------------

class _SceneHandle:
    """Keeps the FP64 copies alive while the C struct points at them."""

    def __init__(self, scene):
        r = scene.robot
        self.dh = _c64(r.dh)
        self.link = _c64(r.link_spheres) if r.link_spheres.size else np.zeros(4)
        self.spheres = _c64(scene.spheres) if scene.spheres.size else np.zeros(4)
        self.boxes = _c64(scene.boxes) if scene.boxes.size else np.zeros(6)
        self.s = OrcScene(int(r.kind), int(r.dof), _ptr(self.dh, _f64p), int(r.spheres_per_link),
                          _ptr(self.link, _f64p), float(r.point_radius),
                          int(scene.spheres.shape[0]), _ptr(self.spheres, _f64p),
                          int(scene.boxes.shape[0]), _ptr(self.boxes, _f64p))
        self.ref = ctypes.byref(self.s)
        self.dof = int(r.dof)


def sample_free(scene, seed: int, restart: int, L: int, M: int, max_attempts: int = 64, eps=EPS_DEFAULT):
    """Layer samples on C_free by rejection (Sec. III's pi_m on C_free): attempt 0 is the uniform sample,
    attempt a >= 1 its own Philox block; returns Q float32 [L][M][dof], the accepted attempt per sample
    (-1: none of max_attempts was free, the last is kept) and an `undecided` flag (an earlier attempt lay in
    the +-eps band)."""
    dof = scene.robot.dof
    lo, hi = _c32(scene.robot.q_lo), _c32(scene.robot.q_hi)
    Q = np.zeros((L, M, dof), np.float32)
    used = np.zeros(L * M, np.int32)
    und = np.zeros(L * M, np.int8)
    h = _SceneHandle(scene)
    lib().orc_sample_free(h.ref, seed, restart, L, M, _ptr(lo, _f32p), _ptr(hi, _f32p), eps, max_attempts,
                          _ptr(Q, _f32p), used.ctypes.data_as(_P(ctypes.c_int32)), _ptr(und, _i8p))
    return Q, used.reshape(L, M), und.reshape(L, M).astype(bool)


def fk_spheres(scene, q) -> np.ndarray:
    h = _SceneHandle(scene)
    S = lib().orc_num_robot_spheres(h.ref)
    out = np.zeros((S, 4))
    qq = _c64(q)
    lib().orc_fk_spheres(h.ref, _ptr(qq, _f64p), _ptr(out, _f64p))
    return out


def config_margin(scene, q) -> float:
    h = _SceneHandle(scene)
    qq = _c64(q)
    return lib().orc_config_margin(h.ref, _ptr(qq, _f64p))


def config_labels(scene, Q, eps=EPS_DEFAULT):
    """Tri-state labels and margins of configurations Q[n][dof] (float32)."""
    h = _SceneHandle(scene)
    q = _c32(Q).reshape(-1, h.dof)
    n = q.shape[0]
    labels = np.zeros(n, np.int8)
    margins = np.zeros(n)
    lib().orc_config_labels(h.ref, n, _ptr(q, _f32p), eps, _ptr(labels, _i8p), _ptr(margins, _f64p))
    return labels, margins


def config_free(scene, Q, eps=EPS_DEFAULT):
    labels, _ = config_labels(scene, Q, eps)
    return labels == FREE


def _bumps(bumps, dof):
    """Weight bumps as float64 [K][dof + 2] (centre, radius s, amplitude a); K = 0 when None."""
    if bumps is None:
        return np.zeros((0, dof + 2)), 0
    b = _c64(bumps).reshape(-1, dof + 2)
    return b, b.shape[0]


def edge_block(scene, A, B, H: int, eps=EPS_DEFAULT, max_len=math.inf, bumps=None):
    """Labels int8 [na][nb] and FP64 costs of every edge A[a] -> B[b].

    Cost: the length, or with weight bumps the weighted length of App.
    "General Costs" (trapezoid rule on the H waypoints; see weighted_length).
    """
    h = _SceneHandle(scene)
    A = _c32(A).reshape(-1, h.dof)
    B = _c32(B).reshape(-1, h.dof)
    labels = np.zeros((A.shape[0], B.shape[0]), np.int8)
    costs = np.zeros((A.shape[0], B.shape[0]))
    wb, K = _bumps(bumps, h.dof)
    lib().orc_edge_block(h.ref, _ptr(A, _f32p), A.shape[0], _ptr(B, _f32p), B.shape[0], H, eps, max_len,
                         _ptr(wb, _f64p), K, _ptr(labels, _i8p), _ptr(costs, _f64p))
    return labels, costs


def weight(q, bumps) -> float:
    """w(q) = 1 + sum_b a_b max(0, 1 - |q - c_b|^2 / s_b^2) (App. "General Costs": 1 <= w <= W, Lipschitz)."""
    q = _c64(q)
    wb, K = _bumps(bumps, q.shape[0])
    return lib().orc_weight(q.shape[0], _ptr(q, _f64p), _ptr(wb, _f64p), K)


def weighted_length(u, v, H: int, bumps) -> float:
    """Integral of w along the straight edge u -> v by the trapezoid rule on its H waypoints:
    |v - u| / (H - 1) * (w_0 / 2 + w_1 + ... + w_{H-2} + w_{H-1} / 2)."""
    u, v = _c32(u), _c32(v)
    wb, K = _bumps(bumps, u.shape[0])
    return lib().orc_weighted_length(u.shape[0], _ptr(u, _f32p), _ptr(v, _f32p), H, _ptr(wb, _f64p), K)


def edge_margins(scene, u, v, H: int) -> np.ndarray:
    h = _SceneHandle(scene)
    u, v = _c32(u), _c32(v)
    out = np.zeros(H)
    lib().orc_edge_margins(h.ref, _ptr(u, _f32p), _ptr(v, _f32p), H, _ptr(out, _f64p))
    return out


# ---------------------------------------------------------------------------
# Informed sampling and expand-samples (AO-GTMP)
# ---------------------------------------------------------------------------

def informed_params(q0, qg, c: float):
    q0, qg = _c32(q0), _c32(qg)
    e = OrcEllipsoid()
    lib().orc_informed_params(q0.shape[0], _ptr(q0, _f32p), _ptr(qg, _f32p), np.float32(c), ctypes.byref(e))
    d = q0.shape[0]
    return dict(centre=np.array(e.centre[:d], np.float32), axis=np.array(e.axis[:d], np.float32),
                r1=np.float32(e.r1), r2=np.float32(e.r2), cmin=np.float32(e.cmin), _raw=e)


def informed_attempt(seed, i, l, attempt, params, q_lo, q_hi):
    lo, hi = _c32(q_lo), _c32(q_hi)
    x = np.zeros(lo.shape[0], np.float32)
    ok = lib().orc_informed_attempt(seed, i, l, attempt, lo.shape[0], ctypes.byref(params["_raw"]),
                                    _ptr(lo, _f32p), _ptr(hi, _f32p), _ptr(x, _f32p))
    return bool(ok), x


def expand_layers(seed, Q_old, M_new, q0, qg, q_lo, q_hi, c_best, max_attempts=1 << 16):
    """expand-samples of Alg. 1: returns (status, Q float32 [L][M_new][dof])."""
    Q_old = _c32(Q_old)
    L, M_old, dof = Q_old.shape
    Q = np.zeros((L, M_new, dof), np.float32)
    Q[:, :M_old] = Q_old
    lo, hi, a, b = _c32(q_lo), _c32(q_hi), _c32(q0), _c32(qg)
    st = lib().orc_expand_layers(seed, L, M_old, M_new, dof, _ptr(lo, _f32p), _ptr(hi, _f32p), _ptr(a, _f32p),
                                 _ptr(b, _f32p), np.float32(c_best), max_attempts, _ptr(Q, _f32p))
    return st, Q


# ---------------------------------------------------------------------------
# Graph search on the layered DAG (Sec. IV-B; Alg. 1 gtmp)
# ---------------------------------------------------------------------------

def layer_vertices(Q, q0, qg):
    """Vertex sets V_0 = {q0}, V_1..V_L = Q[0..L-1], V_{L+1} = {qg} (qg [dof]) or the goal set (qg [G][dof])."""
    goals = _c32(qg)
    goals = goals[None, :] if goals.ndim == 1 else goals
    return [_c32(q0)[None, :]] + [_c32(Q[l]) for l in range(Q.shape[0])] + [goals]


def realize_edges(scene, verts, H, eps=EPS_DEFAULT, max_len=math.inf, bumps=None):
    """Labels and costs of every transition l -> l+1, l = 0..L."""
    return [edge_block(scene, verts[l], verts[l + 1], H, eps, max_len, bumps) for l in range(len(verts) - 1)]


def value_iteration(edges, ambiguous_free: bool, terminal=None):
    """Backward pass J_l(u) = min_v c(u,v) + J_{l+1}(v); returns V, sigma, second.

    J_{L+1} = the goals' terminal values V_g (Alg. 1; `terminal`, default 0).
    V[l] float64 [n_l], sigma[l] int64 [n_l] (-1 if no finite candidate),
    second[l] = the second smallest candidate value (over distinct v).
    """
    n_layers = len(edges) + 1
    V = [None] * n_layers
    sigma = [None] * n_layers
    second = [None] * n_layers
    n_goals = edges[-1][0].shape[1]
    V[-1] = np.zeros(n_goals) if terminal is None else np.asarray(terminal, np.float64).reshape(n_goals)
    sigma[-1] = np.full(V[-1].shape, -1)
    second[-1] = np.full(V[-1].shape, np.inf)
    for l in range(len(edges) - 1, -1, -1):
        labels, costs = edges[l]
        ok = (labels == FREE) | ((labels == AMBIGUOUS) if ambiguous_free else False)
        cand = np.where(ok, costs + V[l + 1][None, :], np.inf)
        arg = np.argmin(cand, axis=1)                      # first index among equal minima
        best = cand[np.arange(cand.shape[0]), arg]
        if cand.shape[1] > 1:
            part = np.sort(cand, axis=1)
            sec = part[:, 1]
        else:
            sec = np.full(cand.shape[0], np.inf)
        V[l] = best
        sigma[l] = np.where(np.isfinite(best), arg, -1)
        second[l] = sec
    return V, sigma, second


def extract_path(sigma):
    """Follow the minimisers from q0: one index per sample layer 1..L (-1 if infeasible)."""
    L = len(sigma) - 2
    path = np.full(L, -1, np.int64)
    i = 0
    if sigma[0][0] < 0:
        return path
    for l in range(0, L):
        i = sigma[l][i]
        path[l] = i
    return path


@dataclass
class Solution:
    V_lo: list
    V_hi: list
    sigma: list
    second: list
    path: np.ndarray
    cost_lo: float
    cost_hi: float
    edges: list
    verts: list


def solve(scene, Q, H: int, eps=EPS_DEFAULT, max_len=math.inf, goals=None, goal_values=None,
          bumps=None) -> Solution:
    """gtmp of Alg. 1 for given samples Q float32 [L][M][dof]; the goal set G with terminal values V_g
    (`goals` [G][dof], `goal_values` [G]) replaces the scene's goal when given; `bumps` makes the edge
    cost the weighted length."""
    verts = layer_vertices(Q, scene.q_start, scene.q_goal if goals is None else goals)
    edges = realize_edges(scene, verts, H, eps, max_len, bumps)
    V_lo, sig_lo, sec_lo = value_iteration(edges, ambiguous_free=True, terminal=goal_values)
    V_hi, _, _ = value_iteration(edges, ambiguous_free=False, terminal=goal_values)
    path = extract_path(sig_lo)
    return Solution(V_lo, V_hi, sig_lo, sec_lo, path, float(V_lo[0][0]), float(V_hi[0][0]), edges, verts)


def path_cost(scene, Q, path, H: int, bumps=None):
    """FP64 cost of the chain q0 -> Q[l][path[l]] -> qg and its worst waypoint margin."""
    verts = [_c32(scene.q_start)] + [_c32(Q[l, int(path[l])]) for l in range(Q.shape[0])] + [_c32(scene.q_goal)]
    total = 0.0
    worst = math.inf
    for a, b in zip(verts[:-1], verts[1:]):
        total += weighted_length(a, b, H, bumps)
        worst = min(worst, float(edge_margins(scene, a, b, H).min()))
    return total, worst


def anytime(scene, seed, R, L, M, H, eps=EPS_DEFAULT, bumps=None):
    """anytime-gtmp of Alg. 1 with R restarts (single class): per-restart solutions."""
    return [solve(scene, sample_uniform(seed, r, L, M, scene.robot.q_lo, scene.robot.q_hi), H, eps, bumps=bumps)
            for r in range(R)]


# ---------------------------------------------------------------------------
# AO-GTMP epochs (Sec. IV-D) and the edge-length limit l_M(r) (Sec. V).
# Within an epoch the layer count is fixed and the samples per layer double
# each stage up to a cap; a new epoch (fresh samples, Philox seed + epoch)
# starts when the layer rule L + 1 >= c / (reach - 2r - varsigma) fails for
# the best cost c, or when the samples have reached their cap.  The limit of
# a stage is l = L_ref / (L + 1) + 2r + varsigma with the best cost so far
# standing in for the reference length.  The float32 values that decide
# edges (the limit) or samples (the informed bound) are formed exactly as the
# CUDA driver forms them: double arithmetic, one rounding to float32.
# ---------------------------------------------------------------------------

def _margin(r, varsigma):
    return 2.0 * float(np.float32(r)) + float(np.float32(varsigma))


def ao_edge_limit(c_best, L, r, varsigma, base=math.inf):
    """Edge-length limit of a stage with L layers (L + 1 edges per chain): l_M(r) of Sec. V, capped by `base`;
    `base` itself while no chain has been found."""
    base = np.float32(base)
    if not math.isfinite(float(c_best)):
        return base
    l = np.float32(float(np.float32(c_best)) / (L + 1) + _margin(r, varsigma))
    return l if l < base else base


def ao_next(L, M, c_best, L_cap, M0, M_max, reach, r, varsigma):
    """(L', M', new_epoch) after a stage: the layer rule of Sec. IV-D first, then saturation of the samples,
    else the samples double."""
    c = float(np.float32(c_best))
    if math.isfinite(float(np.float32(reach))) and math.isfinite(c) and L < L_cap:
        need = math.ceil(c / (float(np.float32(reach)) - _margin(r, varsigma))) - 1
        if need > L:
            return min(max(need, L + 1), L_cap), M0, True
    if M >= M_max:
        return min(L + 1, L_cap), M0, True
    return L, min(2 * M, M_max), False


def ao_run(scene, seed, L0, M0, M_max, stages, H, L_cap, reach=math.inf, r=0.0, varsigma=0.0, limit_edges=False,
           base_limit=math.inf, best_feed=None):
    """AO-GTMP with epochs on the oracle's own solves.  `best_feed[k]` (float32 best cost after stage k, e.g.
    the GPU's) replaces the oracle's own running best where given, so both sides draw the same informed
    samples; the log records what the oracle computed."""
    dof = scene.robot.dof
    log = []
    epoch, L, M = 0, L0, M0
    Q = np.zeros((L, 0, dof), np.float32)
    best_own = math.inf
    c_before = np.float32(np.inf)
    for k in range(stages):
        limit = ao_edge_limit(c_before, L, r, varsigma, base_limit) if limit_edges else np.float32(base_limit)
        st, Q = expand_layers((seed + epoch) % (1 << 64), Q, M, scene.q_start, scene.q_goal, scene.robot.q_lo,
                              scene.robot.q_hi, np.float32(c_before))
        sol = solve(scene, Q, H, max_len=float(limit))
        best_own = min(best_own, sol.cost_lo)
        c_after = np.float32(best_feed[k]) if best_feed is not None else np.float32(best_own)
        log.append(dict(epoch=epoch, L=L, M=M, edge_limit=limit, status=st, solution=sol, Q=Q,
                        stage_cost=sol.cost_lo, stage_cost_hi=sol.cost_hi, best_cost=best_own))
        L2, M2, new = ao_next(L, M, c_after, L_cap, M0, M_max, reach, r, varsigma)
        if new:
            epoch += 1
            Q = np.zeros((L2, 0, dof), np.float32)
        L, M = L2, M2
        c_before = c_after
    return log


# ---------------------------------------------------------------------------
# Class-augmented value iteration (Prop. 1; Alg. 1 with a class-indexed archive)
# for planar scenes.  Label of a start-to-goal chain: the winding numbers of
# the closed loop (chain, then the straight segment qg -> q0) about every
# obstacle's centre, a homology invariant like the h-signature.  It splits
# over the chain's edges: edge (u, v) contributes the winding numbers of the
# triangle u -> v -> qg -> u (0 or +-1 per obstacle), because the triangles'
# extra sides cancel in pairs.  Labels compose by addition.
# ---------------------------------------------------------------------------

def obstacle_centres_2d(scene):
    """Representative point of every obstacle in the plane: disk centres, then box centres (float64)."""
    pts = [(float(s[0]), float(s[1])) for s in np.asarray(scene.spheres, np.float64)]
    pts += [(0.5 * (float(b[0]) + float(b[3])), 0.5 * (float(b[1]) + float(b[4])))
            for b in np.asarray(scene.boxes, np.float64)]
    return pts


def orient2d(a, b, c) -> float:
    """(b - a) x (c - a) in float64.  For float32 coordinates the differences and products are exact and the
    final subtraction is correctly rounded, so the sign is the exact sign."""
    return (float(b[0]) - float(a[0])) * (float(c[1]) - float(a[1])) - \
           (float(b[1]) - float(a[1])) * (float(c[0]) - float(a[0]))


def triangle_winding(a, b, c, p) -> int:
    """Winding number of the closed triangle a -> b -> c -> a about p: the sign of its orientation when p lies
    strictly inside, else 0 (p on the boundary counts as outside)."""
    o = orient2d(a, b, c)
    if o == 0.0:
        return 0
    d1, d2, d3 = orient2d(a, b, p), orient2d(b, c, p), orient2d(c, a, p)
    if o > 0 and d1 > 0 and d2 > 0 and d3 > 0:
        return 1
    if o < 0 and d1 < 0 and d2 < 0 and d3 < 0:
        return -1
    return 0


def edge_class_label(u, v, g, centres) -> tuple:
    """Label of edge (u, v) toward goal g: per obstacle, the winding number of triangle u -> v -> g."""
    return tuple(triangle_winding(u, v, g, p) for p in centres)


def class_value_iteration(edges, verts, centres, ambiguous_free=False):
    """Prop. 1: J_l(u, chi) = min over (v, chi') with kappa(u, v) + chi' = chi of c(u, v) + J_{l+1}(v, chi'),
    from J_{L+1}(qg, 0) = 0.  Returns tables[l][u] = {chi: (cost, v, chi')}; among equal costs the first v
    (lowest index) is kept.  Plain Python loops: small graphs only."""
    g = verts[-1][0]
    zero = (0,) * len(centres)
    n_layers = len(verts)
    tables = [None] * n_layers
    tables[-1] = [{zero: (0.0, -1, None)}]
    for l in range(n_layers - 2, -1, -1):
        labels_e, costs = edges[l]
        ok = (labels_e == FREE) | ((labels_e == AMBIGUOUS) if ambiguous_free else False)
        rows = []
        for i, u in enumerate(verts[l]):
            tab = {}
            for j, v in enumerate(verts[l + 1]):
                if not ok[i, j] or not tables[l + 1][j]:
                    continue
                k = edge_class_label(u, v, g, centres)
                for chi2, (c2, _, _) in tables[l + 1][j].items():
                    chi = tuple(a + b for a, b in zip(k, chi2))
                    c = float(costs[i, j]) + c2
                    if chi not in tab or c < tab[chi][0]:
                        tab[chi] = (c, j, chi2)
            rows.append(tab)
        tables[l] = rows
    return tables


def class_paths(tables):
    """For every label of the start vertex: (cost, chain of sample indices, one per layer 1..L)."""
    out = {}
    L = len(tables) - 2
    for chi, (c, j, chi2) in tables[0][0].items():
        path = []
        for l in range(1, L + 1):
            path.append(j)
            c_l, j, chi2 = tables[l][j][chi2]
        out[chi] = (c, path)
    return out


def polygon_winding(points, p) -> int:
    """Winding number of the closed polygon points[0] -> ... -> points[-1] -> points[0] about p, from the sum
    of the signed angles the edges subtend at p (an independent definition used to pin the labels)."""
    total = 0.0
    n = len(points)
    for k in range(n):
        a = (float(points[k][0]) - p[0], float(points[k][1]) - p[1])
        b = (float(points[(k + 1) % n][0]) - p[0], float(points[(k + 1) % n][1]) - p[1])
        total += math.atan2(a[0] * b[1] - a[1] * b[0], a[0] * b[0] + a[1] * b[1])
    return int(round(total / (2 * math.pi)))
