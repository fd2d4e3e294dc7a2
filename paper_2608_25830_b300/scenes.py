"""Seeded synthetic planning problems (inputs only).

This module draws robots, obstacle sets and start/goal candidates for the
layered-graph planner.  It is the one module that both the CUDA path and the
CPU oracle are fed from, so it holds none of the planner's arithmetic: no
forward kinematics, no waypoint interpolation, no collision predicate, no
value iteration and no Philox stream.  Its random numbers come from numpy's
PCG64 and describe the problem; every random number the planner itself draws
(layer samples, informed samples, heuristic coins) comes from the planner's own
counter-based Philox generator.

Scene recipes (readings of the workloads; the paper's MotionBenchMaker scenes
and street maps are not available, seeded scenes of the same dimensions stand
in for them):

* 2D point robot: configuration = position in [-1, 1]^2, disks with centres
  uniform in the square and radii U[0.05, 0.15]; a disk is redrawn while it
  covers the start or the goal (0.02 clearance).
* DH serial arm, d joints: link lengths a_i ~ U[0.1, 0.3] m, offsets
  d_i ~ U[0, 0.1] m, twists alpha_i uniform in {-pi/2, 0, pi/2}, theta
  offsets 0, joint box [-pi, pi]^d, base at the origin of the obstacle cube.
  Four spheres of radius 0.04 m per link sit at fractions 1/8, 3/8, 5/8, 7/8
  of the segment from the origin of frame i-1 to the origin of frame i, given
  in the frame of link i.
* Arm obstacles in a 1.5 m cube: n obstacles split into floor(2n/3) spheres
  (radius U[0.05, 0.15] m) and the rest axis-aligned boxes (half extents
  U[0.05, 0.15] m), centres uniform in [-0.75, 0.75]^3; an obstacle whose
  bounding ball comes within 0.40 m of the base is redrawn, so that the first
  link (which only turns about the base axis) is always free.
* Arm start/goal: a list of candidate (start, goal) pairs uniform in the joint
  box.  Which pair is used is decided by the caller with an exact
  configuration checker (the first pair whose both ends are collision free).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ROBOT_POINT = 0
ROBOT_DH_ARM = 1


@dataclass
class Robot:
    kind: int                    # ROBOT_POINT or ROBOT_DH_ARM
    dof: int
    dh: np.ndarray               # float32 [dof][4]: d, a, alpha, theta_offset
    link_spheres: np.ndarray     # float32 [dof][spl][4]: x, y, z, r in link frame
    q_lo: np.ndarray             # float32 [dof]
    q_hi: np.ndarray             # float32 [dof]
    point_radius: float = 0.0    # point robot: radius of the robot disk

    @property
    def spheres_per_link(self) -> int:
        return int(self.link_spheres.shape[1]) if self.kind == ROBOT_DH_ARM else 0


@dataclass
class Scene:
    robot: Robot
    spheres: np.ndarray          # float32 [n_s][4]: cx, cy, cz, r
    boxes: np.ndarray            # float32 [n_b][6]: lo x, y, z, hi x, y, z
    q_start: np.ndarray          # float32 [dof]
    q_goal: np.ndarray           # float32 [dof]
    candidates: np.ndarray = field(default=None)  # float32 [K][2][dof] or None
    name: str = ""

    def with_endpoints(self, k: int) -> "Scene":
        """Copy of the scene using candidate pair k as start/goal."""
        c = self.candidates[k]
        return Scene(self.robot, self.spheres, self.boxes, c[0].copy(), c[1].copy(),
                     self.candidates, self.name)


def _f32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def point_robot_2d() -> Robot:
    return Robot(ROBOT_POINT, 2, np.zeros((2, 4), np.float32), np.zeros((2, 0, 4), np.float32),
                 _f32([-1, -1]), _f32([1, 1]), 0.0)


def point2d_scene(seed: int = 0, n_disks: int = 10, rmin: float = 0.05, rmax: float = 0.15,
                  start=(-0.9, -0.9), goal=(0.9, 0.9)) -> Scene:
    """2D point robot among disks (disks are spheres with z = 0)."""
    rng = np.random.default_rng([seed, 2])
    s = np.asarray(start, np.float64)
    g = np.asarray(goal, np.float64)
    disks = []
    while len(disks) < n_disks:
        c = rng.uniform(-1.0, 1.0, 2)
        r = rng.uniform(rmin, rmax)
        if np.hypot(*(c - s)) <= r + 0.02 or np.hypot(*(c - g)) <= r + 0.02:
            continue
        disks.append((c[0], c[1], 0.0, r))
    return Scene(point_robot_2d(), _f32(disks).reshape(-1, 4), np.zeros((0, 6), np.float32),
                 _f32(start), _f32(goal), None, f"point2d-s{seed}-n{n_disks}")


def dh_arm(seed: int, dof: int, spheres_per_link: int = 4, sphere_radius: float = 0.04) -> Robot:
    """Seeded serial arm in standard DH form (see module docstring)."""
    rng = np.random.default_rng([seed, 1, dof])
    a = rng.uniform(0.1, 0.3, dof)
    d = rng.uniform(0.0, 0.1, dof)
    twist_choice = rng.integers(0, 3, dof)          # 0 -> -pi/2, 1 -> 0, 2 -> +pi/2
    alpha = (twist_choice - 1) * (math.pi / 2)
    sin_alpha = (twist_choice - 1).astype(np.float64)   # exact sine of the three twists
    cos_alpha = (twist_choice == 1).astype(np.float64)  # exact cosine of the three twists
    dh = np.stack([d, a, alpha, np.zeros(dof)], 1)
    fr = (np.arange(spheres_per_link) + 0.5) / spheres_per_link
    sph = np.zeros((dof, spheres_per_link, 4))
    for i in range(dof):
        # origin of frame i-1 written in frame i (constant for a revolute DH joint)
        prev = np.array([-a[i], -d[i] * sin_alpha[i], -d[i] * cos_alpha[i]])
        for k, f in enumerate(fr):
            sph[i, k, :3] = (1.0 - f) * prev
            sph[i, k, 3] = sphere_radius
    lo = np.full(dof, -math.pi)
    hi = np.full(dof, math.pi)
    return Robot(ROBOT_DH_ARM, dof, _f32(dh), _f32(sph), _f32(lo), _f32(hi), 0.0)


def arm_obstacles(rng, n: int, keepout: float = 0.40, half: float = 0.75,
                  rmin: float = 0.05, rmax: float = 0.15):
    n_s = (2 * n) // 3
    n_b = n - n_s
    spheres, boxes = [], []
    while len(spheres) < n_s:
        c = rng.uniform(-half, half, 3)
        r = rng.uniform(rmin, rmax)
        if np.linalg.norm(c) - r < keepout:
            continue
        spheres.append((c[0], c[1], c[2], r))
    while len(boxes) < n_b:
        c = rng.uniform(-half, half, 3)
        h = rng.uniform(rmin, rmax, 3)
        if np.linalg.norm(c) - np.linalg.norm(h) < keepout:
            continue
        boxes.append(tuple(c - h) + tuple(c + h))
    return _f32(spheres).reshape(-1, 4), _f32(boxes).reshape(-1, 6)


def arm_scene(seed: int = 0, dof: int = 7, n_obstacles: int = 30, n_candidates: int = 64) -> Scene:
    """DH arm among spheres and boxes in a 1.5 m cube; endpoints chosen by the caller."""
    robot = dh_arm(seed, dof)
    rng = np.random.default_rng([seed, 3, dof, n_obstacles])
    spheres, boxes = arm_obstacles(rng, n_obstacles)
    cand = rng.uniform(-math.pi, math.pi, (n_candidates, 2, dof))
    cand = _f32(cand)
    return Scene(robot, spheres, boxes, cand[0, 0].copy(), cand[0, 1].copy(), cand,
                 f"arm{dof}-s{seed}-n{n_obstacles}")


def pick_endpoints(scene: Scene, config_free) -> Scene:
    """Return the scene with the first candidate pair whose ends are both free.

    ``config_free(q[n][dof]) -> bool[n]`` is supplied by the caller (the exact
    checker of whichever side is being fed); no collision arithmetic lives here.
    """
    if scene.candidates is None:
        return scene
    flat = scene.candidates.reshape(-1, scene.robot.dof)
    free = np.asarray(config_free(flat), bool).reshape(-1, 2)
    ok = np.nonzero(free[:, 0] & free[:, 1])[0]
    if ok.size == 0:
        raise RuntimeError(f"no collision-free start/goal pair among candidates of {scene.name}")
    return scene.with_endpoints(int(ok[0]))


def corridor_scene(w: float = 0.1, t: float = 0.3, x0: float = 0.9) -> Scene:
    """2D point robot in a corridor: the free strip |y| < w, walled off by two
    boxes of thickness t from the chambers |y| > w + t; start (-x0, 0) and
    goal (x0, 0) in the strip.  Every chain must keep each layer vertex in
    the strip (the layerwise-hitting instance of the appendix)."""
    boxes = _f32([[-1.2, w, -1.0, 1.2, w + t, 1.0], [-1.2, -w - t, -1.0, 1.2, -w, 1.0]])
    return Scene(point_robot_2d(), np.zeros((0, 4), np.float32), boxes, _f32([-x0, 0.0]), _f32([x0, 0.0]), None,
                 f"corridor-w{w}-t{t}-x{x0}")


def weight_bumps(scene: Scene, seed: int = 0, K: int = 6, amin: float = 0.5, amax: float = 3.0,
                 smin: float = 0.3, smax: float = 0.6) -> np.ndarray:
    """Seeded weight field for weighted-length costs: float32 [K][dof + 2] rows
    (centre, radius s, amplitude a).  Bump 0 sits at the midpoint of the
    scene's start and goal (so the straight connection is penalised), the rest
    uniformly in the joint box; radii are U[smin, smax] times half the box
    diagonal, amplitudes U[amin, amax]."""
    lo = scene.robot.q_lo.astype(np.float64)
    hi = scene.robot.q_hi.astype(np.float64)
    rng = np.random.default_rng([seed, 6, scene.robot.dof, K])
    half_diag = 0.5 * float(np.linalg.norm(hi - lo))
    cen = rng.uniform(lo, hi, (K, lo.shape[0]))
    cen[0] = 0.5 * (scene.q_start.astype(np.float64) + scene.q_goal)
    rad = rng.uniform(smin, smax, K) * half_diag
    amp = rng.uniform(amin, amax, K)
    return _f32(np.concatenate([cen, rad[:, None], amp[:, None]], axis=1))


# ---------------------------------------------------------------------------
# Workload descriptions (sizes of the five evaluated configurations)
# ---------------------------------------------------------------------------

WORKLOADS = {
    "point2d_m32_l4_h16": dict(kind="point2d", seed=0, n_obs=10, M=32, L=4, H=16),
    "arm7_m1024_l8_h32": dict(kind="arm", dof=7, seed=0, n_obs=30, M=1024, L=8, H=32),
    "arm6_anytime_r64_m256_l6_h32": dict(kind="arm", dof=6, seed=0, n_obs=30, M=256, L=6, H=32, R=64),
    "arm6_ao_m64to4096_l6_h32": dict(kind="arm", dof=6, seed=0, n_obs=30, M0=64, M1=4096, L=6, H=32,
                                     epochs=dict(L0=2, L_cap=8, M0=64, M_max=2048, stages=14, reach=2.5, r=0.1,
                                                 varsigma=0.1, limit_edges=True)),
    "arm7_m4096_l8_h32_n40": dict(kind="arm", dof=7, seed=0, n_obs=40, M=4096, L=8, H=32,
                                  n_train=1 << 21, epochs=3, sigma=0.25, threshold=0.1, protect=0.1,
                                  score_waypoints=1),
    "batched512_h32": dict(kind="batched", seed=0, n=512, H=32),
    "point2d_classes_m32_l4_h16": dict(kind="classes", seed=0, n_obs=10, M=32, L=4, H=16, K=256, R=16),
    "point2d_classes_m64_l4_h16_n16": dict(kind="classes", seed=2, n_obs=16, M=64, L=4, H=16, K=1024, R=16),
}


@dataclass
class BatchProblem:
    scene: Scene
    M: int
    L: int
    H: int
    seed: int


def batch_problems(seed: int = 0, n: int = 512, H: int = 32, Mmin: int = 64, Mmax: int = 2048,
                   Lmin: int = 3, Lmax: int = 12, obs_min: int = 5, obs_max: int = 40):
    """Uneven problem mix: DoF in {2, 7}, M log-uniform, L uniform, 5-40 obstacles."""
    rng = np.random.default_rng([seed, 4])
    out = []
    for p in range(n):
        two_d = bool(rng.integers(0, 2))
        M = int(round(math.exp(rng.uniform(math.log(Mmin), math.log(Mmax)))))
        L = int(rng.integers(Lmin, Lmax + 1))
        n_obs = int(rng.integers(obs_min, obs_max + 1))
        scene_seed = int(rng.integers(0, 2**31 - 1))
        if two_d:
            sc = point2d_scene(scene_seed, n_obs)
        else:
            sc = arm_scene(scene_seed, 7, n_obs, n_candidates=16)
        out.append(BatchProblem(sc, M, L, H, p))
    return out


def nominal_checks(M: int, L: int, H: int) -> int:
    """Waypoint checks of one solve: H per candidate edge, 2M + (L-1) M^2 edges."""
    return H * (2 * M + (L - 1) * M * M)


def nominal_edges(M: int, L: int) -> int:
    return 2 * M + (L - 1) * M * M
