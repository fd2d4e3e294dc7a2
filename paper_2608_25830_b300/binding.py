"""Python binding of the C ABI in include/gtmp.h (argument marshalling only).

Every function here forwards to the function of the same name in libgtmp.so:
host arrays are passed as numpy float32 pointers, device buffers as the data
pointers of CUDA torch tensors, and the stream as the current torch stream.
No planning arithmetic happens in Python; if the shared library has not been
built, importing the binding's loader raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import scenes

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libgtmp.so")

GTMP_OK = 0
STATUS = {0: "GTMP_OK", 1: "GTMP_ERR_INVALID_ARG", 2: "GTMP_ERR_CUDA", 3: "GTMP_ERR_OOM", 4: "GTMP_ERR_TIMEOUT",
          5: "GTMP_ERR_UNSUPPORTED", 6: "GTMP_ERR_NOT_READY"}
EVAL_EARLY_EXIT, EVAL_FULL, EVAL_LAZY = 0, 1, 2
ROBOT_POINT, ROBOT_DH_ARM = 0, 1


class GtmpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class GtmpRobot(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dof", ctypes.c_int32), ("dh", ctypes.POINTER(ctypes.c_float)),
                ("link_spheres", ctypes.POINTER(ctypes.c_float)), ("spheres_per_link", ctypes.c_int32),
                ("q_lo", ctypes.POINTER(ctypes.c_float)), ("q_hi", ctypes.POINTER(ctypes.c_float)),
                ("point_radius", ctypes.c_float)]


class GtmpParams(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("L", ctypes.c_int32), ("H", ctypes.c_int32), ("R", ctypes.c_int32),
                ("max_obstacles", ctypes.c_int32), ("eval_mode", ctypes.c_int32), ("max_edge_len", ctypes.c_float)]


class GtmpProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("fused_launches", ctypes.c_int64), ("fused_ms", ctypes.c_double),
                ("fused_edges", ctypes.c_double), ("minplus_launches", ctypes.c_int64), ("minplus_ms", ctypes.c_double),
                ("minplus_bytes", ctypes.c_double)]


_lib = None
_vp, _i32, _u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
_fp = ctypes.POINTER(ctypes.c_float)


class GtmpSurrogateConfig(ctypes.Structure):
    _fields_ = [("n_train", ctypes.c_int32), ("n_holdout", ctypes.c_int32), ("epochs", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("lr", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("fourier_sigma", ctypes.c_float)]


class GtmpSurrogateStats(ctypes.Structure):
    _fields_ = [("final_loss", ctypes.c_float), ("holdout_accuracy", ctypes.c_float),
                ("holdout_fn_rate", ctypes.c_float), ("holdout_fp_rate", ctypes.c_float),
                ("train_ms", ctypes.c_float)]


class GtmpPruneStats(ctypes.Structure):
    _fields_ = [("edges", ctypes.c_double), ("pruned", ctypes.c_double), ("score_ms", ctypes.c_float),
                ("solve_ms", ctypes.c_float), ("scored", ctypes.c_double), ("band_ms", ctypes.c_float),
                ("lists_ms", ctypes.c_float)]


class GtmpLazyStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("colliding_edges", ctypes.c_int64)]


class GtmpAoSchedule(ctypes.Structure):
    _fields_ = [("L0", ctypes.c_int32), ("M0", ctypes.c_int32), ("M_max", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("reach", ctypes.c_float), ("r", ctypes.c_float), ("varsigma", ctypes.c_float),
                ("limit_edges", ctypes.c_int32)]


class GtmpAoStage(ctypes.Structure):
    _fields_ = [("epoch", ctypes.c_int32), ("L", ctypes.c_int32), ("M", ctypes.c_int32), ("edge_limit", ctypes.c_float),
                ("stage_cost", ctypes.c_float), ("best_cost", ctypes.c_float)]


class GtmpProblem(ctypes.Structure):
    _fields_ = [("robot", GtmpRobot), ("spheres", _fp), ("n_s", ctypes.c_int32), ("boxes", _fp),
                ("n_b", ctypes.c_int32), ("q_start", _fp), ("q_goal", _fp), ("M", ctypes.c_int32),
                ("L", ctypes.c_int32), ("seed", ctypes.c_uint64)]

_SIGNATURES = {
    "gtmp_create": [ctypes.POINTER(GtmpRobot), ctypes.POINTER(GtmpParams), _vp, ctypes.POINTER(_vp)],
    "gtmp_destroy": [_vp],
    "gtmp_set_stream": [_vp, _vp],
    "gtmp_synchronize": [_vp],
    "gtmp_set_obstacles": [_vp, _fp, _i32, _fp, _i32],
    "gtmp_set_endpoints": [_vp, _fp, _fp],
    "gtmp_sample_layers": [_vp, _u64, _i32],
    "gtmp_set_layers": [_vp, _vp, _i32],
    "gtmp_get_layers": [_vp, _vp],
    "gtmp_label_configs": [_vp, _vp, _i32, _vp],
    "gtmp_solve": [_vp, _vp, _vp],
    "gtmp_get_values": [_vp, _i32, _vp, _vp],
    "gtmp_solve_unfused": [_vp, _vp, _vp],
    "gtmp_get_edge_costs": [_vp, _i32, _vp],
    "gtmp_anytime": [_vp, _u64, _i32, _vp, _vp, _vp],
    "aogtmp_expand": [_vp, _u64, _i32, _vp, _vp, _vp, _vp],
    "gtmp_set_num_layers": [_vp, _i32],
    "gtmp_set_max_edge_len": [_vp, ctypes.c_float],
    "aogtmp_run": [_vp, _u64, ctypes.POINTER(GtmpAoSchedule), _vp, _vp, ctypes.POINTER(GtmpAoStage),
                   ctypes.POINTER(_i32)],
    "gtmp_get_M": [_vp, ctypes.POINTER(_i32)],
    "gtmp_profile_enable": [_vp, _i32],
    "gtmp_profile_read": [_vp, ctypes.POINTER(GtmpProfile)],
    "gtmp_batch_create": [ctypes.POINTER(GtmpProblem), _i32, _i32, _vp, ctypes.POINTER(_vp)],
    "gtmp_batch_destroy": [_vp],
    "gtmp_batch_set_stream": [_vp, _vp],
    "gtmp_batch_info": [_vp, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i32),
                        ctypes.POINTER(_i32)],
    "gtmp_batch_solve": [_vp, _vp, _vp],
    "gtmp_batch_synchronize": [_vp],
    "gtmp_batch_set_tiling": [_vp, _i32, _i32],
    "gtmp_batch_set_kind_tiling": [_vp, _i32, _i32, _i32],
    "gtmp_batch_get_tiling": [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)],
    "gtmp_batch_autotune": [_vp, _i32, _vp, _vp, ctypes.POINTER(ctypes.c_float)],
    "gtmp_batch_set_eval_mode": [_vp, _i32],
    "gtmp_batch_inject_stall": [_vp, _i32, _i32],
    "gtmp_solve_classes": [_vp, _i32, _i32, _vp, _vp, _vp, ctypes.POINTER(_i32)],
    "gtmp_set_goals": [_vp, _fp, _fp, _i32],
    "gtmp_set_sampler": [_vp, _i32, _i32],
    "gtmp_set_cost_weight": [_vp, _fp, _i32],
    "gtmp_fp32_fma_peak": [_vp, ctypes.POINTER(ctypes.c_double)],
    "gtmp_joint_sincos": [_vp, _i32, _vp, _vp, _vp],
    "gtmp_cull_grid": [_fp, _i32, _fp, _i32, ctypes.c_float, _i32, ctypes.POINTER(ctypes.c_uint32),
                       ctypes.POINTER(_i32), _fp],
    "gtmp_get_goal_reached": [_vp, _i32, _vp],
    "gtmp_surrogate_train": [_vp, ctypes.POINTER(GtmpSurrogateConfig), ctypes.POINTER(GtmpSurrogateStats)],
    "gtmp_surrogate_predict": [_vp, _vp, _i32, _vp],
    "gtmp_surrogate_get_params": [_vp, _fp, ctypes.c_int64, _fp, ctypes.c_int64],
    "gtmp_solve_pruned": [_vp, ctypes.c_float, _i32, _vp, _vp, ctypes.POINTER(GtmpPruneStats)],
    "gtmp_surrogate_set_protect": [_vp, ctypes.c_float],
    "gtmp_solve_lazy_path": [_vp, _i32, _vp, _vp, ctypes.POINTER(GtmpLazyStats)],
    "gtmp_surrogate_score": [_vp, _i32, ctypes.c_float, _i32, _vp, ctypes.POINTER(ctypes.c_int64)],
    "gtmp_surrogate_set_params": [_vp, _fp, ctypes.c_int64, _fp, ctypes.c_int64],
    "gtmp_surrogate_loss_grad": [_vp, _vp, _vp, _i32, ctypes.POINTER(ctypes.c_double), _fp, ctypes.c_int64],
    "gtmp_umma_gemm_f32": [_vp, _i32, _vp, _i32, _i32, _i32, _i32, _vp, _i32, _vp, _vp],
    "gtmp_solve_noalloc": [ctypes.POINTER(GtmpRobot), _fp, _i32, _fp, _i32, _fp, _fp, _vp, _i32, _i32, _i32,
                           ctypes.c_float, _vp, _vp, _vp, _vp, ctypes.c_char_p, _i32],
}


def lib() -> ctypes.CDLL:
    """Load libgtmp.so (built in-tree by paper_2608_25830_b300/build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                               f"g.build()'` (nvcc, sm_103a); there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.gtmp_last_error.argtypes = [_vp]
        L.gtmp_last_error.restype = ctypes.c_char_p
        L.gtmp_surrogate_param_count.argtypes = []
        L.gtmp_surrogate_param_count.restype = ctypes.c_int64
        L.gtmp_batch_last_error.argtypes = [_vp]
        L.gtmp_batch_last_error.restype = ctypes.c_char_p
        L.gtmp_status_string.argtypes = [ctypes.c_int]
        L.gtmp_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(ctx, status):
    if status != GTMP_OK:
        msg = lib().gtmp_last_error(ctx).decode() if ctx else ""
        raise GtmpError(status, msg)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(_fp)


def _dev(t, dtype=None):
    """Data pointer of a CUDA tensor (checked: device, contiguity, dtype)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if not t.is_contiguous():
        raise ValueError("device buffer must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---------------------------------------------------------------------------
# the C calls, one by one
# ---------------------------------------------------------------------------

def robot_struct(robot: scenes.Robot):
    keep = dict(dh=_f32(robot.dh).reshape(-1), sph=_f32(robot.link_spheres).reshape(-1) if robot.link_spheres.size
                else np.zeros(4, np.float32), lo=_f32(robot.q_lo), hi=_f32(robot.q_hi))
    s = GtmpRobot(robot.kind, robot.dof, _ptr(keep["dh"]), _ptr(keep["sph"]),
                  robot.spheres_per_link if robot.kind == ROBOT_DH_ARM else 0,
                  _ptr(keep["lo"]), _ptr(keep["hi"]), float(robot.point_radius))
    return s, keep


def gtmp_create(robot: scenes.Robot, M, L, H, R=1, max_obstacles=64, eval_mode=EVAL_EARLY_EXIT,
                max_edge_len=math.inf, stream=None):
    rs, keep = robot_struct(robot)
    ps = GtmpParams(M, L, H, R, max_obstacles, eval_mode, max_edge_len)
    out = _vp()
    st = stream if stream is not None else _stream()
    status = lib().gtmp_create(ctypes.byref(rs), ctypes.byref(ps), st, ctypes.byref(out))
    if status != GTMP_OK:
        raise GtmpError(status, "gtmp_create rejected its arguments or the device")
    return out


def gtmp_destroy(ctx):
    _check(None, lib().gtmp_destroy(ctx))


def gtmp_set_stream(ctx, stream=None):
    _check(ctx, lib().gtmp_set_stream(ctx, stream if stream is not None else _stream()))


def gtmp_synchronize(ctx):
    _check(ctx, lib().gtmp_synchronize(ctx))


def gtmp_set_obstacles(ctx, spheres, boxes):
    s = _f32(spheres).reshape(-1, 4)
    b = _f32(boxes).reshape(-1, 6)
    _check(ctx, lib().gtmp_set_obstacles(ctx, _ptr(s), s.shape[0], _ptr(b), b.shape[0]))


def gtmp_set_endpoints(ctx, q_start, q_goal):
    a, b = _f32(q_start), _f32(q_goal)
    _check(ctx, lib().gtmp_set_endpoints(ctx, _ptr(a), _ptr(b)))


def gtmp_sample_layers(ctx, seed, M):
    _check(ctx, lib().gtmp_sample_layers(ctx, seed, M))


def gtmp_set_layers(ctx, dev_Q, M):
    import torch
    _check(ctx, lib().gtmp_set_layers(ctx, _dev(dev_Q, torch.float32), M))


def gtmp_get_layers(ctx, dev_Q):
    import torch
    _check(ctx, lib().gtmp_get_layers(ctx, _dev(dev_Q, torch.float32)))


def gtmp_label_configs(ctx, dev_q, dev_labels):
    import torch
    n = dev_q.shape[0]
    _check(ctx, lib().gtmp_label_configs(ctx, _dev(dev_q, torch.float32), n, _dev(dev_labels, torch.uint8)))


def gtmp_solve(ctx, dev_path, dev_cost):
    import torch
    _check(ctx, lib().gtmp_solve(ctx, _dev(dev_path, torch.int32), _dev(dev_cost, torch.float32)))


def gtmp_get_values(ctx, g, dev_V, dev_sigma):
    import torch
    _check(ctx, lib().gtmp_get_values(ctx, g, _dev(dev_V, torch.float32), _dev(dev_sigma, torch.int32)))


def gtmp_solve_unfused(ctx, dev_path, dev_cost):
    import torch
    _check(ctx, lib().gtmp_solve_unfused(ctx, _dev(dev_path, torch.int32), _dev(dev_cost, torch.float32)))


def gtmp_get_edge_costs(ctx, l, dev_C):
    import torch
    _check(ctx, lib().gtmp_get_edge_costs(ctx, l, _dev(dev_C, torch.float32)))


def gtmp_anytime(ctx, seed, restarts, dev_paths, dev_costs, dev_best):
    import torch
    _check(ctx, lib().gtmp_anytime(ctx, seed, restarts, _dev(dev_paths, torch.int32), _dev(dev_costs, torch.float32),
                                   _dev(dev_best, torch.int32)))


def aogtmp_expand(ctx, seed, M_new, dev_stage_path, dev_stage_cost, dev_best_path, dev_best_cost):
    import torch
    _check(ctx, lib().aogtmp_expand(ctx, seed, M_new, _dev(dev_stage_path, torch.int32),
                                    _dev(dev_stage_cost, torch.float32), _dev(dev_best_path, torch.int32),
                                    _dev(dev_best_cost, torch.float32)))


def gtmp_set_num_layers(ctx, L):
    _check(ctx, lib().gtmp_set_num_layers(ctx, L))


def gtmp_set_max_edge_len(ctx, max_edge_len):
    _check(ctx, lib().gtmp_set_max_edge_len(ctx, max_edge_len))


def aogtmp_run(ctx, seed, schedule, dev_best_chain, dev_best_cost):
    """AO-GTMP with epochs; returns (per-stage records as dicts, layer count of the best chain)."""
    import torch
    log = (GtmpAoStage * schedule.stages)()
    best_layers = _i32()
    _check(ctx, lib().aogtmp_run(ctx, seed, ctypes.byref(schedule), _dev(dev_best_chain, torch.float32),
                                 _dev(dev_best_cost, torch.float32), log, ctypes.byref(best_layers)))
    recs = [dict(epoch=x.epoch, L=x.L, M=x.M, edge_limit=x.edge_limit, stage_cost=x.stage_cost,
                 best_cost=x.best_cost) for x in log]
    return recs, best_layers.value


def gtmp_profile_enable(ctx, enable=True):
    _check(ctx, lib().gtmp_profile_enable(ctx, 1 if enable else 0))


def gtmp_profile_read(ctx):
    out = GtmpProfile()
    _check(ctx, lib().gtmp_profile_read(ctx, ctypes.byref(out)))
    return dict(launches=out.launches, fused_launches=out.fused_launches, fused_ms=out.fused_ms,
                fused_edges=out.fused_edges, minplus_launches=out.minplus_launches, minplus_ms=out.minplus_ms,
                minplus_bytes=out.minplus_bytes)


def gtmp_solve_noalloc(robot: scenes.Robot, spheres, boxes, q_start, q_goal, dev_Q, H, dev_path, dev_cost,
                       dev_status=None, max_edge_len=math.inf, stream=None):
    """Allocation-free solve (see include/gtmp.h): caller passes every input and output."""
    import torch
    rs, keep = robot_struct(robot)
    s = _f32(spheres).reshape(-1, 4)
    b = _f32(boxes).reshape(-1, 6)
    a, g = _f32(q_start), _f32(q_goal)
    L, M = int(dev_Q.shape[0]), int(dev_Q.shape[1])
    msg = ctypes.create_string_buffer(512)
    st = stream if stream is not None else _stream()
    status = lib().gtmp_solve_noalloc(ctypes.byref(rs), _ptr(s), s.shape[0], _ptr(b), b.shape[0], _ptr(a), _ptr(g),
                                      _dev(dev_Q, torch.float32), M, L, H, max_edge_len, st,
                                      _dev(dev_path, torch.int32), _dev(dev_cost, torch.float32),
                                      _dev(dev_status, torch.int32) if dev_status is not None else None,
                                      msg, len(msg))
    if status != GTMP_OK:
        raise GtmpError(status, msg.value.decode())


def gtmp_get_M(ctx):
    m = _i32()
    _check(ctx, lib().gtmp_get_M(ctx, ctypes.byref(m)))
    return m.value


# ---------------------------------------------------------------------------
# A small object wrapper over the same calls
# ---------------------------------------------------------------------------

class Planner:
    """One planning context (robot, capacities, obstacles, endpoints, layers)."""

    def __init__(self, robot: scenes.Robot, M, L, H, R=1, max_obstacles=64, eval_mode=EVAL_EARLY_EXIT,
                 max_edge_len=math.inf):
        import torch
        self.robot, self.M, self.L, self.H, self.R = robot, M, L, H, R
        self.L_cap = L   # capacity; self.L follows gtmp_set_num_layers
        self.dev = torch.device("cuda")
        self.ctx = gtmp_create(robot, M, L, H, R, max_obstacles, eval_mode, max_edge_len)

    def close(self):
        if self.ctx:
            gtmp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scene(self, scene: scenes.Scene):
        gtmp_set_obstacles(self.ctx, scene.spheres, scene.boxes)
        self.n_obstacles = int(np.asarray(scene.spheres).shape[0] + np.asarray(scene.boxes).shape[0])
        gtmp_set_endpoints(self.ctx, scene.q_start, scene.q_goal)

    def ao_run(self, seed, L0, M0, M_max, stages, reach=math.inf, r=0.0, varsigma=0.0, limit_edges=False):
        """AO-GTMP with epochs: (best chain [L capacity + 2][dof] device, best cost device [1], stage log,
        layer count of the best chain)."""
        import torch
        sched = GtmpAoSchedule(L0, M0, M_max, stages, reach, r, varsigma, 1 if limit_edges else 0)
        chain = torch.empty((self.L_cap + 2, self.robot.dof), dtype=torch.float32, device="cuda")
        cost = torch.empty(1, dtype=torch.float32, device="cuda")
        log, best_layers = aogtmp_run(self.ctx, seed, sched, chain, cost)
        self.L = log[-1]["L"]
        return chain, cost, log, best_layers

    def set_num_layers(self, L):
        gtmp_set_num_layers(self.ctx, L)
        self.L = L

    def set_cost_weight(self, bumps):
        gtmp_set_cost_weight(self.ctx, bumps)

    def sample_layers(self, seed, M=None):
        gtmp_sample_layers(self.ctx, seed, M or self.M)

    def set_layers(self, Q):
        gtmp_set_layers(self.ctx, Q, Q.shape[1])

    def get_layers(self):
        import torch
        Q = torch.empty((self.L, gtmp_get_M(self.ctx), self.robot.dof), dtype=torch.float32, device=self.dev)
        gtmp_get_layers(self.ctx, Q)
        return Q

    def solve_classes(self, max_labels=256, max_classes=256):
        """Minimum-cost chain per class of graph 0 (planar point robots): {label tuple: (cost, path)}."""
        import torch
        paths = torch.empty((max_classes, self.L), dtype=torch.int32, device=self.dev)
        costs = torch.empty(max_classes, dtype=torch.float32, device=self.dev)
        labels = torch.empty((max_classes, 16), dtype=torch.int8, device=self.dev)
        n = gtmp_solve_classes(self.ctx, max_labels, max_classes, paths, costs, labels)
        k = min(n, max_classes)
        n_obs = self.n_obstacles
        P, C, Lb = paths[:k].cpu().numpy(), costs[:k].cpu().numpy(), labels[:k].cpu().numpy()
        return {tuple(int(x) for x in Lb[i, :n_obs]): (float(C[i]), P[i].copy()) for i in range(k)}, n

    def anytime_classes(self, seed, restarts, max_labels=256, max_classes=256):
        """anytime-gtmp of Alg. 1 with its class-indexed archive: `restarts` fresh graphs (sample seeds
        seed, seed + 1, ...), each swept class by class on the device; the archive keeps, per label, the
        cheapest chain found so far.  Returns {label: (cost, restart, path)}."""
        archive = {}
        for r in range(restarts):
            self.sample_layers(seed + r, self.M)
            classes, _ = self.solve_classes(max_labels, max_classes)
            for chi, (c, path) in classes.items():
                if chi not in archive or c < archive[chi][0]:
                    archive[chi] = (c, r, path)
        return archive

    def label_configs(self, q):
        import torch
        out = torch.empty(q.shape[0], dtype=torch.uint8, device=self.dev)
        gtmp_label_configs(self.ctx, q.contiguous(), out)
        return out

    def solve(self, unfused=False):
        import torch
        path = torch.empty(self.L, dtype=torch.int32, device=self.dev)
        cost = torch.empty(1, dtype=torch.float32, device=self.dev)
        (gtmp_solve_unfused if unfused else gtmp_solve)(self.ctx, path, cost)
        return path, cost

    def values(self, g=0):
        import torch
        V = torch.empty((self.L + 2, gtmp_get_M(self.ctx)), dtype=torch.float32, device=self.dev)
        S = torch.empty_like(V, dtype=torch.int32)
        gtmp_get_values(self.ctx, g, V, S)
        return V, S

    def edge_costs(self, l):
        import torch
        m = gtmp_get_M(self.ctx)
        rows = 1 if l == 0 else m
        cols = 1 if l == self.L else m
        C = torch.empty((rows, cols), dtype=torch.float32, device=self.dev)
        gtmp_get_edge_costs(self.ctx, l, C)
        return C

    def anytime(self, seed, restarts):
        import torch
        paths = torch.empty((restarts, self.L), dtype=torch.int32, device=self.dev)
        costs = torch.empty(restarts, dtype=torch.float32, device=self.dev)
        best = torch.empty(1, dtype=torch.int32, device=self.dev)
        gtmp_anytime(self.ctx, seed, restarts, paths, costs, best)
        return paths, costs, best

    def synchronize(self):
        gtmp_synchronize(self.ctx)


# ---------------------------------------------------------------------------
# batched planning
# ---------------------------------------------------------------------------

def _bcheck(b, status):
    if status != GTMP_OK:
        msg = lib().gtmp_batch_last_error(b).decode() if b else ""
        raise GtmpError(status, msg)


def gtmp_batch_create(problems, H, stream=None):
    """problems: sequence of (scenes.Scene, M, L, seed)."""
    arr = (GtmpProblem * len(problems))()
    keep = []
    for k, (sc, M, L, seed) in enumerate(problems):
        rs, kr = robot_struct(sc.robot)
        sph = _f32(sc.spheres).reshape(-1, 4)
        box = _f32(sc.boxes).reshape(-1, 6)
        a, g = _f32(sc.q_start), _f32(sc.q_goal)
        keep.append((kr, sph, box, a, g))
        arr[k] = GtmpProblem(rs, _ptr(sph), sph.shape[0], _ptr(box), box.shape[0], _ptr(a), _ptr(g), M, L, seed)
    out = _vp()
    st = stream if stream is not None else _stream()
    status = lib().gtmp_batch_create(arr, len(problems), H, st, ctypes.byref(out))
    if status != GTMP_OK:
        raise GtmpError(status, "gtmp_batch_create rejected its arguments or the device")
    return out


def gtmp_batch_destroy(b):
    _bcheck(None, lib().gtmp_batch_destroy(b))


def gtmp_batch_set_stream(b, stream=None):
    _bcheck(b, lib().gtmp_batch_set_stream(b, stream if stream is not None else _stream()))


def gtmp_batch_info(b):
    """(L_max, nominal checks, work items, kernel launches per solve)."""
    L_max, checks, items, kernels = _i32(), ctypes.c_double(), _i32(), _i32()
    _bcheck(b, lib().gtmp_batch_info(b, ctypes.byref(L_max), ctypes.byref(checks), ctypes.byref(items),
                                     ctypes.byref(kernels)))
    return L_max.value, checks.value, items.value, kernels.value


def gtmp_batch_solve(b, dev_paths, dev_costs):
    import torch
    _bcheck(b, lib().gtmp_batch_solve(b, _dev(dev_paths, torch.int32), _dev(dev_costs, torch.float32)))


def gtmp_batch_synchronize(b):
    _bcheck(b, lib().gtmp_batch_synchronize(b))


def gtmp_batch_set_tiling(b, target_edges, chunk, kind=None):
    """Both robot kinds (kind None) or one (ROBOT_POINT, ROBOT_DH_ARM)."""
    if kind is None:
        _bcheck(b, lib().gtmp_batch_set_tiling(b, target_edges, chunk))
    else:
        _bcheck(b, lib().gtmp_batch_set_kind_tiling(b, kind, target_edges, chunk))


def gtmp_batch_get_tiling(b, kind):
    t, c = _i32(), _i32()
    _bcheck(b, lib().gtmp_batch_get_tiling(b, kind, ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


def gtmp_batch_get_tilings(b):
    """{kind: (target_edges, chunk)} for both robot kinds."""
    return {k: gtmp_batch_get_tiling(b, k) for k in (ROBOT_POINT, ROBOT_DH_ARM)}


def gtmp_batch_set_tilings(b, tilings):
    """Apply a {kind: (target_edges, chunk)} map (as gtmp_batch_get_tilings returns)."""
    for k, (t, c) in tilings.items():
        gtmp_batch_set_tiling(b, t, c, kind=k)


SAMPLER_UNIFORM, SAMPLER_FREE = 0, 1


def gtmp_set_sampler(ctx, sampler, max_attempts=64):
    _check(ctx, lib().gtmp_set_sampler(ctx, sampler, max_attempts))


def gtmp_set_goals(ctx, goals, values=None):
    g = _f32(goals)
    v = None if values is None else _f32(values)
    _check(ctx, lib().gtmp_set_goals(ctx, _ptr(g), None if v is None else _ptr(v), g.shape[0]))


def gtmp_joint_sincos(x):
    """(sin, cos) of a device float32 tensor as the arm kinematics computes them."""
    import torch
    x = x.contiguous()
    s, c = torch.empty_like(x), torch.empty_like(x)
    st = lib().gtmp_joint_sincos(_dev(x, torch.float32), x.numel(), _dev(s, torch.float32), _dev(c, torch.float32),
                                 _stream())
    if st != GTMP_OK:
        raise GtmpError(st, "gtmp_joint_sincos")
    return s, c


def gtmp_fp32_fma_peak(stream=None):
    """Measured FP32 FMA throughput of the current device, TFLOP/s."""
    out = ctypes.c_double()
    st = lib().gtmp_fp32_fma_peak(stream, ctypes.byref(out))
    if st != 0:
        raise RuntimeError(f"gtmp_fp32_fma_peak: {STATUS.get(st, st)}")
    return out.value


def gtmp_cull_grid(spheres, boxes, R_link, max_cells=16384):
    """The early-exit cull grid for these obstacles (host only): (masks [nz][ny][nx] uint32, origin [3], inv)."""
    sp = _f32(spheres).reshape(-1, 4)
    bx = _f32(boxes).reshape(-1, 6)
    masks = np.zeros(max(max_cells, 1), np.uint32)
    dims = (_i32 * 3)()
    oi = np.zeros(4, np.float32)
    st = lib().gtmp_cull_grid(_ptr(sp), sp.shape[0], _ptr(bx), bx.shape[0], R_link, max_cells,
                              masks.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), dims, _ptr(oi))
    if st != 0:
        raise GtmpError(st, "gtmp_cull_grid")
    nx, ny, nz = dims[0], dims[1], dims[2]
    return masks[:nx * ny * nz].reshape(nz, ny, nx), oi[:3].copy(), np.float32(oi[3])


MAX_WEIGHT_BUMPS = 16


def gtmp_set_cost_weight(ctx, bumps):
    """Weighted-length edge cost: bumps [K][dof + 2] = (centre, radius s, amplitude a); None or K = 0: length."""
    if bumps is None or np.asarray(bumps).size == 0:
        _check(ctx, lib().gtmp_set_cost_weight(ctx, None, 0))
        return
    b = _f32(bumps)
    b = b[None, :] if b.ndim == 1 else b
    _check(ctx, lib().gtmp_set_cost_weight(ctx, _ptr(b), b.shape[0]))


def gtmp_get_goal_reached(ctx, graph, dev_goal):
    import torch
    _check(ctx, lib().gtmp_get_goal_reached(ctx, graph, _dev(dev_goal, torch.int32)))


def gtmp_solve_classes(ctx, max_labels, max_classes, dev_paths, dev_costs, dev_labels):
    """Class-augmented sweep (Prop. 1): returns the number of classes found."""
    import torch
    n = _i32()
    _check(ctx, lib().gtmp_solve_classes(ctx, max_labels, max_classes, _dev(dev_paths, torch.int32),
                                         _dev(dev_costs, torch.float32), _dev(dev_labels, torch.int8),
                                         ctypes.byref(n)))
    return n.value


def gtmp_batch_set_eval_mode(b, eval_mode):
    _bcheck(b, lib().gtmp_batch_set_eval_mode(b, eval_mode))


def gtmp_batch_autotune(b, repeats, dev_paths, dev_costs):
    import torch
    ms = ctypes.c_float()
    _bcheck(b, lib().gtmp_batch_autotune(b, repeats, _dev(dev_paths, torch.int32), _dev(dev_costs, torch.float32),
                                         ctypes.byref(ms)))
    return ms.value


class Batch:
    """Many independent problems solved by one persistent launch."""

    def __init__(self, problems, H, eval_mode=None):
        import torch
        self.n = len(problems)
        self.handle = gtmp_batch_create(problems, H)
        if eval_mode is not None:
            gtmp_batch_set_eval_mode(self.handle, eval_mode)
        self.L_max, self.nominal_checks, _, _ = gtmp_batch_info(self.handle)
        self.paths = torch.empty((self.n, self.L_max), dtype=torch.int32, device="cuda")
        self.costs = torch.empty(self.n, dtype=torch.float32, device="cuda")

    @property
    def work_items(self):
        return gtmp_batch_info(self.handle)[2]

    @property
    def kernels_per_solve(self):
        return gtmp_batch_info(self.handle)[3]

    def solve(self):
        gtmp_batch_solve(self.handle, self.paths, self.costs)
        return self.paths, self.costs

    def autotune(self, repeats=2):
        return gtmp_batch_autotune(self.handle, repeats, self.paths, self.costs)

    def synchronize(self):
        gtmp_batch_synchronize(self.handle)

    def close(self):
        if self.handle:
            gtmp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned collision surrogate
# ---------------------------------------------------------------------------

def gtmp_surrogate_train(ctx, n_train=1 << 20, n_holdout=1 << 16, epochs=2, batch=8192, lr=1e-3, seed=1,
                         fourier_sigma=1.0):
    cfg = GtmpSurrogateConfig(n_train, n_holdout, epochs, batch, lr, seed, fourier_sigma)
    st = GtmpSurrogateStats()
    _check(ctx, lib().gtmp_surrogate_train(ctx, ctypes.byref(cfg), ctypes.byref(st)))
    return dict(final_loss=st.final_loss, holdout_accuracy=st.holdout_accuracy, holdout_fn_rate=st.holdout_fn_rate,
                holdout_fp_rate=st.holdout_fp_rate, train_ms=st.train_ms)


def gtmp_surrogate_predict(ctx, dev_q, dev_logits):
    import torch
    _check(ctx, lib().gtmp_surrogate_predict(ctx, _dev(dev_q, torch.float32), dev_q.shape[0],
                                             _dev(dev_logits, torch.float32)))


def gtmp_surrogate_param_count():
    return int(lib().gtmp_surrogate_param_count())


def gtmp_surrogate_get_params(ctx, dof):
    n = gtmp_surrogate_param_count()
    P = np.zeros(n, np.float32)
    B = np.zeros(64 * dof, np.float32)
    _check(ctx, lib().gtmp_surrogate_get_params(ctx, _ptr(P), n, _ptr(B), B.size))
    o = 0
    out = {}
    for name, shape in (("W1", (256, 128)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)),
                        ("W3", (256, 256)), ("b3", (256,)), ("w4", (256,)), ("b4", (1,))):
        size = int(np.prod(shape))
        out[name] = P[o:o + size].reshape(shape)
        o += size
    out["B"] = B.reshape(64, dof)
    return out


def gtmp_solve_pruned(ctx, threshold, dev_path, dev_cost, score_waypoints=1):
    import torch
    st = GtmpPruneStats()
    _check(ctx, lib().gtmp_solve_pruned(ctx, threshold, score_waypoints, _dev(dev_path, torch.int32),
                                        _dev(dev_cost, torch.float32), ctypes.byref(st)))
    return dict(edges=st.edges, pruned=st.pruned, score_ms=st.score_ms, solve_ms=st.solve_ms, scored=st.scored,
                band_ms=st.band_ms, lists_ms=st.lists_ms)


def gtmp_solve_lazy_path(ctx, dev_path, dev_cost, max_iterations=100000):
    """Path-level lazy evaluation: optimistic min-plus sweeps, exact check of the winning chain, repeat."""
    import torch
    st = GtmpLazyStats()
    _check(ctx, lib().gtmp_solve_lazy_path(ctx, max_iterations, _dev(dev_path, torch.int32),
                                           _dev(dev_cost, torch.float32), ctypes.byref(st)))
    return dict(iterations=st.iterations, colliding_edges=st.colliding_edges)


def gtmp_surrogate_set_protect(ctx, band):
    """Protection band of the pruned solve: edges within (1 + band) x their row's best bound are never pruned."""
    _check(ctx, lib().gtmp_surrogate_set_protect(ctx, band))


def gtmp_surrogate_score(ctx, layer, threshold, dev_mask, score_waypoints=1):
    """The scoring kernel's decisions for transition `layer`: dev_mask uint8 [rows][cols] (1 pruned, 0 kept,
    2 not live); returns the live-edge count."""
    import torch
    n = ctypes.c_int64()
    _check(ctx, lib().gtmp_surrogate_score(ctx, layer, threshold, score_waypoints, _dev(dev_mask, torch.uint8),
                                           ctypes.byref(n)))
    return int(n.value)


def gtmp_umma_gemm_f32(A, B, C, err, stream=None):
    """C = A @ B.T on the tcgen05 tensor cores (A [M][K], B [N][K] bf16, C [M][N] float32)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    st = stream if stream is not None else _stream()
    _check(None, lib().gtmp_umma_gemm_f32(_dev(A, torch.bfloat16), A.stride(0), _dev(B, torch.bfloat16), B.stride(0),
                                          M, N, K, _dev(C, torch.float32), C.stride(0), st, _dev(err, torch.int32)))


_PARAM_LAYOUT = (("W1", (256, 128)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)),
                 ("b3", (256,)), ("w4", (256,)), ("b4", (1,)))


def flatten_params(P):
    return np.concatenate([np.asarray(P[k], np.float32).reshape(-1) for k, _ in _PARAM_LAYOUT])


def unflatten_params(v):
    out, o = {}, 0
    for name, shape in _PARAM_LAYOUT:
        size = int(np.prod(shape))
        out[name] = v[o:o + size].reshape(shape)
        o += size
    return out


def gtmp_surrogate_set_params(ctx, P):
    flat = flatten_params(P)
    B = _f32(P["B"]).reshape(-1)
    _check(ctx, lib().gtmp_surrogate_set_params(ctx, _ptr(flat), flat.size, _ptr(B), B.size))


def gtmp_surrogate_loss_grad(ctx, dev_q, dev_labels):
    import torch
    n = gtmp_surrogate_param_count()
    g = np.zeros(n, np.float32)
    loss = ctypes.c_double()
    _check(ctx, lib().gtmp_surrogate_loss_grad(ctx, _dev(dev_q, torch.float32), _dev(dev_labels, torch.uint8),
                                               dev_q.shape[0], ctypes.byref(loss), _ptr(g), n))
    return loss.value, unflatten_params(g)
