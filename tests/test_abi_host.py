"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/gtmp.h declares, and rejects bad arguments before it
touches a device."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2608_25830_b300 import binding, build, scenes

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gtmp.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^GTMP_API\s+[\w\s\*]+?\b((?:gtmp|aogtmp)_\w+)\s*\(", text, flags=re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    names = declared_functions()
    assert len(names) >= 19
    L = binding.lib()
    for n in names:
        assert hasattr(L, n), n
        assert n in binding._SIGNATURES or n in ("gtmp_last_error", "gtmp_status_string", "gtmp_batch_last_error",
                                                 "gtmp_surrogate_param_count"), n


def test_status_strings():
    L = binding.lib()
    for code, name in binding.STATUS.items():
        assert L.gtmp_status_string(code).decode() == name


def _create(robot, **kw):
    p = dict(M=16, L=3, H=8, R=1, max_obstacles=8, eval_mode=0, max_edge_len=math.inf)
    p.update(kw)
    rs, keep = binding.robot_struct(robot)
    ps = binding.GtmpParams(p["M"], p["L"], p["H"], p["R"], p["max_obstacles"], p["eval_mode"], p["max_edge_len"])
    out = ctypes.c_void_p()
    return binding.lib().gtmp_create(ctypes.byref(rs), ctypes.byref(ps), None, ctypes.byref(out)), out


@pytest.mark.parametrize("kw", [dict(M=0), dict(M=20000), dict(L=0), dict(H=1), dict(R=0), dict(eval_mode=7),
                                dict(max_edge_len=0.0), dict(max_edge_len=float("nan")), dict(max_obstacles=-1)])
def test_create_rejects_bad_params(kw):
    st, out = _create(scenes.dh_arm(0, 7), **kw)
    assert st == 1 and not out.value


def test_create_rejects_bad_robots():
    good = scenes.dh_arm(0, 7)
    bad_dof = scenes.Robot(good.kind, 0, good.dh[:0], good.link_spheres[:0], good.q_lo[:0], good.q_hi[:0])
    assert _create(bad_dof)[0] == 1
    box = good.q_lo.copy()
    assert _create(scenes.Robot(good.kind, 7, good.dh, good.link_spheres, good.q_hi, box))[0] == 1   # hi < lo
    nan_dh = good.dh.copy()
    nan_dh[2, 1] = np.nan
    assert _create(scenes.Robot(good.kind, 7, nan_dh, good.link_spheres, good.q_lo, good.q_hi))[0] == 1
    zero_r = good.link_spheres.copy()
    zero_r[1, 2, 3] = 0.0
    assert _create(scenes.Robot(good.kind, 7, good.dh, zero_r, good.q_lo, good.q_hi))[0] == 1
    pt = scenes.point_robot_2d()
    assert _create(scenes.Robot(pt.kind, 4, np.zeros((4, 4), np.float32), np.zeros((4, 0, 4), np.float32),
                                np.full(4, -1, np.float32), np.full(4, 1, np.float32)))[0] == 1


def test_null_context_calls_fail_cleanly():
    L = binding.lib()
    assert L.gtmp_destroy(None) == 0
    assert L.gtmp_synchronize(None) == 1
    assert L.gtmp_solve(None, None, None) == 1
    assert L.gtmp_set_cost_weight(None, None, 0) == 1
    assert L.gtmp_last_error(None).decode() == "null context"
