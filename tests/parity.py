"""Comparison rules between the CUDA planner and the CPU oracle.

Floating-point tolerance: costs and values are sums of at most L+1 float32
edge lengths (each a correctly rounded sqrt of a float32 dot product, relative
error below 1e-6) plus float32 additions, so agreement to REL = 1e-5 relative
leaves an order of magnitude of headroom.  Collision labels are compared only
outside the +-eps (1e-6 m) band in which the oracle calls a waypoint
ambiguous; float32 forward kinematics of the evaluated arms stays within
3e-7 m of FP64.  Minimiser indices are compared only where the best and the
second-best candidate differ by more than REL and no ambiguous edge decides.
"""
import math

import numpy as np

REL = 1e-5


def scene_for(kind, seed=0, dof=7, n_obs=30):
    import oracle
    from paper_2608_25830_b300 import scenes
    if kind == "point2d":
        return scenes.point2d_scene(seed, n_obs)
    sc = scenes.arm_scene(seed, dof, n_obs)
    return scenes.pick_endpoints(sc, lambda q: oracle.config_free(sc, q))


def check_values(V_gpu, V_lo, V_hi, what=""):
    """Per vertex: V_lo (1-REL) <= V_gpu <= V_hi (1+REL), +inf exactly where forced."""
    V_gpu = np.asarray(V_gpu, np.float64)
    V_lo = np.asarray(V_lo, np.float64)
    V_hi = np.asarray(V_hi, np.float64)
    lo_inf = np.isinf(V_lo)
    assert np.all(np.isinf(V_gpu[lo_inf])), f"{what}: GPU finite where no chain exists"
    hi_fin = np.isfinite(V_hi)
    assert np.all(np.isfinite(V_gpu[hi_fin])), f"{what}: GPU +inf where a chain exists"
    fin = np.isfinite(V_gpu)
    assert np.all(V_gpu[fin] >= V_lo[fin] * (1 - REL) - 1e-12), f"{what}: below the lower bound"
    ok_hi = fin & hi_fin
    bad = np.nonzero(V_gpu[ok_hi] > V_hi[ok_hi] * (1 + REL) + 1e-12)[0]
    assert bad.size == 0, f"{what}: above the upper bound at {bad[:5]}"


def decisive(sol, layer):
    """Vertices of `layer` whose minimiser is unique beyond REL and unaffected by ambiguity."""
    best = sol.V_lo[layer]
    sec = sol.second[layer]
    fin = np.isfinite(best)
    with np.errstate(invalid="ignore"):   # inf - inf where a vertex has a single finite candidate
        gap = np.where(fin, sec - best, 0.0)
    same = np.where(fin, np.isclose(sol.V_lo[layer], sol.V_hi[layer], rtol=0, atol=0), False)
    return fin & same & (gap > REL * np.maximum(best, 1e-30))


def compare_solution(sol, V_gpu, S_gpu, path_gpu, cost_gpu, what=""):
    """Values of every layer, minimisers where decisive, the returned cost and path."""
    n_layers = len(sol.V_lo)
    for l in range(n_layers):
        n = len(sol.V_lo[l])
        check_values(V_gpu[l, :n], sol.V_lo[l], sol.V_hi[l], f"{what} layer {l}")
        if l < n_layers - 1:
            d = decisive(sol, l)
            np.testing.assert_array_equal(S_gpu[l, :n][d], sol.sigma[l][d], err_msg=f"{what} sigma layer {l}")
    check_values([cost_gpu], [sol.cost_lo], [sol.cost_hi], f"{what} cost")
    if math.isinf(sol.cost_lo):
        assert list(path_gpu) == [-1] * len(path_gpu)
        return
    # path: identical while every choice along the oracle's chain is decisive
    i = 0
    for l in range(0, n_layers - 2):
        if not decisive(sol, l)[i]:
            break
        assert path_gpu[l] == sol.path[l], f"{what}: path differs at layer {l + 1}"
        i = sol.path[l]
