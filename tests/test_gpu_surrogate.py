"""Collision surrogate on the tcgen05 tensor cores: the forward and backward
passes and the fused scoring kernel against an independent FP64 evaluation of
the same BF16 weights, element by element within the bounds that
`surrogate_bounds` derives from BF16 rounding (and pins on the CPU); training
against the exact checker's labels; and the surrogate-pruned solve (exact
checking of every surviving edge, so returned paths stay collision free)."""
import math

import numpy as np
import pytest

import oracle
import surrogate_bounds as sb
from paper_2608_25830_b300 import binding, scenes

from parity import REL, scene_for

pytestmark = pytest.mark.gpu

# The device computes the Fourier features with the fast __sincosf.  Its
# documented maximum absolute error is 2^-21.41 on [-pi, pi]; beyond, the
# range reduction adds about |z| 2^-23.  The bounds assume 2^-16, over ten
# times either for the |z| <= 16 the tests check.
EPS_SIN = 2.0 ** -16
Z_MAX = 16.0


@pytest.fixture(scope="module")
def trained():
    sc = scene_for("arm", 0, 7, 40)
    p = binding.Planner(sc.robot, 128, 4, 32, max_obstacles=64)
    p.set_scene(sc)
    stats = binding.gtmp_surrogate_train(p.ctx, n_train=1 << 19, n_holdout=1 << 15, epochs=3, batch=1024, lr=1e-3,
                                         seed=3, fourier_sigma=0.25)
    return sc, p, stats


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 256, 448), (1000, 128, 128), (77, 16, 8), (256, 256, 8192)])
def test_tensor_core_gemm_is_exact(M, N, K):
    """bf16 products are exact and the accumulation is float32: compare with an fp64 GEMM of the same inputs."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    binding.gtmp_umma_gemm_f32(A.cuda(), B.cuda(), C, err)
    torch.cuda.synchronize()
    ref = A.double() @ B.double().T
    got = C.cpu().double()
    assert int(err.cpu()[0]) == 0
    bound = 1e-5 * (A.double().abs() @ B.double().abs().T) + 1e-6      # float32 accumulation of K terms
    assert torch.all((got - ref).abs() <= bound), float(((got - ref).abs() / bound).max())


def test_forward_matches_numpy_with_same_bf16_weights(trained):
    """Every logit of the GEMM path within its first-order bound of the FP64 reference."""
    import torch
    sc, p, _ = trained
    rng = np.random.default_rng(0)
    n = 1000                                  # several 128-row tiles and a ragged tail
    q = rng.uniform(sc.robot.q_lo, sc.robot.q_hi, (n, 7)).astype(np.float32)
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    binding.gtmp_surrogate_predict(p.ctx, torch.from_numpy(q).cuda(), z)
    got = z.cpu().numpy().astype(np.float64)
    P = binding.gtmp_surrogate_get_params(p.ctx, 7)
    ref, tau = sb.logit_bound(P, q, EPS_SIN)
    assert np.max(np.abs(sb.reference(P, q)["zf"])) <= Z_MAX
    err = np.abs(got - ref)
    assert np.all(err <= tau), (int(np.sum(err > tau)), float(np.max(err / tau)))
    # the bound has teeth: it decides most logits at the pruning cut (0) and stays well below their size
    assert np.mean(np.abs(ref) > tau) > 0.75, np.mean(np.abs(ref) > tau)
    assert np.median(tau) < 0.25 * np.median(np.abs(ref)), (np.median(tau), np.median(np.abs(ref)))
    print(f"forward: max err/bound {np.max(err / tau):.3f}, median bound {np.median(tau):.3f}")


def test_training_learns_the_exact_labels(trained):
    _, _, st = trained
    # an untrained model scores ln 2 = 0.69; the collision rate of this scene is
    # about 0.29, so always answering "free" is right 71 % of the time
    assert st["final_loss"] < 0.45, st
    assert st["holdout_accuracy"] > 0.77, st
    assert 0.0 <= st["holdout_fn_rate"] <= 1.0 and 0.0 <= st["holdout_fp_rate"] <= 1.0


def test_pruned_solve_is_exactly_checked(trained):
    import torch
    sc, p, _ = trained
    L, H, M = 4, 32, 128
    for seed, kw, thr in ((5, 1, 0.5), (6, 3, 0.5), (7, 1, 0.9)):
        p.sample_layers(seed, M)
        plain_path, plain_cost = p.solve()
        path = torch.empty(L, dtype=torch.int32, device="cuda")
        cost = torch.empty(1, dtype=torch.float32, device="cuda")
        st = binding.gtmp_solve_pruned(p.ctx, thr, path, cost, score_waypoints=kw)
        p.synchronize()
        c0, c1 = float(plain_cost.cpu()[0]), float(cost.cpu()[0])
        assert st["edges"] == 2 * M + (L - 1) * M * M and 0 <= st["pruned"] <= st["edges"]
        if thr == 0.5:
            assert st["pruned"] > 0.05 * st["edges"]
        # a subset of the edges can only make the best chain longer (same per-edge float32 values)
        assert c1 >= c0 or (math.isinf(c0) and math.isinf(c1))
        if math.isfinite(c1):
            Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
            total, worst = oracle.path_cost(sc, Q, path.cpu().numpy(), H)
            assert worst > -oracle.EPS_DEFAULT          # every returned path is collision free
            assert c1 == pytest.approx(total, rel=REL)


def test_lazy_pruned_solve_equals_early_exit_pruned_solve(trained):
    """Same scene, samples and surrogate: the lazy exact pass over the surviving edges returns the early-exit
    pass's path and cost bit for bit (it skips only edges that cannot lower a row's minimum)."""
    import torch
    sc, p, _ = trained
    L, H, M = 4, 32, 128
    lz = binding.Planner(sc.robot, M, L, H, max_obstacles=64, eval_mode=binding.EVAL_LAZY)
    lz.set_scene(sc)
    binding.gtmp_surrogate_set_params(lz.ctx, binding.gtmp_surrogate_get_params(p.ctx, sc.robot.dof))
    for seed, kw, thr in ((5, 1, 0.5), (8, 3, 0.3)):
        out = []
        for pl in (p, lz):
            pl.sample_layers(seed, M)
            path = torch.empty(L, dtype=torch.int32, device="cuda")
            cost = torch.empty(1, dtype=torch.float32, device="cuda")
            st = binding.gtmp_solve_pruned(pl.ctx, thr, path, cost, score_waypoints=kw)
            pl.synchronize()
            out.append((path.cpu().numpy(), float(cost.cpu()[0]), st["pruned"]))
        np.testing.assert_array_equal(out[0][0], out[1][0])
        assert out[0][1] == out[1][1] or (math.isinf(out[0][1]) and math.isinf(out[1][1]))
        assert out[0][2] == out[1][2]
    lz.close()


def test_backward_pass_matches_numpy():
    """One training batch's loss and gradients against an independent fp64 backward pass."""
    import torch
    sc = scene_for("arm", 1, 7, 30)
    p = binding.Planner(sc.robot, 8, 1, 2, max_obstacles=64)
    p.set_scene(sc)
    rng = np.random.default_rng(5)
    P = {"B": rng.normal(0, 0.25, (64, 7)).astype(np.float32)}
    for name, (fo, fi) in (("W1", (256, 128)), ("W2", (256, 256)), ("W3", (256, 256))):
        P[name] = rng.uniform(-1 / math.sqrt(fi), 1 / math.sqrt(fi), (fo, fi)).astype(np.float32)
    for name in ("b1", "b2", "b3"):
        P[name] = rng.uniform(-0.1, 0.1, 256).astype(np.float32)
    P["w4"] = rng.uniform(-1 / 16, 1 / 16, 256).astype(np.float32)
    P["b4"] = np.array([0.05], np.float32)
    binding.gtmp_surrogate_set_params(p.ctx, P)
    n = 512
    q = rng.uniform(sc.robot.q_lo, sc.robot.q_hi, (n, 7)).astype(np.float32)
    qd = torch.from_numpy(q).cuda()
    labels = p.label_configs(qd)
    loss, G = binding.gtmp_surrogate_loss_grad(p.ctx, qd, labels)
    y = labels.cpu().numpy().astype(np.float64)
    ref_loss, dloss, R, tol = sb.gradients(P, q, y, EPS_SIN)
    assert abs(loss - ref_loss) <= dloss, (loss, ref_loss, dloss)
    for k in R:
        err = np.abs(G[k].astype(np.float64).reshape(R[k].shape) - R[k])
        assert np.all(err <= tol[k]), (k, int(np.sum(err > tol[k])), float(np.max(err / tol[k])))


def _live_edges(p, sc, L, V, flags, layer):
    """Live (row, column) pairs of a transition: row vertex free; column vertex free with a finite cost-to-go."""
    rows = np.nonzero(flags[layer] == 0)[0]
    cols = np.nonzero((flags[layer + 1] == 0) & np.isfinite(V[layer + 1, :len(flags[layer + 1])]))[0]
    return rows, cols


def _waypoints(u, v, kw):
    """The float32 configurations the scoring kernel evaluates: fma(t, v - u, u) at t = 1/2 (kw = 1) or
    t = 1/4, 1/2, 3/4 (kw = 3), one rounding each (exact in float64 before it)."""
    d = (v - u).astype(np.float32).astype(np.float64)
    ts = [0.5] if kw == 1 else [0.25, 0.5, 0.75]
    return [(u.astype(np.float64) + t * d).astype(np.float32) for t in ts]


def test_protection_band_keeps_each_rows_best_bounds(trained):
    """With a protection band b, an edge whose bound |v - u| + J(v) is at most (1 + b) times the smallest
    bound of its row (over the live columns) is never pruned, and every other live edge keeps the decision
    it has without the band; the band only ever removes edges from the pruned set.  Edges within 1e-5
    relative of the band's edge are not judged (float32 bound against the host's FP64 one).  Aggressive
    threshold 0.1, M = 120, five transitions."""
    import torch
    sc, p, _ = trained
    L, M, thr, band = 4, 120, 0.1, 0.1
    p.sample_layers(23, M)
    p.solve()
    V, _ = p.values()
    V = V.cpu().numpy()
    Q = p.get_layers().cpu().numpy()
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    flags = [p.label_configs(torch.from_numpy(np.ascontiguousarray(v)).cuda()).cpu().numpy() for v in verts]
    assert binding.lib().gtmp_surrogate_set_protect(p.ctx, -0.5) == 1
    assert binding.lib().gtmp_surrogate_set_protect(p.ctx, float("nan")) == 1
    judged = protected = 0
    try:
        for layer in range(L + 1):
            nr, nc = len(verts[layer]), len(verts[layer + 1])
            masks = []
            for b in (0.0, band):
                binding.gtmp_surrogate_set_protect(p.ctx, b)
                m = torch.full((nr, nc), 7, dtype=torch.uint8, device="cuda")
                binding.gtmp_surrogate_score(p.ctx, layer, thr, m)
                masks.append(m.cpu().numpy())
            off, on = masks
            rows, cols = _live_edges(p, sc, L, V, flags, layer)
            if len(rows) == 0 or len(cols) == 0:
                continue
            assert np.all(on[np.ix_(rows, cols)] <= off[np.ix_(rows, cols)]), f"layer {layer}: band added prunes"
            u = verts[layer][rows].astype(np.float64)
            v = verts[layer + 1][cols].astype(np.float64)
            vj = V[layer + 1, :nc][cols].astype(np.float64)
            bound = np.sqrt(((v[None, :, :] - u[:, None, :]) ** 2).sum(-1)) + vj[None, :]
            lim = (1.0 + band) * bound.min(1, keepdims=True)
            inside = bound <= lim * (1 - 1e-5)
            outside = bound >= lim * (1 + 1e-5)
            sub_on, sub_off = on[np.ix_(rows, cols)], off[np.ix_(rows, cols)]
            assert np.all(sub_on[inside] == 0), f"layer {layer}: {int(np.sum(sub_on[inside]))} band edges pruned"
            np.testing.assert_array_equal(sub_on[outside], sub_off[outside], err_msg=f"layer {layer}")
            judged += int(inside.sum() + outside.sum())
            protected += int(np.sum(inside & (sub_off == 1)))
    finally:
        binding.gtmp_surrogate_set_protect(p.ctx, 0.0)
    assert protected > 0, "the band never overrode a prune: the test has no teeth"
    print(f"protection band: {judged} live edges judged, {protected} prunes overridden")


@pytest.mark.parametrize("kw", [1, 3])
def test_scoring_kernel_decisions_elementwise(trained, kw):
    """Every live edge's prune decision from the fused scoring kernel (gtmp_surrogate_score) against
    (a) the same model through the GEMM path at the same float32 waypoints: the two share the features
    (same FMA order and sincos), the tensor-core accumulation order and the epilogue roundings, and differ
    only in the head's summation order, so the decisions must agree wherever the GEMM logit is farther
    from the cut than two FP32 sums of the head's 256 terms can differ; and (b) the FP64 reference,
    wherever its logit lies outside the first-order bound of surrogate_bounds.  M = 120 (ragged against
    the 128-query tiles), five transitions including the start row and the goal column."""
    import torch
    sc, p, _ = trained
    L, M, thr = 4, 120, 0.5
    cut = math.log(thr / (1 - thr))
    P = binding.gtmp_surrogate_get_params(p.ctx, 7)
    p.sample_layers(21, M)
    p.solve()                                   # vertex labels and cost-to-go that decide liveness
    V, _ = p.values()
    V = V.cpu().numpy()
    Q = p.get_layers().cpu().numpy()
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    flags = [p.label_configs(torch.from_numpy(np.ascontiguousarray(v)).cuda()).cpu().numpy() for v in verts]
    compared_a = compared_b = total = 0
    for layer in range(L + 1):
        nr, nc = len(verts[layer]), len(verts[layer + 1])
        mask = torch.full((nr, nc), 7, dtype=torch.uint8, device="cuda")
        scored = binding.gtmp_surrogate_score(p.ctx, layer, thr, mask, score_waypoints=kw)
        mask = mask.cpu().numpy()
        rows, cols = _live_edges(p, sc, L, V, flags, layer)
        live = np.zeros((nr, nc), bool)
        live[np.ix_(rows, cols)] = True
        assert scored == live.sum()
        np.testing.assert_array_equal(mask[~live], 2, err_msg=f"layer {layer}: non-live edges written")
        assert np.all(mask[live] <= 1), f"layer {layer}: live edge not scored"
        if not live.any():
            continue
        ii, jj = np.nonzero(live)
        got = mask[ii, jj].astype(bool)
        wps = _waypoints(verts[layer][ii], verts[layer + 1][jj], kw)
        # (a) the GEMM path at the same waypoints
        z_gemm, head = [], []
        for w in wps:
            z = torch.empty(len(w), dtype=torch.float32, device="cuda")
            binding.gtmp_surrogate_predict(p.ctx, torch.from_numpy(np.ascontiguousarray(w)).cuda(), z)
            z_gemm.append(z.cpu().numpy().astype(np.float64))
            r = sb.reference(P, w)
            assert np.max(np.abs(r["zf"])) <= Z_MAX
            head.append(2.0 * sb.gamma(256) * 1.5 * (r["h3"] @ np.abs(r["w4"])) + 1e-6)
        zg, hb = np.max(z_gemm, 0), np.max(head, 0)
        want = zg > cut
        sure = np.abs(zg - cut) > hb
        np.testing.assert_array_equal(got[sure], want[sure], err_msg=f"layer {layer}: scoring vs GEMM path")
        compared_a += int(sure.sum())
        # (b) the FP64 reference: prune if any waypoint is surely above the cut, keep if all surely below
        dec = np.stack([sb.decisions(*sb.logit_bound(P, w, EPS_SIN), cut) for w in wps])
        must_prune = np.any(dec == 1, 0)
        must_keep = np.all(dec == 0, 0)
        assert np.all(got[must_prune]), f"layer {layer}: {int(np.sum(~got[must_prune]))} edges not pruned"
        assert not np.any(got[must_keep]), f"layer {layer}: {int(np.sum(got[must_keep]))} edges pruned"
        compared_b += int(must_prune.sum() + must_keep.sum())
        total += len(ii)
    print(f"scoring kw={kw}: {total} live edges, {compared_a} compared with the GEMM path, "
          f"{compared_b} with the FP64 reference")
    assert total > 8000
    assert compared_a >= 0.999 * total, (compared_a, total)
    assert compared_b >= 0.6 * total, (compared_b, total)


@pytest.mark.parametrize("dof", [6, 5])
def test_scoring_kernel_other_joint_counts(dof):
    """The scoring kernel's 6-joint instantiation and its generic one (5 joints: the joint count read at
    run time) against the GEMM path at the same float32 waypoints, edge by edge, wherever the GEMM logit
    is farther from the cut than two FP32 sums of the head's 256 terms can differ (the bound of
    test_scoring_kernel_decisions_elementwise).  M = 100 (one full 128-query tile and a ragged one per
    row block), every transition including the start row and the goal column."""
    import torch
    sc = scene_for("arm", 1, dof, 30)
    L, M, thr = 3, 100, 0.5
    cut = math.log(thr / (1 - thr))
    p = binding.Planner(sc.robot, M, L, 16, max_obstacles=64)
    p.set_scene(sc)
    binding.gtmp_surrogate_train(p.ctx, n_train=1 << 16, n_holdout=1 << 12, epochs=1, batch=1024, lr=1e-3,
                                 seed=5, fourier_sigma=0.25)
    P = binding.gtmp_surrogate_get_params(p.ctx, dof)
    p.sample_layers(9, M)
    p.solve()
    V, _ = p.values()
    V = V.cpu().numpy()
    Q = p.get_layers().cpu().numpy()
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    flags = [p.label_configs(torch.from_numpy(np.ascontiguousarray(v)).cuda()).cpu().numpy() for v in verts]
    compared = total = 0
    for layer in range(L + 1):
        nr, nc = len(verts[layer]), len(verts[layer + 1])
        mask = torch.full((nr, nc), 7, dtype=torch.uint8, device="cuda")
        scored = binding.gtmp_surrogate_score(p.ctx, layer, thr, mask, score_waypoints=1)
        mask = mask.cpu().numpy()
        rows, cols = _live_edges(p, sc, L, V, flags, layer)
        live = np.zeros((nr, nc), bool)
        live[np.ix_(rows, cols)] = True
        assert scored == live.sum()
        np.testing.assert_array_equal(mask[~live], 2, err_msg=f"layer {layer}: non-live edges written")
        if not live.any():
            continue
        ii, jj = np.nonzero(live)
        got = mask[ii, jj].astype(bool)
        (w,) = _waypoints(verts[layer][ii], verts[layer + 1][jj], 1)
        z = torch.empty(len(w), dtype=torch.float32, device="cuda")
        binding.gtmp_surrogate_predict(p.ctx, torch.from_numpy(np.ascontiguousarray(w)).cuda(), z)
        zg = z.cpu().numpy().astype(np.float64)
        r = sb.reference(P, w)
        hb = 2.0 * sb.gamma(256) * 1.5 * (r["h3"] @ np.abs(r["w4"])) + 1e-6
        sure = np.abs(zg - cut) > hb
        np.testing.assert_array_equal(got[sure], (zg > cut)[sure], err_msg=f"dof {dof} layer {layer}")
        compared += int(sure.sum())
        total += len(ii)
    print(f"scoring dof={dof}: {total} live edges, {compared} compared with the GEMM path")
    assert total > 5000
    assert compared >= 0.999 * total, (compared, total)
