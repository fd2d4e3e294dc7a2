"""Collision surrogate on the tcgen05 tensor cores: the forward pass against an
independent numpy evaluation of the same BF16 weights, training against the
exact checker's labels, and the surrogate-pruned solve (exact checking of every
surviving edge, so returned paths stay collision free)."""
import math

import numpy as np
import pytest

import oracle
from paper_2608_25830_b300 import binding, scenes

from parity import REL, scene_for

pytestmark = pytest.mark.gpu


def _bf16(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def reference_logits(P, q):
    """FP64 evaluation of the surrogate with the kernel's BF16 rounding points."""
    z = q.astype(np.float64) @ P["B"].astype(np.float64).T
    phi = _bf16(np.concatenate([np.sin(z), np.cos(z)], 1))
    h1 = _bf16(np.maximum(phi @ _bf16(P["W1"]).T + P["b1"], 0))
    h2 = _bf16(np.maximum(h1 @ _bf16(P["W2"]).T + P["b2"], 0))
    h3 = np.maximum(h2 @ _bf16(P["W3"]).T + P["b3"], 0)
    return h3 @ P["w4"].astype(np.float64) + float(P["b4"][0])


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
    import torch
    sc, p, _ = trained
    rng = np.random.default_rng(0)
    n = 1000                                  # several 128-row tiles and a ragged tail
    q = rng.uniform(sc.robot.q_lo, sc.robot.q_hi, (n, 7)).astype(np.float32)
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    binding.gtmp_surrogate_predict(p.ctx, torch.from_numpy(q).cuda(), z)
    got = z.cpu().numpy().astype(np.float64)
    ref = reference_logits(binding.gtmp_surrogate_get_params(p.ctx, 7), q)
    # the feature map is taken in float32 on the device and in fp64 here, so a
    # bf16 rounding of a feature or hidden unit can land one ulp apart; the
    # logits agree to a few percent and the decisions almost everywhere
    err = np.abs(got - ref)
    assert np.corrcoef(got, ref)[0, 1] > 0.999
    assert np.mean(err <= 0.05 + 0.05 * np.abs(ref)) > 0.99, np.quantile(err, [0.5, 0.99, 1.0])
    assert np.mean((got > 0) == (ref > 0)) > 0.99


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


def reference_gradients(P, q, y):
    """FP64 backward pass of the mean binary cross-entropy, with the kernel's BF16 rounding points."""
    z = q.astype(np.float64) @ P["B"].astype(np.float64).T
    phi = _bf16(np.concatenate([np.sin(z), np.cos(z)], 1))
    W1, W2, W3 = _bf16(P["W1"]), _bf16(P["W2"]), _bf16(P["W3"])
    h1 = _bf16(np.maximum(phi @ W1.T + P["b1"], 0))
    h2 = _bf16(np.maximum(h1 @ W2.T + P["b2"], 0))
    h3f = np.maximum(h2 @ W3.T + P["b3"], 0)
    h3 = _bf16(h3f)
    logit = h3f @ P["w4"].astype(np.float64) + float(P["b4"][0])
    p = 1 / (1 + np.exp(-logit))
    n = len(y)
    loss = np.mean(np.maximum(logit, 0) - logit * y + np.log1p(np.exp(-np.abs(logit))))
    dz = (p - y) / n
    g = {"w4": h3.T @ dz, "b4": np.array([dz.sum()])}
    dA3 = _bf16(dz[:, None] * P["w4"][None, :] * (h3 > 0))
    g["W3"], g["b3"] = dA3.T @ h2, dA3.sum(0)
    dA2 = _bf16((dA3 @ W3) * (h2 > 0))
    g["W2"], g["b2"] = dA2.T @ h1, dA2.sum(0)
    dA1 = _bf16((dA2 @ W2) * (h1 > 0))
    g["W1"], g["b1"] = dA1.T @ phi, dA1.sum(0)
    return loss, g


def test_backward_pass_matches_numpy():
    """One training batch's loss and gradients against an independent fp64 backward pass."""
    import torch
    sc = scene_for("arm", 1, 7, 30)
    p = binding.Planner(sc.robot, 8, 1, 2, max_obstacles=64)
    p.set_scene(sc)
    rng = np.random.default_rng(5)
    P = {"B": rng.normal(0, 1, (64, 7)).astype(np.float32)}
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
    ref_loss, R = reference_gradients(P, q, labels.cpu().numpy().astype(np.float64))
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    binding.gtmp_surrogate_predict(p.ctx, qd, z)
    zr = reference_logits(P, q)
    rels = {k: float(np.linalg.norm(G[k].astype(np.float64) - R[k]) / max(np.linalg.norm(R[k]), 1e-30)) for k in R}
    report = dict(loss=loss, ref_loss=ref_loss, logit_corr=float(np.corrcoef(z.cpu().numpy(), zr)[0, 1]),
                  logit_mean=(float(z.cpu().numpy().mean()), float(zr.mean())), rel=rels)
    assert loss == pytest.approx(ref_loss, rel=1e-2), report
    for k, rel in rels.items():
        assert rel < 3e-2, report


def test_scoring_kernel_prunes_what_the_model_predicts(trained):
    """The fused scoring kernel's decisions against the model evaluated through the GEMM path
    (gtmp_surrogate_predict) at every live edge's midpoint: the pruned counts agree up to decisions within
    rounding of the threshold (features use the fast sincos in the scoring kernel)."""
    import torch
    sc, p, _ = trained
    L, H, M = 4, 32, 128
    thr = 0.5
    p.sample_layers(12, M)
    p.solve()                                   # vertex flags and values of this graph
    st = binding.gtmp_solve_pruned(p.ctx, thr, torch.empty(L, dtype=torch.int32, device="cuda"),
                                   torch.empty(1, dtype=torch.float32, device="cuda"), score_waypoints=1)
    p.synchronize()
    V, _ = p.values()
    V = V.cpu().numpy()
    Q = p.get_layers().cpu().numpy()
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    flags = [p.label_configs(torch.from_numpy(np.ascontiguousarray(v)).cuda()).cpu().numpy() for v in verts]
    # the pruned solve's own value iteration decides which columns are live; its values equal the plain
    # solve's wherever no edge was pruned on the way, so recompute liveness from its own tables
    mids, live_count = [], 0
    for l in range(L + 1):
        rows = np.nonzero(flags[l] == 0)[0]
        cols = np.nonzero((flags[l + 1] == 0) & np.isfinite(V[l + 1, :len(verts[l + 1])]))[0]
        live_count += len(rows) * len(cols)
        if len(rows) and len(cols):
            u = verts[l][rows][:, None, :]
            v = verts[l + 1][cols][None, :, :]
            mids.append((u + np.float32(0.5) * (v - u)).reshape(-1, sc.robot.dof).astype(np.float32))
    q = np.concatenate(mids)
    z = torch.empty(len(q), dtype=torch.float32, device="cuda")
    binding.gtmp_surrogate_predict(p.ctx, torch.from_numpy(q).cuda(), z)
    want = int((z.cpu().numpy() > math.log(thr / (1 - thr))).sum())
    assert st["scored"] == live_count
    assert abs(st["pruned"] - want) <= 0.01 * live_count, (st["pruned"], want, live_count)
