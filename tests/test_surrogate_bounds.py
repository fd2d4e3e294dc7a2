"""Pins of the surrogate's bounded FP64 reference (CPU).

The GPU tests compare the tensor-core surrogate with `surrogate_bounds`
element by element, trusting its bounds.  Here the bounds are checked against
an independent float32 simulation of the device arithmetic: features from a
float32 chain with sin/cos perturbed by up to the allowed error, every layer's
products summed in float32 in a random order, BF16 rounding after the
features and layers 1 and 2.  Every simulated logit and gradient must lie
within its bound, and plausible mistakes planted in the simulation (a
transposed weight matrix, a dropped K chunk, swapped biases, swapped sin and
cos, a flipped gradient sign, a missing ReLU gate) must break the bound."""
import math

import numpy as np
import pytest

import surrogate_bounds as sb

EPS_SIN = 2.0 ** -16


def _params(rng, d=7, scale=1.0):
    P = {"B": rng.normal(0, 0.25, (64, d)).astype(np.float32)}
    for name, (fo, fi) in (("W1", (256, 128)), ("W2", (256, 256)), ("W3", (256, 256))):
        P[name] = (scale * rng.uniform(-1, 1, (fo, fi)) / math.sqrt(fi)).astype(np.float32)
    for name in ("b1", "b2", "b3"):
        P[name] = rng.uniform(-0.1, 0.1, 256).astype(np.float32)
    P["w4"] = rng.uniform(-0.3, 0.3, 256).astype(np.float32)
    P["b4"] = np.array([0.02], np.float32)
    return P


def _f32_dot(x, W, rng):
    """x [n][K] @ W.T [K][N], summed term by term in float32 in a random order."""
    x = x.astype(np.float32)
    W = W.astype(np.float32)
    acc = np.zeros((x.shape[0], W.shape[0]), np.float32)
    for k in rng.permutation(x.shape[1]):
        acc = (acc + x[:, k:k + 1] * W[None, :, k]).astype(np.float32)
    return acc


def simulate(P, q, rng, plant=None):
    """Float32 model of the device's forward arithmetic (one possible execution); optional planted mistake."""
    q = q.astype(np.float32)
    B = P["B"].astype(np.float32)
    z = np.zeros((q.shape[0], 64), np.float32)
    for d in range(q.shape[1]):
        z = (z + B[None, :, d] * q[:, d:d + 1]).astype(np.float32)
    noise = rng.uniform(-0.9, 0.9, (q.shape[0], 128)) * EPS_SIN
    s, c = np.sin(z.astype(np.float64)), np.cos(z.astype(np.float64))
    feats = np.concatenate([c, s] if plant == "sincos_swap" else [s, c], 1)
    phi = sb.bf16((feats + noise).astype(np.float32))
    W1, W2, W3 = sb.bf16(P["W1"]), sb.bf16(P["W2"]), sb.bf16(P["W3"])
    b2, b3 = P["b2"], P["b3"]
    if plant == "transposed":
        W2 = W2.T.copy()
    if plant == "drop_chunk":
        W2 = W2.copy()
        W2[:, 64:128] = 0.0
    if plant == "swap_bias":
        b2, b3 = b3, b2
    h1 = sb.bf16(np.maximum((_f32_dot(phi, W1, rng) + P["b1"]).astype(np.float32), 0))
    h2 = sb.bf16(np.maximum((_f32_dot(h1, W2, rng) + b2).astype(np.float32), 0))
    h3 = np.maximum((_f32_dot(h2, W3, rng) + b3).astype(np.float32), 0)
    z_out = (_f32_dot(h3, P["w4"][None, :], rng)[:, 0] + P["b4"][0]).astype(np.float32)
    return z_out.astype(np.float64), (phi, h1, h2, h3)


def _queries(rng, n=1500, d=7):
    return rng.uniform(-math.pi, math.pi, (n, d)).astype(np.float32)


def test_bf16_rounding_and_spacing():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 3.0], np.float64)
    # BF16 keeps 8 significant bits: the step at 1 is 2^-7 and 1 + 2^-8, the midpoint, rounds to even (1)
    np.testing.assert_array_equal(sb.bf16(x), [1.0, 1.0, 1.0, 3.0])
    np.testing.assert_array_equal(sb.ulp_bf16([1.0, 1.5, 2.0, 0.75]), [2 ** -7, 2 ** -7, 2 ** -6, 2 ** -8])


@pytest.mark.parametrize("seed,scale", [(0, 1.0), (1, 2.0), (2, 4.0)])
def test_logit_bound_holds_for_simulated_device(seed, scale):
    rng = np.random.default_rng(seed)
    P = _params(rng, scale=scale)
    q = _queries(rng)
    z, tau = sb.logit_bound(P, q, EPS_SIN)
    for rep in range(3):
        z_sim, _ = simulate(P, q, np.random.default_rng([seed, rep]))
        err = np.abs(z_sim - z)
        assert np.all(err <= tau), float(np.max(err / tau))
    # the bound decides most queries at cut 0
    assert np.mean(sb.decisions(z, tau, 0.0) >= 0) > 0.6


@pytest.mark.parametrize("plant", ["transposed", "drop_chunk", "swap_bias", "sincos_swap"])
def test_logit_bound_catches_planted_mistakes(plant):
    rng = np.random.default_rng(7)
    P = _params(rng, scale=2.0)
    q = _queries(rng)
    z, tau = sb.logit_bound(P, q, EPS_SIN)
    z_sim, _ = simulate(P, q, np.random.default_rng(8), plant=plant)
    bad = np.abs(z_sim - z) > tau
    assert np.mean(bad) > 0.05, (plant, np.mean(bad))
    dec = sb.decisions(z, tau, 0.0)
    assert np.any((dec >= 0) & (dec != (z_sim > 0))), plant


def _sim_gradients(P, q, y, rng, plant=None):
    """Float32 model of one training batch's gradients (mean binary cross-entropy)."""
    n = len(y)
    z, (phi, h1, h2, h3f) = simulate(P, q, rng)
    p = 1.0 / (1.0 + np.exp(-z))
    g = ((p - y) / n).astype(np.float32)
    if plant == "sign":
        g = -g
    w4 = P["w4"].astype(np.float32)
    W2, W3 = sb.bf16(P["W2"]), sb.bf16(P["W3"])
    h3 = sb.bf16(h3f)
    G = {"w4": _f32_dot(h3.T, g[None, :], rng)[:, 0], "b4": np.array([np.float32(g.sum())])}
    dA3 = sb.bf16(g[:, None] * w4[None, :] * (h3f > 0))
    G["W3"] = _f32_dot(dA3.T, h2.T, rng)
    G["b3"] = dA3.sum(0)
    gate2 = np.ones_like(h2) if plant == "no_gate" else (h2 > 0)
    dA2 = sb.bf16(_f32_dot(dA3, W3.T, rng) * gate2)
    G["W2"] = _f32_dot(dA2.T, h1.T, rng)
    G["b2"] = dA2.sum(0)
    dA1 = sb.bf16(_f32_dot(dA2, W2.T, rng) * (h1 > 0))
    G["W1"] = _f32_dot(dA1.T, phi.T, rng)
    G["b1"] = dA1.sum(0)
    return G


@pytest.mark.parametrize("plant", [None, "sign", "no_gate"])
def test_gradient_tolerance(plant):
    rng = np.random.default_rng(11)
    P = _params(rng)
    q = _queries(rng, n=256)
    y = (rng.uniform(size=256) < 0.3).astype(np.float64)
    loss, dloss, R, tol = sb.gradients(P, q, y, EPS_SIN)
    G = _sim_gradients(P, q, y, np.random.default_rng(12), plant=plant)
    ratio = {k: float(np.max(np.abs(G[k] - R[k]) / (tol[k] + 1e-30))) for k in R}
    if plant is None:
        assert all(v <= 1.0 for v in ratio.values()), ratio
    else:
        assert max(ratio.values()) > 1.0, (plant, ratio)
