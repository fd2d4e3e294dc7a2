"""FP64 reference of the collision surrogate with rigorous per-element error bounds.

The surrogate (Fourier features -> three 256-unit ReLU layers -> logit) runs on
the device with BF16 weights and activations and FP32 accumulation.  The
reference here evaluates the same network in FP64 at the device's rounding
points and, for every output, bounds how far the device's value can lie from
it.  The bound is propagated layer by layer as an absolute error per unit:

* features: the device forms z = B q with a float32 FMA chain (at most
  2 d u sum |B q| from the exact value, u = 2^-24) and takes sin/cos with an
  error of at most `eps_sin`; the float32 result is rounded to BF16.
* a rounding to BF16 of a value known to lie within +-d of the reference's
  unrounded x lands in [bf16(x - d), bf16(x + d)] (rounding is monotone), so
  the rounded values differ by at most bf16(x + d) - bf16(x - d): zero unless
  a rounding boundary lies within d of x.
* a layer's FP32 accumulation of K exact BF16 x BF16 products in any order
  errs by at most gamma = 2 K u times the sum of the absolute products (twice
  the textbook K u, as the tensor core's summation order and internal
  rounding are not specified), the bias add by u times the result; errors of
  the inputs enter through |W|; ReLU is 1-Lipschitz and monotone.

A decision "logit > cut" is therefore fixed wherever |z_ref - cut| exceeds
the output's bound; only there is the device's decision compared.  The
backward pass of the mean binary cross-entropy is bounded the same way, with
the ReLU gate of a unit counted as either open or closed wherever its
interval straddles zero.
"""
import numpy as np

U32 = 2.0 ** -24


def bf16(x):
    """float64 -> float32 -> BF16 (round to nearest even), as float64."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32))
    return t.to(torch.bfloat16).double().numpy()


def round_interval(x, d):
    """Largest difference between BF16 roundings of two values within +-d of x."""
    return bf16(x + d) - bf16(x - d)


def relu_round_interval(x, d):
    return bf16(np.maximum(x + d, 0.0)) - bf16(np.maximum(x - d, 0.0))


def gamma(k):
    return 2.0 * k * U32


def _f64(P):
    return {k: np.asarray(v, np.float64) for k, v in P.items()}


def forward(P, q, eps_sin):
    """Reference and bounds of the forward pass at float32 configurations q [n][d].

    Returns a dict with the reference values (phi, h1, h2 rounded to BF16; h3
    and the logit z unrounded) and their bounds (dphi, dh1, dh2, dh3, dz)."""
    P = _f64(P)
    q = np.asarray(q, np.float32).astype(np.float64)
    B = P["B"]
    W1, W2, W3 = bf16(P["W1"]), bf16(P["W2"]), bf16(P["W3"])
    d = q.shape[1]
    z = q @ B.T
    ez = 2.0 * d * U32 * (np.abs(q) @ np.abs(B).T) + 2.0 * U32 * (np.abs(q) @ np.abs(B).T)
    pre = np.concatenate([np.sin(z), np.cos(z)], 1)
    e_pre = np.concatenate([ez, ez], 1) + eps_sin
    phi = bf16(pre)
    dphi = round_interval(pre, e_pre)

    def layer(x, dx, W, b, K, rounded):
        a = x @ W.T + b
        da = dx @ np.abs(W).T + gamma(K) * ((np.abs(x) + dx) @ np.abs(W).T) + 2.0 * U32 * np.abs(a) + 1e-30
        if rounded:
            return a, bf16(np.maximum(a, 0.0)), relu_round_interval(a, da), da
        return a, np.maximum(a, 0.0), da, da

    a1, h1, dh1, da1 = layer(phi, dphi, W1, P["b1"], 128, True)
    a2, h2, dh2, da2 = layer(h1, dh1, W2, P["b2"], 256, True)
    a3, h3, dh3, da3 = layer(h2, dh2, W3, P["b3"], 256, False)
    w4 = P["w4"]
    zl = h3 @ w4 + float(P["b4"][0])
    dz = dh3 @ np.abs(w4) + gamma(256) * ((h3 + dh3) @ np.abs(w4)) + 2.0 * U32 * np.abs(zl) + 1e-30
    return dict(z_feat=z, phi=phi, dphi=dphi, a1=a1, h1=h1, dh1=dh1, da1=da1, a2=a2, h2=h2, dh2=dh2, da2=da2,
                a3=a3, h3=h3, dh3=dh3, da3=da3, z=zl, dz=dz, W1=W1, W2=W2, W3=W3)


def decisions(z_ref, band, cut):
    """+1 where the device must call the logit above cut, 0 where it must not, -1 where it may go either way."""
    out = np.full(z_ref.shape, -1, np.int8)
    out[z_ref - band > cut] = 1
    out[z_ref + band <= cut] = 0
    return out


def _gate(h, dh):
    """ReLU gate of units with value h (+- dh): 1 open, 0 closed, and whether it is uncertain."""
    lo_open = (h - dh) > 0
    hi_open = (h + dh) > 0
    return lo_open.astype(np.float64), (lo_open != hi_open)


def backward(P, q, y, eps_sin):
    """Reference loss and gradients (mean binary cross-entropy) with per-element bounds.

    Returns (loss, dloss, grads, bounds) with grads/bounds keyed W1 b1 W2 b2 W3 b3 w4 b4."""
    f = forward(P, q, eps_sin)
    P64 = _f64(P)
    w4 = P64["w4"]
    n = len(y)
    y = np.asarray(y, np.float64)
    z, dz_err = f["z"], f["dz"]
    p = 1.0 / (1.0 + np.exp(-z))
    loss = np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z))))
    dloss = np.mean(dz_err) + 1e-6 * abs(loss)             # d loss / d z is within [-1, 1] per sample
    g = (p - y) / n
    dg = dz_err / 4.0 / n + 4.0 * U32 * np.abs(g) + 1e-30  # the sigmoid is 1/4-Lipschitz
    h3f, dh3f = f["h3"], f["dh3"]
    h3 = bf16(h3f)                                           # the transposed copy the w4 gradient reads
    dh3b = relu_round_interval(f["a3"], f["da3"])
    G, E = {}, {}
    G["w4"] = h3.T @ g
    E["w4"] = (np.abs(h3) + dh3b).T @ dg + dh3b.T @ np.abs(g) + gamma(n) * (np.abs(h3).T @ np.abs(g))
    G["b4"] = np.array([g.sum()])
    E["b4"] = np.array([dg.sum() + gamma(n) * np.abs(g).sum()])

    def back(dA_pre_ref, d_pre, gate_h, gate_dh):
        """dA = bf16(dA_pre * gate) with the gate possibly uncertain."""
        open_, unsure = _gate(gate_h, gate_dh)
        ref = bf16(dA_pre_ref * open_)
        # where the gate is unsure the device may have the value or zero
        span = np.where(unsure, np.abs(dA_pre_ref) + d_pre, d_pre * open_)
        err = np.where(unsure, np.abs(dA_pre_ref) + d_pre + np.abs(ref) * 2.0 ** -7,
                       round_interval(dA_pre_ref * open_, span))
        return ref, err

    pre3 = g[:, None] * w4[None, :]
    dpre3 = dg[:, None] * np.abs(w4)[None, :] + U32 * np.abs(pre3)
    dA3, e3 = back(pre3, dpre3, h3f, dh3f)
    W1, W2, W3 = f["W1"], f["W2"], f["W3"]
    h1, dh1, h2, dh2, phi, dphi = f["h1"], f["dh1"], f["h2"], f["dh2"], f["phi"], f["dphi"]

    def wgrad(dA, e, x, dx):
        val = dA.T @ x
        err = e.T @ (np.abs(x) + dx) + np.abs(dA).T @ dx + gamma(n) * (np.abs(dA).T @ np.abs(x))
        return val, err

    def bgrad(dA, e):
        return dA.sum(0), e.sum(0) + gamma(n) * np.abs(dA).sum(0)

    G["W3"], E["W3"] = wgrad(dA3, e3, h2, dh2)
    G["b3"], E["b3"] = bgrad(dA3, e3)
    pre2 = dA3 @ W3
    dpre2 = e3 @ np.abs(W3) + gamma(256) * ((np.abs(dA3) + e3) @ np.abs(W3))
    dA2, e2 = back(pre2, dpre2, h2, dh2)
    G["W2"], E["W2"] = wgrad(dA2, e2, h1, dh1)
    G["b2"], E["b2"] = bgrad(dA2, e2)
    pre1 = dA2 @ W2
    dpre1 = e2 @ np.abs(W2) + gamma(256) * ((np.abs(dA2) + e2) @ np.abs(W2))
    dA1, e1 = back(pre1, dpre1, h1, dh1)
    G["W1"], E["W1"] = wgrad(dA1, e1, phi, dphi)
    G["b1"], E["b1"] = bgrad(dA1, e1)
    return loss, dloss, G, E
