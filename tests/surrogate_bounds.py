"""FP64 reference of the collision surrogate with per-element error bounds.

The surrogate (Fourier features -> three 256-unit ReLU layers -> logit) runs on
the device with BF16 weights and activations and FP32 accumulation.  The
reference here evaluates the same network in FP64 with BF16 rounding at the
device's rounding points (features, h1, h2; the head reads h3 unrounded) and
bounds, element by element, how far the device's result can lie from it.

Logits (`logit_bound`), to first order in the perturbations: the device and
the reference round the same unit to BF16 values at most one BF16 ulp apart
(both rounding errors are below half an ulp of the same binade, or of the
next one up); the features carry besides the device's sin/cos error
(`eps_sin`) and the FP32 FMA chain's error in z = B q (2 (d+1) u sum |B q|,
u = 2^-24); every FP32 accumulation of K exact BF16 x BF16 products errs by
at most gamma = 2 K u times the sum of absolute products (twice the textbook
K u: the tensor core's order of summation is not specified), the bias add by
u.  Each deviation moves the logit by its size times |dz/dx| at that point,
with dz/dx the reference network's own gradient, so the logit bound is the
sum of these products.  A decision "logit > cut" is fixed wherever
|z_ref - cut| exceeds the bound; only there is the device's decision
compared.

Gradients (`gradients`): each element of a weight gradient is a sum over the
batch of products of two BF16 factors (an activation and a back-propagated
error), and a bias gradient a sum of one such factor.  Each factor of the
device differs from the reference's by its own rounding (one BF16 ulp, at
most 2^-7 of its size) plus the first-order effect of earlier roundings (at
most one more such unit per factor, as a BF16 layer carries one rounding of
each input), so a product differs by at most 4 x 2^-7 = 2^-5 of its size and
the sum by 2^-5 of the sum of absolute terms (FP32 accumulation adds 2 n u of
it, far below).  The tolerance is stated per element; test_surrogate_bounds
checks both bounds against a float32 simulation of the device arithmetic and
against planted mistakes.
"""
import numpy as np

U32 = 2.0 ** -24
GRAD_REL = 2.0 ** -5
GATE_REL = 2.0 ** -3


def bf16(x):
    """float64 -> float32 -> BF16 (round to nearest even), as float64."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32))
    return t.to(torch.bfloat16).double().numpy()


def ulp_bf16(x):
    """Spacing of BF16 numbers at |x| (8 significant bits); 2^-133 near zero."""
    a = np.abs(np.asarray(x, np.float64))
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -126)))
    return 2.0 ** (e - 7)


def gamma(k):
    return 2.0 * k * U32


def _f64(P):
    return {k: np.asarray(v, np.float64) for k, v in P.items()}


def reference(P, q):
    """FP64 forward pass at float32 configurations q [n][d] with the device's BF16 rounding points."""
    P = _f64(P)
    q = np.asarray(q, np.float32).astype(np.float64)
    W1, W2, W3 = bf16(P["W1"]), bf16(P["W2"]), bf16(P["W3"])
    zf = q @ P["B"].T
    pre = np.concatenate([np.sin(zf), np.cos(zf)], 1)
    phi = bf16(pre)
    a1 = phi @ W1.T + P["b1"]
    h1 = bf16(np.maximum(a1, 0.0))
    a2 = h1 @ W2.T + P["b2"]
    h2 = bf16(np.maximum(a2, 0.0))
    a3 = h2 @ W3.T + P["b3"]
    h3 = np.maximum(a3, 0.0)
    z = h3 @ P["w4"] + float(P["b4"][0])
    return dict(q=q, zf=zf, pre=pre, phi=phi, a1=a1, h1=h1, a2=a2, h2=h2, a3=a3, h3=h3, z=z,
                W1=W1, W2=W2, W3=W3, w4=P["w4"], B=P["B"])


def logit_bound(P, q, eps_sin, r=None):
    """(z_ref, tau): the reference logit and the first-order bound of the device's deviation, per query."""
    r = r or reference(P, q)
    n = r["z"].shape[0]
    g3 = np.broadcast_to(r["w4"], (n, 256)) * (r["a3"] > 0)          # dz / d a3
    gh2 = g3 @ r["W3"]                                                # dz / d h2
    g2 = gh2 * (r["a2"] > 0)
    gh1 = g2 @ r["W2"]
    g1 = gh1 * (r["a1"] > 0)
    gphi = g1 @ r["W1"]
    ez = 2.0 * (r["q"].shape[1] + 1) * U32 * (np.abs(r["q"]) @ np.abs(r["B"]).T)
    e_phi = ulp_bf16(r["pre"] * (1 + 2.0 ** -7)) + eps_sin + np.concatenate([ez, ez], 1)
    tau = np.sum(np.abs(gphi) * e_phi, 1)
    tau += np.sum(np.abs(gh1) * ulp_bf16(r["h1"] * (1 + 2.0 ** -7)), 1)
    tau += np.sum(np.abs(gh2) * ulp_bf16(r["h2"] * (1 + 2.0 ** -7)), 1)
    acc1 = gamma(128) * (np.abs(r["phi"]) @ np.abs(r["W1"]).T) + U32 * np.abs(r["a1"])
    acc2 = gamma(256) * (np.abs(r["h1"]) @ np.abs(r["W2"]).T) + U32 * np.abs(r["a2"])
    acc3 = gamma(256) * (np.abs(r["h2"]) @ np.abs(r["W3"]).T) + U32 * np.abs(r["a3"])
    tau += np.sum(np.abs(g1) * acc1, 1) + np.sum(np.abs(g2) * acc2, 1) + np.sum(np.abs(g3) * acc3, 1)
    tau += gamma(256) * (r["h3"] @ np.abs(r["w4"])) + U32 * np.abs(r["z"]) + 1e-7
    return r["z"], tau


def decisions(z_ref, band, cut):
    """1 where the device must call the logit above cut, 0 where it must not, -1 where it may go either way."""
    out = np.full(z_ref.shape, -1, np.int8)
    out[z_ref - band > cut] = 1
    out[z_ref + band <= cut] = 0
    return out


def gradients(P, q, y, eps_sin):
    """Mean binary cross-entropy of labels y at q: (loss, dloss, grads, tol) with grads the FP64 reference at
    the device's rounding points and tol the per-element tolerance.

    tol = GRAD_REL * S + T.  S sums over the batch the product of the two factors' magnitudes, each the sum
    of the absolute terms that form it (a factor that is itself a sum of cancelling terms carries the
    roundings of those terms), with the ReLU gate of a unit counted open wherever its pre-activation lies
    within GATE_REL = 2^-3 of its own magnitude of zero (a gate the device may set either way: the
    deviation of a pre-activation is a sum of roundings of its terms, and the first-order logit analysis
    finds these sums far below an eighth of the magnitude).  T carries the
    logit's own deviation (`logit_bound`) into the output error (p - y) / n, which moves by at most a
    quarter of it over n (the sigmoid is 1/4-Lipschitz), and from there through the same magnitudes."""
    r = reference(P, q)
    _, tau = logit_bound(P, q, eps_sin, r)
    P = _f64(P)
    n = len(y)
    y = np.asarray(y, np.float64)
    z = r["z"]
    p = 1.0 / (1.0 + np.exp(-z))
    loss = np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z))))
    dloss = np.mean(tau) + 4.0 * U32 * abs(loss)            # |d loss_i / d z_i| <= 1
    g = (p - y) / n
    eg = tau / 4.0 / n                                     # deviation of the output error per sample
    w4 = r["w4"]
    # magnitudes of the forward factors: |x| plus the absolute terms of their pre-activations
    m1 = np.abs(r["phi"]) @ np.abs(r["W1"]).T + np.abs(P["b1"])
    m2 = np.abs(r["h1"]) @ np.abs(r["W2"]).T + np.abs(P["b2"])
    m3 = np.abs(r["h2"]) @ np.abs(r["W3"]).T + np.abs(P["b3"])
    open1, open2, open3 = r["a1"] > 0, r["a2"] > 0, r["a3"] > 0
    maybe1 = open1 | (np.abs(r["a1"]) <= GATE_REL * m1)
    maybe2 = open2 | (np.abs(r["a2"]) <= GATE_REL * m2)
    maybe3 = open3 | (np.abs(r["a3"]) <= GATE_REL * m3)
    M_h3, M_h2, M_h1 = m3 * maybe3, m2 * maybe2, m1 * maybe1
    M_phi = np.abs(r["phi"]) + 2.0 ** -7                     # features: |sin|, |cos| <= 1
    h3 = bf16(r["h3"])
    G, tol = {}, {}
    ag = np.abs(g)
    G["w4"] = h3.T @ g
    tol["w4"] = GRAD_REL * (M_h3.T @ ag) + M_h3.T @ eg
    G["b4"] = np.array([g.sum()])
    tol["b4"] = np.array([GRAD_REL * ag.sum() + eg.sum()])
    dA3 = bf16(g[:, None] * w4[None, :] * open3)
    M3 = ag[:, None] * np.abs(w4)[None, :] * maybe3
    E3 = eg[:, None] * np.abs(w4)[None, :] * maybe3
    dA2 = bf16((dA3 @ r["W3"]) * open2)
    M2 = (M3 @ np.abs(r["W3"])) * maybe2
    E2 = (E3 @ np.abs(r["W3"])) * maybe2
    dA1 = bf16((dA2 @ r["W2"]) * open1)
    M1 = (M2 @ np.abs(r["W2"])) * maybe1
    E1 = (E2 @ np.abs(r["W2"])) * maybe1
    for k, dA, M, E, x, Mx in (("3", dA3, M3, E3, r["h2"], M_h2), ("2", dA2, M2, E2, r["h1"], M_h1),
                               ("1", dA1, M1, E1, r["phi"], M_phi)):
        G["W" + k] = dA.T @ x
        tol["W" + k] = GRAD_REL * (M.T @ Mx) + E.T @ Mx
        G["b" + k] = dA.sum(0)
        tol["b" + k] = GRAD_REL * M.sum(0) + E.sum(0)
    return loss, dloss, G, tol
