"""FP64 oracle of the learned closure's MLP -- TEST INFRASTRUCTURE ONLY.

The closure (the paper's "material closure" idea of Sec. 1 and Sec. 3.4, made a learned per-cell
model) maps the level-1 state of a cell to the missing level-4 velocity moments:

    features x = (h, u_m, v_m, alpha_1, beta_1, lambda) * in_scale          (6)
    z1 = x W1 + b1,  a1 = gelu(z1)                                          (64)
    z2 = a1 W2 + b2, a2 = gelu(z2)                                          (64)
    y  = (a2 W3 + b3) * out_scale = (alpha_2, alpha_3, alpha_4, beta_2, beta_3, beta_4)

gelu is the tanh form  gelu(z) = z/2 (1 + tanh(c (z + 0.044715 z^3))),  c = sqrt(2/pi).
Loss: mean squared error over the batch and the 6 outputs (in the scaled output space).
Backward pass written out by the chain rule.  bf16_inputs mirrors the inference kernel, which
rounds each layer's input to BF16 (round to nearest even) and accumulates in higher precision.
"""
from __future__ import annotations

import numpy as np

C_GELU = np.sqrt(2.0 / np.pi)
A_GELU = 0.044715
SIZES = (6, 64, 64, 6)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(C_GELU * (z + A_GELU * z**3)))


def gelu_grad(z):
    u = C_GELU * (z + A_GELU * z**3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * C_GELU * (1.0 + 3.0 * A_GELU * z * z)


def round_bf16(a):
    """Round float values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    p = {}
    for i, (a, b) in enumerate(zip(SIZES[:-1], SIZES[1:]), start=1):
        p[f"W{i}"] = rng.normal(0.0, np.sqrt(2.0 / (a + b)), size=(a, b))
        p[f"b{i}"] = np.zeros(b)
    return p


def forward(p, X, bf16_inputs=False):
    """X [n, 6] already scaled.  Returns (Y [n, 6] scaled outputs, cache for backward)."""
    r = round_bf16 if bf16_inputs else (lambda a: a)
    x0 = r(X)
    z1 = x0 @ p["W1"] + p["b1"]
    a1 = gelu(z1)
    x1 = r(a1)
    z2 = x1 @ p["W2"] + p["b2"]
    a2 = gelu(z2)
    x2 = r(a2)
    y = x2 @ p["W3"] + p["b3"]
    return y, (x0, z1, x1, z2, x2)


def loss_and_grads(p, X, T):
    """MSE = mean over batch and outputs of (y - t)^2, and its gradients (FP64, no rounding)."""
    n = X.shape[0]
    y, (x0, z1, a1, z2, a2) = forward(p, X)
    d = y - T
    loss = np.mean(d * d)
    dy = 2.0 * d / (n * y.shape[1])
    g = {"W3": a2.T @ dy, "b3": dy.sum(axis=0)}
    da2 = dy @ p["W3"].T
    dz2 = da2 * gelu_grad(z2)
    g["W2"] = a1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    da1 = dz2 @ p["W2"].T
    dz1 = da1 * gelu_grad(z1)
    g["W1"] = x0.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adam_update(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) on every parameter, in place; t is the 1-based step count."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k]
        mh = m[k] / (1 - beta1**t)
        vh = v[k] / (1 - beta2**t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def pack(p):
    """Flat parameter vector in the library's order: W1 [6x64] row-major, b1, W2 [64x64], b2, W3 [64x6], b3."""
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]])


def unpack(vec):
    p, o = {}, 0
    for i, (a, b) in enumerate(zip(SIZES[:-1], SIZES[1:]), start=1):
        p[f"W{i}"] = np.asarray(vec[o:o + a * b], dtype=np.float64).reshape(a, b)
        o += a * b
        p[f"b{i}"] = np.asarray(vec[o:o + b], dtype=np.float64)
        o += b
    return p


NPARAMS = sum(a * b + b for a, b in zip(SIZES[:-1], SIZES[1:]))
