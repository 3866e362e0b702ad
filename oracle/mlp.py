"""FP64 reference of the moments-to-DOS network -- test infrastructure only.

Not in the paper: the learned part maps noisy low-order KPM moments
(mu_1..mu_{n_in} from few start vectors) to the DOS on a grid.  Network:
    h1 = relu(x W1^T + b1),  h2 = relu(h1 W2^T + b2),  y = h2 W3^T + b3,
loss = mean |y - target| (L1), trained with Adam.

``bf16_round`` emulates round-to-nearest-even to bfloat16 so the reference can
see the same rounded operands (weights, inputs, activations, output gradient)
that the GPU feeds its tensor cores; everything else is FP64.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def init_params(n_in: int, n_hidden: int, n_out: int, seed: int):
    """He-uniform weights, zero biases (any deterministic init works for the tests)."""
    rng = np.random.default_rng(seed)
    def lin(fan_out, fan_in):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=(fan_out, fan_in)), np.zeros(fan_out)
    W1, b1 = lin(n_hidden, n_in)
    W2, b2 = lin(n_hidden, n_hidden)
    W3, b3 = lin(n_out, n_hidden)
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "W3": W3, "b3": b3}


def forward(p, x, bf16: bool = False):
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, W3 = r(p["W1"]), r(p["W2"]), r(p["W3"])
    x = r(x)
    z1 = x @ W1.T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    h1r = r(h1)
    z2 = h1r @ W2.T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    h2r = r(h2)
    y = h2r @ W3.T + p["b3"]
    return y, {"x": x, "h1": h1r, "h2": h2r, "W1": W1, "W2": W2, "W3": W3}


def loss_and_grads(p, x, target, bf16: bool = False):
    """L1 loss and its gradient with respect to every parameter."""
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, c = forward(p, x, bf16)
    B, n_out = y.shape
    diff = y - target
    loss = float(np.abs(diff).sum() / (B * n_out))
    dy = np.sign(diff) / (B * n_out)
    dyr = r(dy)
    g = {"W3": dyr.T @ c["h2"], "b3": dy.sum(axis=0)}
    dh2 = (dyr @ c["W3"]) * (c["h2"] > 0)
    dh2r = r(dh2)
    g["W2"] = dh2r.T @ c["h1"]
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2r @ c["W2"]) * (c["h1"] > 0)
    dh1r = r(dh1)
    g["W1"] = dh1r.T @ c["x"]
    g["b1"] = dh1.sum(axis=0)
    return loss, g


def adam_step(p, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) with bias correction; t counts from 1."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] ** 2
        mh = m[k] / (1 - beta1 ** t)
        vh = v[k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def flatten(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in PARAM_ORDER])


def unflatten(vec, n_in, n_hidden, n_out):
    shapes = {"W1": (n_hidden, n_in), "b1": (n_hidden,), "W2": (n_hidden, n_hidden),
              "b2": (n_hidden,), "W3": (n_out, n_hidden), "b3": (n_out,)}
    out, o = {}, 0
    for k in PARAM_ORDER:
        size = int(np.prod(shapes[k]))
        out[k] = np.asarray(vec[o:o + size], dtype=np.float64).reshape(shapes[k])
        o += size
    return out
