"""The picker network in plain numpy fp64 -- TEST INFRASTRUCTURE ONLY.

Forward, loss and backward of the 24 -> 64 -> 64 -> 3 ReLU network of the
learned variant picker, evaluated in float64 on the exact values of the bf16
parameters, plus one AdamW step. Only tests/ use this module.

Flat parameter order: W1[64][24] b1[64] W2[64][64] b2[64] W3[3][64] b3[3].
xn = (x - mu) / sd; h1 = relu(W1 xn + b1); h2 = relu(W2 h1 + b2);
z = W3 h2 + b3; loss = mean over the batch of logsumexp(z) - z[label].
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 24, 64, 3
SHAPES = (("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NOUT, NH)), ("b3", (NOUT,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """bf16 bit patterns (uint16 or int16) to their exact float values."""
    u = np.asarray(bits).astype(np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def unflatten(p: np.ndarray) -> dict:
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def flatten(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(p: np.ndarray, norm: np.ndarray, x: np.ndarray):
    """Returns (xn, h1, h2, z)."""
    w = unflatten(p)
    mu, sd = np.asarray(norm[:NIN], np.float64), np.asarray(norm[NIN:], np.float64)
    xn = (np.asarray(x, np.float64) - mu) / sd
    h1 = np.maximum(xn @ w["W1"].T + w["b1"], 0.0)
    h2 = np.maximum(h1 @ w["W2"].T + w["b2"], 0.0)
    z = h2 @ w["W3"].T + w["b3"]
    return xn, h1, h2, z


def loss(p, norm, x, label) -> float:
    z = forward(p, norm, x)[3]
    m = z.max(axis=1, keepdims=True)
    lse = np.log(np.exp(z - m).sum(axis=1)) + m[:, 0]
    return float((lse - z[np.arange(len(z)), label]).mean())


def backward(p, norm, x, label) -> np.ndarray:
    """Gradient of loss() with respect to the flat parameter vector."""
    w = unflatten(p)
    xn, h1, h2, z = forward(p, norm, x)
    B = len(z)
    e = np.exp(z - z.max(axis=1, keepdims=True))
    dz = e / e.sum(axis=1, keepdims=True)
    dz[np.arange(B), label] -= 1.0
    dz /= B
    g = {"W3": dz.T @ h2, "b3": dz.sum(axis=0)}
    dh2 = (dz @ w["W3"]) * (h2 > 0)
    g["W2"], g["b2"] = dh2.T @ h1, dh2.sum(axis=0)
    dh1 = (dh2 @ w["W2"]) * (h1 > 0)
    g["W1"], g["b1"] = dh1.T @ xn, dh1.sum(axis=0)
    return flatten(g)


def adamw(master, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step in float64; returns (master, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    master = master - lr * (mh / (np.sqrt(vh) + eps) + wd * master)
    return master, m, v
