"""CPU ORACLE — TEST INFRASTRUCTURE ONLY: FP64 forward/backward of the mode-selector MLP.

The selector maps 8 per-superstep frontier features to scores for the three
exchange modes (push-sparse, push-dense, pull):

    xn = (x - mu) / sd
    h1 = relu(W1 @ xn + b1)        W1: 32x8
    h2 = relu(W2 @ h1 + b2)        W2: 32x32
    z  = W3 @ h2 + b3              W3: 3x32
    mode = argmax(z)

Training loss: sample-weighted softmax cross-entropy,
    L = sum_i s_i * (logsumexp(z_i) - z_i[y_i]) / sum_i s_i.

Everything here is plain numpy in float64. The weights passed in are whatever
the caller supplies (the GPU library rounds its weights to bfloat16; the tests
hand those rounded values to this oracle).
"""
from __future__ import annotations

import numpy as np

SHAPES = {"W1": (32, 8), "b1": (32,), "W2": (32, 32), "b2": (32,), "W3": (3, 32), "b3": (3,)}
ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def forward(params: dict, X: np.ndarray, mu: np.ndarray, sd: np.ndarray):
    """Logits for a batch X[N, 8]; also returns the activations backward needs."""
    X = np.asarray(X, np.float64)
    xn = (X - mu) / sd
    a1 = xn @ params["W1"].T + params["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ params["W2"].T + params["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ params["W3"].T + params["b3"]
    return z, dict(xn=xn, a1=a1, h1=h1, a2=a2, h2=h2)


def loss(z: np.ndarray, y: np.ndarray, s: np.ndarray) -> float:
    zmax = z.max(axis=1, keepdims=True)
    lse = (zmax + np.log(np.exp(z - zmax).sum(axis=1, keepdims=True)))[:, 0]
    ce = lse - z[np.arange(z.shape[0]), y]
    return float((s * ce).sum() / s.sum())


def backward(params: dict, X, y, s, mu, sd):
    """Loss and its gradients with respect to every parameter (FP64)."""
    y = np.asarray(y, np.int64)
    s = np.asarray(s, np.float64)
    z, c = forward(params, X, mu, sd)
    L = loss(z, y, s)
    zmax = z.max(axis=1, keepdims=True)
    p = np.exp(z - zmax)
    p /= p.sum(axis=1, keepdims=True)
    dz = p.copy()
    dz[np.arange(z.shape[0]), y] -= 1.0
    dz *= (s / s.sum())[:, None]
    g = {}
    g["W3"] = dz.T @ c["h2"]
    g["b3"] = dz.sum(axis=0)
    dh2 = dz @ params["W3"]
    da2 = dh2 * (c["a2"] > 0)
    g["W2"] = da2.T @ c["h1"]
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ params["W2"]
    da1 = dh1 * (c["a1"] > 0)
    g["W1"] = da1.T @ c["xn"]
    g["b1"] = da1.sum(axis=0)
    return L, g


def predict(params, X, mu, sd) -> np.ndarray:
    return forward(params, X, mu, sd)[0].argmax(axis=1)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of an IEEE binary32 value; rounding to
    nearest-even adds 0x7FFF plus the lowest kept bit before truncating.
    (NaN inputs are not expected here.)"""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)
