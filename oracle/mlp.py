"""ORACLE (test infrastructure): TaNG's residual MLP in float64, its gradients, and its training math.

Sources in the paper:
  §6.2  feature encoding: the header is cut into 16-bit segments, each taken as a float. A 5-field
        header gives 7 segments: SIP high/low, DIP high/low, SP, DP, PRO.
  §6.1  network: an input FC layer (S -> N), k residual blocks of two N x N FC layers, an output
        FC layer (N -> C), ReLU activations throughout, argmax over the outputs.
  Eq. 1 residual block. The printed equation has unbalanced parentheses; the reading used here is
        B(x) = ReLU( ReLU(x W1 + b1) W2 + b2 + x ), i.e. the skip connection is added before the
        block's last activation.
  Eq. 2 A(z) = max(0, z).
  §6.2  training: cross-entropy loss and the Adam optimiser (PyTorch defaults: beta1 0.9,
        beta2 0.999, eps 1e-8).

Weights follow the x . W convention of Eq. 1: W has shape (inputs, outputs).
The argmax takes the lowest index among equal maxima. The ReLU derivative at 0 is 0.
"""
from __future__ import annotations

import numpy as np

S_FEATURES = 7


def features(headers: np.ndarray) -> np.ndarray:
    """§6.2 encoding: (n, 7) float64 of the 16-bit segments (exact in float32 and float64)."""
    sip = headers["sip"].astype(np.int64)
    dip = headers["dip"].astype(np.int64)
    return np.stack(
        [sip >> 16, sip & 0xFFFF, dip >> 16, dip & 0xFFFF,
         headers["sp"].astype(np.int64), headers["dp"].astype(np.int64), headers["proto"].astype(np.int64)],
        axis=1,
    ).astype(np.float64)


def relu(z):
    return np.maximum(z, 0.0)


def forward(p: dict, X: np.ndarray, keep: bool = False):
    """Logits (n, C) in float64. With keep=True also the per-layer pre-activations for backward."""
    X = np.asarray(X, dtype=np.float64)
    pre0 = X @ p["W0"] + p["b0"]
    h = relu(pre0)
    cache = {"X": X, "pre0": pre0, "h_in": [], "pre1": [], "u": [], "pre2": []}
    for k in range(len(p["W1"])):
        pre1 = h @ p["W1"][k] + p["b1"][k]
        u = relu(pre1)
        pre2 = u @ p["W2"][k] + p["b2"][k] + h
        if keep:
            cache["h_in"].append(h)
            cache["pre1"].append(pre1)
            cache["u"].append(u)
            cache["pre2"].append(pre2)
        h = relu(pre2)
    z = h @ p["Wc"] + p["bc"]
    if keep:
        cache["h_out"] = h
        return z, cache
    return z


def predict(p: dict, X: np.ndarray) -> np.ndarray:
    """Tuple index = argmax of the logits, lowest index on ties."""
    return np.argmax(forward(p, X), axis=1)


def cross_entropy(z: np.ndarray, y: np.ndarray) -> float:
    """Mean over the batch of -log softmax(z)[y]."""
    zmax = z.max(axis=1, keepdims=True)
    lse = np.log(np.exp(z - zmax).sum(axis=1)) + zmax[:, 0]
    return float(np.mean(lse - z[np.arange(len(y)), y]))


def backward(p: dict, X: np.ndarray, y: np.ndarray):
    """(loss, grads) of the mean cross-entropy; grads has the same keys/shapes as p."""
    z, c = forward(p, X, keep=True)
    B = len(y)
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    sm = e / e.sum(axis=1, keepdims=True)
    loss = cross_entropy(z, y)
    dz = sm.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    g = {"W1": [None] * len(p["W1"]), "b1": [None] * len(p["W1"]),
         "W2": [None] * len(p["W1"]), "b2": [None] * len(p["W1"])}
    g["Wc"] = c["h_out"].T @ dz
    g["bc"] = dz.sum(axis=0)
    dh = dz @ p["Wc"].T
    for k in reversed(range(len(p["W1"]))):
        g2 = dh * (c["pre2"][k] > 0)
        g["W2"][k] = c["u"][k].T @ g2
        g["b2"][k] = g2.sum(axis=0)
        du = g2 @ p["W2"][k].T
        g1 = du * (c["pre1"][k] > 0)
        g["W1"][k] = c["h_in"][k].T @ g1
        g["b1"][k] = g1.sum(axis=0)
        dh = g1 @ p["W1"][k].T + g2
    g0 = dh * (c["pre0"] > 0)
    g["W0"] = c["X"].T @ g0
    g["b0"] = g0.sum(axis=0)
    return loss, g


def adam_step(param, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, bias-corrected); returns (param, m, v) as new arrays."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v


def flat_keys(p: dict):
    """(name, index) pairs in the canonical parameter order: W0 b0 {W1 b1 W2 b2}*k Wc bc."""
    out = [("W0", None), ("b0", None)]
    for k in range(len(p["W1"])):
        out += [("W1", k), ("b1", k), ("W2", k), ("b2", k)]
    out += [("Wc", None), ("bc", None)]
    return out


def get(p: dict, key):
    name, k = key
    return p[name] if k is None else p[name][k]
