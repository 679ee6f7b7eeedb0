"""ORACLE (test infrastructure): the §6.1 network evaluated under the library's BF16 and FP8
tensor-core schemes, in float64 with every rounding the scheme defines applied once, exactly.

The paper does not state its inference precision (§5.1.2 only names TensorRT). The library
defines two low-precision schemes on top of §6.1 (Eq. 1-2), documented with tang_load_model:

BF16 scheme
  - the weights of the residual blocks and of the output layer are rounded to BF16 (nearest,
    ties to even); biases and the input layer (W0, b0) stay in FP32;
  - every input of a tensor-core layer is rounded to BF16 after its ReLU: the input layer's
    output h0, each block's inner activation u, and each block's output;
  - products and sums are exact here (float64 of BF16/FP32 values), so the only roundings are the
    ones above; the library's FP32 accumulation differs from this by its summation error.

FP8 (E4M3) scheme
  - activation scale of tensor-core layer input j: s_j = 2^floor(log2(448 / amax_j)) from the
    calibration maxima amax carried by the model blob, so the calibrated range maps into (224, 448];
  - weight scale of a hidden layer: sw = 448 / max|W| in FP32, one per layer; of the output
    layer: one per column c, 448 / max|Wc[:, c]|;
  - weight codes q = E4M3(FP32(W * sw)), dequantisation factor dq = FP32(1 / FP32(s_j * sw));
  - layer inputs are kept in their scaled units: a = E4M3(ReLU(s_j * value)), saturating at 448;
  - hidden layer l (input scale s_l, output scale s_{l+1}): value * s_{l+1} =
    (a @ q) * dq * s_{l+1} + b * s_{l+1} (+ the block input a_in * s_{l+1} / s_{l-1} in the
    second layer of a block, Eq. 1's skip connection);
  - output layer: z = (a @ q) * dq_c + bc.

Weights follow oracle.mlp's x . W convention; p holds the blob's FP32 parameters.
"""
from __future__ import annotations

import numpy as np

from . import quant

E4M3_MAX = 448.0


def _f64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def relu(z):
    return np.maximum(z, 0.0)


def bf16_weights(p: dict) -> dict:
    """The BF16 scheme's parameters: W1, W2, Wc rounded to BF16, everything else FP32, as float64."""
    q = {k: ([_f64(a) for a in v] if isinstance(v, list) else _f64(v)) for k, v in p.items()}
    for k in ("W1", "W2"):
        q[k] = [quant.bf16_round(np.asarray(w, np.float32)).astype(np.float64) for w in p[k]]
    q["Wc"] = quant.bf16_round(np.asarray(p["Wc"], np.float32)).astype(np.float64)
    return q


def forward_bf16(p: dict, X: np.ndarray, keep: bool = False):
    """(logits, magnitude) under the BF16 scheme. magnitude[i, c] = sum_k |h_k| |Wc[k, c]| + |bc[c]|
    over the output layer's (rounded) input h: the scale of that layer's summation error.
    keep=True adds a list with, per layer after the first, (input, weights, partial sums): the
    layer's rounded input, its weight matrix, and the values before the ReLU and rounding as each
    addition leaves them (products summed, + bias, + skip input)."""
    q = bf16_weights(p)
    X = np.asarray(X, dtype=np.float64)
    h = quant.bf16_round64(relu(X @ q["W0"] + q["b0"]))
    steps = []
    for k in range(len(q["W1"])):
        acc = h @ q["W1"][k]
        steps.append((h, q["W1"][k], [acc, acc + q["b1"][k]]))
        u = quant.bf16_round64(relu(acc + q["b1"][k]))
        acc = u @ q["W2"][k]
        steps.append((u, q["W2"][k], [acc, acc + q["b2"][k], acc + q["b2"][k] + h]))
        h = quant.bf16_round64(relu(acc + q["b2"][k] + h))
    acc = h @ q["Wc"]
    steps.append((h, q["Wc"], [acc, acc + q["bc"]]))
    z = acc + q["bc"]
    mag = np.abs(h) @ np.abs(q["Wc"]) + np.abs(q["bc"])
    return (z, mag, steps) if keep else (z, mag)


def act_scales(amax) -> np.ndarray:
    """s_j = 2^floor(log2(448 / amax_j)) for every tensor-core layer input j."""
    a = np.asarray(amax, dtype=np.float32).astype(np.float64)
    return np.ldexp(1.0, np.floor(np.log2(E4M3_MAX / a)).astype(np.int64))


def fp8_weights(p: dict, amax) -> dict:
    """The FP8 scheme's constants: per hidden layer l (2 per block, FC1 then FC2) the E4M3 weight
    values q[l] (in scaled units), dq[l] and the activation scales s; the same for the output layer
    with one weight scale per column."""
    s = act_scales(amax)
    f32 = np.float32
    layers = []
    for k in range(len(p["W1"])):
        layers += [p["W1"][k], p["W2"][k]]
    qs, dqs = [], []
    for l, W in enumerate(layers):
        W = np.asarray(W, f32)
        amax_w = f32(np.abs(W).max())
        sw = f32(448.0) / amax_w if amax_w > 0 else f32(1.0)
        qs.append(quant.e4m3_value(quant.e4m3_bits((W * sw).astype(f32))))
        dqs.append(float(f32(1.0) / (f32(s[l]) * sw)))
    Wc = np.asarray(p["Wc"], f32)
    amax_c = np.abs(Wc).max(axis=0)
    swc = np.where(amax_c > 0, f32(448.0) / np.where(amax_c > 0, amax_c, f32(1.0)), f32(1.0)).astype(f32)
    qc = quant.e4m3_value(quant.e4m3_bits((Wc * swc[None, :]).astype(f32)))
    dqc = (f32(1.0) / (f32(s[len(layers)]) * swc)).astype(np.float64)
    return {"s": s, "q": qs, "dq": dqs, "qc": qc, "dqc": dqc}


def e4m3_act(v) -> np.ndarray:
    """ReLU, then E4M3 (nearest, ties to even, saturating at 448), as float64 values."""
    return quant.e4m3_value(quant.e4m3_bits(relu(v)))


def forward_fp8(p: dict, X: np.ndarray, amax, keep: bool = False):
    """(logits, magnitude) under the FP8 scheme; magnitude[i, c] = dq_c * sum_k |a_k| |q[k, c]| +
    |bc[c]| over the output layer's scaled input a. keep=True adds, per layer after the first,
    (scaled input, weight codes' values, partial results) as in forward_bf16: the sum of products,
    then that sum times the layer's factor plus the scaled bias, then plus the scaled skip input."""
    f = fp8_weights(p, amax)
    s = f["s"]
    X = np.asarray(X, dtype=np.float64)
    W0, b0 = _f64(p["W0"]), _f64(p["b0"])
    a = e4m3_act(s[0] * (X @ W0 + b0))   # layer 0 computed exactly, then scaled by s_0
    steps = []
    for k in range(len(p["W1"])):
        l1, l2 = 2 * k, 2 * k + 1
        b1, b2 = _f64(p["b1"][k]), _f64(p["b2"][k])
        acc = a @ f["q"][l1]
        v = acc * (f["dq"][l1] * s[l1 + 1]) + b1 * s[l1 + 1]
        steps.append((a, f["q"][l1], [acc, v]))
        u = e4m3_act(v)
        acc = u @ f["q"][l2]
        v = acc * (f["dq"][l2] * s[l2 + 1]) + b2 * s[l2 + 1]
        v2 = v + a * (s[l2 + 1] / s[l1])
        steps.append((u, f["q"][l2], [acc, v, v2]))
        a = e4m3_act(v2)
    bc = _f64(p["bc"])
    acc = a @ f["qc"]
    z = acc * f["dqc"][None, :] + bc
    steps.append((a, f["qc"], [acc, z]))
    mag = (np.abs(a) @ np.abs(f["qc"])) * f["dqc"][None, :] + np.abs(bc)
    return (z, mag, steps) if keep else (z, mag)
