"""Seeded model parameters for the network tests (inputs only: no arithmetic of the method).

random_params: PyTorch-style uniform initialisation of the §6.1 network.

exact_bf16_params / exact_fp8_params: networks whose arithmetic is exact in FP32 under the
library's BF16 / FP8 schemes, so that any summation order gives the same value at every layer
and the tensor-core path must reproduce the float64 oracle bit for bit.

BF16-exact: every layer input is a multiple of 2^-8 below 2^16 / 2 (a BF16 rounding of such a
multiple is again one), every weight is 0 or +-1 (the input layer's 2^-8), every bias a multiple
of 2^-8, and each output column has two non-zero weights, so each partial sum is a multiple of
2^-8 of magnitude below 2^16, which FP32 holds exactly. With x >= 0 after every ReLU,
FC1 = ReLU(x_a - x_b + b) <= max x + 4 and FC2 = ReLU(u_c - u_e + b + x_n) <= 2 max x + 8,
so six blocks starting from inputs below 260 stay below 17,200.

FP8-exact: hidden and output weights are 0 or +-7/8 (max |W| = 7/8 makes the weight scale
448 / (7/8) = 512 and every dequantisation factor a power of two), two non-zeros per column;
activation scales are powers of two; biases are multiples of 2^-8 in [-1, 1]. Products of E4M3
activations (multiples of 2^-9, at most 448) with the codes +-448 and the power-of-two rescalings
keep every intermediate value within 24 significant bits.
"""
import numpy as np

S = 7


def random_params(rng, N=512, blocks=6, C=25):
    """PyTorch-style uniform init; W0 scaled by 2^-16 so raw 16-bit features give O(1) activations."""
    def u(shape, fan_in):
        b = 1.0 / np.sqrt(fan_in)
        return rng.uniform(-b, b, shape).astype(np.float32)
    return {
        "W0": (u((S, N), S) / 65536.0).astype(np.float32), "b0": u(N, S),
        "W1": [u((N, N), N) for _ in range(blocks)], "b1": [u(N, N) for _ in range(blocks)],
        "W2": [u((N, N), N) for _ in range(blocks)], "b2": [u(N, N) for _ in range(blocks)],
        "Wc": u((N, C), N), "bc": u(C, N),
    }


def _pair_columns(rng, rows, cols, value):
    """(rows, cols) float32 with +value at one row and -value at another row of every column."""
    W = np.zeros((rows, cols), dtype=np.float32)
    for c in range(cols):
        a, b = rng.choice(rows, size=2, replace=False)
        W[a, c] = value
        W[b, c] = -value
    return W


def _grid(rng, shape, step, lo, hi):
    return (rng.integers(int(lo / step), int(hi / step) + 1, shape) * step).astype(np.float32)


def exact_bf16_params(rng, N=512, blocks=6, C=25):
    if blocks > 6:
        raise ValueError("the exactness bound holds for up to six blocks")
    W0 = np.zeros((S, N), dtype=np.float32)
    W0[rng.integers(0, S, N), np.arange(N)] = 2.0 ** -8
    return {
        "W0": W0, "b0": _grid(rng, N, 2.0 ** -8, -4, 4),
        "W1": [_pair_columns(rng, N, N, 1.0) for _ in range(blocks)],
        "b1": [_grid(rng, N, 2.0 ** -8, -4, 4) for _ in range(blocks)],
        "W2": [_pair_columns(rng, N, N, 1.0) for _ in range(blocks)],
        "b2": [_grid(rng, N, 2.0 ** -8, -4, 4) for _ in range(blocks)],
        "Wc": _pair_columns(rng, N, C, 1.0), "bc": _grid(rng, C, 2.0 ** -8, -4, 4),
    }


def exact_fp8_params(rng, N=512, blocks=6, C=25):
    """(params, amax): amax gives every tensor-core layer input a scale of 1/2, 1 or 2."""
    W0 = np.zeros((S, N), dtype=np.float32)
    W0[rng.integers(0, S, N), np.arange(N)] = 2.0 ** -12
    p = {
        "W0": W0, "b0": _grid(rng, N, 2.0 ** -8, -1, 1),
        "W1": [_pair_columns(rng, N, N, 0.875) for _ in range(blocks)],
        "b1": [_grid(rng, N, 2.0 ** -8, -1, 1) for _ in range(blocks)],
        "W2": [_pair_columns(rng, N, N, 0.875) for _ in range(blocks)],
        "b2": [_grid(rng, N, 2.0 ** -8, -1, 1) for _ in range(blocks)],
        "Wc": _pair_columns(rng, N, C, 0.875), "bc": _grid(rng, C, 2.0 ** -8, -1, 1),
    }
    amax = rng.choice(np.array([896.0, 448.0, 224.0], dtype=np.float32), 2 * blocks + 1)
    return p, amax


def to_f64(p):
    return {k: ([a.astype(np.float64) for a in v] if isinstance(v, list) else v.astype(np.float64)) for k, v in p.items()}
