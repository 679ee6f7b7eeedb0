"""Helpers shared by the GPU tests: device buffers and the exact-tolerance network bound."""
import numpy as np
import torch

import workloads as wl


def to_dev(h: np.ndarray) -> torch.Tensor:
    """Headers (HEADER_DTYPE) -> contiguous CUDA uint8 tensor of shape (n, 16)."""
    a = np.ascontiguousarray(h, dtype=wl.HEADER_DTYPE).view(np.uint8).reshape(len(h), 16)
    return torch.from_numpy(a.copy()).cuda()


def ids_dev(n: int) -> torch.Tensor:
    return torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")[:n]


def ids_host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def abs_forward(p: dict, X: np.ndarray) -> np.ndarray:
    """|x| propagated through |W| and |b| of every layer (ReLU is 1-Lipschitz): the magnitude
    that scales every rounding error of the network, per output logit."""
    a = np.abs(X) @ np.abs(p["W0"]) + np.abs(p["b0"])
    for k in range(len(p["W1"])):
        u = a @ np.abs(p["W1"][k]) + np.abs(p["b1"][k])
        a = u @ np.abs(p["W2"][k]) + np.abs(p["b2"][k]) + a
    return a @ np.abs(p["Wc"]) + np.abs(p["bc"])


def logit_tolerance(p: dict, X: np.ndarray, unit_roundoff: float, act_unit: float = 0.0) -> np.ndarray:
    """Per-logit bound on |z - z64| for a forward that accumulates K-term dot products with unit
    roundoff `unit_roundoff` and rounds each layer input with relative error `act_unit`:
    every one of the L layers adds at most (gamma_{K+1} + act_unit) * |W|.|x| at its output,
    and later layers pass it on through |W|; summed, that is L * (gamma + act_unit) * abs_forward."""
    K = max(p["W0"].shape[1], p["W0"].shape[0])
    L = 2 + 2 * len(p["W1"])
    gamma = (K + 1) * unit_roundoff / (1 - (K + 1) * unit_roundoff)
    return L * (gamma + act_unit) * abs_forward(p, X)


def random_params(rng, N=512, blocks=6, C=25, S=7):
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
