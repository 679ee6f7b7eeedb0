"""Helpers shared by the GPU tests: device buffers and the element-wise logit comparison."""
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


# Unit roundoff of the library's FP32 accumulation: 2^-24 for round-to-nearest; 2^-23 also covers
# an accumulator that truncates, since the tensor core's summation order and rounding are not
# documented.
U_ACC = 2.0 ** -23


def gamma(n: int, u: float = U_ACC) -> float:
    """Higham's gamma_n = n u / (1 - n u): bound on the relative error of an n-term sum."""
    return n * u / (1.0 - n * u)


def compare_logits(z, z_or, mag, K, rho, tile=128):
    """Compare kernel logits z with the oracle's low-precision forward z_or element by element.

    tight = gamma_{K+1} * mag, with mag the oracle's sum of |input| |weight| (+ |bias|) of the
    output layer: the whole difference when every earlier rounding decision of the kernel agrees
    with the oracle's, i.e. the output layer's own K-term FP32 sum and its bias addition.
    A rounding decision taken on the other side of a BF16 / E4M3 boundary (the FP32 sum before it
    lay within its error of the boundary) moves one activation by one unit and shifts later
    values; every logit must stay within tight + rho * max_c |z_or[i, c]|.
    Returns (stats, ok): stats = fraction of packets entirely within tight, worst error / tight
    over those, worst error / allowance over all, and the smallest per-tile fraction within tight."""
    z = np.asarray(z, dtype=np.float64)
    tight = gamma(K + 1) * mag
    err = np.abs(z - z_or)
    rowmax = np.abs(z_or).max(axis=1, keepdims=True)
    allow = tight + rho * rowmax
    in_tight = (err <= tight).all(axis=1)
    n = len(z)
    tiles = [in_tight[t:t + tile].mean() for t in range(0, n - tile + 1, tile)]
    stats = {
        "packets": n,
        "frac_tight": float(in_tight.mean()),
        "worst_tight_ratio": float((err[in_tight] / np.maximum(tight[in_tight], 1e-300)).max()) if in_tight.any() else None,
        "worst_allow_ratio": float((err / allow).max()),
        "min_tile_frac_tight": float(min(tiles)) if tiles else None,
        "median_rel": float(np.median(err.max(axis=1) / rowmax[:, 0])),
    }
    return stats, bool(np.isfinite(z).all() and (err <= allow).all())


def fp32_logit_bound(p64: dict, X: np.ndarray, lam: float = 8.0, kappa: float = 2.0) -> np.ndarray:
    """Per-logit bound on |z - z64| for the FP32 path (CUDA-core FMAs, round to nearest).

    Each FP32 output j of a layer is a chain of n_j = K + 2 rounded operations (K multiply-adds,
    the bias, the skip input), every rounding error at most u |partial sum| <= u M_j with
    M_j = sum_k |x_k| |W_kj| + |b_j| + |skip_j| and u = 2^-24. To first order, logit c moves by
    sum_j g_cj * (errors of output j), with g_cj = dz_c / dpre_j the network's signed sensitivity
    through the later layers and their ReLU masks (from the float64 forward; a ReLU whose input is
    within 1e-4 of its layer's largest |pre-activation| of zero counts as open).
    Modelling the rounding errors as independent, zero-mean and bounded (the probabilistic
    rounding-error analysis of Higham and Mary, SIAM J. Sci. Comput. 41(5), 2019), Hoeffding's
    inequality bounds the sum by lam * u * sqrt(sum_j n_j (g_cj M_j)^2) except with probability
    2 exp(-lam^2 / 2) (about 2.5e-14 at lam = 8) per logit; kappa covers second-order terms."""
    from oracle import mlp
    z, c = mlp.forward(p64, X, keep=True)
    u = 2.0 ** -24
    K = p64["W1"][0].shape[0] if p64["W1"] else p64["W0"].shape[1]
    mask = lambda pre: (pre > -1e-4 * np.abs(pre).max(axis=1, keepdims=True)).astype(np.float64)
    sq = lambda G, M, n: n * np.einsum("pcn,pn->pc", G * G, M * M)
    h_out = c["h_out"]
    Mout = np.abs(h_out) @ np.abs(p64["Wc"]) + np.abs(p64["bc"])
    acc = (K + 1) * Mout * Mout                                                # output layer: g = 1
    G = np.broadcast_to(p64["Wc"].T, (len(X),) + p64["Wc"].T.shape).copy()     # dz/dh, (P, C, N)
    for k in reversed(range(len(p64["W1"]))):
        pre2, pre1, uu, h = c["pre2"][k], c["pre1"][k], c["u"][k], c["h_in"][k]
        G2 = G * mask(pre2)[:, None, :]                                         # dz/dpre2
        acc += sq(G2, np.abs(uu) @ np.abs(p64["W2"][k]) + np.abs(p64["b2"][k]) + np.abs(h), K + 2)
        G1 = (G2 @ p64["W2"][k].T) * mask(pre1)[:, None, :]                     # dz/dpre1
        acc += sq(G1, np.abs(h) @ np.abs(p64["W1"][k]) + np.abs(p64["b1"][k]), K + 1)
        G = G1 @ p64["W1"][k].T + G2                                            # dz/dh (block input)
    G0 = G * mask(c["pre0"])[:, None, :]
    acc += sq(G0, np.abs(X) @ np.abs(p64["W0"]) + np.abs(p64["b0"]), p64["W0"].shape[0] + 1)
    return kappa * lam * u * np.sqrt(acc)


def calibrate(p: dict, X: np.ndarray):
    """Activation maxima of every tensor-core layer input (the blob's FP8 calibration)."""
    from oracle import mlp
    p64 = {k: ([a.astype(np.float64) for a in v] if isinstance(v, list) else v.astype(np.float64)) for k, v in p.items()}
    _, cache = mlp.forward(p64, X, keep=True)
    amax = []
    for k in range(len(p["W1"])):
        amax += [np.abs(cache["h_in"][k]).max(), np.abs(cache["u"][k]).max()]
    amax.append(np.abs(cache["h_out"]).max())
    return np.array(amax, dtype=np.float32)


from nets import random_params  # noqa: E402,F401  (re-exported for the GPU tests)
