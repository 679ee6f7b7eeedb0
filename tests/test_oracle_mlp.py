"""Pins for the oracle's float64 MLP (§6.1, Eq. 1-2), its gradients and training math (§6.2)."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import mlp


def rand_params(rng, S=7, N=8, k=2, C=5, scale=0.5):
    return {
        "W0": rng.normal(0, scale, (S, N)), "b0": rng.normal(0, scale, N),
        "W1": [rng.normal(0, scale, (N, N)) for _ in range(k)], "b1": [rng.normal(0, scale, N) for _ in range(k)],
        "W2": [rng.normal(0, scale, (N, N)) for _ in range(k)], "b2": [rng.normal(0, scale, N) for _ in range(k)],
        "Wc": rng.normal(0, scale, (N, C)), "bc": rng.normal(0, scale, C),
    }


def test_features_segments():
    """§6.2: SIP hi/lo, DIP hi/lo, SP, DP, PRO as 16-bit segment values."""
    h = np.zeros(2, dtype=wl.HEADER_DTYPE)
    h[0] = (0x12345678, 0x9ABCDEF0, 80, 65535, 17, (0, 0, 0))
    h[1] = (0xFFFFFFFF, 0, 0, 1, 255, (0, 0, 0))
    X = mlp.features(h)
    assert X.tolist() == [[0x1234, 0x5678, 0x9ABC, 0xDEF0, 80, 65535, 17], [65535, 65535, 0, 0, 0, 1, 255]]


def test_blocks_reduce_to_closed_forms():
    """Eq. 1 special cases. W1 = W2 = 0: B(x) = ReLU(b2 + x). W1 = W2 = I, b = 0: B(x) = 2x for x >= 0."""
    rng = np.random.default_rng(0)
    p = rand_params(rng, N=6, k=3)
    X = rng.normal(0, 1, (10, 7))
    h0 = np.maximum(X @ p["W0"] + p["b0"], 0)
    q = dict(p)
    q["W1"] = [np.zeros((6, 6))] * 3
    q["W2"] = [np.zeros((6, 6))] * 3
    q["b1"] = [rng.normal(0, 1, 6)] * 3
    want = h0
    for k in range(3):
        want = np.maximum(q["b2"][k] + want, 0)
    np.testing.assert_allclose(mlp.forward(q, X), want @ p["Wc"] + p["bc"], rtol=1e-13, atol=1e-13)
    q = dict(p)
    q["W1"] = [np.eye(6)] * 3
    q["W2"] = [np.eye(6)] * 3
    q["b1"] = [np.zeros(6)] * 3
    q["b2"] = [np.zeros(6)] * 3
    np.testing.assert_allclose(mlp.forward(q, X), (8.0 * h0) @ p["Wc"] + p["bc"], rtol=1e-13, atol=1e-12)


def _torch_net(p):
    class Net(torch.nn.Module):
        def __init__(self):
            super().__init__()
            S, N = p["W0"].shape
            C = p["Wc"].shape[1]
            self.inp = torch.nn.Linear(S, N).double()
            self.l1 = torch.nn.ModuleList([torch.nn.Linear(N, N).double() for _ in p["W1"]])
            self.l2 = torch.nn.ModuleList([torch.nn.Linear(N, N).double() for _ in p["W1"]])
            self.out = torch.nn.Linear(N, C).double()
            with torch.no_grad():
                self.inp.weight.copy_(torch.tensor(p["W0"].T)); self.inp.bias.copy_(torch.tensor(p["b0"]))
                for k in range(len(p["W1"])):
                    self.l1[k].weight.copy_(torch.tensor(p["W1"][k].T)); self.l1[k].bias.copy_(torch.tensor(p["b1"][k]))
                    self.l2[k].weight.copy_(torch.tensor(p["W2"][k].T)); self.l2[k].bias.copy_(torch.tensor(p["b2"][k]))
                self.out.weight.copy_(torch.tensor(p["Wc"].T)); self.out.bias.copy_(torch.tensor(p["bc"]))

        def forward(self, x):
            h = torch.relu(self.inp(x))
            for a, b in zip(self.l1, self.l2):
                h = torch.relu(b(torch.relu(a(h))) + h)
            return self.out(h)
    return Net()


def test_forward_and_backward_match_torch_float64():
    """Library routines (torch.nn.Linear, autograd, F.cross_entropy) in float64."""
    rng = np.random.default_rng(1)
    p = rand_params(rng, N=16, k=3, C=6)
    X = rng.normal(0, 2, (33, 7))
    y = rng.integers(0, 6, 33)
    net = _torch_net(p)
    xt = torch.tensor(X)
    z = net(xt)
    np.testing.assert_allclose(mlp.forward(p, X), z.detach().numpy(), rtol=1e-12, atol=1e-12)
    loss = torch.nn.functional.cross_entropy(z, torch.tensor(y))
    loss.backward()
    l, g = mlp.backward(p, X, y)
    assert abs(l - loss.item()) < 1e-12
    np.testing.assert_allclose(g["W0"], net.inp.weight.grad.numpy().T, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(g["bc"], net.out.bias.grad.numpy(), rtol=1e-10, atol=1e-12)
    for k in range(3):
        np.testing.assert_allclose(g["W1"][k], net.l1[k].weight.grad.numpy().T, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(g["b2"][k], net.l2[k].bias.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_backward_central_differences():
    """Every gradient entry of a tiny network against central finite differences of the loss."""
    rng = np.random.default_rng(2)
    p = rand_params(rng, N=5, k=2, C=4)
    X = rng.normal(0, 1, (9, 7))
    y = rng.integers(0, 4, 9)
    _, g = mlp.backward(p, X, y)
    eps = 1e-6
    for key in mlp.flat_keys(p):
        P = mlp.get(p, key)
        G = mlp.get(g, key)
        for idx in np.ndindex(P.shape):
            old = P[idx]
            P[idx] = old + eps
            lp = mlp.cross_entropy(mlp.forward(p, X), y)
            P[idx] = old - eps
            lm = mlp.cross_entropy(mlp.forward(p, X), y)
            P[idx] = old
            assert abs((lp - lm) / (2 * eps) - G[idx]) < 1e-6, (key, idx)


def test_argmax_ties_lowest_index():
    p = rand_params(np.random.default_rng(3), N=4, k=1, C=3)
    p["Wc"] = np.zeros((4, 3))
    p["bc"] = np.array([1.0, 2.0, 2.0])
    assert mlp.predict(p, np.zeros((2, 7))).tolist() == [1, 1]


def test_adam_closed_form_and_torch():
    """First Adam step moves each parameter by lr*g/(|g|+eps) (bias correction makes m_hat=g, v_hat=g^2)."""
    rng = np.random.default_rng(4)
    w = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    w1, m, v = mlp.adam_step(w, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    np.testing.assert_allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # several steps against torch.optim.Adam in float64
    wt = torch.tensor(w, requires_grad=True)
    opt = torch.optim.Adam([wt], lr=1e-3)
    wo, m, v = w.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        gt = rng.normal(0, 1, 50)
        wt.grad = torch.tensor(gt)
        opt.step()
        wo, m, v = mlp.adam_step(wo, gt, m, v, t, 1e-3)
    np.testing.assert_allclose(wo, wt.detach().numpy(), rtol=0, atol=1e-14)
