"""Pins for the oracle's low-precision forwards (oracle/mlp_lowp.py) and for the exactness of the
test networks the GPU tests compare bit for bit."""
import numpy as np

import workloads as wl
from nets import exact_bf16_params, exact_fp8_params, random_params, to_f64
from oracle import mlp, mlp_lowp, quant


def test_bf16_round64_rounds_once_to_nearest_even():
    # ties go to the even neighbour
    assert quant.bf16_round64([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8)]).tolist() == \
        [1.0, 1.0 + 2.0 ** -6, -1.0]
    # 1 + 2^-8 + 2^-30 lies above the tie, so it rounds up; a detour through float32 would land on
    # the tie 1 + 2^-8 first and then round down to 1 (double rounding)
    x = 1.0 + 2.0 ** -8 + 2.0 ** -30
    assert quant.bf16_round64(x) == 1.0 + 2.0 ** -7
    assert float(quant.bf16_round(np.float32(x))) == 1.0
    # on float32 inputs it agrees with the float32 encoder (pinned against torch's cast)
    rng = np.random.default_rng(0)
    v = (rng.normal(0, 1, 100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    assert (quant.bf16_round64(v.astype(np.float64)) == quant.bf16_round(v).astype(np.float64)).all()


def _one_block(W1, W2, Wc, b0, b1, b2, bc, W0):
    return {"W0": np.asarray(W0, np.float32), "b0": np.asarray(b0, np.float32),
            "W1": [np.asarray(W1, np.float32)], "b1": [np.asarray(b1, np.float32)],
            "W2": [np.asarray(W2, np.float32)], "b2": [np.asarray(b2, np.float32)],
            "Wc": np.asarray(Wc, np.float32), "bc": np.asarray(bc, np.float32)}


def test_bf16_worked_example():
    """One block of width 2, values worked by hand.
    h0 = (257, 100.5) -> BF16 (256, 100.5)  [257 is a tie between 256 and 258: even]
    u = ReLU(h0 W1) = (256, 356.5) -> (256, 356)  [spacing 2 in [256, 512)]
    x = ReLU(u W2 + b2 + h0) = (512, 356 - 300 + 100.5 = 156.5) -> (512, 156)  [tie: even]
    z = x Wc + bc = (512 + 156 + 0.25, 156).
    Without the roundings (oracle.mlp): h0 = (257, 100.5), u = (257, 357.5), x = (514, 158),
    z = (672.25, 158)."""
    W0 = np.zeros((7, 2))
    W0[0, 0] = 1.0
    W0[6, 1] = 1.0
    p = _one_block(W1=[[1, 1], [0, 1]], W2=[[1, 0], [0, 1]], Wc=[[1, 0], [1, 1]],
                   b0=[0, 0.5], b1=[0, 0], b2=[0, -300], bc=[0.25, 0], W0=W0)
    X = np.array([[257, 0, 0, 0, 0, 0, 100]], dtype=np.float64)
    z, mag = mlp_lowp.forward_bf16(p, X)
    assert z.tolist() == [[668.25, 156.0]]
    assert mag.tolist() == [[668.25, 156.0]]
    assert mlp.forward(to_f64(p), X).tolist() == [[672.25, 158.0]]


def test_fp8_worked_example():
    """One block of width 2, one class, activation scales s = (2, 1, 1/2) (amax 224, 448, 896).
    Hidden weights with max |W| = 7/8 get the weight scale 512, so dq = 1 / (512 s_l).
    a0 = E4M3(2 * (10, 3.125)) = (20, 6)            [6.25 is a tie between 6 and 6.5: even]
    FC1: (a0 q1) / 1024 + b1 = (8960, 1344) / 1024 + (0, 1/16) = (8.75, 1.375) -> (9, 1.375)
    FC2: (u q2) / 512 * 1/2 + a0 * (1/2) / 2 = (4032, 4340) / 1024 + (5, 1.5)
         = (8.9375, 5.73828125) -> (9, 5.5)
    z = (a qc) / (512 * 1/2) + bc = (9 * 448 + 5.5 * 224) / 256 + 0.5 = 21.0625."""
    W0 = np.zeros((7, 2))
    W0[0, 0] = 2.0 ** -12
    W0[6, 1] = 1.0 / 32
    p = _one_block(W1=[[0.875, 0], [0, 0.4375]], W2=[[0.875, 0.875], [0, 0.4375]], Wc=[[0.875], [0.4375]],
                   b0=[0, 0], b1=[0, 0.0625], b2=[0, 0], bc=[0.5], W0=W0)
    amax = np.array([224.0, 448.0, 896.0], dtype=np.float32)
    assert mlp_lowp.act_scales(amax).tolist() == [2.0, 1.0, 0.5]
    X = np.array([[40960, 0, 0, 0, 0, 0, 100]], dtype=np.float64)
    z, _ = mlp_lowp.forward_fp8(p, X, amax)
    assert z.tolist() == [[21.0625]]
    f = mlp_lowp.fp8_weights(p, amax)
    assert f["q"][0].tolist() == [[448.0, 0.0], [0.0, 224.0]] and f["dq"][0] == 1.0 / 1024
    assert abs(mlp.forward(to_f64(p), X)[0, 0] - 20.939666748046875) < 1e-12


def test_bf16_forward_equals_plain_forward_when_nothing_needs_rounding():
    """Integer weights and inputs that keep every activation an integer below 256 (all BF16
    values): the BF16 scheme changes nothing, so it must equal oracle.mlp's forward exactly."""
    rng = np.random.default_rng(3)
    N, blocks = 16, 2
    W0 = np.zeros((7, N))
    W0[rng.integers(0, 7, N), np.arange(N)] = 1.0
    p = {"W0": W0.astype(np.float32), "b0": rng.integers(-3, 1, N).astype(np.float32),
         "W1": [], "b1": [], "W2": [], "b2": []}
    for _ in range(blocks):
        for key in ("W1", "W2"):
            W = np.zeros((N, N), np.float32)
            for c in range(N):
                a, b = rng.choice(N, 2, replace=False)
                W[a, c], W[b, c] = 1.0, -1.0
            p[key].append(W)
        p["b1"].append(rng.integers(-3, 1, N).astype(np.float32))
        p["b2"].append(rng.integers(-3, 1, N).astype(np.float32))
    p["Wc"] = rng.integers(-1, 2, (N, 5)).astype(np.float32)
    p["bc"] = rng.integers(-3, 4, 5).astype(np.float32)
    X = rng.integers(0, 32, (500, 7)).astype(np.float64)
    z, _, steps = mlp_lowp.forward_bf16(p, X, keep=True)
    assert max(float(s[0].max()) for s in steps) < 256          # the premise: no rounding anywhere
    assert (z == mlp.forward(to_f64(p), X)).all()


def test_low_precision_forwards_track_the_float64_forward():
    """Random networks: the schemes stay within their precision of the exact forward, and do round."""
    rng = np.random.default_rng(5)
    rules = wl.rules_for_config(0)
    X = mlp.features(wl.trace_for_config(0, rules, seed=4)[:2000])
    p = random_params(rng, N=128, blocks=3, C=25)
    z64, cache = mlp.forward(to_f64(p), X, keep=True)
    amax = []
    for k in range(3):
        amax += [np.abs(cache["h_in"][k]).max(), np.abs(cache["u"][k]).max()]
    amax.append(np.abs(cache["h_out"]).max())
    rowmax = np.abs(z64).max(axis=1)
    for z, lim in ((mlp_lowp.forward_bf16(p, X)[0], 0.03), (mlp_lowp.forward_fp8(p, X, amax)[0], 0.3)):
        rel = np.abs(z - z64).max(axis=1) / rowmax
        assert 0 < np.median(rel) and rel.max() < lim


def _check_exact(steps, quantum, sum_limit):
    """Every layer input is on the grid `quantum`; every output column's sum of |products| stays
    below `sum_limit` (so any summation order is exact); every later partial result is a float32."""
    for inp, W, partial in steps:
        assert (np.abs(inp / quantum - np.rint(inp / quantum)) == 0).all()
        assert (np.abs(inp) @ np.abs(W)).max() < sum_limit
        for v in partial[1:]:
            assert (v.astype(np.float32).astype(np.float64) == v).all()


def test_exact_networks_are_exact_in_fp32():
    rules = wl.rules_for_config(0)
    X = mlp.features(wl.trace_for_config(0, rules, seed=5)[:4096])
    for seed, (N, blocks) in enumerate([(512, 6), (256, 3)]):
        rng = np.random.default_rng(100 + seed)
        p = exact_bf16_params(rng, N=N, blocks=blocks, C=25)
        z, _, steps = mlp_lowp.forward_bf16(p, X, keep=True)
        # partial sums of multiples of 2^-8 below 2^16 need at most 24 significant bits
        _check_exact(steps, 2.0 ** -8, 2.0 ** 16)
        assert len(np.unique(z)) > 100                          # not a degenerate network
        p8, amax = exact_fp8_params(rng, N=N, blocks=blocks, C=25)
        z8, _, steps8 = mlp_lowp.forward_fp8(p8, X, amax, keep=True)
        # E4M3 values are multiples of 2^-9 and the codes +-448 multiples of 2^6: products are
        # multiples of 2^-3, exact in sums below 2^21
        _check_exact(steps8, 2.0 ** -9, 2.0 ** 21)
        assert len(np.unique(z8)) > 100


def test_logit_tolerance_is_below_the_logits_scale():
    """The element-wise acceptance of the tensor-core tests (gpu_util.compare_logits with the RHO
    of test_gpu_tc.py) allows less than 1 % (BF16) and 10 % (FP8) of each packet's largest |logit|,
    on the networks those tests use."""
    from gpu_util import calibrate, gamma
    import ast
    src = open(__file__.replace("test_oracle_mlp_lowp.py", "test_gpu_tc.py")).read()
    rho = ast.literal_eval(src.split("RHO = ", 1)[1].split("\n", 1)[0])
    rules = wl.rules_for_config(0)
    X = mlp.features(wl.trace_for_config(0, rules, seed=5)[:2048])
    p = random_params(np.random.default_rng(77), N=512, blocks=6, C=25)
    amax = calibrate(p, X)
    for prec, lim, (z, mag) in (("bf16", 0.01, mlp_lowp.forward_bf16(p, X)),
                                ("fp8", 0.10, mlp_lowp.forward_fp8(p, X, amax))):
        rowmax = np.abs(z).max(axis=1, keepdims=True)
        tol = gamma(513) * mag + rho[prec] * rowmax
        assert (tol / rowmax).max() < lim, (prec, float((tol / rowmax).max()))
