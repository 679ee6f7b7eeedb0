"""Tensor-core (tcgen05) paths: BF16 / FP8 logits against the float64 oracle forward of the same
quantised weights, and bit-exact rule ids through the fused and staged kernels."""
import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import ids_dev, ids_host, logit_tolerance, random_params, to_dev
from oracle import classify as oc
from oracle import mlp, quant, tss

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U_BF16 = 2.0 ** -8   # BF16 keeps 8 significant bits
U_E4M3 = 2.0 ** -4   # E4M3 keeps 4


@pytest.fixture(scope="module")
def setup():
    ctx = tg.Context(0)
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    T = ctx.ruleset_info(rs)["n_tuples"]
    p = random_params(np.random.default_rng(77), N=512, blocks=6, C=T)
    h = wl.trace_for_config(0, rules, seed=5)
    X = mlp.features(h[:4096])
    p64 = {k: ([a.astype(np.float64) for a in v] if isinstance(v, list) else v.astype(np.float64)) for k, v in p.items()}
    # activation calibration (max |input| of every tensor-core layer) on the oracle side
    _, cache = mlp.forward(p64, X, keep=True)
    amax = []
    for k in range(6):
        amax += [np.abs(cache["h_in"][k]).max(), np.abs(cache["u"][k]).max()]
    amax.append(np.abs(cache["h_out"]).max())
    ctx.load_model(rs, tg.pack_model(p, np.array(amax, dtype=np.float32)))
    yield ctx, rules, rs, T, p, p64, h
    ctx.close()


def bf16_weights(p64):
    q = dict(p64)
    for k in ("W1", "W2"):
        q[k] = [quant.bf16_round(w.astype(np.float32)).astype(np.float64) for w in p64[k]]
    q["Wc"] = quant.bf16_round(p64["Wc"].astype(np.float32)).astype(np.float64)
    return q


def e4m3_weights(p64):
    """E4M3 round-to-nearest-even of W * 448 / max|W|, dequantised: one scale per hidden layer,
    one per output column (Wc[:, c]) for the output layer."""
    def deq(W, per_column=False):
        amax = np.abs(W.astype(np.float32)).max(axis=0)
        if not per_column:
            amax = np.full_like(amax, amax.max())
        sw = np.where(amax > 0, np.float32(448.0) / amax.astype(np.float32), np.float32(1.0)).astype(np.float32)
        q = quant.e4m3_round((W.astype(np.float32) * sw[None, :]).astype(np.float32))
        return q / sw[None, :].astype(np.float64)
    q = dict(p64)
    q["W1"] = [deq(w) for w in p64["W1"]]
    q["W2"] = [deq(w) for w in p64["W2"]]
    q["Wc"] = deq(p64["Wc"], per_column=True)
    return q


def infer(ctx, rs, h, C, precision, variant=None):
    d = to_dev(h)
    z = torch.zeros((len(h), C), dtype=torch.float32, device="cuda")
    t = torch.zeros(len(h), dtype=torch.int32, device="cuda")
    ctx.infer(rs, d, z, t, precision=precision, variant=variant)
    torch.cuda.synchronize()
    return z.cpu().numpy().astype(np.float64), t.cpu().numpy()


@pytest.mark.parametrize("variant", ["1sm", "2sm", "mc2", "mc4", "n256"])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_logits_within_bound(setup, prec, variant):
    ctx, rules, rs, T, p, p64, h = setup
    hs = h[:4096]
    X = mlp.features(hs)
    q = bf16_weights(p64) if prec == "bf16" else e4m3_weights(p64)
    z64 = mlp.forward(q, X)
    z, tup = infer(ctx, rs, hs, T, tg.BF16 if prec == "bf16" else tg.FP8, variant)
    tol = logit_tolerance(q, X, U32, U_BF16 if prec == "bf16" else U_E4M3)
    err = np.abs(z - z64)
    assert np.isfinite(z).all()
    assert (err <= tol).all(), float((err / tol).max())
    assert (tup == np.argmax(z, axis=1)).all()
    # the bound is loose; the typical error is far below it
    rel = err / (np.abs(z64).max(axis=1, keepdims=True) + 1e-30)
    assert np.median(rel) < (0.02 if prec == "bf16" else 0.3)


@pytest.mark.parametrize("variant", ["1sm", "2sm", "mc2", "mc4", "n256"])
@pytest.mark.parametrize("path", ["fused_bf16", "staged_bf16", "fused_fp8", "staged_fp8"])
def test_ids_exact(setup, path, variant):
    ctx, rules, rs, T, p, p64, h = setup
    want = oc.classify(rules, h)
    d = to_dev(h)
    ids = ids_dev(len(h))
    st = ctx.classify(rs, d, ids, path=path, stats=True, variant=variant)
    assert (ids_host(ids) == want).all()
    assert st["packets"] == len(h)
    assert st["pred_hit"] + st["fallback"] == len(h)


@pytest.mark.parametrize("variant", ["1sm", "2sm", "mc2", "mc4", "n256"])
def test_ragged_sizes_and_graph(setup, variant):
    ctx, rules, rs, T, p, p64, h = setup
    for n in (1, 5, 127, 128, 129, 255, 256, 257, 1000, 148 * 128 + 3, 74 * 256 + 129):
        hs = h[:n]
        d = to_dev(hs)
        ids = ids_dev(n)
        ctx.classify(rs, d, ids, path="fused_bf16", variant=variant)
        torch.cuda.synchronize()
        assert (ids_host(ids) == oc.classify(rules, hs)).all(), n
    d = to_dev(h)
    want = oc.classify(rules, h)
    for _ in range(3):
        ids = ids_dev(len(h))
        ctx.classify(rs, d, ids, path="fused_bf16", graph=True, variant=variant)
        torch.cuda.synchronize()
        assert (ids_host(ids) == want).all()


def test_predictions_agree_across_precisions(setup):
    """BF16 and FP32 argmax agree on most packets; disagreements are counted, ids stay exact."""
    ctx, rules, rs, T, p, p64, h = setup
    hs = h[:20000]
    _, t32 = infer(ctx, rs, hs, T, tg.FP32)
    _, t16 = infer(ctx, rs, hs, T, tg.BF16, "1sm")
    assert (t32 == t16).mean() > 0.9
    # the N=128 variants run the same arithmetic on each row
    z16 = infer(ctx, rs, hs, T, tg.BF16, "1sm")[0]
    for v in ("2sm", "mc2", "mc4"):
        zv, tv = infer(ctx, rs, hs, T, tg.BF16, v)
        assert (tv == t16).all(), v
        assert (zv == z16).all(), v
    # the N=256 kernel sums layer 0 on the tensor core (exact products, another FP32 summation
    # order): a BF16 rounding of x may differ by one unit, so logits agree closely, not bitwise
    zv, tv = infer(ctx, rs, hs, T, tg.BF16, "n256")
    scale = np.abs(z16).max(axis=1, keepdims=True) + 1e-30
    assert np.median(np.abs(zv - z16) / scale) < 1e-3
    assert (tv == t16).mean() > 0.998


@pytest.mark.parametrize("width,blocks", [(512, 1), (512, 2), (512, 3), (256, 1), (256, 2), (256, 6)])
def test_other_shapes_on_the_n256_kernel(width, blocks):
    """Networks of 1-3 residual blocks at width 512, and of width 256 (one 256-column chunk per
    layer), run on the N=256 kernel: logits within the bound of the float64 forward of the
    quantised weights (BF16 and FP8), rule ids exact; the N=128 variants, built for width 512 and
    6 blocks, are not used for them."""
    ctx = tg.Context(0)
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    T = ctx.ruleset_info(rs)["n_tuples"]
    p = random_params(np.random.default_rng(100 + blocks + width), N=width, blocks=blocks, C=T)
    h = wl.trace_for_config(0, rules, seed=9)[:20000 + 3]
    X = mlp.features(h[:4096])
    p64 = {k: ([a.astype(np.float64) for a in v] if isinstance(v, list) else v.astype(np.float64)) for k, v in p.items()}
    _, cache = mlp.forward(p64, X, keep=True)
    amax = []
    for k in range(blocks):
        amax += [np.abs(cache["h_in"][k]).max(), np.abs(cache["u"][k]).max()]
    amax.append(np.abs(cache["h_out"]).max())
    ctx.load_model(rs, tg.pack_model(p, np.array(amax, dtype=np.float32)))
    for prec in ("bf16", "fp8"):
        q = bf16_weights(p64) if prec == "bf16" else e4m3_weights(p64)
        z64 = mlp.forward(q, X)
        for variant in (None, "1sm"):  # "1sm" falls back to the N=256 kernel for these shapes
            z, tup = infer(ctx, rs, h[:4096], T, tg.BF16 if prec == "bf16" else tg.FP8, variant)
            tol = logit_tolerance(q, X, U32, U_BF16 if prec == "bf16" else U_E4M3)
            assert np.isfinite(z).all()
            assert (np.abs(z - z64) <= tol).all(), (prec, float((np.abs(z - z64) / tol).max()))
            assert (tup == np.argmax(z, axis=1)).all()
    want = oc.classify(rules, h)
    d = to_dev(h)
    for path in ("fused_bf16", "fused_fp8", "staged_bf16", "plain_fp32"):
        ids = ids_dev(len(h))
        ctx.classify(rs, d, ids, path=path)
        torch.cuda.synchronize()
        assert (ids_host(ids) == want).all(), path
    ctx.close()


def _spread_rules(n, seed):
    """n rules with SIP / DIP prefix lengths uniform in 0..32: hundreds of tuples."""
    rng = np.random.default_rng(seed)
    rules = wl.gen_rules(n, seed)
    for f in ("sip", "dip"):
        rules[f + "_len"] = rng.integers(0, 33, n)
        m = np.array([tss.prefix_mask(int(l)) for l in rules[f + "_len"]], dtype=np.uint64)
        rules[f] = (rules[f].astype(np.uint64) & m).astype(np.uint32)
    return rules


@pytest.mark.parametrize("n_rules,width", [(200, 512), (350, 512), (1500, 512), (350, 256)])
def test_many_tuples_on_the_n256_kernel(n_rules, width):
    """Rulesets with 187, 308 and 824 tuples on the N=256 kernel, whose output layer then runs
    as one chunk of 192 columns, as 256 + 64, and as three of 256 + 64: logits within the bound
    of the float64 forward of the quantised weights, argmax = the first maximum, ids exact (and
    the 308-tuple case at width 256)."""
    ctx = tg.Context(0)
    rules = _spread_rules(n_rules, 300 + n_rules)
    rs = ctx.load_ruleset(rules)
    T = ctx.ruleset_info(rs)["n_tuples"]
    assert T == {200: 187, 350: 308, 1500: 824}[n_rules], T
    blocks = 2
    p = random_params(np.random.default_rng(n_rules + width), N=width, blocks=blocks, C=T)
    h = wl.gen_trace(rules, [("inside", 9000), ("random", 1000)], 31)
    X = mlp.features(h[:4096])
    p64 = {k: ([a.astype(np.float64) for a in v] if isinstance(v, list) else v.astype(np.float64)) for k, v in p.items()}
    _, cache = mlp.forward(p64, X, keep=True)
    amax = []
    for k in range(blocks):
        amax += [np.abs(cache["h_in"][k]).max(), np.abs(cache["u"][k]).max()]
    amax.append(np.abs(cache["h_out"]).max())
    ctx.load_model(rs, tg.pack_model(p, np.array(amax, dtype=np.float32)))
    for prec in ("bf16", "fp8"):
        q = bf16_weights(p64) if prec == "bf16" else e4m3_weights(p64)
        z64 = mlp.forward(q, X)
        for variant in (None, "1sm"):  # "1sm" falls back to the N=256 kernel past 128 classes
            z, tup = infer(ctx, rs, h[:4096], T, tg.BF16 if prec == "bf16" else tg.FP8, variant)
            tol = logit_tolerance(q, X, U32, U_BF16 if prec == "bf16" else U_E4M3)
            assert np.isfinite(z).all()
            assert (np.abs(z - z64) <= tol).all(), (prec, float((np.abs(z - z64) / tol).max()))
            assert (tup == np.argmax(z, axis=1)).all()
    want = oc.classify(rules, h)
    d = to_dev(h)
    for path in ("fused_bf16", "fused_fp8", "staged_bf16", "plain_fp32"):
        ids = ids_dev(len(h))
        ctx.classify(rs, d, ids, path=path)
        torch.cuda.synchronize()
        assert (ids_host(ids) == want).all(), path
    ctx.close()
