"""GPU parity of the network (§6.1) against the float64 oracle forward, per precision and path."""
import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import fp32_logit_bound, ids_dev, ids_host, random_params, to_dev
from oracle import classify as oc
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = tg.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def cfg0(ctx):
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    T = ctx.ruleset_info(rs)["n_tuples"]
    yield ctx, rules, rs, T
    ctx.unload_ruleset(rs)


def run_infer(ctx, rs, h, C, precision):
    d = to_dev(h)
    logits = torch.zeros((len(h), C), dtype=torch.float32, device="cuda")
    tup = torch.zeros(len(h), dtype=torch.int32, device="cuda")
    ctx.infer(rs, d, logits, tup, precision=precision)
    torch.cuda.synchronize()
    return logits.cpu().numpy().astype(np.float64), tup.cpu().numpy()


@pytest.mark.parametrize("shape", [(64, 2), (512, 6)])
def test_fp32_logits_within_bound(cfg0, shape):
    """FP32 path against the float64 forward, element by element, within the per-logit bound of
    gpu_util.fp32_logit_bound; the bound itself stays far below the logits' scale, and an oracle
    with its output biases moved by 0.1 % of that scale (planted on the CPU) falls outside it."""
    ctx, rules, rs, T = cfg0
    N, blocks = shape
    p = random_params(np.random.default_rng(N), N=N, blocks=blocks, C=T)
    ctx.load_model(rs, tg.pack_model(p))
    h = wl.trace_for_config(0, rules, seed=11)[:1024 + 37 if N == 512 else 20000]
    X = mlp.features(h)
    p64 = {k: ([a.astype(np.float64) for a in v] if isinstance(v, list) else v.astype(np.float64)) for k, v in p.items()}
    z64 = mlp.forward(p64, X)
    z, tup = run_infer(ctx, rs, h, T, tg.FP32)
    tol = fp32_logit_bound(p64, X)
    err = np.abs(z - z64)
    rowmax = np.abs(z64).max(axis=1, keepdims=True)
    print(shape, "worst err / bound %.3g, bound / row max <= %.3g" % ((err / tol).max(), (tol / rowmax).max()))
    assert (err <= tol).all(), float((err / tol).max())
    assert (tol / rowmax).max() < 1e-3
    q = dict(p64)
    q["bc"] = p64["bc"] + 1e-3 * np.median(rowmax)
    assert (np.abs(z - mlp.forward(q, X)) > tol).any()
    # the argmax is taken on the kernel's own logits (lowest index on ties)
    assert (tup == np.argmax(z, axis=1)).all()


def test_plain_path_ids_exact_and_counters(cfg0):
    ctx, rules, rs, T = cfg0
    p = random_params(np.random.default_rng(5), N=64, blocks=2, C=T)
    ctx.load_model(rs, tg.pack_model(p))
    h = wl.trace_for_config(0, rules)
    want = oc.classify(rules, h)
    d = to_dev(h)
    ids = ids_dev(len(h))
    st = ctx.classify(rs, d, ids, path="plain_fp32", stats=True)
    assert (ids_host(ids) == want).all()
    assert st["packets"] == len(h)
    assert st["pred_hit"] + st["fallback"] == len(h)
    # graph replay of the 17-launch plain path
    ids2 = ids_dev(len(h))
    ctx.classify(rs, d, ids2, path="plain_fp32", graph=True)
    ctx.classify(rs, d, ids2, path="plain_fp32", graph=True)
    torch.cuda.synchronize()
    assert (ids_host(ids2) == want).all()


def test_model_shape_checks(cfg0):
    ctx, rules, rs, T = cfg0
    p = random_params(np.random.default_rng(1), N=32, blocks=1, C=T + 1)
    with pytest.raises(tg.TangError):
        ctx.load_model(rs, tg.pack_model(p))
    p = random_params(np.random.default_rng(1), N=32, blocks=1, C=T)
    blob = tg.pack_model(p)
    with pytest.raises(tg.TangError):
        ctx.load_model(rs, blob[:-4])
