"""Seeded random configurations of the fused tensor-core kernel against the oracle: width 256 or
512, 1-3 residual blocks, rulesets from tens to hundreds of tuples (one or several output
chunks), batch sizes from one packet to several tiles per CTA, BF16 and FP8, the one-kernel and
the split form. Rule ids must equal the linear scan's, and the predicted tuple must be the first
maximum of the logits the same
call returns; the logits of the first 4,096 packets must match the oracle's low-precision
forward element by element, as in test_gpu_tc.py."""
import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import calibrate, compare_logits, ids_dev, ids_host, random_params, to_dev
from oracle import classify as oc
from oracle import mlp, mlp_lowp, tss
from test_gpu_tc import PHI, PHI_TILE, RHO

pytestmark = pytest.mark.gpu


def _rules(rng, seed):
    n = int(rng.choice([60, 300, 900]))
    rules = wl.gen_rules(n, seed)
    if rng.random() < 0.5:  # prefix lengths uniform in 0..32: many tuples
        for f in ("sip", "dip"):
            rules[f + "_len"] = rng.integers(0, 33, n)
            m = np.array([tss.prefix_mask(int(l)) for l in rules[f + "_len"]], dtype=np.uint64)
            rules[f] = (rules[f].astype(np.uint64) & m).astype(np.uint32)
    rules["priority"] = rng.permutation(n)
    return rules


@pytest.mark.parametrize("seed", range(6))
def test_random_shapes_match_the_oracle(seed):
    rng = np.random.default_rng(1000 + seed)
    ctx = tg.Context(0)
    rules = _rules(rng, 2000 + seed)
    rs = ctx.load_ruleset(rules)
    T = ctx.ruleset_info(rs)["n_tuples"]
    width = int(rng.choice([256, 512]))
    blocks = int(rng.integers(1, 4))
    p = random_params(rng, N=width, blocks=blocks, C=T)
    calib = wl.gen_trace(rules, [("inside", 2048)], 3000 + seed)
    amax = calibrate(p, mlp.features(calib))
    ctx.load_model(rs, tg.pack_model(p, amax))
    n = int(rng.choice([1, 97, 128 * 148 + 5, 128 * 148 * 3 + 77]))
    h = wl.gen_trace(rules, [("inside", n - n // 8), ("random", n // 8)], 4000 + seed)
    want = oc.classify(rules, h)
    d = to_dev(h)
    for path, prec in (("fused_bf16", tg.BF16), ("fused_fp8", tg.FP8)):
        for variant in (None, "split"):  # the one persistent kernel, and network + search kernels
            ids = ids_dev(n)
            ctx.classify(rs, d, ids, path=path, variant=variant)
            torch.cuda.synchronize()
            assert (ids_host(ids) == want).all(), (seed, path, variant, width, blocks, T, n)
        z = torch.zeros((n, T), dtype=torch.float32, device="cuda")
        t = torch.zeros(n, dtype=torch.int32, device="cuda")
        ctx.infer(rs, d, z, t, precision=prec)
        torch.cuda.synchronize()
        zz = z.cpu().numpy()
        assert np.isfinite(zz).all()
        assert (t.cpu().numpy() == np.argmax(zz, axis=1)).all(), (seed, path)
        m = min(n, 4096)
        X = mlp.features(h[:m])
        key = "bf16" if prec == tg.BF16 else "fp8"
        z_or, mag = mlp_lowp.forward_bf16(p, X) if key == "bf16" else mlp_lowp.forward_fp8(p, X, amax)
        stats, ok = compare_logits(zz[:m], z_or, mag, K=width, rho=RHO[key])
        print(seed, width, blocks, T, n, key, stats)
        assert ok and (m < 128 or stats["frac_tight"] >= PHI[key]), (seed, key, stats)
        assert stats["min_tile_frac_tight"] is None or stats["min_tile_frac_tight"] >= PHI_TILE[key], (seed, key, stats)
    ctx.close()
