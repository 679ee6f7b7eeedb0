"""Tensor-core (tcgen05) paths: BF16 / FP8 logits element by element against the oracle's forward
under the same roundings (oracle/mlp_lowp.py), bit for bit on networks whose FP32 arithmetic is
exact, and bit-exact rule ids through the fused and staged kernels."""
import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import calibrate, compare_logits, ids_dev, ids_host, to_dev
from nets import exact_bf16_params, exact_fp8_params, random_params
from oracle import classify as oc
from oracle import mlp, mlp_lowp, tss

pytestmark = pytest.mark.gpu

# Element-wise acceptance of the random-weight networks (see compare_logits): every logit within
# the output layer's own FP32 summation bound plus RHO of the packet's largest |logit| (rounding
# decisions taken on the other side of a BF16 / E4M3 boundary), and at least PHI of the packets
# (and PHI_TILE of every 128-packet tile) entirely within the summation bound. Measured on a B300
# over every shape these tests run: at most 0.51 % (BF16) and 6.4 % (FP8) of the row maximum, at
# least 86.8 % / 99.8 % of the packets and 80 % / 99.2 % of every tile within the summation bound.
RHO = {"bf16": 0.008, "fp8": 0.08}
PHI = {"bf16": 0.6, "fp8": 0.9}
PHI_TILE = {"bf16": 0.4, "fp8": 0.8}
PREC = {"bf16": tg.BF16, "fp8": tg.FP8}


def lowp(prec, p, X, amax):
    return mlp_lowp.forward_bf16(p, X) if prec == "bf16" else mlp_lowp.forward_fp8(p, X, amax)


# the fused kernel on one SM per tile, and on CTA pairs (cta_group::2)
VARIANTS = ["n256", "pair"]


def infer(ctx, rs, h, C, precision, variant=None):
    d = to_dev(h)
    z = torch.zeros((len(h), C), dtype=torch.float32, device="cuda")
    t = torch.zeros(len(h), dtype=torch.int32, device="cuda")
    ctx.infer(rs, d, z, t, precision=precision, variant=variant)
    torch.cuda.synchronize()
    return z.cpu().numpy(), t.cpu().numpy()


def accepted(stats, ok, prec):
    return ok and stats["frac_tight"] >= PHI[prec] and (stats["min_tile_frac_tight"] is None or
                                                         stats["min_tile_frac_tight"] >= PHI_TILE[prec])


@pytest.fixture(scope="module")
def setup():
    ctx = tg.Context(0)
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    T = ctx.ruleset_info(rs)["n_tuples"]
    p = random_params(np.random.default_rng(77), N=512, blocks=6, C=T)
    h = wl.trace_for_config(0, rules, seed=5)
    amax = calibrate(p, mlp.features(h[:4096]))
    ctx.load_model(rs, tg.pack_model(p, amax))
    yield ctx, rules, rs, T, p, amax, h
    ctx.close()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_logits_match_the_oracle_element_by_element(setup, prec, variant):
    ctx, rules, rs, T, p, amax, h = setup
    hs = h[:4096 + 37]                      # 32 full tiles and a ragged one
    X = mlp.features(hs)
    z, tup = infer(ctx, rs, hs, T, PREC[prec], variant)
    z_or, mag = lowp(prec, p, X, amax)
    stats, ok = compare_logits(z, z_or, mag, K=512, rho=RHO[prec])
    print(prec, stats)
    assert accepted(stats, ok, prec), stats
    assert (tup == np.argmax(z, axis=1)).all()


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_comparison_catches_planted_oracle_faults(setup, prec):
    """The comparison above must fail when the oracle differs from the kernel by 1 % of the logit
    scale in one place: the output biases, or one 64-column unit of a hidden layer's biases
    (planted in the oracle's copy of the parameters, on the CPU)."""
    ctx, rules, rs, T, p, amax, h = setup
    hs = h[:4096]
    X = mlp.features(hs)
    z, _ = infer(ctx, rs, hs, T, PREC[prec])
    z_or, mag = lowp(prec, p, X, amax)
    assert accepted(*compare_logits(z, z_or, mag, K=512, rho=RHO[prec]), prec)
    scale = float(np.median(np.abs(z_or).max(axis=1)))
    faults = []
    q = {k: (list(v) if isinstance(v, list) else v.copy()) for k, v in p.items()}
    q["bc"] = (p["bc"] + np.float32(0.01 * scale)).astype(np.float32)
    faults.append(("output biases", q))
    q = {k: (list(v) if isinstance(v, list) else v.copy()) for k, v in p.items()}
    b = p["b2"][5].copy()
    # one 64-column unit of the last block's second chunk, shifted so that the logits move by
    # about 1 % of their scale: 64 shifts through output weights of rms |Wc|
    b[320:384] += np.float32(0.01 * scale / (8.0 * np.sqrt(np.mean(p["Wc"].astype(np.float64) ** 2))))
    q["b2"] = p["b2"][:5] + [b]
    faults.append(("hidden unit biases", q))
    for name, q in faults:
        zq, mq = lowp(prec, q, X, amax)
        stats, ok = compare_logits(z, zq, mq, K=512, rho=RHO[prec])
        assert not accepted(stats, ok, prec), (name, stats)


def _spread_rules(n, seed):
    """n rules with SIP / DIP prefix lengths uniform in 0..32: hundreds of tuples."""
    rng = np.random.default_rng(seed)
    rules = wl.gen_rules(n, seed)
    for f in ("sip", "dip"):
        rules[f + "_len"] = rng.integers(0, 33, n)
        m = np.array([tss.prefix_mask(int(l)) for l in rules[f + "_len"]], dtype=np.uint64)
        rules[f] = (rules[f].astype(np.uint64) & m).astype(np.uint32)
    return rules


# (rules, width, blocks): 25 tuples (config 0) at several shapes; 187 tuples (one 192-column output
# chunk), 308 (256 + 64) and 824 (3 x 256 + 64)
EXACT_CASES = [("cfg0", 512, 6), ("cfg0", 512, 1), ("cfg0", 256, 6), ("cfg0", 256, 2),
               (200, 512, 2), (350, 512, 2), (1500, 512, 1), (350, 256, 2)]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case", EXACT_CASES, ids=[f"{r}-{w}x{b}" for r, w, b in EXACT_CASES])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_exact_networks_bit_for_bit(prec, case, variant):
    """On networks whose every FP32 sum is exact (tests/nets.py, checked on the CPU), the kernel's
    logits equal the oracle's bit for bit, and its tuple is the first maximum; with a change of
    2^-8 planted in the oracle's last output bias, the comparison fails."""
    which, width, blocks = case
    ctx = tg.Context(0)
    rules = wl.rules_for_config(0) if which == "cfg0" else _spread_rules(which, 300 + which)
    rs = ctx.load_ruleset(rules)
    T = ctx.ruleset_info(rs)["n_tuples"]
    if which != "cfg0":
        assert T == {200: 187, 350: 308, 1500: 824}[which], T
    rng = np.random.default_rng(7000 + width + blocks + T)
    if prec == "bf16":
        p, amax = exact_bf16_params(rng, N=width, blocks=blocks, C=T), None
    else:
        p, amax = exact_fp8_params(rng, N=width, blocks=blocks, C=T)
    ctx.load_model(rs, tg.pack_model(p, amax))
    h = wl.gen_trace(rules, [("inside", 2000), ("random", 309)], 41 + T)   # 18 tiles and a ragged one
    X = mlp.features(h)
    z, tup = infer(ctx, rs, h, T, PREC[prec], variant)
    z_or, _ = lowp(prec, p, X, amax)
    assert (z_or.astype(np.float32).astype(np.float64) == z_or).all()      # the oracle's values are FP32 values
    bad = np.argwhere(z.astype(np.float64) != z_or)
    assert len(bad) == 0, (len(bad), bad[:5].tolist())
    assert (tup == np.argmax(z_or, axis=1)).all()
    # a planted fault of one unit in the last output column's bias is seen
    q = dict(p)
    q["bc"] = p["bc"].copy()
    q["bc"][T - 1] += np.float32(2.0 ** -8)
    zq, _ = lowp(prec, q, X, amax)
    assert (z.astype(np.float64) != zq).any()
    ctx.close()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("path", ["fused_bf16", "staged_bf16", "fused_fp8", "staged_fp8"])
def test_ids_exact(setup, path, variant):
    ctx, rules, rs, T, p, amax, h = setup
    want = oc.classify(rules, h)
    d = to_dev(h)
    ids = ids_dev(len(h))
    st = ctx.classify(rs, d, ids, path=path, stats=True, variant=variant)
    assert (ids_host(ids) == want).all()
    assert st["packets"] == len(h)
    assert st["pred_hit"] + st["fallback"] == len(h)


@pytest.mark.parametrize("path", ["fused_bf16", "fused_fp8"])
def test_split_form_matches_the_one_kernel_form(setup, path):
    """The fused path as two kernels (TANG_FUSED_SPLIT): the network kernel leaves each packet's
    predicted tuple in its id, the search kernel replaces it with the rule id. Ids equal the
    oracle's, and every counter equals the one-kernel form's: the same predictions reach the same
    search. Also refused where it does not apply."""
    ctx, rules, rs, T, p, amax, h = setup
    want = oc.classify(rules, h)
    d = to_dev(h)
    st = {}
    for v in ("n256", "split"):
        ids = ids_dev(len(h))
        st[v] = ctx.classify(rs, d, ids, path=path, stats=True, variant=v)
        assert (ids_host(ids) == want).all(), v
    assert st["split"] == st["n256"]
    # host buffers (the pipelined copy-in / compute / copy-out path)
    out = np.full(len(h), 7, dtype=np.uint32)
    ctx.classify(rs, h, out, path=path, variant="split")
    assert (out == want).all()
    # the paper's post-verification: not exact, but the same predictions give the same ids
    paper = {}
    for v in ("n256", "split"):
        ids = ids_dev(len(h))
        ctx.classify(rs, d, ids, path=path, variant=v, paper=True)
        torch.cuda.synchronize()
        paper[v] = ids_host(ids).copy()
    assert (paper["split"] == paper["n256"]).all()
    with pytest.raises(tg.TangError):
        ctx.classify(rs, d, ids_dev(len(h)), path="staged_bf16", variant="split")


@pytest.mark.parametrize("variant", VARIANTS + ["split"])
def test_ragged_sizes_and_graph(setup, variant):
    ctx, rules, rs, T, p, amax, h = setup
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
    ctx, rules, rs, T, p, amax, h = setup
    hs = h[:20000]
    _, t32 = infer(ctx, rs, hs, T, tg.FP32)
    _, t16 = infer(ctx, rs, hs, T, tg.BF16)
    _, t8 = infer(ctx, rs, hs, T, tg.FP8)
    print("argmax flips vs FP32: BF16 %.4f, FP8 %.4f" % ((t32 != t16).mean(), (t32 != t8).mean()))
    assert (t32 == t16).mean() > 0.9
    assert (t32 == t8).mean() > 0.5


@pytest.mark.parametrize("width,blocks", [(512, 1), (512, 2), (512, 3), (256, 1), (256, 2), (256, 6)])
def test_other_shapes(width, blocks):
    """Networks of 1-3 residual blocks at width 512, and of width 256 (one 256-column chunk per
    layer): logits element by element against the oracle's low-precision forward, rule ids exact."""
    ctx = tg.Context(0)
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    T = ctx.ruleset_info(rs)["n_tuples"]
    p = random_params(np.random.default_rng(100 + blocks + width), N=width, blocks=blocks, C=T)
    h = wl.trace_for_config(0, rules, seed=9)[:20000 + 3]
    X = mlp.features(h[:4096])
    amax = calibrate(p, X)
    ctx.load_model(rs, tg.pack_model(p, amax))
    for prec in ("bf16", "fp8"):
        z_or, mag = lowp(prec, p, X, amax)
        for variant in VARIANTS:
            z, tup = infer(ctx, rs, h[:4096], T, PREC[prec], variant)
            stats, ok = compare_logits(z, z_or, mag, K=width, rho=RHO[prec])
            print(width, blocks, prec, variant, stats)
            assert accepted(stats, ok, prec), (prec, variant, stats)
            assert (tup == np.argmax(z, axis=1)).all()
    want = oc.classify(rules, h)
    d = to_dev(h)
    for path, variant in (("fused_bf16", "n256"), ("fused_fp8", "n256"), ("fused_bf16", "pair"),
                          ("fused_fp8", "pair"), ("staged_bf16", None), ("plain_fp32", None)):
        ids = ids_dev(len(h))
        ctx.classify(rs, d, ids, path=path, variant=variant)
        torch.cuda.synchronize()
        assert (ids_host(ids) == want).all(), (path, variant)
    ctx.close()


@pytest.mark.parametrize("n_rules,width", [(200, 512), (350, 512), (1500, 512), (350, 256)])
def test_many_tuples(n_rules, width):
    """Rulesets with 187, 308 and 824 tuples, whose output layer runs as one chunk of 192
    columns, as 256 + 64, and as three of 256 + 64: logits element by element against the oracle,
    argmax = the first maximum, ids exact (and the 308-tuple case at width 256)."""
    ctx = tg.Context(0)
    rules = _spread_rules(n_rules, 300 + n_rules)
    rs = ctx.load_ruleset(rules)
    T = ctx.ruleset_info(rs)["n_tuples"]
    assert T == {200: 187, 350: 308, 1500: 824}[n_rules], T
    blocks = 2
    p = random_params(np.random.default_rng(n_rules + width), N=width, blocks=blocks, C=T)
    h = wl.gen_trace(rules, [("inside", 9000), ("random", 1000)], 31)
    X = mlp.features(h[:4096])
    amax = calibrate(p, X)
    ctx.load_model(rs, tg.pack_model(p, amax))
    for prec in ("bf16", "fp8"):
        z_or, mag = lowp(prec, p, X, amax)
        for variant in VARIANTS:
            z, tup = infer(ctx, rs, h[:4096], T, PREC[prec], variant)
            stats, ok = compare_logits(z, z_or, mag, K=width, rho=RHO[prec])
            print(n_rules, width, prec, variant, stats)
            assert accepted(stats, ok, prec), (prec, variant, stats)
            assert (tup == np.argmax(z, axis=1)).all()
        if T > 256:
            # a 1 % shift of the second output chunk's biases in the oracle is caught
            q = dict(p)
            q["bc"] = p["bc"].copy()
            q["bc"][256:] += np.float32(0.01 * np.median(np.abs(z_or).max(axis=1)))
            zq, mq = lowp(prec, q, X, amax)
            assert not accepted(*compare_logits(z, zq, mq, K=width, rho=RHO[prec]), prec)
    want = oc.classify(rules, h)
    d = to_dev(h)
    for path, variant in (("fused_bf16", "n256"), ("fused_fp8", "n256"), ("fused_bf16", "pair"),
                          ("fused_fp8", "pair"), ("staged_bf16", None), ("plain_fp32", None)):
        ids = ids_dev(len(h))
        ctx.classify(rs, d, ids, path=path, variant=variant)
        torch.cuda.synchronize()
        assert (ids_host(ids) == want).all(), (path, variant)
    ctx.close()
