"""The paper's CPU-GPU pipeline (§5.1.2, Fig. 4): network on the GPU over CUDA streams, search on
host threads. Rule ids against the oracle (exact and paper mode), host search counters against the
search kernel's on the same predictions, ragged sizes, updates."""
import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import ids_dev, ids_host, to_dev
from oracle import classify as oc
from oracle import tss

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    ctx = tg.Context(0)
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    h = wl.gen_trace(rules, [("inside", 16384)], 3)
    blob, _ = ctx.train(rs, h, N=512, blocks=6, batch=8192, epochs=1, max_rounds=1, alpha=10, holdout=0.05, seed=4)
    ctx.load_model(rs, blob)
    yield ctx, rules, rs
    ctx.close()


def predictions(ctx, rs, h, precision):
    t = torch.empty(len(h), dtype=torch.int32, device="cuda")
    ctx.infer(rs, to_dev(h), tuples=t, precision=precision)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("prec", [tg.BF16, tg.FP8, tg.FP32])
def test_hybrid_exact_and_paper_mode(setup, prec):
    ctx, rules, rs = setup
    _, tor = tss.build_tuples(rules)
    h = wl.trace_for_config(0, rules, seed=11)[:50000 + 13]
    want = oc.classify(rules, h)
    ids = np.zeros(len(h), dtype=np.uint32)
    st = ctx.classify_hybrid(rs, h, ids, batch=8192, streams=4, threads=4, precision=prec, stats=True)
    assert (ids == want).all()
    assert st["packets"] == len(h) and st["matched"] == int((want != wl.NO_MATCH).sum())
    pred = predictions(ctx, rs, h, prec)
    ids[:] = 0
    ctx.classify_hybrid(rs, h, ids, batch=8192, streams=4, threads=4, precision=prec, paper=True)
    assert (ids == oc.paper_classify(rules, h, pred, tor)).all()
    # the host search does the search kernel's work on the same predictions
    ids_d = ids_dev(len(h))
    st_d = ctx.search(rs, to_dev(h), torch.tensor(pred, dtype=torch.int32, device="cuda"), ids_d, stats=True)
    for k in ("probes", "rule_reads", "slot_reads", "pred_hit", "fallback", "nn_correct"):
        assert st[k] == st_d[k], k


def test_hybrid_ragged_batches_streams_threads(setup):
    ctx, rules, rs = setup
    h = wl.trace_for_config(0, rules, seed=12)
    for n, batch, streams, threads in ((1, 8192, 4, 0), (8191, 8192, 4, 3), (8193, 8192, 4, 16),
                                       (3 * 1000 + 5, 1000, 3, 2), (70000, 4096, 1, 8), (777, 128, 16, 1)):
        hs = h[:n]
        ids = np.zeros(n, dtype=np.uint32)
        ctx.classify_hybrid(rs, hs, ids, batch=batch, streams=streams, threads=threads)
        assert (ids == oc.classify(rules, hs)).all(), (n, batch, streams, threads)
    ctx.classify_hybrid(rs, h[:0], np.zeros(0, dtype=np.uint32))
    with pytest.raises(tg.TangError):
        ctx.classify_hybrid(rs, h[:10], np.zeros(10, dtype=np.uint32), precision=7)


def test_hybrid_after_updates_and_many_tuples(setup):
    ctx, rules, rs0 = setup
    rng = np.random.default_rng(8)
    rules2 = wl.gen_rules(900, 51)
    rules2["sip_len"] = rng.integers(0, 33, len(rules2))
    rules2["dip_len"] = rng.integers(0, 33, len(rules2))
    for f in ("sip", "dip"):
        m = np.array([tss.prefix_mask(int(l)) for l in rules2[f + "_len"]], dtype=np.uint64)
        rules2[f] = (rules2[f].astype(np.uint64) & m).astype(np.uint32)
    rules2["priority"] = rng.permutation(len(rules2))
    rs = ctx.load_ruleset(rules2)
    T = ctx.ruleset_info(rs)["n_tuples"]
    assert T > 64
    blob, _ = ctx.train(rs, wl.gen_trace(rules2, [("inside", 8192)], 5), N=512, blocks=6, batch=8192, epochs=1,
                        max_rounds=1, alpha=10, holdout=0.05, seed=6)
    ctx.load_model(rs, blob)
    live = {int(r["id"]): r for r in rules2}
    fresh = wl.gen_rules(300, 52, first_id=10 ** 6)
    fresh["priority"] = rng.integers(0, 900, 300)
    for r in fresh:
        ctx.insert_rule(rs, r)
        live[int(r["id"])] = r
    for rid in rng.choice(rules2["id"], 200, replace=False):
        ctx.delete_rule(rs, int(rid))
        del live[int(rid)]
    cur = np.array(list(live.values()), dtype=wl.RULE_DTYPE)
    h = wl.gen_trace(cur, [("inside", 20000), ("random", 2000)], 7)
    ids = np.zeros(len(h), dtype=np.uint32)
    # hundreds of tuples: the tensor-core network runs its output layer in 256-column chunks
    want = oc.classify(cur, h)
    for prec in (tg.BF16, tg.FP32):
        ids[:] = 0
        ctx.classify_hybrid(rs, h, ids, batch=4096, streams=2, precision=prec)
        assert (ids == want).all(), prec
    ctx.unload_ruleset(rs)
