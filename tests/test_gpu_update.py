"""GPU tests of the paper-mode post-verification (§5.1.1 as printed), the hot swap of a model under
captured CUDA graphs, and the deferred update of §5.2.2: monitor windows, incremental training from
the deployed model, and the full rebuild + retraining. Rule ids are checked against the oracle."""
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
def ctx():
    c = tg.Context(0)
    yield c
    c.close()


def quick_blob(ctx, rs, rules, seed, epochs=1, n=16384, **kw):
    h = wl.gen_trace(rules, [("inside", n)], seed)
    blob, rep = ctx.train(rs, h, N=512, blocks=6, batch=8192, epochs=epochs, max_rounds=1, alpha=10, holdout=0.05,
                          seed=seed, **kw)
    return blob, rep


def predictions(ctx, rs, d, n, precision):
    t = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.infer(rs, d, tuples=t, precision=precision)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.int64)


def run(ctx, rs, d, n, **kw):
    ids = ids_dev(n)
    st = ctx.classify(rs, d, ids, **kw)
    torch.cuda.synchronize()
    return ids_host(ids), st


def skewed_ruleset_with_many_tuples(seed, n):
    rng = np.random.default_rng(seed)
    rules = wl.gen_rules(n, seed)
    rules["sip_len"] = rng.integers(0, 33, n)
    rules["dip_len"] = rng.integers(0, 33, n)
    for f in ("sip", "dip"):
        m = np.array([tss.prefix_mask(int(l)) for l in rules[f + "_len"]], dtype=np.uint64)
        rules[f] = (rules[f].astype(np.uint64) & m).astype(np.uint32)
    rules["priority"] = rng.permutation(n)
    return rules


@pytest.mark.parametrize("kind", ["config0", "many_tuples"])
def test_paper_mode_search_matches_oracle(ctx, kind):
    """Stage 2 alone with given predictions: bit-exact against the oracle's paper-mode definition,
    and the exact search is unaffected by the flag being off."""
    rules = wl.rules_for_config(0) if kind == "config0" else skewed_ruleset_with_many_tuples(8, 700)
    rs = ctx.load_ruleset(rules)
    tuples, tor = tss.build_tuples(rules)
    T = len(tuples)
    h = wl.gen_trace(rules, [("inside", 30000), ("random", 3000)], 21)
    d = to_dev(h)
    exact, pos = oc.classify(rules, h, return_index=True)
    truth = np.where(pos >= 0, tor[np.maximum(pos, 0)], -1)
    rng = np.random.default_rng(3)
    for name, pred in (("random", rng.integers(-3, T + 3, len(h))), ("true", truth), ("none", np.full(len(h), -1)),
                       ("constant", np.full(len(h), int(np.bincount(tor).argmax())))):
        pt = torch.tensor(pred, dtype=torch.int32, device="cuda")
        ids = ids_dev(len(h))
        st_p = ctx.search(rs, d, pt, ids, paper=True, stats=True)
        torch.cuda.synchronize()
        want = oc.paper_classify(rules, h, pred, tor)
        assert (ids_host(ids) == want).all(), name
        st_e = ctx.search(rs, d, pt, ids, stats=True)
        torch.cuda.synchronize()
        assert (ids_host(ids) == exact).all(), name
        assert st_p["probes"] <= st_e["probes"], name
        if name in ("random", "constant"):
            assert (want != exact).any(), name
    ctx.unload_ruleset(rs)


def test_paper_mode_through_network_paths(ctx):
    """Fused, staged and plain paths in paper mode equal the oracle's paper mode applied to the
    network's own predictions (stage 1 alone gives them); exact mode still equals the oracle."""
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    _, tor = tss.build_tuples(rules)
    blob, _ = quick_blob(ctx, rs, rules, seed=5)
    ctx.load_model(rs, blob)
    h = wl.trace_for_config(0, rules, seed=6)[: 40000 + 77]
    d = to_dev(h)
    exact = oc.classify(rules, h)
    for path, prec in (("fused_bf16", tg.BF16), ("staged_bf16", tg.BF16), ("fused_fp8", tg.FP8),
                       ("plain_fp32", tg.FP32)):
        pred = predictions(ctx, rs, d, len(h), prec)
        got, st = run(ctx, rs, d, len(h), path=path, paper=True, stats=True)
        assert (got == oc.paper_classify(rules, h, pred, tor)).all(), path
        assert st["packets"] == len(h)
        got, _ = run(ctx, rs, d, len(h), path=path)
        assert (got == exact).all(), path
        got, _ = run(ctx, rs, d, len(h), path=path, paper=True, graph=True)
        got, _ = run(ctx, rs, d, len(h), path=path, paper=True, graph=True)
        assert (got == oc.paper_classify(rules, h, pred, tor)).all(), path + " graph"
    ctx.unload_ruleset(rs)


def test_hot_swap_keeps_graphs(ctx):
    """A same-shape model replaces the live one inside its buffers: captured graphs are kept and
    their next replay uses the new weights. A model of another shape drops them."""
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    tuples, tor = tss.build_tuples(rules)
    T = len(tuples)
    blob_a, _ = quick_blob(ctx, rs, rules, seed=7)
    p, amax = tg.unpack_model(blob_a)
    # model B predicts one tuple for every packet: zero output weights, a bias that picks t_star
    t_star = int(np.bincount(tor, minlength=T).argmax())
    pb = dict(p)
    pb["Wc"] = np.zeros_like(p["Wc"])
    pb["bc"] = np.zeros_like(p["bc"])
    pb["bc"][t_star] = 10.0
    blob_b = tg.pack_model(pb, amax)
    h = wl.trace_for_config(0, rules, seed=8)[:30000]
    d = to_dev(h)
    ctx.load_model(rs, blob_a)
    ids = ids_dev(len(h))
    ids_exact = ids_dev(len(h))
    for _ in range(2):
        ctx.classify(rs, d, ids, path="fused_bf16", graph=True, paper=True)
        ctx.classify(rs, d, ids_exact, path="fused_bf16", graph=True)
    torch.cuda.synchronize()
    n_graphs = ctx.graph_count()
    assert n_graphs >= 2
    pred_a = predictions(ctx, rs, d, len(h), tg.BF16)
    assert (ids_host(ids) == oc.paper_classify(rules, h, pred_a, tor)).all()
    want_b = oc.paper_classify(rules, h, np.full(len(h), t_star), tor)
    assert (want_b != ids_host(ids)).any()  # B's answers differ from A's
    for blob, want in ((blob_b, want_b), (blob_a, oc.paper_classify(rules, h, pred_a, tor))):
        ctx.load_model(rs, blob)
        assert ctx.graph_count() == n_graphs
        ctx.classify(rs, d, ids, path="fused_bf16", graph=True, paper=True)  # replay
        ctx.classify(rs, d, ids_exact, path="fused_bf16", graph=True)
        torch.cuda.synchronize()
        assert (ids_host(ids) == want).all()
        assert (ids_host(ids_exact) == oc.classify(rules, h)).all()
    # another shape: the graphs go, the next call re-captures
    rng = np.random.default_rng(0)
    small = {"W0": rng.normal(size=(7, 64)).astype(np.float32) / 65536, "b0": np.zeros(64, np.float32),
             "W1": [rng.normal(size=(64, 64)).astype(np.float32) / 8] * 2, "b1": [np.zeros(64, np.float32)] * 2,
             "W2": [rng.normal(size=(64, 64)).astype(np.float32) / 8] * 2, "b2": [np.zeros(64, np.float32)] * 2,
             "Wc": rng.normal(size=(64, T)).astype(np.float32), "bc": np.zeros(T, np.float32)}
    ctx.load_model(rs, tg.pack_model(small))
    assert ctx.graph_count() == 0
    got, _ = run(ctx, rs, d, len(h), path="plain_fp32", graph=True)
    assert (got == oc.classify(rules, h)).all()
    ctx.unload_ruleset(rs)


def test_finetune_starts_from_the_deployed_model(ctx):
    """With a zero learning rate, incremental training returns the deployed parameters bit for bit
    (the 2^-16 feature prescale leaves W0 and comes back exactly)."""
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    blob, _ = quick_blob(ctx, rs, rules, seed=9)
    ctx.load_model(rs, blob)
    h = wl.gen_trace(rules, [("inside", 9000)], 10)
    out, rep = ctx.finetune(rs, h, epochs=1, max_rounds=1, alpha=1, lr=0.0, holdout=0.1, seed=1)
    assert rep["epochs_run"] == 1
    p0, _ = tg.unpack_model(blob)
    p1, amax1 = tg.unpack_model(out)
    for k in ("W0", "b0", "Wc", "bc"):
        assert np.array_equal(p0[k], p1[k]), k
    for k in ("W1", "b1", "W2", "b2"):
        assert all(np.array_equal(a, b) for a, b in zip(p0[k], p1[k])), k
    assert (amax1 > 0).all()
    ctx.unload_ruleset(rs)


def test_finetune_follows_rule_drift(ctx):
    """Immediate updates delete half of the rules and insert 64 top-priority rules that claim a
    quarter of the SIP space for tuple (8, 0), so about a quarter of the packets change tuple.
    Incremental training on packets of the current ruleset raises the network's tuple accuracy on
    them; the rule ids stay exact throughout, and the swap keeps the captured graphs."""
    rules = wl.gen_rules(8192, seed=30)
    rs = ctx.load_ruleset(rules)
    tuples, _ = tss.build_tuples(rules)
    assert (8, 0) in tuples
    blob, rep = quick_blob(ctx, rs, rules, seed=31, epochs=1000, n=65536, time_budget_s=4.0)
    ctx.load_model(rs, blob)
    rng = np.random.default_rng(32)
    live = {int(r["id"]): r.copy() for r in rules}
    for rid in rng.choice(rules["id"], 4096, replace=False):
        ctx.delete_rule(rs, int(rid))
        del live[int(rid)]
    fresh = np.zeros(64, dtype=wl.RULE_DTYPE)
    fresh["sip"] = (np.arange(64, dtype=np.uint64) << np.uint64(24)).astype(np.uint32)
    fresh["sip_len"], fresh["dip_len"] = 8, 0
    fresh["sp_hi"], fresh["dp_hi"], fresh["proto_wild"] = 65535, 65535, 1
    fresh["priority"] = 0
    fresh["id"] = 10 ** 6 + np.arange(64)
    for r in fresh:
        ctx.insert_rule(rs, r)
        live[int(r["id"])] = r
    assert ctx.suboptimal_count(rs) == 0  # (8, 0) is a tuple: immediate update places them exactly
    cur = np.array(list(live.values()), dtype=wl.RULE_DTYPE)
    ev = wl.gen_trace(cur, [("inside", 60000)], 34)
    d = to_dev(ev)
    want = oc.classify(cur, ev)
    got, st0 = run(ctx, rs, d, len(ev), path="staged_bf16", stats=True)
    assert (got == want).all()
    acc0 = st0["nn_correct"] / st0["matched"]
    run(ctx, rs, d, len(ev), path="fused_bf16", graph=True)
    n_graphs = ctx.graph_count()
    out, rep = ctx.finetune(rs, wl.gen_trace(cur, [("inside", 65536)], 35), epochs=1000, max_rounds=1, alpha=100,
                            holdout=0.05, time_budget_s=4.0, seed=36)
    ctx.load_model(rs, out)
    assert ctx.graph_count() == n_graphs
    got, st1 = run(ctx, rs, d, len(ev), path="staged_bf16", stats=True)
    assert (got == want).all()
    acc1 = st1["nn_correct"] / st1["matched"]
    assert acc1 > acc0 + 0.05, (acc0, acc1, rep)
    got, _ = run(ctx, rs, d, len(ev), path="fused_bf16", graph=True)
    assert (got == want).all()
    ctx.unload_ruleset(rs)


def test_rebuild_and_full_retraining(ctx):
    """Rules whose lengths have no tuple go to coarser tuples (counted); the rebuild moves them to
    tuples of their own lengths (new tuples, counter reset, conflict sets recomputed), drops the
    model whose classes no longer fit, and the retraining path of du_apply deploys a new one."""
    rules = wl.rules_for_config(0, n_rules=2000)
    rs = ctx.load_ruleset(rules)
    ctx.load_model(rs, quick_blob(ctx, rs, rules, seed=40)[0])
    T0 = ctx.ruleset_info(rs)["n_tuples"]
    odd = wl.gen_rules(300, seed=41, first_id=10 ** 6)
    rng = np.random.default_rng(42)
    odd["sip_len"] = rng.choice([4, 12, 20, 28], 300)
    odd["dip_len"] = rng.choice([4, 12, 20, 28], 300)
    for f in ("sip", "dip"):
        m = np.array([tss.prefix_mask(int(l)) for l in odd[f + "_len"]], dtype=np.uint64)
        odd[f] = (odd[f].astype(np.uint64) & m).astype(np.uint32)
    odd["priority"] = rng.integers(0, 2000, 300)
    for r in odd:
        ctx.insert_rule(rs, r)
    assert ctx.suboptimal_count(rs) == 300
    cur = np.concatenate([rules, odd])
    h = wl.gen_trace(cur, [("inside", 30000), ("random", 2000)], 43)
    d = to_dev(h)
    want = oc.classify(cur, h)
    assert (run(ctx, rs, d, len(h), path="fused_bf16")[0] == want).all()
    kept = ctx.rebuild_ruleset(rs)
    assert not kept
    assert ctx.suboptimal_count(rs) == 0
    tuples, tor = tss.build_tuples(cur)
    info = ctx.ruleset_info(rs)
    assert info["n_tuples"] == len(tuples) > T0 and info["n_rules"] == len(cur)
    for t, (ls, ld) in enumerate(tuples):
        assert ctx.tuple_get(rs, t)[:2] == (ls, ld)
    words = tss.conflict_words(cur, tor, len(tuples))
    for i in range(0, len(cur), 7):
        t, w = ctx.rule_conflicts(rs, int(cur["id"][i]))
        assert t == tor[i] and (w == words[i]).all(), i
    assert (run(ctx, rs, d, len(h), path="no_nn")[0] == want).all()
    with pytest.raises(tg.TangError):
        run(ctx, rs, d, len(h), path="fused_bf16")  # the old model went with its tuple list
    # the retraining branch of the deferred update: rebuild (unchanged now) + train + deploy
    rep = ctx.du_apply(rs, "retrain", wl.gen_trace(cur, [("inside", 16384)], 44), N=512, blocks=6, epochs=1,
                       max_rounds=1, alpha=10, holdout=0.05, seed=45)
    assert rep["epochs_run"] >= 1
    for path in ("fused_bf16", "fused_fp8", "staged_bf16", "plain_fp32"):
        assert (run(ctx, rs, d, len(h), path=path)[0] == want).all(), path
    # a rebuild that keeps the tuple list keeps the model and the graphs
    run(ctx, rs, d, len(h), path="fused_bf16", graph=True)
    n_graphs = ctx.graph_count()
    assert ctx.rebuild_ruleset(rs) and ctx.graph_count() == n_graphs
    got, _ = run(ctx, rs, d, len(h), path="fused_bf16", graph=True)
    assert (got == want).all()
    ctx.unload_ruleset(rs)


def test_monitor_windows_and_decisions(ctx):
    """Window bookkeeping of §5.2.2: the first window is the baseline; later windows trigger by the
    relative drop; the counter picks retraining; an incremental update is a hot swap."""
    rules = wl.rules_for_config(0, n_rules=3000)
    rs = ctx.load_ruleset(rules)
    ctx.load_model(rs, quick_blob(ctx, rs, rules, seed=50)[0])
    ctx.du_observe(rs, 600, 0.5)
    ctx.du_observe(rs, 400, 0.5)
    w = ctx.du_close_window(rs, tau=0.05, theta=10)
    assert w["window"] == 0 and w["decision"] == "none" and w["th_base"] == w["th_cur"] == 1000.0
    ctx.du_observe(rs, 1000, 1.04)
    assert ctx.du_close_window(rs, tau=0.05, theta=10)["decision"] == "none"
    ctx.du_observe(rs, 1000, 1.2)
    w = ctx.du_close_window(rs, tau=0.05, theta=10)
    assert w["window"] == 2 and w["decision"] == "incremental" and w["th_base"] == 1000.0
    with pytest.raises(tg.TangError):
        ctx.du_close_window(rs, tau=0.05, theta=10)  # empty window
    odd = wl.gen_rules(11, seed=51, first_id=10 ** 6)
    odd["sip_len"], odd["dip_len"] = 12, 20
    odd["sip"] &= np.uint32(0xFFF00000)
    odd["dip"] &= np.uint32(0xFFFFF000)
    for r in odd:
        ctx.insert_rule(rs, r)
    ctx.du_observe(rs, 1000, 1.2)
    w = ctx.du_close_window(rs, tau=0.05, theta=10)
    assert w["suboptimal"] == 11 and w["decision"] == "retrain"
    h = wl.trace_for_config(0, rules, seed=52)[:20000]
    d = to_dev(h)
    run(ctx, rs, d, len(h), path="fused_bf16", graph=True)
    n_graphs = ctx.graph_count()
    samples = wl.gen_trace(np.concatenate([rules, odd]), [("inside", 16384)], 53)
    ctx.du_apply(rs, "incremental", samples, epochs=1, max_rounds=1, alpha=10, holdout=0.05, seed=54)
    assert ctx.graph_count() == n_graphs
    want = oc.classify(np.concatenate([rules, odd]), h)
    assert (run(ctx, rs, d, len(h), path="fused_bf16", graph=True)[0] == want).all()
    ctx.du_apply(rs, "retrain", samples, N=512, blocks=6, epochs=1, max_rounds=1, alpha=10, holdout=0.05, seed=55)
    assert ctx.suboptimal_count(rs) == 0
    ctx.du_observe(rs, 1000, 2.0)
    w = ctx.du_close_window(rs, tau=0.05, theta=10)
    assert w["window"] == 0 and w["th_base"] == 500.0  # a new baseline after the full retraining
    assert (run(ctx, rs, d, len(h), path="fused_bf16")[0] == want).all()
    ctx.unload_ruleset(rs)
