"""GPU parity of the tuple space, conflict sets and the exact search against the oracle."""
import itertools

import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from golden_io import table1
from gpu_util import ids_dev, ids_host, random_params, to_dev
from oracle import classify as oc
from oracle import tss

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = tg.Context(0)
    yield c
    c.close()


def classify_dev(ctx, rs, h, path="no_nn", **kw):
    d = to_dev(h)
    ids = ids_dev(len(h))
    st = ctx.classify(rs, d, ids, path=path, **kw)
    torch.cuda.synchronize()
    return ids_host(ids), st


def check_tables(ctx, rs, rules):
    tuples, tor = tss.build_tuples(rules)
    info = ctx.ruleset_info(rs)
    assert info["n_tuples"] == len(tuples)
    for t, (ls, ld) in enumerate(tuples):
        assert ctx.tuple_get(rs, t)[:2] == (ls, ld)
    words = tss.conflict_words(rules, tor, len(tuples))
    for i in range(len(rules)):
        t, w = ctx.rule_conflicts(rs, int(rules["id"][i]))
        assert t == tor[i]
        assert (w == words[i]).all(), i
    return tuples, tor


def test_table1_tuples_conflicts_and_every_point(ctx):
    rules, *_ = table1()
    rs = ctx.load_ruleset(rules)
    check_tables(ctx, rs, rules)
    h = np.zeros(64, dtype=wl.HEADER_DTYPE)
    for k, (x, y) in enumerate(itertools.product(range(8), range(8))):
        h["sip"][k], h["dip"][k] = x << 29, y << 29
    got, _ = classify_dev(ctx, rs, h)
    assert (got == oc.classify(rules, h)).all()
    ctx.unload_ruleset(rs)


@pytest.mark.parametrize("cfg", [0, 1])
def test_conflicts_and_no_nn_parity(ctx, cfg):
    rules = wl.rules_for_config(cfg, n_rules=1024 if cfg == 0 else 2048)
    rs = ctx.load_ruleset(rules)
    check_tables(ctx, rs, rules)
    h = wl.trace_for_config(cfg, rules, scale=0.1 if cfg == 0 else 0.02)
    got, st = classify_dev(ctx, rs, h, stats=True)
    want = oc.classify(rules, h)
    assert (got == want).all()
    assert st["packets"] == len(h) and st["matched"] == int((want != wl.NO_MATCH).sum())
    ctx.unload_ruleset(rs)


def test_more_than_32_tuples(ctx):
    """Uniform prefix lengths 0..32 give hundreds of tuples: multi-word conflict sets."""
    rng = np.random.default_rng(4)
    rules = wl.gen_rules(600, 41)
    rules["sip_len"] = rng.integers(0, 33, len(rules))
    rules["dip_len"] = rng.integers(0, 33, len(rules))
    for f in ("sip", "dip"):
        m = np.array([tss.prefix_mask(int(l)) for l in rules[f + "_len"]], dtype=np.uint64)
        rules[f] = (rules[f].astype(np.uint64) & m).astype(np.uint32)
    rules["priority"] = rng.permutation(len(rules))
    rs = ctx.load_ruleset(rules)
    tuples, tor = check_tables(ctx, rs, rules)
    assert len(tuples) > 64
    h = wl.gen_trace(rules, [("inside", 20000), ("random", 2000)], 3)
    want = oc.classify(rules, h)
    got, _ = classify_dev(ctx, rs, h)
    assert (got == want).all()
    pred = torch.tensor(rng.integers(-3, len(tuples) + 3, len(h)), dtype=torch.int32, device="cuda")
    ids = ids_dev(len(h))
    ctx.search(rs, to_dev(h), pred, ids)
    assert (ids_host(ids) == want).all()
    ctx.unload_ruleset(rs)


def test_search_any_prediction_is_exact_and_probe_counts_match_oracle(ctx):
    rng = np.random.default_rng(9)
    rules = wl.gen_rules(300, 17, len_weights=[0.3, 0.3, 0.2, 0.1, 0.1])
    rules["priority"] = rng.permutation(len(rules))
    rs = ctx.load_ruleset(rules)
    tuples, tor = tss.build_tuples(rules)
    h = wl.gen_trace(rules, [("inside", 1500), ("random", 300)], 5)
    want, pos = oc.classify(rules, h, return_index=True)
    o = tss.TwoStageSearch(rules, tuples, tor)
    truth = np.where(pos >= 0, tor[np.maximum(pos, 0)], 0)
    for name, pred in (("random", rng.integers(0, len(tuples), len(h))), ("true", truth),
                       ("none", np.full(len(h), -1))):
        ids = ids_dev(len(h))
        st = ctx.search(rs, to_dev(h), torch.tensor(pred, dtype=torch.int32, device="cuda"), ids, stats=True)
        assert (ids_host(ids) == want).all(), name
        probes = sum(o.search(h[k], None if pred[k] < 0 else int(pred[k]))[1] for k in range(len(h)))
        assert st["probes"] == probes, name
        if name == "true":
            assert st["nn_correct"] == int((want != wl.NO_MATCH).sum())
    ctx.unload_ruleset(rs)


def test_edge_cases(ctx):
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    for n in (1, 7, 255, 257, 4099):
        h = wl.trace_for_config(0, rules, seed=n)[:n]
        got, _ = classify_dev(ctx, rs, h)
        assert (got == oc.classify(rules, h)).all(), n
    ids = ids_dev(0)
    ctx.classify(rs, to_dev(wl.trace_for_config(0, rules)[:1])[:0], ids, path="no_nn")
    empty = ctx.load_ruleset(rules[:0])
    got, _ = classify_dev(ctx, empty, wl.trace_for_config(0, rules)[:1000])
    assert (got == wl.NO_MATCH).all()
    with pytest.raises(tg.TangError):
        bad = rules.copy()
        bad["id"][5] = bad["id"][6]
        ctx.load_ruleset(bad)
    with pytest.raises(tg.TangError):
        bad = rules.copy()
        bad["sip_len"][3] = 33
        ctx.load_ruleset(bad)
    with pytest.raises(tg.TangError):
        ctx.classify(rs, to_dev(wl.trace_for_config(0, rules)[:10]), ids_dev(10), path="plain_fp32")  # no model
    ctx.unload_ruleset(rs)
    ctx.unload_ruleset(empty)


def test_graph_replay_and_host_pipeline(ctx):
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    h = wl.trace_for_config(0, rules)
    want = oc.classify(rules, h)
    d = to_dev(h)
    for _ in range(3):
        ids = ids_dev(len(h))
        ctx.classify(rs, d, ids, path="no_nn", graph=True)
        torch.cuda.synchronize()
        assert (ids_host(ids) == want).all()
    # host mode: pageable numpy buffers, and pinned ones
    out = np.zeros(len(h), dtype=np.uint32)
    ctx.classify(rs, h, out, path="no_nn")
    assert (out == want).all()
    ph = torch.empty(len(h) * 16, dtype=torch.uint8, pin_memory=True).numpy()
    ph[:] = h.view(np.uint8).reshape(-1)
    pout = torch.zeros(len(h), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    ctx.classify(rs, ph.view(wl.HEADER_DTYPE), pout, path="no_nn")
    assert (pout == want).all()
    ctx.unload_ruleset(rs)


def test_updates_stay_exact(ctx):
    """Immediate update (§5.2.1): inserts and deletes; every epoch is re-checked against the oracle."""
    rules = wl.rules_for_config(0, n_rules=3000)
    rs = ctx.load_ruleset(rules)
    tuples, _ = tss.build_tuples(rules)
    live = {int(r["id"]): r.copy() for r in rules}
    ops = wl.gen_update_stream(rules, 600, seed=3, update_frac=0.5, batch_lo=2000, batch_hi=6000)
    checked = 0
    for op in ops:
        if op[0] == "insert":
            r = op[1]
            ctx.insert_rule(rs, r)
            live[int(r["id"])] = r
            t, _ = ctx.rule_conflicts(rs, int(r["id"]))
            assert t == tss.restricted_insert_tuple(tuples, int(r["sip_len"]), int(r["dip_len"]))
        elif op[0] == "delete":
            ctx.delete_rule(rs, op[1])
            del live[op[1]]
        else:
            cur = np.array(list(live.values()), dtype=wl.RULE_DTYPE)
            h = wl.gen_trace(cur, [("inside", op[1] // 2), ("random", op[1] // 8)], op[2])
            want = oc.classify(cur, h)
            got, _ = classify_dev(ctx, rs, h)
            assert (got == want).all()
            pred = torch.randint(0, len(tuples), (len(h),), dtype=torch.int32, device="cuda")
            ids = ids_dev(len(h))
            ctx.search(rs, to_dev(h), pred, ids)
            torch.cuda.synchronize()
            assert (ids_host(ids) == want).all()
            checked += 1
    assert checked > 10
    # conflict sets after updates contain the exact ones (deletes leave supersets)
    cur = np.array(list(live.values()), dtype=wl.RULE_DTYPE)
    tor = np.array([ctx.rule_conflicts(rs, int(i))[0] for i in cur["id"]])
    exact = tss.conflict_words(cur, tor, len(tuples))
    for i in range(len(cur)):
        _, w = ctx.rule_conflicts(rs, int(cur["id"][i]))
        assert ((w & exact[i]) == exact[i]).all()
    with pytest.raises(tg.TangError):
        ctx.delete_rule(rs, 10 ** 9)
    with pytest.raises(tg.TangError):
        ctx.insert_rule(rs, cur[0])  # id already live
    assert ctx.suboptimal_count(rs) >= 0
    ctx.unload_ruleset(rs)


def test_graph_replay_sees_updates_after_table_growth(ctx):
    """A graph captured before many inserts (which relocate runs, grow the rule pool and rehash
    tuple tables) replays correctly afterwards: kernels read the tables through a descriptor."""
    rules = wl.rules_for_config(0, n_rules=800)
    rs = ctx.load_ruleset(rules)
    h = wl.trace_for_config(0, rules, seed=4)[:20000]
    d = to_dev(h)
    ids = ids_dev(len(h))
    for _ in range(2):
        ctx.classify(rs, d, ids, path="no_nn", graph=True)
    torch.cuda.synchronize()
    assert (ids_host(ids) == oc.classify(rules, h)).all()
    fresh = wl.gen_rules(6000, 77)
    fresh["id"] += 10 ** 6
    fresh["priority"] = np.random.default_rng(1).integers(0, 800, len(fresh))
    for r in fresh:
        ctx.insert_rule(rs, r)
    info = ctx.ruleset_info(rs)
    assert info["n_rules"] == 6800
    ctx.classify(rs, d, ids, path="no_nn", graph=True)  # replay of the graph captured above
    torch.cuda.synchronize()
    cur = np.concatenate([rules, fresh])
    assert (ids_host(ids) == oc.classify(cur, h)).all()
    ctx.unload_ruleset(rs)


def long_run_rules(n_plain, n_wild, seed):
    """n_plain rules of the config-0 generator plus n_wild rules with both prefixes wildcarded
    (tuple (0,0): one hash key, one run of n_wild+ rules) whose exact ports and protocol few
    packets match. The wildcard rules take priorities among the best quarter: a packet whose
    answer lies below them compares it with every rule of the run."""
    rng = np.random.default_rng(seed)
    plain = wl.gen_rules(n_plain, seed)
    both = (plain["sip_len"] == 0) & (plain["dip_len"] == 0)
    plain["sip_len"][both] = 8                 # the (0,0) key holds the wildcard rules below only
    plain["sip"][both] &= np.uint32(0xFF000000)
    wild = wl.gen_rules(n_wild, seed + 1)
    wild["sip_len"] = 0
    wild["dip_len"] = 0
    wild["sip"] = 0
    wild["dip"] = 0
    for f in ("sp", "dp"):
        v = rng.integers(0, 65536, n_wild)
        wild[f + "_lo"] = v
        wild[f + "_hi"] = v
    wild["proto_wild"] = 0
    wild["proto"] = 17
    rules = np.concatenate([plain, wild])
    rules["id"] = np.arange(len(rules))
    rules["priority"] = rng.permutation(len(rules))
    rules["priority"][n_plain:] = rng.integers(0, len(rules) // 4, n_wild)
    return rules


def test_long_runs_scanned_by_the_warp(ctx):
    """A (0,0) run of more than 6,000 rules (a long in-bucket comparison, §5.1.1): the lanes of a
    warp scan it together; ids equal the oracle's on every path, with and without the
    cooperative scan, probe counts equal the oracle's two-stage search, and the cooperative scan
    reads the same rules as the serial one."""
    rules = long_run_rules(20000, 6000, 41)
    rs = ctx.load_ruleset(rules)
    tuples, tor = tss.build_tuples(rules)
    t00 = [k for k, t in enumerate(tuples) if tuple(t) == (0, 0)][0]
    assert int((tor == t00).sum()) >= 6000
    T = ctx.ruleset_info(rs)["n_tuples"]
    ctx.load_model(rs, tg.pack_model(random_params(np.random.default_rng(3), N=256, blocks=1, C=T)))
    wild = rules[tor == t00]
    h = np.concatenate([wl.gen_trace(rules, [("inside", 30000), ("random", 8000)], 7),
                        wl.gen_trace(wild, [("inside", 2000)], 8)])
    want = oc.classify(rules, h)
    d = to_dev(h)
    reads = {}
    for path in ("no_nn", "fused_bf16", "staged_bf16"):
        for serial in (False, True):
            ids = ids_dev(len(h))
            st = ctx.classify(rs, d, ids, path=path, stats=True, serial=serial)
            assert (ids_host(ids) == want).all(), (path, serial)
            reads[(path, serial)] = (st["probes"], st["rule_reads"])
        assert reads[(path, False)] == reads[(path, True)], path
    # the fused path as two kernels (the search with the whole GPU), and whatever the autotuner
    # picks between the forms on this batch
    ids = ids_dev(len(h))
    st = ctx.classify(rs, d, ids, path="fused_bf16", stats=True, variant="split")
    assert (ids_host(ids) == want).all()
    assert (st["probes"], st["rule_reads"]) == reads[("fused_bf16", False)]
    ctx.autotune(rs, d, path="fused_bf16")
    print("autotune on long runs:", ctx.autotune_get(rs, "fused_bf16"))
    ids = ids_dev(len(h))
    ctx.classify(rs, d, ids, path="fused_bf16", graph=True)
    torch.cuda.synchronize()
    assert (ids_host(ids) == want).all()
    # predictions chosen at random: the same ids, and the oracle's probe count
    o = tss.TwoStageSearch(rules, tuples, tor)
    sub = np.arange(0, len(h), 20)
    pred = np.random.default_rng(2).integers(0, len(tuples), len(sub))
    ids = ids_dev(len(sub))
    st = ctx.search(rs, to_dev(h[sub]), torch.tensor(pred, dtype=torch.int32, device="cuda"), ids, stats=True)
    assert (ids_host(ids) == want[sub]).all()
    assert st["probes"] == sum(o.search(h[k], int(pred[i]))[1] for i, k in enumerate(sub))
    ctx.unload_ruleset(rs)
