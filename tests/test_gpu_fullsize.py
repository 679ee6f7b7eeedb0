"""Parity at the benchmark's full sizes, in the launch configuration bench.py times, on every
packet: the oracle classifies the whole trace and each path's ids must equal it."""
import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import ids_dev, ids_host, to_dev
from oracle import classify as oc

pytestmark = pytest.mark.gpu


def quick_model(ctx, rs, rules, seed):
    h = wl.gen_trace(rules, [("inside", 16384)], seed)
    blob, _ = ctx.train(rs, h, N=512, blocks=6, batch=8192, epochs=1, max_rounds=1, alpha=10, holdout=0.05, seed=seed)
    ctx.load_model(rs, blob)


def test_512k_rules_16m_packets_every_packet():
    """Config 2: 524,288 rules, 16,777,216 packets; fused BF16 and FP8 (graph replay, as timed),
    the search alone, and the plain FP32 form."""
    rules = wl.rules_for_config(2)
    trace = wl.trace_for_config(2, rules)
    want = oc.classify(rules, trace)
    with tg.Context(0) as ctx:
        rs = ctx.load_ruleset(rules)
        quick_model(ctx, rs, rules, 2)
        d = to_dev(trace)
        for path in ("fused_bf16", "fused_fp8", "no_nn", "plain_fp32"):
            ids = ids_dev(len(trace))
            graph = path != "plain_fp32"
            for _ in range(2 if graph else 1):  # eager + captured, then a replay
                ctx.classify(rs, d, ids, path=path, graph=graph)
            if graph:
                ids.fill_(-1)
                ctx.classify(rs, d, ids, path=path, graph=True)
            torch.cuda.synchronize()
            got = ids_host(ids)
            bad = np.flatnonzero(got != want)
            assert len(bad) == 0, (path, len(bad), bad[:5].tolist())


def test_64k_skewed_every_packet_and_flips():
    """Config 1: 65,536 skewed rules, 1M Zipf(1.0) packets; FP32 and BF16 (and FP8) networks give
    the oracle's ids on every packet; their tuple predictions may differ, and the flips are counted."""
    rules = wl.rules_for_config(1)
    trace = wl.trace_for_config(1, rules)
    want = oc.classify(rules, trace)
    with tg.Context(0) as ctx:
        rs = ctx.load_ruleset(rules)
        quick_model(ctx, rs, rules, 1)
        d = to_dev(trace)
        for path in ("plain_fp32", "staged_bf16", "fused_bf16", "fused_fp8"):
            ids = ids_dev(len(trace))
            st = ctx.classify(rs, d, ids, path=path, stats=True)
            assert (ids_host(ids) == want).all(), path
            assert st["packets"] == len(trace)
        t = {}
        for name, prec in (("fp32", tg.FP32), ("bf16", tg.BF16), ("fp8", tg.FP8)):
            t[name] = torch.zeros(len(trace), dtype=torch.int32, device="cuda")
            ctx.infer(rs, d, None, t[name], precision=prec)
        torch.cuda.synchronize()
        flips = {k: float((t[k] != t["fp32"]).float().mean()) for k in ("bf16", "fp8")}
        print("config 1 argmax flips vs FP32:", flips)
        assert flips["bf16"] < 0.1, flips  # precision-induced mispredictions are counted, ids stay exact


def test_1m_rules_update_stream_every_batch():
    """Config 4: 1,048,576 rules under an operation stream of 10 % inserts / deletes and lookup
    batches of 4k-256k packets (graph-captured classification, as timed); after every update epoch,
    every packet of the lookup batch is checked against the oracle re-run on the live rules."""
    rules = wl.rules_for_config(4)
    ops = wl.gen_update_stream(rules, 60, seed=3)
    inserted = np.array([op[1] for op in ops if op[0] == "insert"], dtype=wl.RULE_DTYPE)
    pool = np.concatenate([rules, inserted])           # every rule that is ever live
    where = {int(i): k for k, i in enumerate(pool["id"])}
    alive = np.zeros(len(pool), dtype=bool)
    alive[:len(rules)] = True
    with tg.Context(0) as ctx:
        rs = ctx.load_ruleset(rules)
        quick_model(ctx, rs, rules, 4)
        batches = updates = 0
        d_buf = torch.zeros((262_144, 16), dtype=torch.uint8, device="cuda")
        ids = ids_dev(262_144)
        cur = rules
        for op in ops:
            if op[0] in ("insert", "delete"):
                if op[0] == "insert":
                    ctx.insert_rule(rs, op[1])
                    alive[where[int(op[1]["id"])]] = True
                else:
                    ctx.delete_rule(rs, op[1])
                    alive[where[op[1]]] = False
                cur = pool[alive]
                updates += 1
            else:
                n = op[1]
                h = wl.gen_trace(cur, [("inside", n - n // 2), ("zipf", n // 2, 1.2)], op[2])
                d_buf[:len(h)].copy_(to_dev(h))
                ctx.classify(rs, d_buf[:len(h)], ids[:len(h)], path="fused_bf16", graph=True)
                torch.cuda.synchronize()
                got = ids_host(ids[:len(h)])
                assert (got == oc.classify(cur, h)).all(), batches
                batches += 1
        assert batches >= 40 and updates >= 2


@pytest.mark.parametrize("variant", [None, "split"])
def test_updates_wait_for_classifications_in_flight(variant):
    """A large classification issued on a side stream, then deletes and inserts with no host
    synchronisation: the classification sees the ruleset as it was (every id equals the oracle's
    on the pre-update rules), and one issued after the updates sees the new ruleset. Also for the
    split form, whose search kernel runs after the network kernel on the same stream."""
    rules = wl.rules_for_config(2)
    trace = wl.trace_for_config(2, rules, scale=0.25)
    rng = np.random.default_rng(5)
    with tg.Context(0) as ctx:
        rs = ctx.load_ruleset(rules)
        quick_model(ctx, rs, rules, 6)
        d = to_dev(trace)
        before = oc.classify(rules, trace)
        # the rules the trace hits most often: deleting them changes many answers
        hot = np.unique(before[before != tg.NO_MATCH], return_counts=True)
        victims = hot[0][np.argsort(-hot[1])[:300]]
        fresh = wl.gen_rules(300, 991)
        fresh["id"] += 1 << 22
        fresh["priority"] = rng.integers(0, 1000, len(fresh))
        side = torch.cuda.Stream()
        ids_old = ids_dev(len(trace))
        torch.cuda.synchronize()
        for _ in range(2):
            with torch.cuda.stream(side):
                ctx.classify(rs, d, ids_old, path="fused_bf16", stream=side.cuda_stream, variant=variant)
            for v in victims:
                ctx.delete_rule(rs, int(v))
            for r in fresh:
                ctx.insert_rule(rs, r)
            ids_new = ids_dev(len(trace))
            side.wait_stream(torch.cuda.current_stream())   # the buffer's fill comes first
            with torch.cuda.stream(side):
                ctx.classify(rs, d, ids_new, path="fused_bf16", stream=side.cuda_stream, variant=variant)
            torch.cuda.synchronize()
            assert (ids_host(ids_old) == before).all()
            keep = ~np.isin(rules["id"], victims)
            rules = np.concatenate([rules[keep], fresh])
            before = oc.classify(rules, trace)
            assert (ids_host(ids_new) == before).all()
            # the second round deletes the rules the first one inserted and inserts another set
            victims = fresh["id"].copy()
            fresh = wl.gen_rules(300, 992)
            fresh["id"] += 1 << 23
            fresh["priority"] = rng.integers(0, 1000, len(fresh))
