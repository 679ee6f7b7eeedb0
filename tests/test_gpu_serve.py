"""Continuous-batching serving over several resident rulesets, memory admission, and the autotuner."""
import time

import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import ids_dev, ids_host, random_params, to_dev
from oracle import classify as oc

pytestmark = pytest.mark.gpu


def load_rulesets(ctx, sizes, seed0=0):
    out = []
    for k, n in enumerate(sizes):
        rules = wl.gen_rules(n, seed0 + k)
        rs = ctx.load_ruleset(rules)
        T = ctx.ruleset_info(rs)["n_tuples"]
        ctx.load_model(rs, tg.pack_model(random_params(np.random.default_rng(k), C=T)))
        out.append((rs, rules))
    return out


def test_requests_same_alone_and_in_the_mix():
    rng = np.random.default_rng(0)
    with tg.Context(0) as ctx:
        sets = load_rulesets(ctx, [1000, 4000, 16000, 65536])
        reqs = []
        for k in range(60):
            which = int(rng.integers(0, len(sets)))
            n = int(np.exp(rng.uniform(0, np.log(20001))))
            rules = sets[which][1]
            h = wl.gen_trace(rules, [("inside", n - n // 10), ("random", n // 10)], 100 + k)
            reqs.append((which, h))
        # alone: one synchronous device call per request
        alone = []
        for which, h in reqs:
            ids = ids_dev(len(h))
            ctx.classify(sets[which][0], to_dev(h), ids, path="fused_bf16")
            torch.cuda.synchronize()
            alone.append(ids_host(ids).copy())
        # in the mix: all requests submitted with small gaps while others are in flight
        ctx.serve_start(max_inflight=4, max_batch=16384, path="fused_bf16")
        outs, handles = [], []
        for which, h in reqs:
            out = np.full(len(h), 7, dtype=np.uint32)
            outs.append(out)
            handles.append(ctx.serve_submit(sets[which][0], h, out))
            time.sleep(float(rng.uniform(0, 0.002)))
        stats = [ctx.serve_poll(r, wait_ms=20000) for r in handles]
        ctx.serve_stop()
        for k, ((which, h), out, st) in enumerate(zip(reqs, outs, stats)):
            assert st is not None, k
            assert st["submit_s"] <= st["start_s"] <= st["done_s"]
            assert (out == alone[k]).all(), k
            assert (out == oc.classify(sets[which][1], h)).all(), k


def test_memory_admission_caps_slots():
    with tg.Context(0, pool_bytes=256 << 20) as ctx:
        (rs, rules), = load_rulesets(ctx, [2000])
        used0, cap = ctx.memory_usage()
        assert cap == 256 << 20 and used0 < cap
        # 8 slots of 4M packets (80 MB each) cannot all be admitted; the engine starts with fewer
        ctx.serve_start(max_inflight=8, max_batch=1 << 22, path="fused_bf16")
        used1, _ = ctx.memory_usage()
        assert used1 <= cap
        slots = (used1 - used0) // ((1 << 22) * 20)
        assert 1 <= slots < 8
        h = wl.gen_trace(rules, [("inside", 50000)], 4)
        out = np.zeros(len(h), dtype=np.uint32)
        req = ctx.serve_submit(rs, h, out)
        assert ctx.serve_poll(req, wait_ms=20000) is not None
        assert (out == oc.classify(rules, h)).all()
        ctx.serve_stop()
        with pytest.raises(tg.TangError):
            ctx.serve_start(max_inflight=1, max_batch=1 << 30, path="fused_bf16")  # no slot fits


def test_serving_rejects_paths_with_shared_scratch():
    with tg.Context(0) as ctx:
        with pytest.raises(tg.TangError):
            ctx.serve_start(path="plain_fp32")


def test_autotune_keeps_ids_exact():
    with tg.Context(0) as ctx:
        (rs, rules), = load_rulesets(ctx, [20000])
        h = wl.gen_trace(rules, [("inside", 200000)], 8)
        d = to_dev(h)
        want = oc.classify(rules, h)
        for path in ("no_nn", "fused_bf16"):
            ctx.autotune(rs, d, path=path)
            choice = ctx.autotune_get(rs, path)
            assert choice["ms"] > 0
            if path == "fused_bf16":
                assert choice["variant"] in ("1sm", "2sm", "mc2", "mc4", "n256")
            else:
                assert choice["search_threads"] in (128, 256, 512) and choice["search_bps"] in (2, 4, 8, 16)
            ids = ids_dev(len(h))
            ctx.classify(rs, d, ids, path=path, graph=True)
            ctx.classify(rs, d, ids, path=path, graph=True)
            torch.cuda.synchronize()
            assert (ids_host(ids) == want).all(), path


def test_tuned_shapes_restore_in_a_new_context():
    """A launch shape saved from autotune_get and set in a fresh context (a restart) is the one
    the new context reports and runs, with exact ids; values out of range are refused."""
    saved = {}
    with tg.Context(0) as ctx:
        (rs, rules), = load_rulesets(ctx, [20000])
        h = wl.gen_trace(rules, [("inside", 100000)], 9)
        d = to_dev(h)
        for path in ("no_nn", "fused_bf16"):
            ctx.autotune(rs, d, path=path)
            saved[path] = ctx.autotune_get(rs, path)
    with tg.Context(0) as ctx:
        (rs, rules2), = load_rulesets(ctx, [20000])
        assert (rules2 == rules).all()
        d = to_dev(h)
        want = oc.classify(rules, h)
        for path, c in saved.items():
            ctx.autotune_set(rs, path, variant=c["variant"], grid=c["grid"], search_threads=c["search_threads"],
                             search_bps=c["search_bps"])
            got = ctx.autotune_get(rs, path)
            assert {k: got[k] for k in ("variant", "grid", "search_threads", "search_bps")} == \
                   {k: c[k] for k in ("variant", "grid", "search_threads", "search_bps")}
            ids = ids_dev(len(h))
            ctx.classify(rs, d, ids, path=path, graph=True)
            torch.cuda.synchronize()
            assert (ids_host(ids) == want).all(), path
        for bad in ({"variant": 6}, {"grid": 100000}, {"search_threads": 96}, {"search_threads": 512, "search_bps": 8}):
            with pytest.raises(tg.TangError):
                ctx.autotune_set(rs, "no_nn", **bad)
