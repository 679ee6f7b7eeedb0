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


def test_config3_rulesets_every_request():
    """The serving configuration at full size: four resident rulesets of 16k, 64k, 256k and 512k
    rules, Poisson arrivals with batch sizes log-uniform in [1, 65536], paced submission while
    others are in flight; every id of every request equals the oracle's."""
    sizes = [16_384, 65_536, 262_144, 524_288]
    with tg.Context(0) as ctx:
        sets, pools = [], []
        for k, n in enumerate(sizes):
            rules = wl.gen_rules(n, 10 + k)
            rs = ctx.load_ruleset(rules)
            T = ctx.ruleset_info(rs)["n_tuples"]
            ctx.load_model(rs, tg.pack_model(random_params(np.random.default_rng(k), C=T)))
            sets.append((rs, rules))
            pools.append(wl.gen_trace(rules, [("inside", 1 << 17), ("zipf", 1 << 17, 1.2)], 30 + k))
        arrivals = wl.gen_serving_arrivals(400, len(sets), 2000.0, seed=5)
        ctx.serve_start(max_inflight=8, max_batch=262_144, path="fused_bf16")
        outs, handles, reqs = [], [], []
        t0 = time.perf_counter()
        for t_arr, which, size, seed in arrivals:
            delay = t0 + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            off = seed % (len(pools[which]) - size)
            h = pools[which][off:off + size]
            outs.append(np.full(size, 7, dtype=np.uint32))
            reqs.append((which, h))
            handles.append(ctx.serve_submit(sets[which][0], h, outs[-1]))
        for r in handles:
            assert ctx.serve_poll(r, wait_ms=60000) is not None
        info = ctx.serve_info()
        ctx.serve_stop()
        assert info["packets"] == sum(len(h) for _, h in reqs)
        for k in range(len(sets)):
            idx = [i for i, (w, _) in enumerate(reqs) if w == k]
            if not idx:
                continue
            got = np.concatenate([outs[i] for i in idx])
            want = oc.classify(sets[k][1], np.concatenate([reqs[i][1] for i in idx]))
            assert (got == want).all(), sizes[k]


@pytest.mark.parametrize("form", ["tuned", "split"])
def test_requests_same_alone_and_in_the_mix(form):
    """Each request's ids are the same alone and in the mix, and the oracle's. "split": every
    ruleset's fused path set to the two-kernel form, whose search reads the predictions from each
    request's own id buffer, so concurrent slots share no scratch."""
    rng = np.random.default_rng(0)
    with tg.Context(0) as ctx:
        sets = load_rulesets(ctx, [1000, 4000, 16000, 65536])
        if form == "split":
            for rs, _ in sets:
                ctx.autotune_set(rs, "fused_bf16", variant="split")
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


def _serve_wave(ctx, work, max_batch):
    """Submit every (ruleset, rules, headers) request at once, wait, check the ids against the
    oracle, and return the engine's counters."""
    outs, handles = [], []
    for rs, rules, h in work:
        outs.append(np.full(len(h), 7, dtype=np.uint32))
        handles.append(ctx.serve_submit(rs, h, outs[-1]))
    for r in handles:
        assert ctx.serve_poll(r, wait_ms=60000) is not None
    for (rs, rules, h), out in zip(work, outs):
        assert (out == oc.classify(rules, h)).all()
    return ctx.serve_info()


def _wait_released(ctx, timeout_s=2.0):
    t0 = time.time()
    while ctx.serve_info()["slots_admitted"] and time.time() - t0 < timeout_s:
        time.sleep(0.01)
    return ctx.serve_info()["slots_admitted"]


def test_admission_follows_free_memory():
    """Slots are admitted against the pool's free memory when work needs them and given back when
    idle; a large ruleset loaded while the engine runs leaves room for fewer slots, and the engine
    then admits fewer (refusing the rest), with every id equal to the oracle's."""
    rules = wl.rules_for_config(0, n_rules=4000)
    hog_rules = wl.rules_for_config(2, seed=5)
    # sizes from a probe context: the serving context's own use, and the big ruleset's
    with tg.Context(0) as probe:
        rs = probe.load_ruleset(rules)
        T = probe.ruleset_info(rs)["n_tuples"]
        probe.load_model(rs, tg.pack_model(random_params(np.random.default_rng(2), N=256, blocks=2, C=T)))
        u1 = probe.memory_usage()[0]
        probe.load_ruleset(hog_rules)
        hog = probe.memory_usage()[0] - u1
    # free memory F = 1.8 x the big ruleset: F holds 3 slots of S = 0.53 x the ruleset before it
    # is loaded and 1 slot after it (F - ruleset = 1.5 S)
    slot_bytes = int(hog * 0.8 / 1.5)
    max_batch = slot_bytes // 20
    pool = u1 + int(1.8 * hog)
    with tg.Context(0, pool_bytes=pool) as ctx:
        rs = ctx.load_ruleset(rules)
        ctx.load_model(rs, tg.pack_model(random_params(np.random.default_rng(2), N=256, blocks=2, C=T)))
        used0, cap = ctx.memory_usage()
        free1 = cap - used0
        limit1 = min(8, free1 // (20 * max_batch))
        assert limit1 == 3, (free1, max_batch)
        ctx.serve_start(max_inflight=8, max_batch=max_batch, path="fused_bf16")
        assert ctx.memory_usage()[0] == used0          # nothing is admitted before work arrives
        work = [(rs, rules, wl.gen_trace(rules, [("inside", max_batch // 2)], 100 + k)) for k in range(12)]
        info1 = _serve_wave(ctx, work, max_batch)
        assert 2 <= info1["slots_admitted_peak"] <= limit1, info1
        assert _wait_released(ctx) == 0                 # idle slots give their memory back
        assert ctx.memory_usage()[0] == used0
        # mid-serving: the big ruleset takes most of the free memory
        rs2 = ctx.load_ruleset(hog_rules)
        free2 = cap - ctx.memory_usage()[0]
        limit2 = free2 // (20 * max_batch)
        assert limit2 == 1, (free2, max_batch)
        # the peak counter restarts only with the engine; count this wave's refusals
        before = ctx.serve_info()
        work2 = [(rs, rules, wl.gen_trace(rules, [("inside", max_batch // 2)], 200 + k)) for k in range(8)]
        info2 = _serve_wave(ctx, work2, max_batch)
        assert info2["admissions_refused"] > before["admissions_refused"], info2
        assert info2["slots_busy"] == 0
        assert _wait_released(ctx) == 0
        ctx.serve_stop()
        # with the engine restarted, its peak shows the lower limit
        ctx.serve_start(max_inflight=8, max_batch=max_batch, path="fused_bf16")
        info3 = _serve_wave(ctx, work2, max_batch)
        assert info3["slots_admitted_peak"] == 1 and info3["admissions_refused"] >= 1, info3
        ctx.serve_stop()
        ctx.unload_ruleset(rs2)
        with pytest.raises(tg.TangError):
            ctx.serve_start(max_inflight=1, max_batch=1 << 30, path="fused_bf16")  # one slot exceeds the pool


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
                assert choice["variant"] in ("n256", "pair", "split")
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
        for bad in ({"variant": 7}, {"variant": 8}, {"variant": 1}, {"grid": 100000}, {"search_threads": 96},
                    {"search_threads": 512, "search_bps": 8}):
            with pytest.raises(tg.TangError):
                ctx.autotune_set(rs, "no_nn", **bad)
        # the split form exists for the fused paths only
        ctx.autotune_set(rs, "fused_fp8", variant="split")
        assert ctx.autotune_get(rs, "fused_fp8")["variant"] == "split"
        with pytest.raises(tg.TangError):
            ctx.autotune_set(rs, "staged_bf16", variant="split")
