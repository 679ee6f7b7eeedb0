"""Failure handling without faulting the GPU: a bounded device wait that runs out is reported as
TANG_ETIMEOUT and leaves the context usable; memory admission refuses what the pool cannot hold;
malformed input is refused on the host. Checkpointing a ruleset: the exported live rules reload
into the same classifier."""
import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import ids_dev, ids_host, to_dev
from oracle import classify as oc

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_survives():
    with tg.Context(0) as ctx:
        for limit in (20, 100):
            rc, ms = ctx.selftest_wait_timeout(limit)
            assert rc == tg._native.ETIMEOUT
            # the first warp gave up at its limit; the second left on the abort flag long before 10 s
            assert limit * 0.9 <= ms < limit + 1000, (limit, ms)
        rules = wl.rules_for_config(0)
        rs = ctx.load_ruleset(rules)
        h = wl.trace_for_config(0, rules, seed=2)[:5000]
        ids = ids_dev(len(h))
        st = ctx.classify(rs, to_dev(h), ids, path="no_nn", stats=True)  # synchronising: reports OK
        assert st["packets"] == len(h)
        assert (ids_host(ids) == oc.classify(rules, h)).all()
        assert ctx.selftest_wait_timeout(0)[0] == tg._native.EINVAL


def test_memory_admission_and_host_validation():
    rules = wl.rules_for_config(0, n_rules=4096)
    with tg.Context(0, pool_bytes=8 << 20) as ctx:
        with pytest.raises(tg.TangError) as e:
            ctx.load_ruleset(wl.gen_rules(200000, 5))  # its tables do not fit in 8 MB
        assert e.value.code == tg._native.ENOMEM
        rs = ctx.load_ruleset(rules)  # a small one still does
        used, cap = ctx.memory_usage()
        assert 0 < used <= cap == 8 << 20
        bad = rules[:10].copy()
        bad["sp_lo"][3], bad["sp_hi"][3] = 9, 8
        with pytest.raises(tg.TangError) as e:
            ctx.load_ruleset(bad)
        assert e.value.code == tg._native.EINVAL
        with pytest.raises(tg.TangError) as e:
            ctx.delete_rule(rs, 10 ** 9)
        assert e.value.code == tg._native.ENOTFOUND
        with pytest.raises(tg.TangError) as e:
            ctx.insert_rule(rs, rules[0])
        assert e.value.code == tg._native.EEXIST


def test_export_reload_round_trip():
    with tg.Context(0) as ctx:
        rules = wl.rules_for_config(0, n_rules=3000)
        rs = ctx.load_ruleset(rules)
        rng = np.random.default_rng(3)
        live = {int(r["id"]): r.copy() for r in rules}
        for rid in rng.choice(rules["id"], 500, replace=False):
            ctx.delete_rule(rs, int(rid))
            del live[int(rid)]
        fresh = wl.gen_rules(400, 9, first_id=10 ** 6)
        fresh["sip_len"][:50] = 12  # lengths without a tuple: restricted insertion
        fresh["sip"][:50] &= np.uint32(0xFFF00000)
        fresh["priority"] = rng.integers(0, 3000, 400)
        for r in fresh:
            ctx.insert_rule(rs, r)
            live[int(r["id"])] = r
        exp = ctx.export_rules(rs)
        cur = np.array(list(live.values()), dtype=wl.RULE_DTYPE)
        order = np.lexsort((cur["id"], cur["priority"]))
        assert len(exp) == len(cur)
        for f in ("sip_len", "dip_len", "sp_lo", "sp_hi", "dp_lo", "dp_hi", "proto_wild", "priority", "id"):
            assert (exp[f] == cur[f][order]).all(), f
        assert (exp["sip"] == cur["sip"][order]).all() and (exp["dip"] == cur["dip"][order]).all()
        rs2 = ctx.load_ruleset(exp)
        h = wl.gen_trace(cur, [("inside", 20000), ("random", 2000)], 4)
        d = to_dev(h)
        a, b = ids_dev(len(h)), ids_dev(len(h))
        ctx.classify(rs, d, a, path="no_nn")
        ctx.classify(rs2, d, b, path="no_nn")
        torch.cuda.synchronize()
        want = oc.classify(cur, h)
        assert (ids_host(a) == want).all() and (ids_host(b) == want).all()
