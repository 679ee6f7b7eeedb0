"""The allocation-free classify entry point, called through the C ABI.

Some callers cannot allocate device memory during a call: code running inside a custom allocator
or an allocation hook, processes with a fixed device-memory budget, and loops that cannot absorb
cudaMalloc's synchronisation. tang_classify_noalloc gives them the staged BF16 classification with
its inter-kernel scratch in a static device array. Its ids must equal the oracle's and those of
tang_classify's staged BF16 path, call after call, with the context's memory pool untouched.
This file is collected last so that a failure here cannot hide others.
"""
import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import ids_dev, ids_host, random_params, to_dev
from oracle import classify as oc
from paper_2601_03187_b300._native import lib

pytestmark = pytest.mark.gpu

MAX_PACKETS = 1048576  # TANG_NOALLOC_MAX_PACKETS


def _spread_rules(n, seed):
    """n rules whose SIP / DIP prefix lengths are uniform in 0..32 (hundreds of tuples)."""
    rng = np.random.default_rng(seed)
    rules = wl.gen_rules(n, seed)
    for f in ("sip", "dip"):
        lens = rng.integers(0, 33, n)
        rules[f + "_len"] = lens
        mask = np.where(lens == 0, 0, (0xFFFFFFFF << (32 - lens)) & 0xFFFFFFFF).astype(np.uint64)
        rules[f] = (rules[f].astype(np.uint64) & mask).astype(np.uint32)
    return rules


# config 0 at the paper's width; a 308-tuple ruleset (two output chunks) at width 256
CASES = [("cfg0", 512, 6), ("spread", 256, 2)]


@pytest.mark.parametrize("case", CASES, ids=["cfg0-512x6", "308tuples-256x2"])
def test_noalloc_matches_oracle_and_staged_classify(case):
    which, width, blocks = case
    rules = wl.rules_for_config(0) if which == "cfg0" else _spread_rules(350, 650)
    with tg.Context(0) as ctx:
        rs = ctx.load_ruleset(rules)
        T = ctx.ruleset_info(rs)["n_tuples"]
        ctx.load_model(rs, tg.pack_model(random_params(np.random.default_rng(3), N=width, blocks=blocks, C=T)))
        h = wl.gen_trace(rules, [("inside", 90000), ("random", 10000 + 37)], 9)
        d = to_dev(h)
        n = len(h)
        want = oc.classify(rules, h)
        ref = ids_dev(n)
        ctx.classify(rs, d, ref, path="staged_bf16")
        torch.cuda.synchronize()
        assert (ids_host(ref) == want).all()
        stream = torch.cuda.current_stream().cuda_stream or 1
        used0 = ctx.memory_usage()
        for call in range(2):
            out = ids_dev(n)
            rc = lib.tang_classify_noalloc(ctx.handle, rs, d.data_ptr(), n, out.data_ptr(), stream)
            assert rc == 0, lib.tang_last_error(ctx.handle)
            torch.cuda.synchronize()
            got = ids_host(out)
            assert (got == want).all(), call
            assert (got == ids_host(ref)).all(), call
        assert ctx.memory_usage() == used0          # nothing allocated from the context's pool
        # a batch beyond the static array's capacity is refused, not truncated
        big = lib.tang_classify_noalloc(ctx.handle, rs, d.data_ptr(), MAX_PACKETS + 1, ref.data_ptr(), stream)
        assert big == tg._native.EINVAL
        assert b"exceeds" in lib.tang_last_error(ctx.handle)


def test_noalloc_at_its_maximum_batch():
    rules = wl.rules_for_config(0)
    with tg.Context(0) as ctx:
        rs = ctx.load_ruleset(rules)
        T = ctx.ruleset_info(rs)["n_tuples"]
        ctx.load_model(rs, tg.pack_model(random_params(np.random.default_rng(4), N=512, blocks=6, C=T)))
        h = wl.gen_trace(rules, [("inside", MAX_PACKETS - MAX_PACKETS // 8), ("random", MAX_PACKETS // 8)], 10)
        assert len(h) == MAX_PACKETS
        d = to_dev(h)
        want = oc.classify(rules, h)
        stream = torch.cuda.current_stream().cuda_stream or 1
        used0 = ctx.memory_usage()
        for call in range(2):
            out = ids_dev(MAX_PACKETS)
            rc = lib.tang_classify_noalloc(ctx.handle, rs, d.data_ptr(), MAX_PACKETS, out.data_ptr(), stream)
            assert rc == 0, lib.tang_last_error(ctx.handle)
            torch.cuda.synchronize()
            assert (ids_host(out) == want).all(), call
        assert ctx.memory_usage() == used0
