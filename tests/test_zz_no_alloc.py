"""The allocation-free classify entry point, called through the C ABI.

Some callers cannot allocate device memory during a call (custom allocators, processes with a
fixed device-memory budget, loops that cannot absorb cudaMalloc's synchronisation).
tang_classify_noalloc gives them the staged BF16 classification with its inter-kernel scratch in
a static device array. This file is collected last so that a failure here cannot hide others.
"""
import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import ids_dev, ids_host, random_params, to_dev
from paper_2601_03187_b300._native import lib

pytestmark = pytest.mark.gpu


def test_noalloc_matches_staged_classify_on_two_calls():
    rules = wl.rules_for_config(0)
    with tg.Context(0) as ctx:
        rs = ctx.load_ruleset(rules)
        T = ctx.ruleset_info(rs)["n_tuples"]
        ctx.load_model(rs, tg.pack_model(random_params(np.random.default_rng(3), C=T)))
        h = wl.trace_for_config(0, rules, seed=9)
        d = to_dev(h)
        n = len(h)
        ref = ids_dev(n)
        ctx.classify(rs, d, ref, path="staged_bf16")
        torch.cuda.synchronize()
        want = ids_host(ref)
        stream = torch.cuda.current_stream().cuda_stream or 1
        for call in range(2):
            out = ids_dev(n)
            rc = lib.tang_classify_noalloc(ctx.handle, rs, d.data_ptr(), n, out.data_ptr(), stream)
            assert rc == 0, lib.tang_last_error(ctx.handle)
            torch.cuda.synchronize()
            assert (ids_host(out) == want).all(), call
        # a batch beyond the static array's capacity is refused, not truncated
        big = tg._native.lib.tang_classify_noalloc(ctx.handle, rs, d.data_ptr(), 1048577, ref.data_ptr(), stream)
        assert big == tg._native.EINVAL
        assert b"exceeds" in lib.tang_last_error(ctx.handle)
