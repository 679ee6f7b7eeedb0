"""The checked build (TANG_CHECKED): every table index the search forms is tested before the
access. Run the GPU suite against it with TANG_LIBRARY=.../libtang_checked.so; no index is then
out of range. This file also makes the check fire on purpose, with the descriptor's pool size
narrowed so that every rule index counts as out of range while the memory stays allocated, and
checks that the error is reported, that nothing else broke and that the real size restores exact
results. Against other builds it is skipped."""
import numpy as np
import pytest
import torch

import paper_2601_03187_b300 as tg
import workloads as wl
from gpu_util import ids_dev, ids_host, random_params, to_dev
from oracle import classify as oc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not tg.checked_build(), reason="needs the TANG_CHECKED build of the library")]


def test_out_of_range_index_is_reported_and_skipped():
    ctx = tg.Context(0)
    rules = wl.rules_for_config(0)
    rs = ctx.load_ruleset(rules)
    T = ctx.ruleset_info(rs)["n_tuples"]
    ctx.load_model(rs, tg.pack_model(random_params(np.random.default_rng(5), C=T), np.full(13, 8.0, np.float32)))
    h = wl.trace_for_config(0, rules, seed=21)[:20000]
    want = oc.classify(rules, h)
    d = to_dev(h)
    for path in ("no_nn", "fused_bf16", "staged_bf16"):
        ids = ids_dev(len(h))
        ctx.classify(rs, d, ids, path=path, stats=True)
        assert (ids_host(ids) == want).all(), path
        ctx.debug_set_pool_view(rs, 0)
        with pytest.raises(tg.TangError) as e:
            ctx.classify(rs, d, ids_dev(len(h)), path=path, stats=True)
        assert e.value.code == -5 and "out of range" in str(e.value), path  # TANG_EDEVICE
        ctx.debug_set_pool_view(rs, None)
        ids = ids_dev(len(h))
        ctx.classify(rs, d, ids, path=path, stats=True)
        torch.cuda.synchronize()
        assert (ids_host(ids) == want).all(), path
    ctx.close()
