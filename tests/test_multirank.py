"""The bench's multi-rank host logic on CPU: two gloo ranks, as torchrun launches them.

Packets are independent and every rank holds the whole ruleset, so N > 1 runs N independent
replicas with no collective on the data path. What ranks share is the timing: a barrier on both
sides of the timed region, the slowest rank's time as the job's, the whole job's packets over
that time as the value, and a reference arm that only rank 0 runs."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "TANG_BENCH_BACKEND": "gloo"})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    w, r, local = bench.dist_setup()
    res = {"world": w, "rank": r, "local": local, "backend": dist.get_backend()}
    # rank r "took" 1 + r seconds: every rank must report the slowest rank's time
    res["dt_max"] = bench.max_over_ranks(1.0 + r, w)
    res["value"] = bench.job_mpkts(1_000_000, 3, res["dt_max"], w)
    bench.barrier(w)

    class Args:
        steps, warmup = 1, 0

    buf = io.StringIO()
    with redirect_stdout(buf):
        if r != 0:
            bench.run_reference(Args, w, r)  # ranks other than 0 do no work and print nothing
    res["reference_output"] = buf.getvalue()
    bench.barrier(w)
    dist.destroy_process_group()
    out.put(res)


def test_two_gloo_ranks_time_and_aggregate_as_torchrun_would():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda d: d["rank"])
    assert [d["rank"] for d in res] == [0, 1] and all(d["world"] == 2 for d in res)
    assert all(d["backend"] == "gloo" for d in res)
    # the job's time is the slowest rank's, seen identically by both ranks
    assert all(d["dt_max"] == 2.0 for d in res)
    # whole-job throughput: 2 ranks x 3 steps x 1M packets over 2 s
    assert all(abs(d["value"] - 3.0) < 1e-12 for d in res)
    assert res[1]["reference_output"] == ""


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.job_mpkts(16_777_216, 10, 0.8, 1) == 16_777_216 * 10 / 0.8 / 1e6
    bench.barrier(1)
