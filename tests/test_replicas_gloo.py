"""The multi-GPU path is replicas only (no data-path collective): each rank runs the whole step on
its own GPU, and bench.py's host logic joins them with a barrier and a max over ranks of the
timed seconds.  This checks that logic with two CPU ranks on the gloo backend (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), ICWF_BENCH_GLOO="1")
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_init()
    bench.barrier(w)
    slowest = bench.max_over_ranks(1.0 + r, w)      # rank 1 is the slow one: 2 s
    rate = bench.whole_job_rate(w, 1024 * 10, slowest)
    q.put((r, w, local, slowest, rate))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_barrier_and_max():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=90) for _ in range(ws))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, local, slowest, rate in out:
        assert w == 2 and local == r
        assert slowest == 2.0                      # the max over ranks, seen by every rank
        assert rate == 2 * 1024 * 10 / 2.0          # all ranks' units over the slowest time


def test_single_process_needs_no_process_group():
    import bench
    assert bench.dist_init() == (0, 1, 0) or os.environ.get("WORLD_SIZE", "1") != "1"
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1, 100, 2.0) == 50.0
