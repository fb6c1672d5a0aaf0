"""bench.py's multi-rank host logic on two gloo ranks (CPU): barriers,
max-over-ranks timing, whole-job sums, gathered latency samples, and the
reference arm doing no work off rank 0."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    R = bench.Replicas(backend="gloo")
    R.barrier()
    seconds = 2.0 + rank          # rank 1 is the slower replica
    t = R.max(seconds)
    units = R.sum(100.0 * (rank + 1))
    lat = R.gather([10.0 * rank + 1, 10.0 * rank + 2])
    rate = bench.whole_job_rate(50.0, R.world, t)
    # the reference arm returns at once on every rank but 0
    ref = "skipped"
    if rank != 0:
        bench.reference_arm(None)
        ref = "returned"
    R.close()
    q.put((rank, t, units, lat, rate, ref))


@pytest.mark.timeout(120)
def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, t, units, lat, rate, ref = q.get(timeout=100)
        out[rank] = (t, units, lat, rate, ref)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank in range(world):
        t, units, lat, rate, ref = out[rank]
        assert t == 3.0                       # max over ranks
        assert units == 300.0                 # sum over ranks
        assert lat == [1.0, 2.0, 11.0, 12.0]  # rank order
        assert rate == pytest.approx(2 * 50.0 / 3.0)
    assert out[1][4] == "returned"


def test_single_process_reductions_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        R = bench.Replicas()
        assert (R.world, R.rank) == (1, 0)
        assert R.max(2.5) == 2.5 and R.sum(4.0) == 4.0 and R.gather([3, 1]) == [3, 1]
        R.barrier()
        R.close()
        assert bench.percentile([1.0, 2.0, 3.0, 4.0, 5.0], 0.5) == 3.0
        assert bench.percentile([1.0, 2.0, 3.0, 4.0, 5.0], 0.99) == 5.0
    finally:
        os.environ.update(env)
