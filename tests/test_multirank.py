"""Host logic of bench.py on several GPUs, exercised with two gloo ranks on CPU.

bench.py under torchrun runs one replica of the workload per GPU (the chains
are independent Markov chains: no data exchange).  Each rank seeds its own
chains, the reported step time is the maximum over ranks and the value counts
the updates of every rank.  No GPU is needed for any of this."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ms, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        slow = bench.max_over_ranks(ms[rank], dist, "cpu")
        q.put((rank, slow, bench.rank_seed(rank), bench.job_value(world, slow)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_the_whole_job():
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ms = [640.0, 655.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, seed, value in out:
        assert slow == max(ms)  # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * bench.updates_per_sweep(bench.W["chains"]) / 0.6555)
    seeds = [o[2] for o in out]
    assert len(set(seeds)) == 2


def test_ranks_sample_independent_chains():
    """Different rank seeds give different initial fields for the same chain
    index (the Philox key differs), so the replicas are independent."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import dqmc as o
    f0 = o.initial_field(bench.rank_seed(0), 3, 16, 8)
    f1 = o.initial_field(bench.rank_seed(1), 3, 16, 8)
    assert f0.shape == f1.shape
    assert not np.array_equal(f0, f1)
    # about half of the spins differ, as for independent fields
    assert 0.3 < np.mean(f0 != f1) < 0.7
