"""Host logic of bench.py on several GPUs, exercised with two gloo ranks on CPU.

bench.py under torchrun runs one replica of the workload per GPU (the chains
are independent Markov chains: no data exchange).  Each rank holds its own
block of global chain ids, the reported step time is the maximum over ranks
and the value counts the updates of every rank.  No GPU is needed for any of
this."""
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
        q.put((rank, slow, bench.rank_chain_offset(rank), bench.job_value(world, slow)))
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
    for rank, slow, offset, value in out:
        assert slow == max(ms)  # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * bench.updates_per_sweep(bench.W["chains"]) / 0.6555)
    # the ranks' chain blocks tile 0 .. 2C - 1 without overlap
    assert [o[2] for o in out] == [0, bench.W["chains"]]


def test_ranks_sample_independent_chains():
    """Local chain 3 of rank 1 is global chain C + 3: its initial field (the
    Philox counter carries the global id) differs from rank 0's chain 3, so
    the replicas are independent, and equals the field that chain has in a
    single run of 2C chains."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import dqmc as o
    f0 = o.initial_field(0, bench.rank_chain_offset(0) + 3, 16, 8)
    f1 = o.initial_field(0, bench.rank_chain_offset(1) + 3, 16, 8)
    assert np.array_equal(f1, o.initial_field(0, bench.W["chains"] + 3, 16, 8))
    assert f0.shape == f1.shape
    assert not np.array_equal(f0, f1)
    # about half of the spins differ, as for independent fields
    assert 0.3 < np.mean(f0 != f1) < 0.7
