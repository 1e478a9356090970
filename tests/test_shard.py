"""Multi-rank host logic on CPU (gloo, world size 2): packet-id shards cover
the job without overlap, timings reduce by max, tallies by sum."""
import os

import pytest

from paper_2608_09340_gb300 import shard


def test_step_ranges_partition_the_job():
    world, per, steps = 3, 7, 5
    seen = []
    for s in range(steps):
        for r in range(world):
            lo, n = shard.step_range(s, r, world, per, first=11)
            seen.extend(range(lo, lo + n))
    assert sorted(seen) == list(range(11, 11 + world * per * steps))
    with pytest.raises(ValueError):
        shard.step_range(0, 3, 3, 1)


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = shard.max_over_ranks(1.5 + rank)
        t = torch.tensor([rank + 1.0, 10.0 * rank], dtype=torch.float64)
        shard.sum_over_ranks(t)
        q.put((rank, m, t.tolist()))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, t in out:
        assert m == 2.5
        assert t == [3.0, 10.0]


def _oracle_rank(rank, world, port, q):
    """One rank of a sharded job, with the FP64 oracle standing in for the
    device walk: run this rank's packet-id shards, then the tally exchange."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = W.slab(tau0=300.0, n_packets=0, bins=(-20.0, 20.0, 40), tallies=("scatmap",))
        spec = np.zeros(42, dtype=np.int64)
        scat = np.zeros(p.ncell, dtype=np.int64)
        for step in range(3):
            lo, n = shard.step_range(step, rank, world, 50)
            r = oracle.run(p, n=n, first=lo, nthreads=1)
            spec += r["spec_c"].astype(np.int64)
            scat += r["scat"].astype(np.int64)
        ts = [torch.from_numpy(spec), torch.from_numpy(scat)]
        shard.reduce_tallies(ts)
        q.put((rank, ts[0].tolist(), ts[1].tolist()))
    finally:
        dist.destroy_process_group()


def test_sharded_job_equals_one_process():
    """Two gloo ranks, three steps of 50 packets each: after the exchange,
    both ranks hold exactly the tallies of one process running all 300 ids."""
    import socket
    import numpy as np
    import torch.multiprocessing as mp
    import oracle
    import workloads as W
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    p = W.slab(tau0=300.0, n_packets=0, bins=(-20.0, 20.0, 40), tallies=("scatmap",))
    ref = oracle.run(p, n=300, first=0, nthreads=2)
    for rank, spec, scat in out:
        assert spec == ref["spec_c"].astype(np.int64).tolist()
        assert scat == ref["scat"].astype(np.int64).tolist()
