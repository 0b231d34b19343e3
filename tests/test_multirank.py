"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

Every rank integrates its own independent instances (weak scaling); the only
cross-rank operations are the harness's: the slowest rank's time and the sum
of the work.  Checked here without a GPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.workload_instances("yig_wire", rank)
    seeds = torch.tensor([I.seed % (1 << 62) for I in w.instances], dtype=torch.int64)
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    ms, work = bench.reduce_over_ranks(dist, "cpu", 10.0 + rank, 1000.0 * (rank + 1))
    q.put((rank, [g.tolist() for g in gathered], ms, work, [I.omega_c for I in w.instances]))
    dist.destroy_process_group()


def test_two_ranks_shard_independent_instances():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, gathered, ms, work, wcs in res:
        assert ms == 11.0            # the slowest rank sets the time
        assert work == 3000.0        # work adds up over ranks
        s0, s1 = set(gathered[0]), set(gathered[1])
        assert len(s0) == 21 and len(s1) == 21 and not (s0 & s1)   # distinct instances per rank
    # the same sweep of cavity frequencies on every rank
    assert res[0][4] == res[1][4]
