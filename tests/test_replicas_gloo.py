"""The multi-rank path of bench.py on CPU: world_size 2 over gloo.  The method does not
shard (each rank steps its own independent lattice), so the only cross-rank work is the
benchmark bookkeeping: distinct replica seeds, the slowest rank's time, the whole-job rate."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import time

    import torch
    import torch.distributed as dist

    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L = oracle.Lattice(8, 8, seed=bench.replica_seed(42, rank))
    L.set_params(1e-4, 0.01, 0.8, 1.0, 1.0, oracle.NOISE_LW)
    t0 = time.perf_counter()
    L.step(5 + 5 * rank)                         # the ranks take different times
    ms = (time.perf_counter() - t0) * 1e3
    ms_max = bench.max_over_ranks(dist, ms, "cpu")
    mine = torch.tensor([float(np.abs(L.f - L.model.fbar()[:, None, None]).sum())], dtype=torch.float64)
    everyone = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(everyone, mine)
    q.put((rank, ms, ms_max, bench.whole_job_mlups(world, 64, 10, ms_max), [float(e) for e in everyone]))
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ms = [o[1] for o in out]
    for rank, _, ms_max, rate, sums in out:
        assert ms_max == pytest.approx(max(ms))              # every rank sees the slowest time
        assert rate == pytest.approx(2 * 64 * 10 / (max(ms) / 1e3) / 1e6)
        assert sums[0] != sums[1]                           # independent replicas
