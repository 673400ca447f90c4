"""Multi-process path of the benchmark on CPU (gloo, world size 2).

The GN step does not shard: N GPUs run N independent replicas, each fitting its
own seeded profile, and the reported time is the slowest rank's.  This checks
the host-side pieces of that path: distinct per-rank inputs, identical shapes,
and the max-over-ranks reduction.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.replica_workload("ccf_stable", rank)
    fits = bench.replica_workload("batched", rank)
    ms = bench.max_over_ranks(10.0 + rank, "cpu")
    out[rank] = (w.theta[:8].copy(), w.y[0, -8:].copy(), w.theta.shape, ms, len(fits), fits[0].lam)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_replicas_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    a, b = out[0], out[1]
    assert a[2] == b[2]                      # same architecture on every rank
    assert not np.array_equal(a[0], b[0])    # ... but each rank's own seeded initialisation
    assert not np.array_equal(a[1], b[1])    # ... and its own collocation points
    assert a[3] == b[3] == 11.0              # every rank reports the slowest rank's time
    assert a[4] == b[4] == 64 and a[5] != b[5]


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
