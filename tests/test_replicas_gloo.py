"""The multi-GPU path is replicas only: each rank solves its own right-hand
sides and the job reports the slowest rank's time.  The reduction and the
per-rank inputs are checked with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [1000.0, 3000.0][rank]           # rank 1 is the slow one
    ms_step, value = bench.replica_reduce(ms, 2, 12, world, dist, "cpu")
    out[rank] = (ms_step, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms_step, value = res[r]
        assert ms_step == 1500.0                    # max over ranks, per step
        assert abs(value - 1.5 / 24) < 1e-15        # 12 x 2 solves in that time


def test_ranks_get_distinct_sources(monkeypatch):
    """Every rank draws its own seeded right-hand sides (no two ranks repeat a
    system), reproducibly."""
    import bench
    import paper_1205_2933_gb300.inputs as I
    monkeypatch.setattr(bench, "DIMS", (2, 2, 2, 2))
    monkeypatch.setattr(bench, "LS", 2)
    monkeypatch.setattr(bench.I, "heatbath_links", lambda dims, *a, **k: I.unit_links(dims))
    _, b0 = bench.gen_inputs(3, rank=0)
    _, b1 = bench.gen_inputs(3, rank=1)
    _, b0again = bench.gen_inputs(3, rank=0)
    assert np.array_equal(b0, b0again)
    for i in range(3):
        for j in range(3):
            assert not np.allclose(b0[i], b1[j])
