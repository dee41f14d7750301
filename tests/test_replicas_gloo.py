"""Multi-process host logic of the replica runs (one process per GPU, no data
exchange): two gloo ranks on CPU check the barrier, the max-over-ranks time and
sum-over-ranks work that the benchmark reports, and that each rank draws its
own workload replicate."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist

    from paper_1403_4099_gb300 import runtime, synth
    r = runtime.ranks_from_env()
    assert (r.rank, r.world, r.local) == (rank, world, rank)
    runtime.init_dist(r, "gloo")
    try:
        runtime.barrier(r)
        # uneven per-rank time and work: the job takes the slowest rank's time
        # and the sum of the work
        secs, units = runtime.aggregate(r, 1.0 + 0.5 * rank, 100.0 * (rank + 1))
        # each rank's replicate of the workload is its own seeded draw
        pl = synth.small16(replicate=r.rank)
        digest = torch.tensor([float(np.abs(pl.R).sum())], dtype=torch.float64)
        allv = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(allv, digest)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([secs, units] + [float(v.item()) for v in allv]))
        runtime.barrier(r)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate_gloo(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    port = _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"r{k}.npy") for k in range(world)]
    for v in res:
        assert v[0] == pytest.approx(1.5)          # max of 1.0, 1.5
        assert v[1] == pytest.approx(300.0)        # 100 + 200
        assert v[2] != v[3]                        # replicates differ
    np.testing.assert_array_equal(res[0], res[1])  # every rank sees the same totals


def test_single_rank_aggregate_is_identity():
    from paper_1403_4099_gb300 import runtime
    r = runtime.Ranks(0, 1, 0)
    assert runtime.aggregate(r, 2.5, 7.0) == (2.5, 7.0)
    runtime.barrier(r)  # no process group needed at world size 1
