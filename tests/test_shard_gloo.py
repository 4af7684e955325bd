"""Multi-rank host logic on CPU with the gloo backend (world size 2): every
rank draws its own shard of a workload (weak scaling), the shards are disjoint
and equal to the serial draw of the same instances, and the job time is the
maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    from paper_2512_09058_gb300 import inputs, shard
    idx = list(shard.shard_indices(3, rank))
    b = inputs.make_batch("uneven4096", idx, workers=1)
    sig = torch.tensor([float(b.Q.sum()), float(b.N.sum()), float(idx[0])], dtype=torch.float64)
    gathered = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, sig)
    ms = shard.reduce_time_ms(10.0 * (rank + 1), dist, device="cpu")
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.stack([g.numpy() for g in gathered]))
        np.save(os.path.join(out_dir, "ms.npy"), np.array([ms]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_with_gloo(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    gathered = np.load(tmp_path / "gathered.npy")
    ms = float(np.load(tmp_path / "ms.npy")[0])
    from paper_2512_09058_gb300 import inputs, shard
    for r in range(world):
        ref = inputs.make_batch("uneven4096", list(range(3 * r, 3 * r + 3)), workers=1)
        assert gathered[r][0] == pytest.approx(float(ref.Q.sum()), rel=0, abs=0)
        assert gathered[r][1] == float(ref.N.sum())
        assert gathered[r][2] == 3 * r
    assert ms == 20.0
    assert shard.job_throughput(3, world, ms) == pytest.approx(6 / 0.02)
