"""Host logic of the replicas-only multi-GPU bench, on CPU with two gloo
ranks: the job time is the slowest rank's, the work the sum over ranks, and
each replica draws its own seeded batch."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    from paper_2403_16341_gb300 import inputs as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, solved = bench.reduce_over_ranks(dist, 10.0 + 5.0 * rank, 100 + rank, torch.device("cpu"))
    b = I.cubic_batch(8, 16, seed=bench.shard_seed(rank), config_id=1, b_half_width=5.0)
    digest = torch.tensor([float(b.params.sum())], dtype=torch.float64)
    gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, digest)
    out[rank] = (ms, solved, [float(g.item()) for g in gathered])
    dist.destroy_process_group()


def test_two_replicas_reduce_time_and_work():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            ms, solved, digests = out[r]
            assert ms == 15.0 and solved == 201
            assert not np.isclose(digests[0], digests[1])  # distinct seeded batches
