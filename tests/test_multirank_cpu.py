"""The multi-GPU path (replicas): each rank solves its own shard and the job
reports the max-over-ranks step time and the summed KKT solves.  Covered on
CPU with world_size 2 over gloo (no GPU, no kernels)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2506_07823_b300 import synth
    ms, kkt = bench.aggregate(10.0 + rank, 100.0 * (rank + 1), torch.device("cpu"))
    # shards: distinct problems per rank, identical problems for equal seeds
    insts, _, Nv, _, x0 = synth.srbd_batch(4, seed=bench.rank_seed(rank, 4), Ns_choices=bench.HORIZONS)
    gathered = [None] * world
    dist.all_gather_object(gathered, x0.tolist())
    out[rank] = (ms, kkt, gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_and_sharding():
    ctx = tmp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms, kkt, gathered = out[r]
        assert ms == 11.0            # max over ranks
        assert kkt == 300.0          # sum over ranks
        a, b = np.asarray(gathered[0]), np.asarray(gathered[1])
        assert a.shape == b.shape and not np.allclose(a, b)


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate(3.5, 7.0, torch.device("cpu")) == (3.5, 7.0)
