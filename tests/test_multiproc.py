"""The N > 1 path on CPU: two gloo ranks, each with its own seeded batch,
no data-path collective, a barrier and a max-reduction of the time."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle
    from paper_2607_28897_gb300 import inputs, ranks

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, _, w = ranks.world()
    a = inputs.limbs(ranks.rank_seed(5, r), 4, 32)
    b = inputs.limbs(ranks.rank_seed(6, r), 4, 32)
    p = oracle.batch_mul(a, b)  # each rank's own work, no collective
    dist.barrier()
    t = ranks.max_over_ranks(1.0 + r, dist)
    out[r] = (int(a[0, 0]), int(p[0, 0]), t, w)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp

    import oracle

    oracle.build()
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0][3] == out[1][3] == 2
    assert out[0][0] != out[1][0]  # disjoint seeded batches
    assert out[0][2] == out[1][2] == 2.0  # max over ranks
