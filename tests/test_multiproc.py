"""The N > 1 paths on CPU (gloo ranks; every GPU call here gets one GPU):

* weak scaling: each rank its own seeded batch, no data-path collective, a
  barrier and a max-reduction of the time;
* one ragged batch split over ranks by estimated cost (ranks.partition):
  each rank computes its share, rank 0 gathers the results, and they equal
  the results of the whole batch computed by one rank."""
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


def _init(rank, world, port):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _worker(rank, world, port, out):
    import oracle
    from paper_2607_28897_gb300 import inputs, ranks

    dist = _init(rank, world, port)
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


def _run_ops(ops, pool, nout):
    """The oracle on every operation of a batch, into an output pool."""
    import oracle

    out = np.zeros(nout, dtype=np.uint64)
    for o in ops:
        a = pool[o["a"]:o["a"] + o["na"]]
        b = pool[o["b"]:o["b"] + o["nb"]]
        if o["op"] in (1, 2):
            r, _ = (oracle.add if o["op"] == 1 else oracle.sub)(a, b)
            out[o["o1"]:o["o1"] + r.size] = r
        elif o["op"] == 3:
            r = oracle.mul(a, b)
            out[o["o1"]:o["o1"] + r.size] = r
        else:
            q, r, _ = oracle.divmod_(a, b)
            out[o["o1"]:o["o1"] + q.size] = q
            out[o["o2"]:o["o2"] + r.size] = r
    return out


def _batch():
    from paper_2607_28897_gb300 import inputs

    ops, nin, nout = inputs.ragged_ops(61, 90, min_limbs=4, max_limbs=300)
    return ops, inputs.ragged_pool(62, ops, nin), nout


def _partition_worker(rank, world, port, out):
    from paper_2607_28897_gb300 import ranks

    dist = _init(rank, world, port)
    ops, pool, nout = _batch()
    parts = ranks.partition(ops, world)  # the same split on every rank, no exchange
    sub, sub_pool, sub_nout, out_map = ranks.sub_batch(ops, parts[rank], pool)
    mine = _run_ops(sub, sub_pool, sub_nout)
    gathered = [None] * world if rank == 0 else None
    dist.gather_object((mine, out_map), gathered, dst=0)
    if rank == 0:
        full = np.zeros(nout, dtype=np.uint64)
        for res, omap in gathered:
            for o_orig, o_sub, n in omap:
                full[o_orig:o_orig + n] = res[o_sub:o_sub + n]
        out["full"] = full.tobytes()
        out["loads"] = [float(ranks.op_cost(ops[p]).sum()) for p in parts]
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_batch_equals_single_rank():
    import torch.multiprocessing as mp

    import oracle
    from paper_2607_28897_gb300 import ranks

    oracle.build()
    ops, pool, nout = _batch()
    parts = ranks.partition(ops, 2)
    assert sorted(np.concatenate(parts).tolist()) == list(range(len(ops)))
    cost = ranks.op_cost(ops)
    loads = [cost[p].sum() for p in parts]
    assert max(loads) - min(loads) <= cost.max()  # the greedy split's bound
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_partition_worker, args=(2, port, out), nprocs=2, join=True)
    single = _run_ops(ops, pool, nout)
    assert np.array_equal(np.frombuffer(out["full"], dtype=np.uint64), single)


def test_partition_balances_costs():
    """The split follows the cost model: on the batched workload's size law
    the heaviest rank carries at most the mean load plus the cost of one
    operation, for 2, 4 and 8 ranks."""
    from paper_2607_28897_gb300 import inputs, ranks

    ops, _, _ = inputs.ragged_ops(63, 400)
    for world in (2, 4, 8):
        parts = ranks.partition(ops, world)
        cost = ranks.op_cost(ops)
        loads = np.array([cost[p].sum() for p in parts])
        assert loads.max() - loads.min() <= cost.max()
        assert loads.max() <= cost.sum() / world + cost.max()
