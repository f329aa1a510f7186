"""Multi-process (one process per GPU) helpers for the weak-scaling launch.

Instances are independent (the paper batches with map2 badd asss bsss,
Sec. V-A), so every rank runs its own batch with no collective on the data
path.  The only collectives are the timing barrier and a max-reduction of
the elapsed time over ranks.
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's synthetic batch: disjoint streams per rank."""
    return base + 1000 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (identity without a process
    group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# One ragged batch split over ranks by cost (strong scaling of a fixed batch)
# ---------------------------------------------------------------------------
OP_ADD, OP_SUB, OP_MUL, OP_DIVMOD = 1, 2, 3, 4


def op_cost(ops):
    """Estimated work of each operation of a ragged batch (bigint_op
    descriptors): n for an addition or subtraction (linear), n_a n_b limb
    products for a product, and for a division about two products of the
    quotient by the divisor plus the Newton steps' products on the divisor
    (all quadratic)."""
    import numpy as np

    op = ops["op"]
    na = ops["na"].astype(np.float64)
    nb = ops["nb"].astype(np.float64)
    nq = np.maximum(na - nb + 1.0, 1.0)
    cost = np.where(op == OP_MUL, na * nb, na)
    div = op == OP_DIVMOD
    cost = np.where(div, 2.0 * nq * nb + 1.4 * nb * np.minimum(nb, nq) + na, cost)
    return cost


def partition(ops, world: int):
    """Splits a batch's operations over `world` ranks so that their
    estimated costs are balanced: largest first, each to the rank with the
    least work so far (the longest-processing-time rule).  Returns one
    sorted index array per rank; every operation is in exactly one of them.
    Deterministic, so every rank computes the same split on its own and no
    rank has to send the plan to the others."""
    import heapq

    import numpy as np

    cost = op_cost(ops)
    order = np.argsort(-cost, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + float(cost[i]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def sub_batch(ops, idx, pool):
    """The operations `idx` of a batch as a batch of their own: operands
    copied back to back into a new input pool, results laid out back to back
    in a new output pool.  Returns (sub_ops, sub_pool, out_limbs, out_map)
    where out_map[k] = (offset of op idx[k]'s results in the original output
    pool, offset in the new one, result limbs)."""
    import numpy as np

    sub = ops[idx].copy()
    nq = np.maximum(sub["na"] - sub["nb"] + 1, 1)
    res = np.where(sub["op"] == OP_MUL, sub["na"] + sub["nb"],
                   np.where(sub["op"] == OP_DIVMOD, nq + sub["nb"], sub["na"]))
    pieces, pos, opos, out_map = [], 0, 0, []
    for k, i in enumerate(idx):
        o = ops[i]
        pieces.append(pool[o["a"]:o["a"] + o["na"]])
        pieces.append(pool[o["b"]:o["b"] + o["nb"]])
        sub["a"][k], sub["b"][k] = pos, pos + o["na"]
        pos += int(o["na"] + o["nb"])
        sub["o1"][k] = opos
        sub["o2"][k] = opos + nq[k] if o["op"] == OP_DIVMOD else 0
        out_map.append((int(o["o1"]), opos, int(res[k])))
        opos += int(res[k])
    sub_pool = np.concatenate(pieces) if pieces else pool[:0]
    return sub, sub_pool, opos, out_map
