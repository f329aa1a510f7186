"""Continuous-batching request loop over the batched (persistent) form.

Requests (a multiply or a division of two integers given as limb arrays in
pinned host memory) arrive over time.  The loop admits every request that
has arrived into the next batch as soon as a launch slot and HBM budget are
free: it copies the batch's operands to the device, builds the batch plan,
launches it on one of several CUDA streams and copies the results back, so
batches launched while others are still running overlap on the GPU.
Operands, Newton iterates (the division scratch) and results stay on the
device while a batch is in flight.  Latency of a request is the time from its
arrival to the device-side completion event of its batch (results back in
host memory).

The comparison form, ``run_per_request``, launches every request on its own
(one uniform-entry-point call per request) in arrival order on one stream.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import Batch, BATCH_PERSISTENT, OP_DIVMOD, OP_MUL, load, divmod as _divmod, mul as _mul
from . import inputs


@dataclass
class Workload:
    """Requests: ops (bigint_op layout, offsets into `pool`), arrival times
    (seconds from the start) and the pinned host pool of operand limbs."""
    ops: np.ndarray
    arrival: np.ndarray
    pool: object  # pinned torch int64 tensor
    out_limbs: np.ndarray = field(default=None)


def make_workload(seed: int, count: int, rate: float, device="cuda", mix_mul=0.5,
                  min_limbs: int = 512, max_limbs: int = 8192):
    """Poisson arrivals at `rate` req/s; each request a mul or a divmod (a
    divisor of n limbs, a dividend of [n, 2n] limbs) with n from the 2^15..
    2^19-bit size law."""
    import torch

    ops, nin, _ = inputs.ragged_ops(seed, count, min_limbs=min_limbs, max_limbs=max_limbs,
                                    mix=(mix_mul, 0.0, 0.0, 1.0 - mix_mul))
    gaps = -np.log1p(-((inputs.uniform(seed + 9, count) >> np.uint64(11)).astype(np.float64)
                       / float(1 << 53))) / rate
    arrival = np.cumsum(gaps)
    pool = inputs.ragged_pool(seed + 5, ops, nin, device=device).cpu().pin_memory()
    nq = np.maximum(ops["na"] - ops["nb"] + 1, 1)
    out_limbs = np.where(ops["op"] == OP_MUL, ops["na"] + ops["nb"], nq + ops["nb"])
    return Workload(ops=ops, arrival=arrival, pool=pool, out_limbs=out_limbs)


class _InFlight:
    def __init__(self, idx, batch, dev_in, dev_out, host_out, status, done, nbytes):
        self.idx, self.batch, self.dev_in, self.dev_out = idx, batch, dev_in, dev_out
        self.host_out, self.status, self.done, self.nbytes = host_out, status, done, nbytes


def run_continuous(w: Workload, budget_bytes=64 << 30, streams=3, max_batch=2048,
                   keep_results=False):
    """Serves the workload; returns a dict with throughput, p50/p99 latency,
    per-request statuses and (optionally) the results."""
    import torch

    load()
    n = len(w.ops)
    ss = [torch.cuda.Stream() for _ in range(streams)]
    origin = torch.cuda.Event(enable_timing=True)
    origin.record()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    latency = np.zeros(n)
    statuses = np.zeros(n, dtype=np.int32)
    results = {} if keep_results else None
    inflight, in_use, nxt, done_count, si = [], 0, 0, 0, 0
    a_off = w.ops["a"]
    in_end = w.ops["b"] + w.ops["nb"]
    while done_count < n:
        now = time.perf_counter() - t0
        # retire finished batches
        still = []
        for f in inflight:
            if f.done.query():
                t_done = origin.elapsed_time(f.done) * 1e-3
                latency[f.idx] = t_done - w.arrival[f.idx]
                statuses[f.idx] = f.status.numpy()
                if keep_results:
                    out = f.host_out.numpy().view(np.uint64)
                    for k, i in enumerate(f.idx):
                        o = f.batch.ops[k]
                        results[int(i)] = out[o["o1"]:o["o1"] + w.out_limbs[i]].copy()
                in_use -= f.nbytes
                done_count += len(f.idx)
            else:
                still.append(f)
        inflight = still
        # admit: every request that has arrived, while a slot and budget are free
        if nxt < n and w.arrival[nxt] <= now and len(inflight) < streams:
            hi = int(np.searchsorted(w.arrival, now, side="right"))
            hi = min(hi, nxt + max_batch)
            idx = np.arange(nxt, hi)
            sub = w.ops[idx].copy()
            base = int(a_off[idx[0]])
            in_limbs = int(in_end[idx[-1]]) - base
            sub["a"] -= base
            sub["b"] -= base
            o = np.concatenate([[0], np.cumsum(w.out_limbs[idx])[:-1]])
            sub["o1"] = o
            nq = np.maximum(sub["na"] - sub["nb"] + 1, 1)
            sub["o2"] = np.where(sub["op"] == OP_DIVMOD, o + nq, 0)
            out_limbs = int(w.out_limbs[idx].sum())
            io_bytes = 8 * (in_limbs + out_limbs)
            if in_use + io_bytes <= budget_bytes or not inflight:
                s = ss[si % streams]
                si += 1
                with torch.cuda.stream(s):
                    batch = Batch(sub, stream=s)
                    nbytes = io_bytes + batch.workspace_bytes
                    dev_in = torch.empty(in_limbs, dtype=torch.int64, device="cuda")
                    dev_in.copy_(w.pool[base:base + in_limbs], non_blocking=True)
                    dev_out = torch.empty(out_limbs, dtype=torch.int64, device="cuda")
                    st = torch.empty(len(idx), dtype=torch.int32, device="cuda")
                    batch.launch(dev_in, dev_out, st, mode=BATCH_PERSISTENT, stream=s)
                    host_out = torch.empty(out_limbs if keep_results else 1,
                                           dtype=torch.int64).pin_memory()
                    if keep_results:
                        host_out.copy_(dev_out, non_blocking=True)
                    host_st = torch.empty(len(idx), dtype=torch.int32).pin_memory()
                    host_st.copy_(st, non_blocking=True)
                    done = torch.cuda.Event(enable_timing=True)
                    done.record(s)
                inflight.append(_InFlight(idx, batch, dev_in, dev_out, host_out, host_st, done,
                                          nbytes))
                in_use += nbytes
                nxt = hi
                continue
        if not inflight and nxt < n and w.arrival[nxt] > now:
            time.sleep(min(w.arrival[nxt] - now, 0.001))
        elif inflight:
            time.sleep(0.0001)
    total = time.perf_counter() - t0
    return {"requests": n, "seconds": total, "throughput": n / total,
            "p50_ms": float(np.percentile(latency, 50) * 1e3),
            "p99_ms": float(np.percentile(latency, 99) * 1e3),
            "status": statuses, "results": results}


def run_per_request(w: Workload, limit: int | None = None):
    """The plain form: one uniform-entry-point call per request, in arrival
    order, on one stream; a request launches once it has arrived."""
    import torch

    n = len(w.ops) if limit is None else min(limit, len(w.ops))
    origin = torch.cuda.Event(enable_timing=True)
    origin.record()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    events = []
    for i in range(n):
        now = time.perf_counter() - t0
        if w.arrival[i] > now:
            time.sleep(w.arrival[i] - now)
        o = w.ops[i]
        a = w.pool[o["a"]:o["a"] + o["na"]].to("cuda", non_blocking=True).view(1, -1)
        b = w.pool[o["b"]:o["b"] + o["nb"]].to("cuda", non_blocking=True).view(1, -1)
        if o["op"] == OP_MUL:
            r = _mul(a, b)
            r.to("cpu", non_blocking=True)
        else:
            q, r, _ = _divmod(a, b)
            q.to("cpu", non_blocking=True)
            r.to("cpu", non_blocking=True)
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        events.append(e)
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    lat = np.array([origin.elapsed_time(e) * 1e-3 - w.arrival[i] for i, e in enumerate(events)])
    return {"requests": n, "seconds": total, "throughput": n / total,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3)}
