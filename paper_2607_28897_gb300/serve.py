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

from . import Batch, BATCH_PERSISTENT, OP_DIVMOD, OP_MUL, load, op_dtype, divmod as _divmod
from . import mul_split as _mul_split
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
    def __init__(self, idx, batch, dev_in, dev_out, host_out, status, done, nbytes, stream):
        self.idx, self.batch, self.dev_in, self.dev_out = idx, batch, dev_in, dev_out
        self.host_out, self.status, self.done, self.nbytes = host_out, status, done, nbytes
        self.stream = stream


def _sub_batch(w: Workload, lo: int, hi: int):
    """Descriptors of requests [lo, hi) re-based onto their own input and
    output pools; returns (ops, input base, input limbs, output limbs)."""
    idx = np.arange(lo, hi)
    sub = w.ops[idx].copy()
    base = int(w.ops["a"][lo])
    in_limbs = int(w.ops["b"][hi - 1] + w.ops["nb"][hi - 1]) - base
    sub["a"] -= base
    sub["b"] -= base
    o = np.concatenate([[0], np.cumsum(w.out_limbs[idx])[:-1]])
    sub["o1"] = o
    nq = np.maximum(sub["na"] - sub["nb"] + 1, 1)
    sub["o2"] = np.where(sub["op"] == OP_DIVMOD, o + nq, 0)
    return sub, base, in_limbs, int(w.out_limbs[idx].sum())


def run_continuous(w: Workload, budget_bytes=64 << 30, streams=3, max_batch=2048,
                   keep_results=False):
    """Serves the workload; returns a dict with throughput, p50/p99 latency,
    per-request statuses, the number of batches launched and (optionally)
    the results.

    Admission: every request that has arrived joins the next batch while a
    stream has no batch in flight and the batch's device bytes -- operands,
    results and the batch workspace (the division scratch that holds the
    Newton iterates) -- fit the HBM budget next to the batches in flight.
    A batch over the budget is halved until it fits; with nothing in
    flight, a single request is admitted even if it alone exceeds the
    budget (nothing else could make room for it)."""
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
    inflight, in_use, nxt, done_count, batches, peak = [], 0, 0, 0, 0, 0
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
        # admit: every request that has arrived, while a stream is free and
        # the batch fits the budget
        busy = {id(f.stream) for f in inflight}
        free = [s for s in ss if id(s) not in busy]
        if nxt < n and w.arrival[nxt] <= now and free:
            hi = int(np.searchsorted(w.arrival, now, side="right"))
            hi = min(hi, nxt + max_batch)
            while True:
                sub, base, in_limbs, out_limbs = _sub_batch(w, nxt, hi)
                batch = Batch(sub, allocate=False)
                nbytes = 8 * (in_limbs + out_limbs) + batch.workspace_bytes
                if in_use + nbytes <= budget_bytes or hi - nxt == 1:
                    break
                batch.close()
                hi = nxt + (hi - nxt) // 2
            if in_use + nbytes <= budget_bytes or not inflight:
                s = free[0]
                idx = np.arange(nxt, hi)
                with torch.cuda.stream(s):
                    batch.allocate(stream=s)
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
                                          nbytes, s))
                in_use += nbytes
                peak = max(peak, in_use)
                batches += 1
                nxt = hi
                continue
            batch.close()
        if not inflight and nxt < n and w.arrival[nxt] > now:
            time.sleep(min(w.arrival[nxt] - now, 0.001))
        elif inflight:
            time.sleep(0.0001)
    total = time.perf_counter() - t0
    return {"requests": n, "seconds": total, "throughput": n / total,
            "p50_ms": float(np.percentile(latency, 50) * 1e3),
            "p99_ms": float(np.percentile(latency, 99) * 1e3),
            "status": statuses, "results": results, "batches": batches,
            "peak_bytes_in_flight": peak}


def run_per_request(w: Workload, limit: int | None = None):
    """The plain form: one uniform-entry-point call per request, in arrival
    order, on one stream; a request launches once it has arrived.  A product
    with several output tiles spreads them over CTAs (bigint_mul_split)."""
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
            r = _mul_split(a, b)
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


class Server:
    """Request-level API over the batched form: ``submit(op, a, b)`` returns
    a ticket, ``poll(ticket)`` says whether its result is ready, ``wait``
    returns it as device tensors (``(product,)`` for OP_MUL, ``(q, r)`` for
    OP_DIVMOD, ``(sum,)`` / ``(difference,)`` for OP_ADD / OP_SUB; results
    stay on the device until the caller copies them).

    Pending requests are launched as one ragged batch (persistent form, one
    launch) on a stream with no batch in flight, when the batch's operand,
    result and workspace bytes fit the HBM budget next to the batches in
    flight (admission; a request whose operands and results alone exceed the
    budget is refused with BigIntError).  Batches on different streams
    overlap on the GPU."""

    def __init__(self, budget_bytes: int = 64 << 30, streams: int = 3, max_batch: int = 2048,
                 device="cuda"):
        import torch

        load()
        self.budget = budget_bytes
        self.max_batch = max_batch
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.batches_launched = 0
        self.peak_in_use = 0
        self._pending = []   # (ticket, op, a, b)
        self._inflight = []  # dicts: tickets, event, bytes, keep-alive tensors
        self._done = {}      # ticket -> tuple of result tensors
        self._ticket = 0
        self._in_use = 0

    @staticmethod
    def _out_limbs(op, na, nb):
        if op == OP_MUL:
            return na + nb, 0
        if op == OP_DIVMOD:
            return max(na - nb + 1, 1), nb
        return na, 0

    def submit(self, op: int, a, b) -> int:
        """Queue one operation on 1-D limb tensors (int64/uint64, host or
        device); returns its ticket."""
        from . import BigIntError, EINVAL, ENOMEM, OP_ADD, OP_SUB

        if op not in (OP_ADD, OP_SUB, OP_MUL, OP_DIVMOD):
            raise BigIntError(EINVAL, "submit: unknown op")
        if a.dim() != 1 or b.dim() != 1:
            raise BigIntError(EINVAL, "submit: operands must be 1-D limb tensors")
        if op in (OP_ADD, OP_SUB) and a.numel() != b.numel():
            raise BigIntError(EINVAL, "submit: add/sub need operands of equal length")
        o1, o2 = self._out_limbs(op, a.numel(), b.numel())
        if 8 * (a.numel() + b.numel() + o1 + o2) > self.budget:
            raise BigIntError(ENOMEM, "submit: request larger than the HBM budget")
        t = self._ticket
        self._ticket += 1
        self._pending.append((t, op, a, b))
        self._pump()
        return t

    def _retire(self):
        still = []
        for f in self._inflight:
            if f["event"].query():
                for t, res in f["results"].items():
                    self._done[t] = res
                self._in_use -= f["bytes"]
            else:
                still.append(f)
        self._inflight = still

    def _pump(self):
        import numpy as np
        import torch

        self._retire()
        while self._pending and len(self._inflight) < len(self.streams):
            take, in_limbs, out_limbs = [], 0, 0
            for t, op, a, b in self._pending[: self.max_batch]:
                o1, o2 = self._out_limbs(op, a.numel(), b.numel())
                add_in, add_out = a.numel() + b.numel(), o1 + o2
                if take and 8 * (in_limbs + add_in + out_limbs + add_out) + self._in_use > self.budget:
                    break
                take.append((t, op, a, b))
                in_limbs += add_in
                out_limbs += add_out
            # the batch's workspace (division scratch) counts against the
            # budget too: drop requests from the end until everything fits
            while True:
                ops = np.zeros(len(take), dtype=op_dtype())
                pos = oo = 0
                for k, (t, op, a, b) in enumerate(take):
                    o1, o2 = self._out_limbs(op, a.numel(), b.numel())
                    ops[k] = (op, a.numel(), b.numel(), 0, pos, pos + a.numel(), oo,
                              oo + o1 if op == OP_DIVMOD else 0)
                    pos += a.numel() + b.numel()
                    oo += o1 + o2
                batch = Batch(ops, device=self.device, allocate=False)
                nbytes = 8 * (pos + oo) + batch.workspace_bytes
                if nbytes + self._in_use <= self.budget or len(take) == 1:
                    break
                batch.close()
                take = take[: len(take) // 2]
            if nbytes + self._in_use > self.budget and self._inflight:
                batch.close()
                return  # wait for a batch to retire
            self._pending = self._pending[len(take):]
            busy = {id(f["stream"]) for f in self._inflight}
            s = next(x for x in self.streams if id(x) not in busy)
            with torch.cuda.stream(s):
                batch.allocate(device=self.device, stream=s)
                pool = torch.cat([x.to(self.device, dtype=torch.int64, non_blocking=True).view(-1)
                                  for _, _, a, b in take for x in (a, b)])
                out = torch.empty(max(oo, 1), dtype=torch.int64, device=self.device)
                status = torch.empty(len(take), dtype=torch.int32, device=self.device)
                batch.launch(pool, out, status, mode=BATCH_PERSISTENT, stream=s)
                ev = torch.cuda.Event()
                ev.record(s)
            results = {}
            for k, (t, op, a, b) in enumerate(take):
                o = ops[k]
                o1, o2 = self._out_limbs(op, a.numel(), b.numel())
                r1 = out[int(o["o1"]):int(o["o1"]) + o1]
                results[t] = (r1, out[int(o["o2"]):int(o["o2"]) + o2]) if op == OP_DIVMOD else (r1,)
            self._in_use += nbytes
            self.peak_in_use = max(self.peak_in_use, self._in_use)
            self.batches_launched += 1
            self._inflight.append({"event": ev, "results": results, "bytes": nbytes, "stream": s,
                                   "keep": (pool, out, status, batch)})

    def poll(self, ticket: int) -> bool:
        self._pump()
        return ticket in self._done

    def wait(self, ticket: int):
        """The result tensors of a ticket (blocks until its batch is done)."""
        from . import BigIntError, EINVAL

        while ticket not in self._done:
            self._pump()
            if ticket in self._done:
                break
            if not self._inflight:
                if any(t == ticket for t, *_ in self._pending):
                    continue
                raise BigIntError(EINVAL, f"wait: unknown ticket {ticket}")
            self._inflight[0]["event"].synchronize()
        return self._done.pop(ticket)
