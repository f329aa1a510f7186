#!/usr/bin/env python
"""Benchmark of the batched big-integer hot path on GB300.

One step = one pass of every step of the path over its synthetic batch:
  * add, sub and full-product mul at 2^15 .. 2^19 bits (512 .. 8192 limbs),
    each operand array 2^32 bits (batch 2^26 / n) -- the paper's
    Bits x Insts = 2^32 size sweep (Sec. VI, Tables I and II);
  * divmod of a 2n-limb dividend by an n-limb divisor at n = 512, 2048, 8192
    (batches 4096, 1024, 256) -- Newton shifted-inverse division (Table III).
The headline value is limb-Gops/s: output limbs for add/sub, limb products
(n_a n_b) for mul, (n_u - n_v + 1) n_v limb-product equivalents for divmod,
summed over the step and divided by the device time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 run under torch.distributed.run; every rank processes the same
per-GPU batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import platform
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("bigint mul & divmod ops/s and limb-Gops/s at 2^15–2^19 bits; "
          "% of int-mul/HBM peak")
UNIT = "limb-Gops/s"
SWEEP = (512, 1024, 2048, 4096, 8192)
DIV = ((512, 4096), (2048, 1024), (8192, 256))
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--sizes", default=",".join(str(n) for n in SWEEP))
    p.add_argument("--workload", default="sweep", choices=["sweep", "batched", "serving", "programs"],
                   help="sweep: the headline step (default); batched: the ragged mixed-op "
                        "batch in one persistent launch vs one launch per size class; "
                        "serving: continuous batching vs per-request launches")
    p.add_argument("--batch-ops", type=int, default=200000)
    p.add_argument("--requests", type=int, default=100000,
                   help="requests per rate of --workload serving")
    p.add_argument("--serving-requests", type=int, default=10000,
                   help="requests per rate of the serving block in the default line")
    p.add_argument("--no-forms", action="store_true",
                   help="leave the batched and serving blocks out of the default line")
    p.add_argument("--rates", default="5000,20000,50000,100000,200000")
    return p.parse_args()


# --------------------------------------------------------------------------
# workload accounting (shared by both arms)
# --------------------------------------------------------------------------
def sweep_batch(n: int) -> int:
    return (1 << 26) // n


def step_units(sizes):
    """(name, batch, limb-ops per instance) of every op in one step."""
    ops = []
    for n in sizes:
        b = sweep_batch(n)
        ops.append((f"add_{n}", b, n))
        ops.append((f"sub_{n}", b, n))
        ops.append((f"mul_{n}", b, n * n))
    for n, b in DIV:
        ops.append((f"divmod_{2 * n}_{n}", b, (n + 1) * n))
    return ops


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 8]
        sm, smax, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax = max(smax, float(r[1]))
            except ValueError:
                continue
            for name, val in zip(names, r[4:8]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample of the same workload
# --------------------------------------------------------------------------
_SAMPLE_INPUTS = {}


def _sample_inputs(kind, n, k):
    """Seeded sample operands, kept across calls (up to 64 MB each) so that
    repeated reference steps time the oracle rather than the generator."""
    from paper_2607_28897_gb300 import inputs

    key = (kind, n, k)
    if key in _SAMPLE_INPUTS:
        return _SAMPLE_INPUTS[key]
    if kind == "divmod":
        ab = inputs.config_div(n, k)
    else:
        ab = (inputs.limbs(11 + n, k, n, True), inputs.limbs(12 + n, k, n, True))
    if ab[0].nbytes <= (64 << 20):
        _SAMPLE_INPUTS[key] = ab
    return ab


def oracle_sample_rate(sizes, budget_s: float):
    """Times the plain CPU oracle on a bounded sample of every op of the step,
    extrapolates the time of a full step, and returns the limb-Gops/s a full
    step would reach, the host threads used and a description.  Additions
    and subtractions take at most 1/16 of their batch (their time is linear
    in the batch, and generating full 512 MiB operands would dominate)."""
    import oracle

    oracle.build()
    ops = step_units(sizes)
    per_op = budget_s / len(ops)
    total_ops, total_time, desc = 0.0, 0.0, []
    for name, batch, units in ops:
        kind = name.split("_")[0]
        if kind == "divmod":
            n = int(name.split("_")[2])
        else:
            n = int(name.split("_")[1])
        cap = max(1, batch // 16) if kind in ("add", "sub") else batch
        k = 1
        while True:
            k = min(k, cap)
            if kind == "divmod":
                u, v = _sample_inputs(kind, n, k)
                t0 = time.perf_counter()
                oracle.batch_divmod(u, v)
            else:
                a, b = _sample_inputs(kind, n, k)
                t0 = time.perf_counter()
                if kind == "add":
                    oracle.batch_add(a, b)
                elif kind == "sub":
                    oracle.batch_sub(a, b)
                else:
                    oracle.batch_mul(a, b)
            dt = time.perf_counter() - t0
            if dt >= per_op or k >= cap or dt * (2 * batch / k) < 0.05:
                break
            k = int(min(cap, max(2 * k, k * per_op / max(dt, 1e-6) * 0.8)))
        full = dt * batch / k
        total_ops += batch * units
        total_time += full
        desc.append(f"{name}:{k}/{batch}")
    return total_ops / total_time / 1e9, oracle.num_threads(), " ".join(desc)


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


# --------------------------------------------------------------------------
# committed ncu traffic of the multiply kernel, valid only for its source
# --------------------------------------------------------------------------
def kernel_source_hash(files=("tccore.cuh", "tcmul.cu", "mul.cu", "blockops.cuh",
                              "common.cuh")) -> str:
    """Hash of the multiply kernel's code: // comments, blank lines and
    indentation do not count, so a comment edit keeps a profile valid."""
    h = hashlib.sha256()
    for f in files:
        for line in open(os.path.join(ROOT, "paper_2607_28897_gb300", "csrc", f)):
            code = line.split("//", 1)[0].strip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def committed_traffic():
    """key = value lines of profiles/mul_tc_traffic.txt (DRAM bytes per
    multiply launch from an ncu capture), or None once the kernel source
    changed."""
    path = os.path.join(ROOT, "profiles", "mul_tc_traffic.txt")
    d = {}
    try:
        for line in open(path):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                d[k.strip()] = v.strip()
    except OSError:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return {k: float(v) for k, v in d.items() if k.startswith("bytes_per_launch")}


# --------------------------------------------------------------------------
# reference arm: the oracle, K timed steps of a bounded sample
# --------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    sizes = [int(s) for s in args.sizes.split(",")]
    for _ in range(args.warmup):
        oracle_sample_rate(sizes, 2.0)
    vals, t0 = [], time.perf_counter()
    threads, desc = 1, ""
    for _ in range(args.steps):
        v, threads, desc = oracle_sample_rate(sizes, 8.0)
        vals.append(v)
    elapsed = time.perf_counter() - t0
    value = sum(vals) / len(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed * 1e3 / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(sizes),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": desc, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(sizes):
    return {
        "workload": ("add/sub/mul sweep at 2^15..2^19 bits, 2^32 bits per operand array "
                     "(batch 2^26/n), + divmod 2n/n limbs at n=512/2048/8192 "
                     "(batch 4096/1024/256)"),
        "sweep_limbs": list(sizes),
        "mul_form": {str(n): kara_form(n) for n in sizes},
        "div": [list(d) for d in DIV],
        "l2": "sweep operands (512 MiB each) exceed L2; L2 flushed (256 MiB write) before each step",
        "parallelism": "instances: one CTA per instance, batches sharded per GPU",
    }


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "programs":
        return run_programs(args)
    if args.workload == "serving":
        run_serving(args)
        return

    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs, ranks

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    bi.load()
    sizes = [int(s) for s in args.sizes.split(",")]

    # ---- inputs, resident in HBM before timing (seeded, per rank)
    seed_off = ranks.rank_seed(0, rank)
    sweep = {}
    for n in sizes:
        a, b = inputs.config_sweep_torch(n, seed=2 + seed_off, device=dev)
        # subtraction operands ordered a >= b (top limbs decide for random data)
        top_a = a[:, -1] ^ (-(1 << 63))  # unsigned order as signed order
        top_b = b[:, -1] ^ (-(1 << 63))
        sw = top_a < top_b
        sa = torch.where(sw[:, None], b, a)
        sb = torch.where(sw[:, None], a, b)
        batch = a.shape[0]
        sweep[n] = dict(a=a, b=b, sa=sa, sb=sb,
                        s=torch.empty_like(a), d=torch.empty_like(a),
                        p=torch.empty((batch, 2 * n), dtype=torch.int64, device=dev),
                        c=torch.empty(batch, dtype=torch.uint8, device=dev),
                        # the full product through bigint_mul_kara's measured choice
                        # (Karatsuba levels over the batched products from 4096
                        # limbs; bigint_mul's own path below)
                        kws=torch.empty(max(bi.mul_kara_workspace_bytes(batch, n), 256),
                                        dtype=torch.uint8, device=dev))
    import numpy as np

    divs = {}
    for n, batch in DIV:
        u, v = inputs.config_div(n, batch, seed=3 + seed_off)
        du = torch.from_numpy(u.view(np.int64)).to(dev)
        dv = torch.from_numpy(v.view(np.int64)).to(dev)
        ws = torch.empty(bi.divmod_workspace_bytes(batch, 2 * n, n), dtype=torch.uint8, device=dev)
        divs[n] = dict(u=du, v=dv, ws=ws,
                       q=torch.empty((batch, n + 1), dtype=torch.int64, device=dev),
                       r=torch.empty((batch, n), dtype=torch.int64, device=dev),
                       st=torch.empty(batch, dtype=torch.int32, device=dev))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    mul_events = {n: [] for n in sizes}
    add_events = {n: [] for n in sizes}
    # the three divisions are independent and none fills the GPU to its end
    # (2^20 / 2^19 bits: 256 one-SM instances, two waves on 152 SMs), so they
    # run side by side on streams of their own after the sweep, the largest
    # first: the smaller ones take the SMs the larger ones leave idle in
    # their last wave.  (Started with the sweep instead, they shortened the
    # step by 0.3 %, and the sweep's launches, timed below inside the step,
    # would share the GPU with them.)
    div_streams = [torch.cuda.Stream(device=dev) for _ in DIV]

    def one_step(record):
        flush.fill_(1)
        for n in sizes:
            S = sweep[n]
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            bi.add(S["a"], S["b"], out=S["s"], carry=S["c"])
            if record:
                e1 = torch.cuda.Event(enable_timing=True)
                e1.record(stream)
                add_events[n].append((e0, e1))
            bi.sub(S["sa"], S["sb"], out=S["d"], borrow=S["c"])
            if record:
                e2 = torch.cuda.Event(enable_timing=True)
                e2.record(stream)
            bi.mul_kara(S["a"], S["b"], out=S["p"], workspace=S["kws"])
            if record:
                e3 = torch.cuda.Event(enable_timing=True)
                e3.record(stream)
                mul_events[n].append((e2, e3))
        fork = torch.cuda.Event()
        fork.record(stream)
        joins = []
        for (n, batch), ds in zip(sorted(DIV, reverse=True), div_streams):
            D = divs[n]
            ds.wait_event(fork)
            bi.divmod(D["u"], D["v"], q=D["q"], r=D["r"], status=D["st"], workspace=D["ws"],
                      stream=ds)
            j = torch.cuda.Event()
            j.record(ds)
            joins.append(j)
        for j in joins:
            stream.wait_event(j)

    for _ in range(max(args.warmup, 3)):
        one_step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    k0 = bi.kernel_launches()
    for _ in range(args.steps):
        one_step(True)
    launches = bi.kernel_launches() - k0  # every kernel the library enqueued
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms_total = ranks.max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    ops = step_units(sizes)
    limb_ops_step = sum(b * u for _, b, u in ops)
    value = world * limb_ops_step * args.steps / (ms_total * 1e-3) / 1e9

    # ---- per-op breakdown from a separately timed pass (one launch each)
    breakdown = {}

    def time_op(fn, reps=1):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        s0.record(stream)
        for _ in range(reps):
            fn()
        s1.record(stream)
        s1.synchronize()
        return s0.elapsed_time(s1) / reps

    for n in sizes:
        S = sweep[n]
        b = S["a"].shape[0]
        # the spans of each op inside the timed steps (CUDA events)
        t_add = sum(e0.elapsed_time(e1) for e0, e1 in add_events[n]) / len(add_events[n])
        t_mul = sum(e0.elapsed_time(e1) for e0, e1 in mul_events[n]) / len(mul_events[n])
        breakdown[f"add_{n}"] = {"ms": t_add, "ops_per_s": b / (t_add * 1e-3),
                                 "GB_s": 24.0 * b * n / (t_add * 1e-3) / 1e9}
        breakdown[f"mul_{n}"] = {"ms": t_mul, "ops_per_s": b / (t_mul * 1e-3),
                                 "limb_gops": b * n * n / (t_mul * 1e-3) / 1e9,
                                 "form": kara_form(n)}
        if kara_levels(n) > 0:  # the schoolbook product alone, for the roofline
            breakdown[f"mul_{n}"]["schoolbook_ms"] = time_op(
                lambda: bi.mul(S["a"], S["b"], out=S["p"]))
    for n, batch in DIV:
        D = divs[n]
        t = time_op(lambda: bi.divmod(D["u"], D["v"], q=D["q"], r=D["r"], status=D["st"],
                                      workspace=D["ws"]))
        breakdown[f"divmod_{2 * n}_{n}"] = {"ms": t, "ops_per_s": batch / (t * 1e-3),
                                            "limb_gops": batch * (n + 1) * n / (t * 1e-3) / 1e9}

    # ---- single-product latency (serving): one product on one CTA against
    #      its output tiles spread over CTAs (bigint_mul_split)
    latency = {}
    for n in (4096, 8192):
        a1, b1 = sweep[n]["a"][:1], sweep[n]["b"][:1]
        o1 = torch.empty((1, 2 * n), dtype=torch.int64, device=dev)
        ws1 = torch.empty(max(1, bi.mul_split_workspace_bytes(1, n, n)), dtype=torch.uint8,
                          device=dev)
        row = {"form": "split-K: (tile, group) units over the SMs, column sums added atomically"}
        for name, fn in (("mul_us", lambda: bi.mul(a1, b1, out=o1, stream=stream)),
                         ("mul_split_us", lambda: bi.mul_split(a1, b1, out=o1, workspace=ws1,
                                                               stream=stream))):
            for _ in range(3):
                fn()
            row[name] = round(time_op(fn, reps=20) * 1e3, 1)
        latency[f"mul_{n}x{n}_one_product"] = row
    # one 2^20 / 2^19-bit division alone: the step-batched form (every
    # product one launch over the whole GPU) against one CTA per division
    if 8192 in divs:
        D = divs[8192]
        u1, v1 = D["u"][1:2], D["v"][1:2]
        q1 = torch.empty((1, 8193), dtype=torch.int64, device=dev)
        r1 = torch.empty((1, 8192), dtype=torch.int64, device=dev)
        s1 = torch.empty(1, dtype=torch.int32, device=dev)
        w1 = torch.empty(bi.divmod_workspace_bytes(1, 16384, 8192), dtype=torch.uint8, device=dev)
        row = {}
        for name, variant in (("steps_us", 0), ("one_cta_us", 1)):
            bi.set_variant(1, variant)
            fn = lambda: bi.divmod(u1, v1, q=q1, r=r1, status=s1, workspace=w1, stream=stream)
            for _ in range(2):
                fn()
            row[name] = round(time_op(fn, reps=5) * 1e3, 1)
        bi.set_variant(1, 0)
        latency["divmod_16384_8192_one_division"] = row

    # ---- roofline of the dominant kernel: the multiply launch at the largest
    #      size (2^19 bits), the longest launch of the step
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    nmax = max(sizes)
    vmax = bi.mul_variant_for(nmax, nmax)

    def mul_units(n):
        """Limb products the multiply algorithm the library picks performs
        for one n x n product (Karatsuba: three (n/2+1)-limb half products;
        the tensor-core product is a schoolbook product)."""
        v = bi.mul_variant_for(n, n)
        if v in (10, 11):
            hh = n - n // 2
            return (n // 2) ** 2 + hh * hh + (hh + 1) ** 2
        return n * n

    def school_ms(n):  # the tensor-core (schoolbook) product's own time
        row = breakdown[f"mul_{n}"]
        return row.get("schoolbook_ms", row["ms"])

    # the dominant kernel as the step runs it: the tensor-core product at the
    # leaf size of the largest Karatsuba product (2048 limbs: the 2^17-bit
    # sweep product and every leaf of the 2^18- and 2^19-bit products), its
    # sweep launch timed inside the step
    nk = nmax >> kara_levels(nmax)
    if nk not in sizes:
        nk = nmax
    mul_ms = breakdown[f"mul_{nk}"]["ms"] if kara_levels(nk) == 0 else school_ms(nk)
    all_ms = sum(school_ms(n) for n in sizes)
    tr = committed_traffic()
    vk = bi.mul_variant_for(nk, nk)
    kernel = (f"{'k_mul_tc<256, 8, 1, 128>' if vk == 12 else 'k_mul_kara' if vk in (10, 11) else 'k_mul'}"
              f" (variant {vk}), {nk}-limb operands, batch {sweep_batch(nk)}: the launch shape "
              f"of the step's tensor-core products (the {nk}-limb sweep product and the leaves "
              f"of the Karatsuba products)")
    if vmax == 12:
        # tensor bound: 2 flops per fp16 digit product of the 8-bit schoolbook
        # convolution, (8 n)^2 per n x n product.  The step holds the maximum
        # SM clock (no power cap: see "clocks"), so the burst peak -- a GEMM
        # timed alone at that clock -- is the denominator; the fraction of
        # the sustained (power-capped) peak and of the nominal dense rate
        # are given beside it.
        def tc_flops(n):
            return 2.0 * (8 * n) ** 2 * sweep_batch(n)

        burst = float(peaks.get("bf16_tflops", 1900.0))
        sustained = float(peaks.get("bf16_tflops_sustained", 1700.0))
        peak = burst
        achieved = tc_flops(nk) / (mul_ms * 1e-3) / 1e12
        tc_sizes = [n for n in sizes if bi.mul_variant_for(n, n) == 12]
        tc_ms = sum(school_ms(n) for n in tc_sizes)
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "traffic": tr.get(f"bytes_per_launch_{nk}") if tr else None,
                    "kernel": kernel,
                    "algorithmic_work": "2 x (8 n)^2 flops per n x n product: fp16 products of "
                                        "base-256 digits, accumulated in fp32",
                    "frac_all_sizes": (sum(tc_flops(n) for n in tc_sizes) / (tc_ms * 1e-3) / 1e12
                                       / peak) if tc_sizes else None,
                    "frac_by_size": {str(n): tc_flops(n) / (school_ms(n) * 1e-3)
                                     / 1e12 / peak for n in tc_sizes},
                    "timing_basis": (f"achieved: the {nk}-limb product's span inside the timed "
                                     "step; frac_by_size: the schoolbook tensor-core product of "
                                     "each size (the 4096- and 8192-limb ones timed alone, since "
                                     "the step runs them as Karatsuba levels over 2048-limb "
                                     "products of this kernel)"),
                    "frac_of_sustained": achieved / sustained,
                    # the sustained peak scaled from its own median SM clock to
                    # the clock this step held (time x median SM MHz)
                    "frac_clock_normalized": (
                        achieved / (sustained * clk["sm_mhz"] /
                                    float(peaks["clocks_under_load"]["sm_mhz_median"]))
                        if clk and peaks.get("clocks_under_load", {}).get("sm_mhz_median")
                        else None),
                    "frac_of_nominal_2250": achieved / 2250.0,
                    "peak_basis": ("of measured: MEASURED_PEAKS.json bf16_tflops (burst: a GEMM "
                                   "timed alone; fp16 and bf16 share the nominal dense rate), "
                                   "the basis for a step that held the maximum SM clock; "
                                   "frac_of_sustained divides by bf16_tflops_sustained "
                                   "(measured power-capped), frac_clock_normalized by that "
                                   "peak scaled by this step's median SM clock over the "
                                   "median clock of its measurement")
                    if "bf16_tflops" in peaks else "of fallback: 1900 TFLOP/s burst"}
    else:
        ipc, probe_mhz = bi.probe_int_throughput(0)  # IMAD.WIDE per SM per clock
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clk["sm_mhz"] if clk else probe_mhz
        peak = ipc * sms * mhz * 1e6 / 1e12  # T IMAD.WIDE / s at the clock under load
        mul_work = 4.0 * sweep_batch(nmax) * mul_units(nmax)  # 4 IMAD.WIDE per limb product
        achieved = mul_work / (mul_ms * 1e-3) / 1e12
        all_work = sum(4.0 * sweep_batch(n) * mul_units(n) for n in sizes)
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak,
                    "unit": "T IMAD.WIDE-equivalent/s (4 per limb product)",
                    "frac": achieved / peak, "traffic": None, "kernel": kernel,
                    "algorithmic_work": "4 IMAD.WIDE-equivalents per limb product the algorithm "
                                        "performs",
                    "frac_all_sizes": all_work / (all_ms * 1e-3) / 1e12 / peak,
                    "peak_basis": (f"measured {ipc:.1f} IMAD.WIDE/clk/SM x {sms} SMs x "
                                   f"{mhz:.0f} MHz (median SM clock in the timed region)")}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    add_bytes = sum(24.0 * sweep_batch(n) * n for n in sizes)
    add_ms = sum(breakdown[f"add_{n}"]["ms"] for n in sizes)
    roofline_add = {"bound": "hbm", "achieved": add_bytes / (add_ms * 1e-3) / 1e9,
                    "peak": hbm_peak, "unit": "GB/s",
                    "frac": add_bytes / (add_ms * 1e-3) / 1e9 / hbm_peak,
                    "peak_basis": "MEASURED_PEAKS.json hbm_gbs (measured copy)"
                    if "hbm_gbs" in peaks else "fallback 6800 GB/s", "kernel": "k_addsub"}

    # ---- end to end through the C ABI with host buffers
    e2e = run_e2e(args, torch, bi, sweep, divs, sizes, dev, stream, limb_ops_step, world, dist)

    # ---- the batched form (200k ragged instances) and the serving loop
    #      (continuous batching at Poisson rates), outside the timed step
    batched = serving = None
    if not args.no_forms:
        batched = batched_block(torch, bi, args.batch_ops, 3, rank, world, dist, dev)
        if world == 1:
            serving = serving_block(torch, bi, [float(r) for r in args.rates.split(",")],
                                    args.serving_requests, 1000)

    # ---- the autotuner against the built-in choice, on an eighth of each
    #      sweep batch (the built-in table is restored afterwards)
    tuning = tuning_block(torch, bi, sweep, sizes) if not args.no_forms else None

    # ---- CPU baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, th, desc = oracle_sample_rate(sizes, 20.0)
        cpu = {"value": v, "unit": UNIT, "cores": th, "kind": "oracle", "sample": desc,
               "cpu": cpu_model()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": workload_config(sizes), "roofline": roofline,
            "roofline_add": roofline_add, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "breakdown": breakdown,
            "latency": latency, "batched": batched, "serving": serving, "tuning": tuning,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def tuning_block(torch, bi, sweep, sizes):
    """bigint_tune on an eighth of each sweep batch: the variant it picks
    against the built-in one, with the product's time under each."""
    import tempfile

    def best_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        out = 1e30
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out = min(out, e0.elapsed_time(e1))
        return out

    res = {}
    try:
        for n in sizes:
            k = max(1, sweep_batch(n) // 8)
            a, b, p = sweep[n]["a"][:k], sweep[n]["b"][:k], sweep[n]["p"][:k]
            v0 = bi.mul_variant_for(n, n)
            t0 = best_ms(lambda: bi.mul(a, b, out=p))
            v1 = bi.tune(a, b, out=p)
            t1 = best_ms(lambda: bi.mul(a, b, out=p))
            res[str(n)] = {"batch": k, "builtin_variant": v0, "builtin_ms": round(t0, 3),
                           "tuned_variant": v1, "tuned_ms": round(t1, 3)}
    finally:
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "t.json")
            bi.save_tuning(path)
            table = json.load(open(path))
            table["mul_variant_by_class"] = [0] * 32
            json.dump(table, open(path, "w"))
            bi.load_tuning(path)
    return res


def bind_to_gpu_cpus(torch, dev):
    """Restricts this process to the CPUs next to the GPU (the PCI device's
    local_cpulist in sysfs), so that the pinned host buffers allocated
    afterwards sit in the GPU's NUMA-local memory, as a deployment binds a
    GPU's feeder process.  Returns what was done (or why not)."""
    try:
        props = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
        path = f"/sys/bus/pci/devices/{bus}/local_cpulist"
        text = open(path).read().strip()
        cpus = set()
        for part in text.split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return {"bound": False, "why": f"no usable CPU in {text}"}
        os.sched_setaffinity(0, cpus)
        return {"bound": True, "pci": bus, "cpus": text}
    except (OSError, AttributeError, ValueError) as e:
        return {"bound": False, "why": type(e).__name__}


def run_e2e(args, torch, bi, sweep, divs, sizes, dev, stream, limb_ops_step, world, dist):
    """Same step through the library's host-buffer entry points
    (bigint_host_async for add, sub, mul and divmod, then bigint_host_sync):
    every call copies its inputs from pinned host memory and its results
    (with carries and statuses) back to pinned host memory inside the timed
    region; the library overlaps the copies of one chunk or call with the
    kernels of the next.  Timed on the host clock; calls_ms are enqueue
    times, "sync" the wait for the step's work."""
    steps = max(1, args.e2e_steps)
    all_cpus = os.sched_getaffinity(0)
    numa = bind_to_gpu_cpus(torch, dev)
    try:
        return _run_e2e(args, torch, bi, sweep, divs, sizes, dev, limb_ops_step, world, dist,
                        steps, numa)
    finally:  # the CPU baseline that follows uses every host core again
        os.sched_setaffinity(0, all_cpus)


def _run_e2e(args, torch, bi, sweep, divs, sizes, dev, limb_ops_step, world, dist, steps, numa):

    def pinned_like(t, dtype=None):
        return torch.empty(tuple(t.shape), dtype=dtype or t.dtype).pin_memory()

    host_in, host_out, ws = {}, {}, {}
    h2d = d2h = 0
    for n in sizes:
        S = sweep[n]
        b = S["a"].shape[0]
        host_in[n] = tuple(S[k].cpu().pin_memory() for k in ("a", "b", "sa", "sb"))
        host_out[n] = (pinned_like(S["s"]), pinned_like(S["d"]), pinned_like(S["p"]),
                       torch.empty(b, dtype=torch.uint8).pin_memory(),
                       torch.empty(b, dtype=torch.uint8).pin_memory())
        chunk = max(1, (b + 3) // 4)
        # one workspace per call, so that enqueued calls do not wait for each
        # other, with a staging slot per chunk (2 x two slots): no chunk waits
        # for an earlier chunk's copy-out
        ws[n] = {op: torch.empty(2 * bi.host_workspace_bytes(op, chunk, n, n), dtype=torch.uint8,
                                 device=dev) for op in (bi.OP_ADD, bi.OP_SUB, bi.OP_MUL)}
        a_bytes = S["a"].numel() * 8
        h2d += 6 * a_bytes  # add: a, b; sub: sa, sb; mul: a, b
        d2h += 2 * a_bytes + 2 * b + S["p"].numel() * 8
    hdiv = {}
    for n, batch in DIV:
        D = divs[n]
        hu, hv = D["u"].cpu().pin_memory(), D["v"].cpu().pin_memory()
        hq, hr = pinned_like(D["q"]), pinned_like(D["r"])
        hst = torch.empty(batch, dtype=torch.int32).pin_memory()
        chunk = max(1, (batch + 3) // 4)
        wsd = torch.empty(2 * bi.host_workspace_bytes(bi.OP_DIVMOD, chunk, 2 * n, n),
                          dtype=torch.uint8, device=dev)
        hdiv[n] = (hu, hv, hq, hr, hst, wsd)
        h2d += (hu.numel() + hv.numel()) * 8
        d2h += (hq.numel() + hr.numel()) * 8 + 4 * batch

    calls_ms = {}

    def timed(name, fn):
        c0 = time.perf_counter()
        fn()
        calls_ms[name] = calls_ms.get(name, 0.0) + (time.perf_counter() - c0) * 1e3

    def step():
        # every call is enqueued (sync=False): the copies of one call overlap
        # the kernels of the next; one host_sync ends the step.  Longest
        # kernels first: while the 2^19-bit products run, the copies of the
        # copy-bound additions behind them stream in (in the opposite order
        # the additions' copies, 4.8 ms each, wait with an idle GPU)
        for n in sorted(sizes, reverse=True):
            ha, hb, hsa, hsb = host_in[n]
            hs, hd, hp, hc, hbw = host_out[n]
            w = ws[n]
            timed(f"mul_{n}", lambda: bi.mul_host(ha, hb, out=hp, workspace=w[bi.OP_MUL],
                                                  sync=False))
            timed(f"add_{n}", lambda: bi.add_host(ha, hb, out=hs, carry=hc,
                                                  workspace=w[bi.OP_ADD], sync=False))
            timed(f"sub_{n}", lambda: bi.sub_host(hsa, hsb, out=hd, borrow=hbw,
                                                  workspace=w[bi.OP_SUB], sync=False))
        for n, _ in DIV:
            hu, hv, hq, hr, hst, wsd = hdiv[n]
            timed(f"divmod_{2 * n}_{n}",
                  lambda: bi.divmod_host(hu, hv, q=hq, r=hr, status=hst, workspace=wsd,
                                         sync=False))
        timed("sync", bi.host_sync)

    # the host link's copy rate on this machine (differs between machines),
    # measured outside the timed region on 512 MiB pinned buffers
    probe_h = torch.empty(1 << 26, dtype=torch.int64).pin_memory()
    probe_d = torch.empty(1 << 26, dtype=torch.int64, device=dev)

    def copy_gbs(fn, nbytes=probe_h.numel() * 8):
        fn()
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        return 3 * nbytes / (time.perf_counter() - c0) / 1e9

    h2d_gbs = copy_gbs(lambda: probe_d.copy_(probe_h, non_blocking=True))
    d2h_gbs = copy_gbs(lambda: probe_h.copy_(probe_d, non_blocking=True))
    # both directions at once (as the step's copies run): bytes moved both
    # ways per second
    probe_h2 = torch.empty_like(probe_h).pin_memory()
    probe_d2 = torch.empty_like(probe_d)
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def both():
        with torch.cuda.stream(s_in):
            probe_d.copy_(probe_h, non_blocking=True)
        with torch.cuda.stream(s_out):
            probe_h2.copy_(probe_d2, non_blocking=True)

    both_gbs = 2 * copy_gbs(both)
    del probe_h, probe_d, probe_h2, probe_d2
    # the same rates on the step's own largest pinned buffers (where they were
    # placed can differ from a freshly pinned probe buffer)
    nbig = max(sizes)
    own_h, own_o = host_in[nbig][0], host_out[nbig][2]
    own_d = torch.empty_like(sweep[nbig]["a"])
    own_p = torch.empty_like(sweep[nbig]["p"])
    own_h2d = copy_gbs(lambda: own_d.copy_(own_h, non_blocking=True), own_h.numel() * 8)
    own_d2h = copy_gbs(lambda: own_o.copy_(own_p, non_blocking=True), own_o.numel() * 8)
    del own_d, own_p

    step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    calls_ms.clear()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    from paper_2607_28897_gb300 import ranks

    dt = ranks.max_over_ranks(time.perf_counter() - t0, dist, dev)
    return {"value": world * limb_ops_step * steps / dt / 1e9, "unit": UNIT, "host_binding": numa,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "path": "bigint_host_async + bigint_host_sync (C ABI, pinned host buffers, copies "
                    "overlapped with kernels)",
            "host_link_gbs": {"h2d": round(h2d_gbs, 1), "d2h": round(d2h_gbs, 1),
                              "both_directions_at_once": round(both_gbs, 1),
                              "h2d_step_buffer": round(own_h2d, 1),
                              "d2h_step_buffer": round(own_d2h, 1)},
            "copy_bound_ms_per_step": round((h2d + d2h) / (both_gbs * 1e9) * 1e3, 1),
            "calls_ms": {k: round(v / steps, 2) for k, v in calls_ms.items()}}

def batched_block(torch, bi, count, reps, rank=0, world=1, dist=None, dev=None):
    """The batched form: `count` ragged instances (sizes log-uniform over
    2^15..2^19 bits; 40 % mul, 15 % add, 15 % sub, 30 % divmod) in one
    persistent launch with a device-side work queue, in the steps form
    (large divisions grouped into padded shape classes and divided
    step-batched, the rest persistent), the faster of the two tuned and
    replayed as a CUDA graph, against one launch per (op, size class).  With
    several ranks the batch is split by estimated cost (ranks.partition) and
    every rank runs its share (strong scaling of the fixed batch); times are
    the maximum over ranks."""
    import numpy as np

    from paper_2607_28897_gb300 import inputs, ranks

    ops, nin, nout = inputs.ragged_ops(4, count)
    pool = inputs.ragged_pool(5, ops, nin, device=dev or "cuda")
    if world > 1:
        part = ranks.partition(ops, world)[rank]
        host_pool = pool.cpu().numpy().view(np.uint64)
        ops, sub_pool, nout, _ = ranks.sub_batch(ops, part, host_pool)
        pool = torch.from_numpy(sub_pool.view(np.int64)).to(dev or "cuda")
    out = torch.zeros(max(nout, 1), dtype=torch.int64, device=pool.device)
    st = torch.zeros(max(len(ops), 1), dtype=torch.int32, device=pool.device)
    B = bi.Batch(ops, device=pool.device)

    def best_of(fn, reps):
        fn()
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return ranks.max_over_ranks(min(times), dist, dev)

    # SM clocks sampled from here to the last timed pass; about a second of
    # the persistent form first, so that they have settled under load
    clk = ClockSampler(dev.index if dev is not None and dev.index is not None else 0)
    clk.start()
    t_end = time.perf_counter() + 1.0
    while time.perf_counter() < t_end:
        B.launch(pool, out, st, mode=bi.BATCH_PERSISTENT)
        torch.cuda.synchronize()
    t_class = best_of(lambda: B.launch(pool, out, st, mode=bi.BATCH_PER_CLASS), reps)
    ref = out.clone()
    t_pers = best_of(lambda: B.launch(pool, out, st, mode=bi.BATCH_PERSISTENT), reps)
    same = bool(torch.equal(out, ref))
    t_steps = best_of(lambda: B.launch(pool, out, st, mode=bi.BATCH_STEPS), reps)
    same = same and bool(torch.equal(out, ref))
    threads = B.tune(pool, out, st)
    # the faster of the persistent and the steps form, tuned, as a CUDA graph
    mode = bi.BATCH_STEPS if t_steps < t_pers else bi.BATCH_PERSISTENT
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        B.launch(pool, out, st, mode=mode, stream=s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            B.launch(pool, out, st, mode=mode, stream=s)
    t_graph = best_of(lambda: g.replay(), reps)
    clocks = clk.stop()
    same = same and bool(torch.equal(out, ref))
    bad_status = int((st[:len(ops)] < 0).sum().item()) if len(ops) else 0
    del pool, out, st, ref, g
    B.close()
    torch.cuda.empty_cache()
    best = min(t_pers, t_steps, t_graph)
    return {"workload": f"{count} ragged instances, 2^15..2^19 bits log-uniform, 40% mul / 15% "
                        "add / 15% sub / 30% divmod (n_u in [n_v, 2 n_v])",
            "ops_per_s": count / (best * 1e-3), "per_class_ms": t_class,
            "persistent_ms": t_pers, "steps_ms": t_steps,
            "graph_form": "steps" if mode == bi.BATCH_STEPS else "persistent",
            "tuned_graph_ms": t_graph,
            "tuned_threads": threads, "speedup_vs_per_class": t_class / best, "clocks": clocks,
            "results_identical_across_forms": same, "negative_statuses": bad_status,
            "scaling": "strong" if world > 1 else None,
            "ranks": world}


def run_batched(args):
    """The batched form alone, as its own JSON line."""
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import ranks

    rank, local, world = ranks.world()
    dist, dev = None, torch.device("cuda", local)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    bi.load()
    blk = batched_block(torch, bi, args.batch_ops, max(args.steps, 1), rank, world, dist, dev)
    if rank == 0:
        line = {"metric": "batched form: ragged mixed-op instances per second",
                "value": blk["ops_per_s"], "unit": "ops/s", "n_gpus": world,
                "higher_is_better": True, "data": "synthetic",
                "scaling": "strong" if world > 1 else "weak",
                "config": {"workload": blk["workload"]}, **blk}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def kara_levels(n):
    """Karatsuba levels bigint_mul_kara's measured choice runs for square
    n-limb products (the library's rule: two from 8192 limbs, one from 4096,
    each level halving n exactly)."""
    L = 2 if n >= 8192 else (1 if n >= 4096 else 0)
    while L > 0 and n % (1 << L):
        L -= 1
    return L


def kara_form(n):
    L = kara_levels(n)
    if L == 0:
        return "tensor-core schoolbook product (bigint_mul)"
    return (f"Karatsuba, {L} level{'s' if L > 1 else ''} over {n >> L}-limb tensor-core "
            "products (bigint_mul_kara)")


def run_programs(args):
    """Tables I and II of Sec. VI on the sweep shapes (2^32 bits per operand
    array): 1-Add vs the fused 6-Add (GB/s over the 3 n 8 bytes one addition
    must move), and the full product (1-Mul) vs the fused Poly
    (a a + b)(b b + b) + a b mod B^n (ms per launch), CUDA events, best of
    the timed repetitions."""
    import torch

    import paper_2607_28897_gb300 as bi

    bi.load()
    sizes = [int(x) for x in args.sizes.split(",")]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def best_of(fn, reps):
        fn()
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return min(times)

    reps = max(args.steps, 1)
    rows = []
    for n in sizes:
        b = sweep_batch(n)
        g = torch.Generator(device="cuda")
        g.manual_seed(n)
        a = torch.randint(-2**62, 2**62, (b, n), dtype=torch.int64, device="cuda", generator=g)
        y = torch.randint(-2**62, 2**62, (b, n), dtype=torch.int64, device="cuda", generator=g)
        s = torch.empty_like(a)
        c = torch.empty(b, dtype=torch.uint8, device="cuda")
        bytes_ = 24.0 * b * n
        t1 = best_of(lambda: bi.add(a, y, out=s, carry=c), reps)
        t6 = best_of(lambda: bi.add_chain(a, y, 6, out=s, carry=c), reps)
        p = torch.empty((b, 2 * n), dtype=torch.int64, device="cuda")
        tm = best_of(lambda: bi.mul(a, y, out=p), reps)
        del p
        ws = torch.empty(bi.poly_workspace_bytes(b, n), dtype=torch.uint8, device="cuda")
        tp = best_of(lambda: bi.poly(a, y, out=s, workspace=ws), reps)
        rows.append({"limbs": n, "batch": b, "add1_GBs": bytes_ / (t1 * 1e-3) / 1e9,
                     "add6_GBs": bytes_ / (t6 * 1e-3) / 1e9, "mul_full_ms": tm, "poly_ms": tp,
                     "poly_over_mul": tp / tm})
        del a, y, s, c, ws
    line = {"metric": "fused programs: 6-Add GB/s and Poly ms (Tables I, II shapes)",
            "value": min(r["add6_GBs"] / r["add1_GBs"] for r in rows), "unit": "6-Add/1-Add",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "2^32 bits per operand array at 2^15..2^19 bits; 6-Add = a + 6 b "
                                   "(six fused additions), Poly = (a a + b)(b b + b) + a b mod B^n"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def serving_block(torch, bi, rates, requests, per_request_sample):
    """Continuous batching against one launch per request at Poisson
    arrival rates: throughput and p50/p99 latency per rate."""
    from paper_2607_28897_gb300 import serve

    res = []
    for rate in rates:
        w = serve.make_workload(41, requests, rate)
        # warm-up over the whole size range, so that the device and pinned
        # host allocators have grown to the sizes the timed run asks for
        serve.run_continuous(serve.make_workload(42, 2000, rate))
        c = serve.run_continuous(w)
        p = serve.run_per_request(w, limit=min(requests, per_request_sample))
        res.append({"rate": rate,
                    "continuous": {k: c[k] for k in ("throughput", "p50_ms", "p99_ms", "batches")},
                    "continuous_negative_statuses": int((c["status"] < 0).sum()),
                    "per_request": {k: p[k] for k in ("throughput", "p50_ms", "p99_ms")},
                    "per_request_sample": p["requests"]})
        del w
        torch.cuda.empty_cache()
    return {"workload": f"{requests} requests per rate, Poisson arrivals, 50% mul / 50% divmod, "
                        "sizes 2^15..2^19 bits log-uniform, HBM budget 64 GiB",
            "rates": res}


def run_serving(args):
    """Continuous batching against per-request launches at Poisson arrival
    rates; throughput and p50/p99 latency."""
    import torch

    import paper_2607_28897_gb300 as bi

    bi.load()
    blk = serving_block(torch, bi, [float(r) for r in args.rates.split(",")], args.requests,
                        5000)
    line = {"metric": "serving: requests/s and p50/p99 latency",
            "value": max(r["continuous"]["throughput"] for r in blk["rates"]),
            "unit": "req/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": blk["workload"]}, **blk}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
