#!/usr/bin/env python
"""Benchmark of the fused GI-preconditioned cascaded stream-collide step.

Workload (default): 4096 x 4096 lid-driven cavity, U = 0.1, Re = 1000,
gamma = 0.5, FP32 storage and collision, started from rest.  A "step" is one
full time step of the domain (one launch of the stream-collide kernel).

Prints one JSON line (rank 0).  value = cell updates per second over all
ranks (MLUPS); each rank advances its own replica of the domain (the path is
data-parallel over independent domains; no collective on the data path), so
scaling is weak.  Inputs (1.2 GB of populations per replica) exceed the 129 MB
L2, so no L2 flush is needed between steps.

The default line also carries "batch": the batch study (steady solves/s of
the FP16 batch against the plain FP32 solver one domain at a time) on the first
--batch-domains cavities of the seeded 256-cavity set, with the FP16 results'
error against the oracle's stored steady states.

--impl reference times the FP64 CPU oracle on the host cores instead.

Other workloads (--workload, each prints its own JSON line): batch (the batch
study on --batch-count domains, with FP64-storage GPU references across the
sizes), serve (a Poisson stream of steady-solve requests into the batch engine:
latency percentiles per request kind, aggregate MLUPS), precision (storage
formats to steady state on a scaled obstacle channel, against FP64 storage),
gamma (steps to steady state per preconditioning parameter), cylinder (wake
length and drag of the square cylinder in a channel, Re 5-60).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and steady-state solves/sec (FP16-storage batched vs plain FP32) at L2≤1e-3"
BYTES_PER_CELL = {"f32": 72, "f16": 36, "bf16": 36, "f64": 144}
STORAGE_CODE = {"f32": 0, "f16": 1, "bf16": 2, "f64": 3}
KERNEL_SOURCES = ["paper_1806_10251_gb300/csrc/stream_collide_x2.cuh",
                  "paper_1806_10251_gb300/csrc/collide_x2.cuh",
                  "paper_1806_10251_gb300/csrc/f32x2.cuh",
                  "paper_1806_10251_gb300/csrc/stream_collide.cuh",
                  "paper_1806_10251_gb300/csrc/d2q9_collide.cuh",
                  "paper_1806_10251_gb300/csrc/open_bc.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=list(STORAGE_CODE), default="f32")
    ap.add_argument("--n", "--side", dest="n", type=int, default=4096,
                    help="cavity side (--side also under torchrun, whose parser takes --n as an abbreviation)")
    ap.add_argument("--gamma", type=float, default=0.5)
    ap.add_argument("--Re", type=float, default=1000.0)
    ap.add_argument("--gi-mode", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-domains", type=int, default=32,
                    help="default line: the batch study (FP16 batch vs plain FP32 steady solves/s) on the first N "
                         "cavities of the seeded 256-cavity set; 0 leaves it out")
    ap.add_argument("--batch-refs", type=int, default=0,
                    help="default line: FP64-storage GPU references of the batch study besides the oracle ones")
    ap.add_argument("--reference-budget-s", type=float, default=150.0,
                    help="--impl reference: stop the timed oracle steps after this many seconds")
    ap.add_argument("--e2e-check-every", type=int, default=100)
    ap.add_argument("--cells-per-item", type=int, default=0,
                    help="rows per work item of the step kernel (0 = automatic)")
    ap.add_argument("--workload", choices=["cavity", "batch", "serve", "precision", "gamma", "cylinder"], default="cavity",
                    help="cavity: the timed step of one large domain (default); batch: steady solves/s of "
                         "independent cavities, FP16 batch against the plain FP32 solver one domain at a time; "
                         "serve: a Poisson stream of steady-solve requests into the batch engine")
    ap.add_argument("--batch-count", type=int, default=256, help="batch: first N cavities of the seeded set")
    ap.add_argument("--tol", type=float, default=1e-3, help="batch/serve: steady when r < tol between checks")
    ap.add_argument("--check-every", type=int, default=1000)
    ap.add_argument("--max-steps", type=int, default=400000)
    ap.add_argument("--accuracy-sample", type=int, default=3,
                    help="batch: domains spread over the sizes whose results are compared with an FP64-storage "
                         "GPU steady state (besides the oracle steady states stored for the smallest ones)")
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--rate", type=float, default=2.0, help="serve: mean arrivals per second")
    ap.add_argument("--request-max-steps", type=int, default=100000,
                    help="serve: steps after which a request is returned as not converged")
    ap.add_argument("--cyl-d", type=int, default=16, help="cylinder: side of the square cylinder in cells")
    ap.add_argument("--serve-wall-s", type=float, default=600.0,
                    help="serve: the session ends this long after the first arrival (what is left is cancelled)")
    ap.add_argument("--admission", type=int, choices=[0, 1], default=1,
                    help="serve: 0 first come first served, 1 smallest domain first")
    ap.add_argument("--max-running-cells", type=float, default=32e6,
                    help="serve: admit while the running domains hold at most this many cells (0: no cap)")
    ap.add_argument("--lid-mach", type=float, default=0.05, help="gamma: lid speed over c_s")
    ap.add_argument("--side-min", type=int, default=128)
    ap.add_argument("--side-max", type=int, default=512)
    ap.add_argument("--scale", type=int, default=16,
                    help="precision: linear scale-down of the 8192 x 2048 obstacle channel")
    return ap.parse_args()


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fp:
            h.update(fp.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fp:
            d = json.load(fp)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(storage: str, n: int, rows_per_item=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", f"stream_collide_{storage}_cavity{n}.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_sources_sha256") != kernel_hash():
        return None
    if rows_per_item is not None and vals.get("rows_per_item") not in (None, str(rows_per_item)):
        return None  # another work decomposition than the one the counters were taken on
    try:
        return int(float(vals["dram_bytes_per_launch"]))
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.proc = None
        self.device_id = device_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.device_id:
            cmd += ["-i", self.device_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        sm, mx, reasons = [], [], set()
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, dist, device):
    """The job's time is its slowest rank's: the max of a per-rank float over
    all ranks (the value itself when there is one rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(cells_per_rank, steps, world, seconds):
    """Whole-job cell updates per second (MLUPS): every rank advances its own
    replica for the same number of steps (weak scaling)."""
    return cells_per_rank * steps * world / seconds / 1e6


def cpu_baseline(case_fn, seconds_target=15.0):
    """The FP64 oracle as it stands, on the host cores, over a bounded sample."""
    import oracle as orc
    c = case_fn()
    d = orc.Domain(c.nx, c.ny, c.nu, c.gamma, c.sides)
    d.init_equilibrium()
    d.step(1)  # first touch
    t = time.perf_counter()
    d.step(1)
    one = time.perf_counter() - t
    n = max(1, min(50, int(seconds_target / max(one, 1e-6))))
    t = time.perf_counter()
    d.step(n)
    el = time.perf_counter() - t
    return {"value": c.cells * n / el / 1e6, "unit": "MLUPS", "cores": orc.get_threads(), "kind": "oracle",
            "sample": f"{c.name}: {n} oracle steps of the full domain (FP64, OpenMP over rows)"}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle as orc
    import workloads as wl
    # the same workload as the GPU arm: each step is one oracle step of the whole
    # domain (about 0.2 s for 4096^2 on 16 cores); the timed sample stops at the
    # step count or the time budget, whichever comes first
    side = args.n
    c = wl.cavity(side, args.Re, 0.1, args.gamma)
    d = orc.Domain(c.nx, c.ny, c.nu, c.gamma, c.sides, gi_mode=args.gi_mode)
    d.init_equilibrium()
    d.step(args.warmup)
    done = 0
    t = time.perf_counter()
    while done < args.steps:
        d.step(1)
        done += 1
        if time.perf_counter() - t > args.reference_budget_s:
            break
    el = time.perf_counter() - t
    v = c.cells * done / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "steps_timed": done, "warmup": args.warmup, "ms_per_step": el / done * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"lid-driven cavity {side}x{side}, U=0.1, Re={args.Re:g}, "
                                   f"gamma={args.gamma:g}, GI mode {args.gi_mode}, from rest", "storage": "f64"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": orc.get_threads(), "kind": "oracle",
                             "sample": f"{done} of {args.steps} oracle steps of the whole {side}x{side} cavity "
                                       f"after {args.warmup} warm-up steps (time budget "
                                       f"{args.reference_budget_s:g} s)"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def rel_l2(u, v, uo, vo, mask=None):
    import numpy as np
    if mask is None:
        mask = np.ones(u.shape, bool)
    d = ((u - uo) ** 2 + (v - vo) ** 2)[mask].sum()
    n = (uo ** 2 + vo ** 2)[mask].sum()
    return float(np.sqrt(d / n))


BATCH_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "batch_sample_steady.npz")


def check_interval(case, K, transits=8.0):
    """Steps between a domain's convergence checks: about `transits` crossings
    of the domain at the preconditioned convection speed U/gamma (n gamma / U
    steps each), at least K and a multiple of K.  A residual taken over an
    interval shorter than the slowest decay time stops a large domain far from
    its steady state (on the GB300 runs, r < 1e-3 between checks 10 000 steps
    apart left 1024^2 cavities 2.5e-3 away); over this interval the remaining
    distance is a small fraction of r."""
    import math
    n = max(case.nx, case.ny)
    t = transits * n * case.gamma / max(case.U, 1e-12)
    return int(K * max(1, math.ceil(t / K)))


def batch_study(count, K, tol, mx, n_fp64_refs=3, ref_tol=1e-7):
    """Steady solves per second on the first `count` cavities of the seeded set
    (sides 64 + 32k, k ~ U{0..30}; Re ~ U[100, 1000]; gamma ~ U[0.2, 1.0];
    U = 0.1): (a) the plain FP32 path one domain at a time (lbm_run_to_steady:
    one launch per step, no graph), (b) one FP16 batch (lbm_batch_*: all domains
    in lockstep under a captured CUDA graph).  Both stop a domain at the first
    check where r < tol (checks K steps apart).  Accuracy of both arms: the L2
    error of u against the FP64 oracle's steady state for the set's smallest
    cavities (stored by tests/golden/make_batch_sample_steady.py) and against
    FP64-storage GPU runs driven to r < ref_tol (the FP64 GPU path equals the
    oracle to 1e-12 per step) for n_fp64_refs domains spread over the sizes."""
    import numpy as np
    import torch

    import workloads as wl
    from paper_1806_10251_gb300 import lbm

    cases = wl.batch_cavities(256, seed=0)[:count]
    cells = sum(c.cells for c in cases)
    golden = {}
    if os.path.exists(BATCH_GOLDEN):
        z = np.load(BATCH_GOLDEN)
        golden = {int(i): (z[f"ux_{int(i)}"].astype(np.float64), z[f"uy_{int(i)}"].astype(np.float64))
                  for i in z["indices"] if int(i) < count}
    others = sorted((i for i in range(count) if i not in golden), key=lambda i: cases[i].cells)
    spread = sorted({others[int(round(q * (len(others) - 1)))] for q in np.linspace(0, 1, n_fp64_refs)}) \
        if others and n_fp64_refs > 0 else []
    sample = sorted(set(golden) | set(spread))
    # (a) plain FP32, sequential
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res_a, fields_a = [], {}
    kk = [check_interval(c, K) for c in cases]
    for i, c in enumerate(cases):
        g = lbm.Solver(c.nx, c.ny, c.nu, c.gamma, c.U)
        st, steps, r = g.run_to_steady(tol, kk[i], mx, raise_on_error=False)
        res_a.append((st, steps, r))
        if i in sample:
            fields_a[i] = g.fields()[1:]
        g.close()
    t_a = time.perf_counter() - t0
    upd_a = sum(c.cells * x[1] for c, x in zip(cases, res_a))
    # (b) FP16 batch
    b = lbm.Batch(64 << 30, storage=lbm.STORAGE_F16)
    b.set_option("check_every", K)
    t0 = time.perf_counter()
    ids = [b.submit_case(c, tol=tol, max_steps=mx, check_every=k) for c, k in zip(cases, kk)]
    b.run()
    t_b = time.perf_counter() - t0
    res_b = [b.poll(i)[1] for i in ids]
    stats = b.stats()
    fields_b = {i: b.fields(ids[i], cases[i].nx, cases[i].ny)[1:] for i in sample}
    b.close()
    acc = []
    for i in sample:
        c = cases[i]
        if i in golden:
            uo, vo = golden[i]
            ref = "fp64 oracle"
        else:
            g = lbm.Solver(c.nx, c.ny, c.nu, c.gamma, c.U)
            g.set_option("storage", lbm.STORAGE_F64)
            st, steps, r = g.run_to_steady(ref_tol, kk[i], 4_000_000, raise_on_error=False)
            _, uo, vo = g.fields()
            g.close()
            ref = f"fp64-storage GPU, r={r:.1e}"
        conv_a, conv_b = res_a[i][0] == 0, res_b[i].state == lbm.REQ_CONVERGED
        acc.append({"index": i, "side": c.nx, "Re": round(c.meta["Re"], 1), "gamma": round(c.gamma, 3),
                    "reference": ref,
                    "l2_fp16_batch": rel_l2(*fields_b[i], uo, vo) if conv_b else None,
                    "l2_fp32_plain": rel_l2(*fields_a[i], uo, vo) if conv_a else None})
    conv_a = sum(1 for x in res_a if x[0] == 0)
    conv_b = sum(1 for x in res_b if x.state == lbm.REQ_CONVERGED)
    l2b = [x["l2_fp16_batch"] for x in acc if x["l2_fp16_batch"] is not None]
    return {"metric": "steady solves/s (FP16 batch vs plain FP32)", "unit": "solves/s",
            "value": count / t_b, "plain_fp32": {"value": count / t_a, "seconds": t_a, "converged": conv_a,
                                                "steps": sum(x[1] for x in res_a), "mlups": upd_a / t_a / 1e6},
            "fp16_batch": {"value": count / t_b, "seconds": t_b, "converged": conv_b,
                           "steps": sum(x.steps for x in res_b), "launches": stats["launches"],
                           "mlups": stats["cell_updates"] / t_b / 1e6},
            "speedup": t_a / t_b, "max_l2_fp16_batch": max(l2b) if l2b else None,
            "config": {"domains": count, "cells": cells, "tol": tol, "check_every": K,
                       "check_rule": "per domain: K * ceil(8 n gamma / (U K)) steps, both arms", "max_steps": mx,
                       "set": "batch_cavities(256, seed=0)" + (f"[:{count}]" if count < 256 else ""),
                       "gi_mode": "full", "storage_b": "f16 (stochastic rounding)", "storage_a": "f32"},
            "accuracy_sample": acc}


def run_batch(args, rank):
    """--workload batch: the batch study on the first --batch-count domains."""
    import torch
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    line = batch_study(args.batch_count, args.check_every, args.tol, args.max_steps, args.accuracy_sample)
    line.update({"workload": "batch", "higher_is_better": True, "data": "synthetic"})
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args, rank):
    """Serving: a Poisson stream of steady-solve requests (cavity or obstacle
    channel, p = 1/2; side on multiples of 32 in [side-min, side-max]; Re ~
    U[50, 1000]; gamma ~ U[0.2, 1.0]; FP16 storage) submitted at their arrival
    times to the batch engine running on a background thread (continuous
    batching: admission by device footprint as memory frees up).  Each request
    carries a step cap and the check interval of the batch study
    (check_interval); the session ends --serve-wall-s after the first arrival,
    cancelling what is still queued or running then.  Reports converged / not
    converged / diverged / cancelled counts per kind, the arrival-to-done
    latency percentiles of all requests and of the converged ones, queue waits,
    the aggregate MLUPS and the queue depth."""
    import numpy as np
    import torch

    import workloads as wl
    from paper_1806_10251_gb300 import lbm
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    reqs = wl.poisson_requests(count=args.requests, rate=args.rate, seed=0, side_min=args.side_min,
                               side_max=args.side_max)
    budget = 24 << 30
    b = lbm.Batch(budget, storage=lbm.STORAGE_F16)
    b.set_option("check_every", args.check_every)
    b.set_option("admission", args.admission)
    b.set_option("max_running_cells", args.max_running_cells)
    b.start()
    t0 = time.perf_counter()
    ids, kinds, pending, done = [], {}, set(), {}
    depth = []

    def harvest():
        for rid in list(pending):
            fin, res = b.poll(rid)
            if fin:
                done[rid] = res
                pending.discard(rid)
                b.release(rid)

    for ta, c in reqs:
        while True:
            now = time.perf_counter() - t0
            if now >= ta:
                break
            harvest()
            time.sleep(min(0.002, ta - now))
        rid = b.submit_case(c, tol=args.tol, max_steps=args.request_max_steps,
                            check_every=check_interval(c, args.check_every))
        ids.append(rid)
        kinds[rid] = "cavity" if c.name.startswith("cavity") else "channel"
        pending.add(rid)
        st = b.stats()
        depth.append((st["running"], st["queued"]))
    cancelled_at = None
    while pending:
        harvest()
        if cancelled_at is None and time.perf_counter() - t0 > args.serve_wall_s:
            cancelled_at = time.perf_counter() - t0
            for rid in list(pending):
                try:
                    b.cancel(rid)
                except lbm.LbmError:
                    pass  # finished meanwhile
        time.sleep(0.002)
    wall = time.perf_counter() - t0
    stats = b.stats()
    b.stop()
    b.close()
    names = {lbm.REQ_CONVERGED: "converged", lbm.REQ_NOT_CONVERGED: "not_converged",
             lbm.REQ_DIVERGED: "diverged", lbm.REQ_CANCELLED: "cancelled", lbm.REQ_FAILED: "failed"}

    def pct(x):
        x = np.asarray(x)
        return ({"p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99)), "n": int(x.size)}
                if x.size else {"n": 0})

    lat = {i: done[i].t_done - done[i].t_submit for i in ids}
    per_kind = {}
    for kind in ("cavity", "channel"):
        mine = [i for i in ids if kinds[i] == kind]
        counts = {v: 0 for v in names.values()}
        for i in mine:
            counts[names.get(done[i].state, "failed")] += 1
        per_kind[kind] = {"requests": len(mine), **counts,
                          "latency_converged_s": pct([lat[i] for i in mine if done[i].state == lbm.REQ_CONVERGED])}
    queue = [done[i].t_admit - done[i].t_submit for i in ids if done[i].t_admit > 0]
    conv = [lat[i] for i in ids if done[i].state == lbm.REQ_CONVERGED]
    line = {"metric": "arrival-to-steady latency and aggregate MLUPS (serving, FP16 batch engine)",
            "workload": "serve", "value": pct(conv).get("p50"), "unit": "s (p50 latency of converged requests)",
            "higher_is_better": False,
            "latency_all_s": pct(list(lat.values())), "latency_converged_s": pct(conv),
            "queue_wait_s": pct(queue), "per_kind": per_kind,
            "aggregate_mlups": stats["cell_updates"] / wall / 1e6, "wall_s": wall,
            "cancelled_at_s": cancelled_at,
            "max_running": int(max(d[0] for d in depth)), "max_queued": int(max(d[1] for d in depth)),
            "requests": len(ids),
            "config": {"rate_per_s": args.rate, "requests": args.requests, "side": [args.side_min, args.side_max],
                       "request_max_steps": args.request_max_steps, "session_wall_s": args.serve_wall_s,
                       "tol": args.tol, "check_every": args.check_every,
                       "admission": ["first come first served", "smallest domain first"][args.admission],
                       "max_running_cells": args.max_running_cells, "ticks": stats["ticks"],
                       "check_rule": "per request: check_interval (8 transits)", "budget_bytes": budget,
                       "stream": "poisson_requests(seed=0)"},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_cylinder(args, rank):
    """Flow past the square cylinder in a channel (Sec. 6: 50 D x 8 D, cylinder
    at 12.5 D, parabolic inflow of peak U = 0.1, convective outflow, gamma =
    0.5): for each Reynolds number (U D / nu) the steady field (FP32, r < 2e-7
    between checks 1000 steps apart), the recirculation length behind the rear
    face on the channel axis against the printed correlation L_r / D = -0.065 +
    0.0554 Re (5 < Re < 60), and the drag coefficient from the momentum
    exchange, C_D = 2 gamma F_x / (rho0 U^2 D) (the preconditioned momentum
    equation divides every flux by gamma)."""
    import numpy as np
    import torch

    import workloads as wl
    from paper_1806_10251_gb300 import lbm
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    rows = []
    for Re in (5.0, 10.0, 20.0, 30.0, 40.0, 50.0, 60.0):
        c = wl.square_cylinder(args.cyl_d, Re, 0.1, 0.5)
        g = lbm.solver_from_case(c)
        t = time.perf_counter()
        st, steps, r = g.run_to_steady(2e-7, 1000, 3_000_000, raise_on_error=False)
        sec = time.perf_counter() - t
        _, u, _ = g.fields()
        F = g.drag()
        m = c.meta
        ya = int(m["y_axis"])
        ax = 0.5 * (u[ya, :] + u[ya + 1, :])
        k = int(np.ceil(m["x_rear"]))
        Lr = 0.0
        if ax[k] < 0:
            while k < c.nx - 1 and not (ax[k] < 0 <= ax[k + 1]):
                k += 1
            Lr = (k + (-ax[k]) / (ax[k + 1] - ax[k]) - m["x_rear"]) / m["D"]
        g.close()
        rows.append({"Re": Re, "Lr_over_D": Lr, "correlation": -0.065 + 0.0554 * Re,
                     "C_D": 2 * c.gamma * F[0] / (0.1 ** 2 * m["D"]), "C_L": 2 * c.gamma * F[1] / (0.1 ** 2 * m["D"]),
                     "steps": steps, "residual": r, "status": st, "seconds": sec})
    line = {"metric": "square-cylinder wake length and drag (Sec. 6)", "workload": "cylinder",
            "value": float(np.mean([abs(x["Lr_over_D"] / x["correlation"] - 1) for x in rows if x["Re"] >= 10])),
            "unit": "mean relative deviation of L_r/D from the correlation (Re 10-60)", "higher_is_better": False,
            "rows": rows, "config": {"D": args.cyl_d, "U": 0.1, "gamma": 0.5, "storage": "f32", "gi_mode": "full",
                                     "channel": "50 D x 8 D, cylinder at 12.5 D"},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args, rank):
    """Storage precision on a geometry-scaled copy of the obstacle channel
    (8192 x 2048, square obstacle of side 128 centred at (1024, 1024), walls in
    y, periodic in x, body force F_x = 8 nu U0 / H^2, Re = 40 on the obstacle,
    U0 = 0.05, gamma = 0.3), every length divided by --scale.  Each storage
    runs to its steady criterion (checks 10 000 steps apart); errors are relative
    L2 against the FP64-storage run (the GPU FP64 path matches the oracle to
    1e-12 per step): u over fluid cells, rho as sum (rho - rho64)^2 over
    sum (rho64 - mean rho64)^2."""
    import numpy as np
    import torch

    import workloads as wl
    from paper_1806_10251_gb300 import lbm
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    k = args.scale
    c = wl.channel_obstacle(nx=8192 // k, ny=2048 // k, D=128 // k, Re=40.0, U0=0.05, gamma=0.3, xc=1024 // k)
    fluid = c.solid == 0
    runs = [("f64", 3, 1, 1e-10), ("f32", 0, 1, 2e-7), ("f16", 1, 1, 1e-3), ("bf16", 2, 1, 1e-2),
            ("f16_nearest", 1, 0, 1e-3)]
    out, ref = [], None
    for name, st, sr, tol in runs:
        g = lbm.solver_from_case(c, storage=st)
        if st in (1, 2):
            g.set_option("stochastic_rounding", sr)
        t0 = time.perf_counter()
        status, steps, r = g.run_to_steady(tol, args.check_every, args.max_steps, raise_on_error=False)
        dt = time.perf_counter() - t0
        rho, ux, uy = g.fields()
        g.close()
        if ref is None:
            ref = (rho, ux, uy)
        r64, u64, v64 = ref
        l2u = rel_l2(ux, uy, u64, v64, fluid)
        d = rho - r64
        l2r = float(np.sqrt((d[fluid] ** 2).sum() / ((r64[fluid] - r64[fluid].mean()) ** 2).sum()))
        du = float(max(np.abs(ux - u64)[fluid].max(), np.abs(uy - v64)[fluid].max()) / c.U)
        out.append({"storage": name, "status": int(status), "steps": int(steps), "residual": float(r), "tol": tol,
                    "seconds": dt, "l2_u": l2u, "l2_rho": l2r, "max_du_over_U0": du,
                    "u_max": float(np.abs(ux[fluid]).max())})
    line = {"metric": "steady-state error of u and rho per storage format against FP64 storage",
            "workload": "precision", "value": out[2]["l2_u"], "unit": "relative L2 of u (FP16)",
            "higher_is_better": False, "runs": out,
            "config": {"case": c.name, "scale": k, "nx": c.nx, "ny": c.ny, "nu": c.nu, "Fx": c.Fx,
                       "gamma": c.gamma, "check_every": args.check_every, "max_steps": args.max_steps},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_gamma(args, rank):
    """Convergence acceleration by preconditioning (the paper's steady-state
    claim): the lid-driven cavity of side --n at --Re with the lid at Mach
    --lid-mach (U = Ma c_s), for gamma = 1, 0.5, 0.25, 0.1, 0.05, all in one FP32
    batch started from rest; a domain stops at the first check (--check-every
    steps apart) with r < --tol.  Reports the steps to steady state per gamma,
    their ratio to gamma = 1, and the relative L2 distance of each steady field
    from the gamma = 1 one (the steady state does not depend on gamma up to the
    discretisation)."""
    import numpy as np
    import torch

    import workloads as wl
    from paper_1806_10251_gb300 import lbm
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    U = args.lid_mach / np.sqrt(3.0)
    gammas = [1.0, 0.5, 0.25, 0.1, 0.05]
    cases = [wl.cavity(args.n, args.Re, U, g) for g in gammas]
    b = lbm.Batch(16 << 30, storage=lbm.STORAGE_F32)
    b.set_option("check_every", args.check_every)
    ids = [b.submit_case(c, tol=args.tol, max_steps=args.max_steps) for c in cases]
    t0 = time.perf_counter()
    b.run()
    wall = time.perf_counter() - t0
    res = [b.poll(i)[1] for i in ids]
    fields = [b.fields(i, c.nx, c.ny) for i, c in zip(ids, cases)]
    b.close()
    _, u1, v1 = fields[0]
    base, base_conv = res[0].steps, res[0].state == lbm.REQ_CONVERGED
    runs = []
    for g, r, (_, u, v) in zip(gammas, res, fields):
        conv = r.state == lbm.REQ_CONVERGED
        run = {"gamma": g, "state": int(r.state), "converged": conv, "steps": int(r.steps),
               "residual": float(r.residual), "l2_vs_gamma1": rel_l2(u, v, u1, v1) if conv else None}
        if conv:
            # gamma = 1 not converged within max_steps: the ratio is a lower bound
            run["speedup_vs_gamma1" if base_conv else "speedup_vs_gamma1_at_least"] = base / r.steps
        if r.state == lbm.REQ_DIVERGED:
            # retry alone with the strain-solve guard (reading A8; the batch kernel has no guard)
            c = wl.cavity(args.n, args.Re, U, g)
            sg = lbm.solver_from_case(c, guard=1)
            st, steps, rr = sg.run_to_steady(args.tol, args.check_every, args.max_steps, raise_on_error=False)
            _, ug, vg = sg.fields()
            run["with_guard"] = {"status": int(st), "steps": int(steps), "residual": float(rr),
                                 "guard_events": int(sg.guard_count),
                                 "l2_vs_gamma1": rel_l2(ug, vg, u1, v1) if st == 0 else None}
            if st == 0:
                run["with_guard"]["speedup_vs_gamma1" if base_conv else "speedup_vs_gamma1_at_least"] = base / steps
            sg.close()
        runs.append(run)
    line = {"metric": "steps to steady state per gamma (preconditioned convergence acceleration)",
            "workload": "gamma", "value": max(r.get("speedup_vs_gamma1", r.get("speedup_vs_gamma1_at_least", 0.0))
                                              for r in runs),
            "unit": "x fewer steps than gamma = 1 (best converged gamma; a lower bound if gamma = 1 did not converge)",
            "higher_is_better": True, "runs": runs, "wall_s": wall,
            "config": {"n": args.n, "Re": args.Re, "U": U, "lid_mach": args.lid_mach, "tol": args.tol,
                       "check_every": args.check_every, "max_steps": args.max_steps, "storage": "f32", "gi_mode": "full"},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "batch":
        return run_batch(args, rank)
    if args.workload == "serve":
        return run_serve(args, rank)
    if args.workload == "precision":
        return run_precision(args, rank)
    if args.workload == "gamma":
        return run_gamma(args, rank)
    if args.workload == "cylinder":
        return run_cylinder(args, rank)

    import numpy as np
    import torch

    import workloads as wl
    from paper_1806_10251_gb300 import lbm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    lbm.use_torch_allocator()
    case = wl.cavity(args.n, args.Re, 0.1, args.gamma)
    g = lbm.Solver(case.nx, case.ny, case.nu, case.gamma, case.U)
    g.set_option("gi_mode", args.gi_mode)
    if args.storage != "f32":
        g.set_option("storage", STORAGE_CODE[args.storage])
    if args.cells_per_item:
        g.set_option("cells_per_item", args.cells_per_item)
    # A dedicated stream: its handle is non-zero, so the library launches on it
    # and the CUDA events below time exactly those launches.
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    g.set_stream(stream.cuda_stream)

    # ---- device-resident throughput (value) --------------------------------
    for _ in range(args.warmup):
        g.step(1)
    torch.cuda.synchronize()
    barrier()
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        dev_id = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
    except Exception:
        dev_id = None
    clocks = ClockSampler(dev_id)
    clocks.start()
    time.sleep(0.3)
    l0 = g.kernel_launches
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        g.step(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = g.kernel_launches - l0
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    cells = case.cells
    value = job_mlups(cells, args.steps, world, ms / 1e3)
    per_launch_s = ms / 1e3 / args.steps
    bpc = BYTES_PER_CELL[args.storage]
    achieved = bpc * cells / per_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    r, _ = g.residual()
    assert np.isfinite(r), "non-finite state after the timed steps"

    # ---- end to end through the public API with pinned host buffers --------
    ce = max(1, min(args.e2e_check_every, args.steps))
    nchunks = max(1, args.steps // ce)
    e2e_steps = nchunks * ce
    pin = lambda: torch.empty((case.ny, case.nx), dtype=torch.float64, pin_memory=True).numpy()
    rho0, ux0, uy0 = pin(), pin(), pin()
    rho0[:] = 1.0
    ux0[:] = 0.0
    uy0[:] = 0.0
    outs = (pin(), pin(), pin())
    g2 = lbm.Solver(case.nx, case.ny, case.nu, case.gamma, case.U)
    g2.set_option("gi_mode", args.gi_mode)
    if args.storage != "f32":
        g2.set_option("storage", STORAGE_CODE[args.storage])
    if args.cells_per_item:
        g2.set_option("cells_per_item", args.cells_per_item)
    g2.set_stream(stream.cuda_stream)
    g2.init_fields(rho0, ux0, uy0)
    g2.step(args.warmup)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    g2.init_fields(rho0, ux0, uy0)
    for _ in range(nchunks):
        g2.step(ce)
        g2.residual()
    g2.fields(out=outs)
    t1 = time.perf_counter()
    e2e_s = max_over_ranks(t1 - t0, dist, "cuda")
    field_bytes = 3 * cells * 8
    e2e = {"value": job_mlups(cells, e2e_steps, world, e2e_s), "unit": "MLUPS",
           "h2d_bytes_per_step": field_bytes / e2e_steps,
           "d2h_bytes_per_step": (field_bytes + nchunks * 40) / e2e_steps,
           "calls": f"lbm_init_fields + {nchunks} x (lbm_step({ce}) + lbm_residual) + lbm_fields, pinned host arrays"}
    g2.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage != "f64" else "f64",
            "data": "synthetic",
            "config": {"workload": f"lid-driven cavity {args.n}x{args.n}, U=0.1, Re={args.Re:g}, "
                                   f"gamma={args.gamma:g}, GI mode {args.gi_mode}, from rest",
                       "storage": args.storage, "replicas": world,
                       "rows_per_item": int(g.get_option("cells_per_item")),
                       "grid": int(g.get_option("grid")),
                       "l2": "no flush: populations (per replica) exceed the 129 MB L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": profiled_traffic(args.storage, args.n, int(g.get_option("cells_per_item"))),
                         "bytes_per_cell": bpc,
                         "kernel": "stream_collide_kernel" if args.storage == "f64" else "stream_collide_x2_kernel"},
            "gpu_launches": launches,
            "e2e": e2e,
            "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(lambda: wl.cavity(args.n, args.Re, 0.1, args.gamma))
        if world == 1 and args.batch_domains > 0:
            # the headline's second half: a bounded prefix of the seeded batch set
            line["batch"] = batch_study(args.batch_domains, 10000, 1e-3, 1_000_000, n_fp64_refs=args.batch_refs)
        print(json.dumps(line), flush=True)
    g.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
