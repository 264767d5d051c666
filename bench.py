#!/usr/bin/env python
"""Benchmark: CPTR-preconditioned FGMRES to a 1e-6 relative residual.

One step = one pass of the whole hot path on one system: cptr_setup
(Quasi-IMPES decoupling, system-AMG hierarchy, ILU(0) factors and schedules)
followed by cptr_solve (FGMRES(m) with the Eq. 3 preconditioner until
||b - A x|| <= 1e-6 ||b||).  Default workload: the 200x200x100 Cartesian system
(4,000,000 cells, 16M unknowns, 4x4 blocks, layered log-normal permeability
with sigma 2 and 10x vertical anisotropy, a 40 K cold plume, Peclet 1,
FGMRES(50)), synthetic and seeded; --config c3 (1M-point kNN cloud) and c2
(64x64x32) select the others.  value = solves per second over all ranks (each
rank solves its own replica).

Timing: W warm-up steps, then K steps each bracketed by CUDA events on the
library's stream, with a 512 MiB device write between steps to flush L2 (the
matrix alone is larger than L2 on the default workload).  Under torchrun every
rank does the same; the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CPTR-GMRES time-to-1e-6 residual & HBM GB/s; served p50/p99 latency vs plain FP64"
WORKLOADS = {
    "c4": ("cartesian 200x200x100 (4000000 cells, 16M DoF), 4x4 BSR thermal Jacobian, layered "
           "log-normal permeability sigma=2, 10x vertical anisotropy, 40 K cold plume, Pe=1, "
           "seed 1004; step = cptr_setup + cptr_solve (FGMRES(50), tol 1e-6)"),
    "c3": ("kNN cloud 200x200x25 jittered lattice (1000000 points, 4M DoF), k in 6..12, 4x4 BSR "
           "thermal Jacobian, Pe=10, seed 1003; step = cptr_setup + cptr_solve (FGMRES(30), "
           "tol 1e-6)"),
    "c2": ("cartesian 64x64x32 (131072 cells, 524288 DoF), 4x4 BSR thermal Jacobian, Pe=1, "
           "seed 1002; step = cptr_setup + cptr_solve (FGMRES(30), tol 1e-6)"),
}
RESTART = {"c2": 30, "c3": 30, "c4": 50}
# bounded CPU samples of each workload: the same generator on fewer layers
SLAB = {"c4": (10, 3), "c3": (4, 2), "c2": (32, 8)}  # (cpu_baseline layers, reference-arm layers)
FULL_LAYERS = {"c4": 100, "c3": 25, "c2": 32}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c4", choices=["c4", "c3", "c2"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--pe", type=float, default=None)
    ap.add_argument("--agg", type=int, default=0, choices=[0, 1, 2],
                    help="aggregate first AMG level of the headline solver (cptr_params.agg)")
    ap.add_argument("--coarsen", type=int, default=0, choices=[0, 1],
                    help="AMG coarsening of the headline solver: 0 PMIS, 1 HMIS")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip every leg after the headline")
    ap.add_argument("--serve-requests", type=int, default=512,
                    help="requests of the serving leg (0 skips it)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-batch-cells", type=int, default=0,
                    help="requests of at most this many cells are solved in batched launches")
    ap.add_argument("--serve-distinct", type=int, default=64,
                    help="distinct systems behind the serving requests")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving leg and print its JSON")
    ap.add_argument("--batch-systems", type=int, default=304,
                    help="systems of the batched-solve leg (0 skips it)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched-solve leg and print its JSON")
    ap.add_argument("--layers", type=int, default=0,
                    help="the workload's generator on this many layers (0: all); a smaller "
                         "case of the same structure for profiler captures")
    ap.add_argument("--profile-apply", type=int, default=0,
                    help="set up once, apply the preconditioner this many times and exit "
                         "(a bounded launch sequence for profiler captures)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1])); smax.append(float(p[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[5 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def host_cpu():
    """Core count and CPU model of this host (the CPU baseline's hardware)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def ncu_traffic(kernel_name: str, workload: str):
    """DRAM bytes per launch of a kernel from a committed ncu summary, if the
    summary was taken from the current source of that kernel on this workload."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[workload][kernel_name]
        src = os.path.join(ROOT, e["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return e["dram_bytes_per_launch"] if h == e["source_sha256_16"] else None
    except (OSError, KeyError, ValueError, TypeError):
        return None


def _replay(P, systems, rhs, arrivals, params, slots, batch_cells=0):
    """Submits request k (system k mod len(systems), right-hand side rhs[k]) at
    arrivals[k] seconds from the start to a server with `slots` slots; returns
    the arrival-to-result latencies (s), the makespan (s) and the iterations."""
    import numpy as np
    srv = P.cptr_server_create(96 << 30, slots, params)
    pending, lat, t_sub, iters = {}, [], {}, []
    t0 = time.perf_counter()
    k = 0
    try:
        P.cptr_server_set_limits(srv, 4096, batch_cells)
        while k < len(arrivals) or pending:
            now = time.perf_counter() - t0
            while k < len(arrivals) and arrivals[k] <= now:
                s = systems[k % len(systems)]
                rid = P.cptr_submit(srv, s.n_cells, s.rowptr, s.col, s.vals, rhs[k])
                pending[rid] = np.empty(4 * s.n_cells)
                t_sub[rid] = t0 + arrivals[k]
                k += 1
            for rid in list(pending):
                st, info = P.cptr_poll(srv, rid, pending[rid])
                if st != P._lib.PENDING:
                    if st not in (P._lib.OK, P._lib.ERR_MAXIT):
                        raise RuntimeError(f"serving request failed with status {st}: "
                                           f"{P.cptr_server_last_error(srv)}")
                    lat.append(time.perf_counter() - t_sub[rid])
                    iters.append(info["iters"])
                    del pending[rid]
            time.sleep(0.0002)
    finally:
        P.cptr_server_destroy(srv)
    return lat, time.perf_counter() - t0, iters


def c5_workload(n_requests=512, distinct=64):
    """The serving workload: n_requests Poisson arrivals (seed 1005, unit rate:
    scaled to the offered load by the caller) over `distinct` seeded systems,
    log-uniform in [8k, 500k] cells, 50/50 Cartesian / kNN, Peclet log-uniform in
    [0.01, 100]; request k solves system k mod distinct with its own N(0, 1)
    right-hand side.  Systems are generated by a process pool (spawn)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import numpy as np
    from synth.jacobian import build_request, serving_mix
    reqs = serving_mix(n_requests=n_requests, seed=1005, min_cells=8000, max_cells=500000)
    descs = reqs[:distinct]
    workers = max(1, min(16, (os.cpu_count() or 2) - 1, len(descs)))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        systems = list(ex.map(build_request, descs))
    rng = np.random.default_rng(1005)
    rhs = [rng.standard_normal(4 * systems[k % distinct].n_cells) for k in range(n_requests)]
    return np.array([r["t"] for r in reqs]), systems, rhs


def serving_leg(P, n_requests, slots=4, batch_cells=0, distinct=64):
    """Continuous batching on the serving workload (c5_workload) in mixed
    precision with `slots` slots (requests of at most batch_cells cells solved
    in batched launches), offered at 80% of the capacity measured with every
    request queued at once; the same arrival process served one request at a
    time in plain FP64 (no graphs, no batching) is the comparison, at the same
    offered load and at 80% of its own capacity."""
    import numpy as np
    t_gen = time.perf_counter()
    gaps, systems, rhs = c5_workload(n_requests, distinct)
    t_gen = time.perf_counter() - t_gen
    mixed = P.params(precision=P.MIXED)
    plain = P.params(precision=P.FP64, use_graphs=0)
    n = len(gaps)
    _replay(P, systems[:4], rhs[:4], [0.0] * 4, mixed, slots, batch_cells)  # warm-up
    _, t_cap, _ = _replay(P, systems, rhs, [0.0] * n, mixed, slots, batch_cells)
    capacity = n / t_cap
    rate = 0.8 * capacity
    lat, span, its = _replay(P, systems, rhs, list(gaps / rate), mixed, slots, batch_cells)
    lat64, span64, its64 = _replay(P, systems, rhs, list(gaps / rate), plain, 1)
    _, t_cap64, _ = _replay(P, systems, rhs, [0.0] * n, plain, 1)
    cap64 = n / t_cap64
    lat64s, span64s, _ = _replay(P, systems, rhs, list(gaps / (0.8 * cap64)), plain, 1)
    pct = lambda v, q: 1e3 * float(np.percentile(v, q))
    cells = [s.n_cells for s in systems]
    return {"requests": n, "distinct_systems": len(systems),
            "cells": [int(min(cells)), int(max(cells))],
            "mean_cells": float(np.mean([cells[k % len(cells)] for k in range(n)])),
            "slots": slots, "batch_max_cells": batch_cells,
            "capacity_solves_per_s": capacity, "rate_per_s": rate,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "solves_per_s": len(lat) / span,
            "mean_iters": float(np.mean(its)),
            "fp64_plain_one_at_a_time": {
                "capacity_solves_per_s": cap64,
                "same_offered_load": {"rate_per_s": rate, "p50_ms": pct(lat64, 50),
                                      "p99_ms": pct(lat64, 99),
                                      "solves_per_s": len(lat64) / span64},
                "own_80pct_load": {"rate_per_s": 0.8 * cap64,
                                   "p50_ms": pct(lat64s, 50), "p99_ms": pct(lat64s, 99),
                                   "solves_per_s": len(lat64s) / span64s},
                "mean_iters": float(np.mean(its64))},
            "capacity_ratio_vs_fp64_one_at_a_time": capacity / cap64,
            "generation_s": t_gen,
            "what": "arrival-to-result latency through cptr_submit/cptr_poll (host buffers); "
                    "each request: create + setup + solve + destroy, on its slot's stream "
                    "or, when small, solved in the next batched launch"}


def batch_leg(P, n_systems=304, seed=1006, reps=3):
    """Many small systems of uneven size solved in one launch (cptr_solve_batch,
    one thread block per system) against the same systems solved one after
    another through cptr_solve, in mixed precision and in plain FP64.  Systems:
    log-uniform 2k-30k cells, 50/50 Cartesian / kNN, Peclet log-uniform in
    [0.01, 100], each with its own right-hand side; all set up before timing
    (solve phase only).  Wall time of the whole call (host buffers)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import numpy as np
    from synth.jacobian import build_request, serving_mix
    descs = serving_mix(n_requests=n_systems, seed=seed, min_cells=2000, max_cells=30000)
    workers = max(1, min(16, (os.cpu_count() or 2) - 1, len(descs)))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        systems = list(ex.map(build_request, descs))
    cells = [s.n_cells for s in systems]
    out = {"systems": len(systems), "cells": [int(min(cells)), int(max(cells))],
           "mean_cells": float(np.mean(cells))}

    def timed(fn):
        best = None
        for _ in range(reps):
            t = time.perf_counter()
            r = fn()
            dt = time.perf_counter() - t
            best = dt if best is None or dt < best else best
        return best, r

    for name, prec in (("mixed", P.MIXED), ("fp64", P.FP64)):
        gs = [P.Solver.from_system(s, precision=prec, tri_tune=0).setup() for s in systems]
        try:
            xs = [np.zeros(4 * s.n_cells) for s in systems]

            def batched():
                for x in xs:
                    x[:] = 0.0
                return P.cptr_solve_batch([g.h for g in gs], [s.rhs for s in systems], xs)

            def one_by_one():
                its = []
                for g, s, x in zip(gs, systems, xs):
                    x[:] = 0.0
                    _, info = g.solve(s.rhs, x)
                    its.append(info["iters"])
                return its

            tb, (st, infos) = timed(batched)
            res = max(float(np.linalg.norm(s.rhs - _bsr_mv(s, x)) / np.linalg.norm(s.rhs))
                      for s, x in zip(systems, xs))
            ts, its = timed(one_by_one)
            out[name] = {"batched_solves_per_s": len(systems) / tb,
                         "one_by_one_solves_per_s": len(systems) / ts,
                         "speedup": ts / tb, "status": st,
                         "iters_batched": [int(np.min([i["iters"] for i in infos])),
                                           int(np.max([i["iters"] for i in infos]))],
                         "iters_one_by_one": [int(np.min(its)), int(np.max(its))],
                         "max_rel_resid_batched": res}
        finally:
            for g in gs:
                g.close()
    out["batched_mixed_vs_fp64_one_by_one"] = (out["mixed"]["batched_solves_per_s"] /
                                               out["fp64"]["one_by_one_solves_per_s"])
    return out


def _bsr_mv(s, x):
    import numpy as np
    rows = np.repeat(np.arange(s.n_cells), np.diff(s.rowptr))
    prod = np.einsum("bij,bj->bi", s.vals.reshape(-1, 4, 4), x.reshape(-1, 4)[s.col])
    y = np.zeros((s.n_cells, 4))
    np.add.at(y, rows, prod)
    return y.ravel()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def kernel_roof(ms: float, nbytes: float, flops: float, fp64: bool, peak_gbs: float,
                fma: dict) -> dict:
    """One kernel's place on the roofline: achieved GB/s and TFLOP/s, each as a
    fraction of its measured roof (copy bandwidth; FMA rate of the kernel's
    precision), and the roof with the larger time floor.  Without a measured
    FMA rate (fma holds an error) the compute floor is zero and HBM the roof."""
    fp = "fp64" if fp64 else "fp32"
    rate = fma.get(fp + "_tflops", float("inf"))
    t_hbm, t_fma = nbytes / (peak_gbs * 1e6), flops / (rate * 1e9)  # ms at each roof
    return {"ms": ms, "bytes": nbytes, "GBps": nbytes / (ms * 1e6),
            "frac": nbytes / (ms * 1e6) / peak_gbs, "flops": flops, "fp": fp,
            "TFLOPs": flops / (ms * 1e9), "fma_frac": flops / (ms * 1e9) / rate,
            "roof": "hbm" if t_hbm >= t_fma else fp, "roof_frac": max(t_hbm, t_fma) / ms}


def max_over_ranks(v: float, device) -> float:
    """The largest value over the ranks of the default process group (any
    backend), or v itself without one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, slowest_ms: float) -> float:
    """Solves per second of the whole job: every rank solves `steps` systems
    (its own replica) and the job lasts as long as its slowest rank."""
    return world * steps / (slowest_ms / 1e3)


def oracle_sample(config: str, layers: int, full_iters: int | None, reps: int = 1):
    """The FP64 CPU oracle (one thread) on the workload's generator with `layers`
    layers instead of the full count: setup + solve wall seconds per rep, scaled
    to the full workload by the cell count (and, for the solve, by the ratio of
    the full workload's iteration count to the sample's, when known)."""
    import oracle
    from synth import config_slab
    oracle.build()
    s = config_slab(config, layers)
    scale = FULL_LAYERS[config] / layers
    out = []
    for _ in range(reps):
        t0 = time.perf_counter()
        o = oracle.Oracle.from_system(s, restart=RESTART[config]).setup()
        t1 = time.perf_counter()
        _, info = o.solve(s.rhs)
        t2 = time.perf_counter()
        it_scale = (full_iters / info["iters"]) if full_iters and info["iters"] else 1.0
        out.append({"setup_s": t1 - t0, "solve_s": t2 - t1, "iters": info["iters"],
                    "scaled_s": scale * ((t1 - t0) + (t2 - t1) * it_scale)})
    return s.n_cells, scale, out


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The FP64 CPU oracle on the host cores, same workload and metric; each
    step is a bounded sample (the workload's generator on fewer layers) whose
    time is scaled to the full workload by the cell count."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    layers = SLAB[args.config][1]
    n_s, scale, runs = oracle_sample(args.config, layers, None, args.warmup + args.steps)
    runs = runs[args.warmup:]
    tot = sum(r["scaled_s"] for r in runs)
    value = len(runs) / tot
    cpu = host_cpu()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / len(runs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config] + " (FP64 CPU oracle)",
                   "parallelism": "single core"},
        "iters_sample": runs[-1]["iters"],
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "host": cpu,
                         "sample": f"each step: oracle setup + FGMRES on the workload's generator "
                                   f"with {layers} of {FULL_LAYERS[args.config]} layers "
                                   f"({n_s} cells), time scaled x{scale:g} by the cell count"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def timed_steps(P, torch, stream, flush, h, b, x, n):
    """n steps of setup + solve, each bracketed by CUDA events after an L2 flush."""
    ms, infos = [], []
    with torch.cuda.stream(stream):
        for _ in range(n):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            x.zero_()
            e0.record(stream)
            P.cptr_setup(h)
            _, info = P.cptr_solve(h, b, x)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
    return ms, infos


def form_leg(P, torch, stream, flush, s, b, dev, restart, reps=3, **kw):
    """Setup + solve of one solver form (extra keyword parameters), first rep untimed."""
    with P.Solver.from_system(s, restart=restart, **kw) as g:
        P.cptr_set_stream(g.h, stream.cuda_stream)
        x = torch.zeros_like(b)
        ms, infos = timed_steps(P, torch, stream, flush, g.h, b, x, reps + 1)
        xh = x.cpu().numpy()
    ms, infos = ms[1:], infos[1:]
    return {"ms_per_step": statistics.mean(ms),
            "setup_ms": 1e3 * statistics.mean(i["setup_s"] for i in infos),
            "solve_ms": 1e3 * statistics.mean(i["solve_s"] for i in infos),
            "iters": infos[-1]["iters"], "status": infos[-1]["status"]}, xh


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2308_11892_gb300 import build as _build
    _build.build()
    import paper_2308_11892_gb300 as P
    from synth import config_system

    if args.batch_only:
        if rank == 0:
            print(json.dumps({"batch": batch_leg(P, args.batch_systems)}), flush=True)
        return 0
    if args.serve_only:
        if rank == 0:
            print(json.dumps({"serving": serving_leg(P, args.serve_requests, args.serve_slots,
                                                     args.serve_batch_cells,
                                                     args.serve_distinct)}), flush=True)
        return 0
    cfg = args.config
    amg = {"agg": args.agg, "coarsen": args.coarsen}
    m = RESTART[cfg]
    if args.layers:
        from synth import config_slab
        s = config_slab(cfg, args.layers)
    else:
        s = config_system(cfg, pe=args.pe)
    if args.profile_apply:
        prec = P.MIXED if args.precision == "mixed" else P.FP64
        with P.Solver.from_system(s, precision=prec, restart=m, **amg).setup() as g:
            b = torch.from_numpy(s.rhs).to(dev)
            out = torch.zeros_like(b)
            for _ in range(args.profile_apply):
                P.cptr_apply(g.h, P.APPLY_PRECOND, b, out)
            torch.cuda.synchronize()
            print(json.dumps({"profile_apply": args.profile_apply, "cells": s.n_cells,
                              "tri_schedule": P.cptr_get_info(g.h)["tri_schedule"]}))
        return 0
    prec = P.MIXED if args.precision == "mixed" else P.FP64
    stream = torch.cuda.Stream(device=dev)
    solver = P.Solver.from_system(s, precision=prec, restart=m, **amg)
    P.cptr_set_stream(solver.h, stream.cuda_stream)
    b = torch.from_numpy(s.rhs).to(dev)
    x = torch.zeros_like(b)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    timed_steps(P, torch, stream, flush, solver.h, b, x, args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    if rank == 0:
        clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = P.cptr_get_info(solver.h)["launches"]
    step_ms, infos = timed_steps(P, torch, stream, flush, solver.h, b, x, args.steps)
    torch.cuda.synchronize()
    launches = P.cptr_get_info(solver.h)["launches"] - launches0
    if world > 1:
        torch.distributed.barrier()
    tot_ms = sum(step_ms)
    clk = clocks.stop() if rank == 0 else None
    tot_ms = max_over_ranks(tot_ms, dev)
    value = job_throughput(world, args.steps, tot_ms)
    last = infos[-1]
    x_host = x.cpu().numpy()

    extras = {}
    if rank == 0 and not args.no_extras:
        import oracle
        oracle.build()
        o = oracle.Oracle.from_system(s, restart=m)
        rel = float(np.linalg.norm(s.rhs - o.spmv(x_host)) / np.linalg.norm(s.rhs))
        del o
        extras["true_rel_resid"] = rel
        # ---- where the setup goes: one more setup with phase timing (synchronising)
        P.cptr_setup_timing(solver.h, True)
        with torch.cuda.stream(stream):
            P.cptr_setup(solver.h)
        torch.cuda.synchronize()
        ph = P.cptr_setup_phases(solver.h)
        P.cptr_setup_timing(solver.h, False)
        with torch.cuda.stream(stream):
            P.cptr_setup(solver.h)
            x.zero_()
            P.cptr_solve(solver.h, b, x)
        torch.cuda.synchronize()
        extras["setup_phases_ms"] = {k: round(v, 3) for k, v in ph.items()}
        # ---- roofline: every profiled kernel, dominant = largest time per solve
        peak, peak_kind = measured_peaks()
        its = last["iters"]
        per_solve = {P.KERNEL_SPMV: its + 1, P.KERNEL_ILU_FWD: its, P.KERNEL_ILU_BWD: its,
                     P.KERNEL_VC_PRE0: its, P.KERNEL_CORRECTION: its, P.KERNEL_MDOT: its}
        tri = {0: "k_ilu_{}", 1: "k_tri_cluster<{}>", 2: "k_tri_strip<{}>",
               3: "k_tri_chain<{}>"}.get(last["tri_schedule"], "k_tri_chunk<{}>")
        names = {P.KERNEL_SPMV: "k_bsr_spmv", P.KERNEL_ILU_FWD: tri.format("fwd"),
                 P.KERNEL_ILU_BWD: tri.format("bwd"), P.KERNEL_VC_PRE0: "k_vc_pre",
                 P.KERNEL_CORRECTION: "k_correction", P.KERNEL_MDOT: "k_cgs_dot"}
        kern = {}
        step_avg = tot_ms / args.steps
        # the compute roof: this device's FMA rate in each precision, measured
        # by the library's FMA-chain kernel (every result checked on the host)
        try:
            fma = {"fp64_tflops": P.cptr_fma_rate(True, 4096, reps=5, stream=stream.cuda_stream),
                   "fp32_tflops": P.cptr_fma_rate(False, 1 << 17, reps=5,
                                                  stream=stream.cuda_stream),
                   "kernel": "k_fma_chains: 8 independent FMA chains per thread, 8 x 256 "
                             "threads per SM, CUDA events, every thread's result checked"}
        except P.CPTRError as e:  # the compute roof is auxiliary: keep the HBM one
            fma = {"error": str(e)}
        extras["fma_rate"] = fma
        with torch.cuda.stream(stream):
            for k, cnt in per_solve.items():
                ms, nbytes = P.cptr_profile_kernel(solver.h, k, 10)
                fl, f64 = P.cptr_kernel_flops(solver.h, k)
                kern[names[k]] = dict(kernel_roof(ms, nbytes, fl, f64, peak, fma),
                                      per_solve=cnt, ms_per_solve=ms * cnt,
                                      share_of_step=ms * cnt / step_avg,
                                      traffic=ncu_traffic(names[k], cfg))
        dom = max(kern, key=lambda k: kern[k]["ms_per_solve"])
        d = kern[dom]
        if d["roof"] == "hbm":
            extras["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": d["GBps"],
                                  "peak": peak, "unit": "GB/s", "frac": d["frac"],
                                  "traffic": ncu_traffic(dom, cfg),
                                  "algorithmic_bytes": d["bytes"], "avg_launch_ms": d["ms"],
                                  "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"}
        else:
            extras["roofline"] = {"bound": "alu", "kernel": dom, "achieved": d["TFLOPs"],
                                  "peak": fma[d["fp"] + "_tflops"], "unit": "TFLOP/s",
                                  "frac": d["fma_frac"], "traffic": ncu_traffic(dom, cfg),
                                  "algorithmic_flops": d["flops"], "avg_launch_ms": d["ms"],
                                  "peak_source": f"measured {d['fp']} FMA rate (fma_rate)"}
        extras["kernels"] = {k: {kk: (round(vv, 6) if isinstance(vv, float) else vv)
                                 for kk, vv in v.items()} for k, v in kern.items()}
        extras["setup_share_of_step"] = {k: round(v / step_avg, 4) for k, v in ph.items()}
        # ---- the FP64 forms: graph-captured (same engine) and plain (no graphs,
        # the comparison point of the target), each with its setup/solve split
        f64, x64 = form_leg(P, torch, stream, flush, s, b, dev, m, precision=P.FP64, **amg)
        plain, xp = form_leg(P, torch, stream, flush, s, b, dev, m, precision=P.FP64,
                             use_graphs=0, **amg)
        mixed_setup = 1e3 * statistics.mean(i["setup_s"] for i in infos)
        mixed_solve = 1e3 * statistics.mean(i["solve_s"] for i in infos)
        extras["mixed"] = {"ms_per_step": step_avg, "setup_ms": mixed_setup,
                           "solve_ms": mixed_solve, "iters": last["iters"]}
        extras["fp64"] = f64
        extras["fp64_plain"] = dict(plain, speedup_of_value=plain["ms_per_step"] / step_avg,
                                    solve_speedup=plain["solve_ms"] / mixed_solve)
        extras["mixed_vs_fp64_x_relerr"] = float(np.linalg.norm(x_host - xp) /
                                                 np.linalg.norm(xp))
        del x64, xp
        # ---- end to end through the C ABI with host buffers (copies timed)
        # Newton-loop use: one context per system; every step uploads the new
        # Jacobian values and rhs from pinned host memory, rebuilds the
        # preconditioner, solves and reads x back (all inside the timed region)
        vals_h = torch.from_numpy(np.ascontiguousarray(s.vals)).pin_memory()
        rhs_h = torch.from_numpy(s.rhs).pin_memory()
        x_h = torch.zeros(4 * s.n_cells, dtype=torch.float64).pin_memory()
        e2e_t = []
        with P.Solver.from_system(s, precision=prec, restart=m, **amg) as ge:
            for k in range(6):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                P.cptr_update_values(ge.h, vals_h)
                ge.setup()
                x_h.zero_()
                ge.solve(rhs_h, x_h)
                if k > 0:
                    e2e_t.append(time.perf_counter() - t0)
        h2d = vals_h.numel() * 8 + rhs_h.numel() * 8 + x_h.numel() * 8
        extras["e2e"] = {"value": 1.0 / statistics.median(e2e_t), "unit": "solves/s",
                         "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(x_h.numel() * 8),
                         "what": "cptr_update_values(pinned host values) + cptr_setup + "
                                 "cptr_solve(pinned host rhs and x) on one context, wall clock, "
                                 "median of 5"}
        del vals_h
        cold = []
        for k in range(2):
            xh = np.zeros(4 * s.n_cells)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with P.Solver.from_system(s, precision=prec, restart=m, **amg) as ge:
                ge.setup()
                ge.solve(s.rhs, xh)
            cold.append(time.perf_counter() - t0)
        extras["e2e_cold"] = {"value": 1.0 / statistics.median(cold), "unit": "solves/s",
                              "what": "cptr_create(host BSR) + cptr_setup + cptr_solve + "
                                      "cptr_destroy per system, wall clock, median of 2"}
        # ---- the other workloads: mixed and plain FP64 setup + solve each
        others = {}
        for oc in [c for c in ("c4", "c3", "c2") if c != cfg]:
            so = config_system(oc)
            bo = torch.from_numpy(so.rhs).to(dev)
            mx, xm = form_leg(P, torch, stream, flush, so, bo, dev, RESTART[oc],
                              precision=P.MIXED)
            pl, xq = form_leg(P, torch, stream, flush, so, bo, dev, RESTART[oc],
                              precision=P.FP64, use_graphs=0)
            others[oc] = {"workload": WORKLOADS[oc], "mixed": mx, "fp64_plain": pl,
                          "mixed_vs_fp64_x_relerr":
                              float(np.linalg.norm(xm - xq) / np.linalg.norm(xq)),
                          "speedup_of_step": pl["ms_per_step"] / mx["ms_per_step"]}
            del so, bo
        extras["other_workloads"] = others
        # ---- first MGR reduction (Section 3.4), one aggregate level (reading R8)
        # and CPR vs CPTR over the Peclet sweep, on the 64x64x32 grid
        extras.update(c2_variant_legs(P, torch, stream, flush, dev, prec, np))
        # ---- many small systems in one launch vs one after another
        if args.batch_systems > 0:
            extras["batched_small_systems"] = batch_leg(P, args.batch_systems)
        # ---- serving: continuous batching vs one-at-a-time plain FP64
        if args.serve_requests > 0:
            extras["serving"] = serving_leg(P, args.serve_requests, args.serve_slots,
                                            args.serve_batch_cells, args.serve_distinct)
        # ---- CPU baseline: the oracle on one host core, bounded sample
        layers = SLAB[cfg][0]
        n_s, scale, runs = oracle_sample(cfg, layers, last["iters"])
        r0 = runs[0]
        extras["cpu_baseline"] = {
            "value": 1.0 / r0["scaled_s"], "unit": "solves/s", "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": f"single-threaded FP64 C oracle, setup + FGMRES({m}) on the workload's "
                      f"generator with {layers} of {FULL_LAYERS[cfg]} layers ({n_s} cells): "
                      f"setup {r0['setup_s']:.2f} s, solve {r0['solve_s']:.2f} s in "
                      f"{r0['iters']} iterations; scaled x{scale:g} by the cell count and the "
                      f"solve by {last['iters']}/{r0['iters']} iterations"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == P.MIXED else "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[cfg], "precision": args.precision,
                       "l2": "flushed between steps (512 MiB device write); inputs larger "
                             "than L2",
                       "parallelism": f"replicas x{world}",
                       "amg": {"agg": args.agg, "coarsen": "hmis" if args.coarsen else "pmis"}},
            "iters": last["iters"], "rel_resid": last["rel_resid"],
            "setup_ms": 1e3 * last["setup_s"], "solve_ms": 1e3 * last["solve_s"],
            "amg_levels": last["amg_levels"], "ilu_levels": last["ilu_levels"],
            "op_complexity": last["op_complexity"], "tri_schedule": last["tri_schedule"],
            "step_ms": [round(v, 4) for v in step_ms],
            "gpu_launches": int(launches) * world,
            "clocks": clk,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def c2_variant_legs(P, torch, stream, flush, dev, prec, np):
    """The variants on the 64x64x32 grid: the first MGR reduction (Section 3.4)
    reduced and unreduced, one aggregate level on the first AMG level (reading
    R8) against the default, HMIS against PMIS coarsening (Section 3.1), and
    CPR and CPTR3 against CPTR over the Peclet sweep (Sections 3.1-3.3, 5.3)."""
    from synth import config_system, with_volume_constraint
    out = {}
    s = config_system("c2")
    b = torch.from_numpy(s.rhs).to(dev)
    sm = with_volume_constraint(s, seed=7)
    bm = torch.from_numpy(sm.rhs).to(dev)
    rows_m = np.repeat(np.arange(sm.n_cells), np.diff(sm.rowptr))
    vm = sm.vals.reshape(-1, 4, 4)

    def full_resid(xv):
        ax = np.zeros((sm.n_cells, 4))
        np.add.at(ax, rows_m, np.einsum("bij,bj->bi", vm, xv.reshape(-1, 4)[sm.col]))
        return float(np.linalg.norm(sm.rhs - ax.ravel()) / np.linalg.norm(sm.rhs))

    mgr = {"workload": "64x64x32 grid with a local volume-constraint row 2 "
                       "(synth.with_volume_constraint, seed 7)"}
    for label, mflag in (("reduced", 1), ("unreduced", 0)):
        r, xm = form_leg(P, torch, stream, flush, sm, bm, dev, 30, precision=prec, mgr=mflag)
        r["true_rel_resid"] = full_resid(xm)
        mgr[label] = r
    out["mgr"] = mgr
    agg = {}
    for aflag in (2, 1, 0):
        with P.Solver.from_system(s, precision=prec, agg=aflag) as ga:
            P.cptr_set_stream(ga.h, stream.cuda_stream)
            xa = torch.zeros_like(b)
            ms, infos = timed_steps(P, torch, stream, flush, ga.h, b, xa, 4)
            ia = infos[-1]
            agg[{2: "agg_multipass", 1: "agg", 0: "default"}[aflag]] = {
                "ms_per_step": statistics.mean(ms[1:]), "setup_ms": ia["setup_s"] * 1e3,
                "iters": ia["iters"], "amg_levels": ia["amg_levels"],
                "op_complexity": ia["op_complexity"], "status": ia["status"]}
    out["aggressive_first_level"] = agg
    coarsen = {}
    for name, cflag in (("hmis", P.COARSEN_HMIS), ("pmis", P.COARSEN_PMIS)):
        with P.Solver.from_system(s, precision=prec, coarsen=cflag) as gc:
            P.cptr_set_stream(gc.h, stream.cuda_stream)
            xc = torch.zeros_like(b)
            ms, infos = timed_steps(P, torch, stream, flush, gc.h, b, xc, 4)
            ic = infos[-1]
            coarsen[name] = {
                "ms_per_step": statistics.mean(ms[1:]), "setup_ms": ic["setup_s"] * 1e3,
                "solve_ms": ic["solve_s"] * 1e3, "iters": ic["iters"],
                "amg_levels": ic["amg_levels"], "op_complexity": ic["op_complexity"],
                "status": ic["status"]}
    out["hmis_vs_pmis"] = coarsen
    cmp = {}
    for pe in (0.01, 1.0, 100.0):
        sp = config_system("c2", pe=pe)
        bs = torch.from_numpy(sp.rhs).to(dev)
        for name, kw in (("cptr", {}), ("cpr", {"e0": 0, "e1": -1}),
                         ("cptr3", {"precond": P.PREC_CPTR3})):
            r, _ = form_leg(P, torch, stream, flush, sp, bs, dev, 30, reps=1, precision=prec,
                            **kw)
            cmp[f"{name}_pe{pe:g}"] = r
    out["cpr_vs_cptr"] = cmp
    return out


if __name__ == "__main__":
    sys.exit(main())
