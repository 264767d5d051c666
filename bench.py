#!/usr/bin/env python
"""Benchmark: CPTR-preconditioned FGMRES to a 1e-6 relative residual.

One step = one pass of the whole hot path on one system: cptr_setup
(Quasi-IMPES decoupling, system-AMG hierarchy, ILU(0) factors and schedules)
followed by cptr_solve (FGMRES(30) with the Eq. 3 preconditioner until
||b - A x|| <= 1e-6 ||b||).  Workload: the 64x64x32 Cartesian system
(131,072 cells, 524,288 unknowns, 4x4 blocks, Peclet 1), synthetic and seeded.
value = solves per second over all ranks (each rank solves its own replica).

Timing: W warm-up steps, then K steps each bracketed by CUDA events on the
library's stream, with a 512 MiB device write between steps to flush L2.
Under torchrun every rank does the same; the max over ranks is reported.
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
WORKLOAD = ("cartesian 64x64x32 (131072 cells, 524288 DoF), 4x4 BSR thermal Jacobian, Pe=1, "
            "seed 1002; step = cptr_setup + cptr_solve (FGMRES(30), tol 1e-6)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--pe", type=float, default=1.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the e2e, FP64, roofline, serving and CPU-baseline legs")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests of the serving leg (0 skips it)")
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


def ncu_traffic(kernel_name: str):
    """DRAM bytes per launch of a kernel from a committed ncu summary, if the
    summary was taken from the current source of that kernel."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel_name]
        src = os.path.join(ROOT, e["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return e["dram_bytes_per_launch"] if h == e["source_sha256_16"] else None
    except (OSError, KeyError, ValueError):
        return None


def _replay(P, systems, arrivals, params, slots):
    """Submits each system at its arrival time (seconds from start) to a server
    with `slots` slots; returns per-request latencies (s) and the makespan."""
    import numpy as np
    srv = P.cptr_server_create(64 << 30, slots, params)
    pending, lat, t_sub = {}, [], {}
    t0 = time.perf_counter()
    k = 0
    try:
        while k < len(systems) or pending:
            now = time.perf_counter() - t0
            while k < len(systems) and arrivals[k] <= now:
                s = systems[k]
                rid = P.cptr_submit(srv, s.n_cells, s.rowptr, s.col, s.vals, s.rhs)
                pending[rid] = np.zeros(4 * s.n_cells)
                t_sub[rid] = t0 + arrivals[k]
                k += 1
            for rid in list(pending):
                st, info = P.cptr_poll(srv, rid, pending[rid])
                if st != P._lib.PENDING:
                    if st not in (P._lib.OK, P._lib.ERR_MAXIT):
                        raise RuntimeError(f"serving request failed with status {st}")
                    lat.append(time.perf_counter() - t_sub[rid])
                    del pending[rid]
            time.sleep(0.0002)
    finally:
        P.cptr_server_destroy(srv)
    return lat, time.perf_counter() - t0


def serving_leg(P, n_requests):
    """Poisson arrivals of seeded systems (Cartesian and kNN, 8k-128k cells, Pe
    log-uniform in [0.01, 100]) served with 4 slots in mixed precision, at 80% of
    the capacity measured with every request queued at once; the same arrival
    process served one at a time in plain FP64 is the comparison."""
    import numpy as np
    from synth.jacobian import build_request, serving_mix
    reqs = serving_mix(n_requests=n_requests, seed=1005, min_cells=8000, max_cells=128000)
    systems = [build_request(r) for r in reqs]
    mixed = P.params(precision=P.MIXED)
    plain = P.params(precision=P.FP64, use_graphs=0)
    _replay(P, systems[:4], [0.0] * 4, mixed, 4)                # warm-up
    _, t_cap = _replay(P, systems, [0.0] * len(systems), mixed, 4)
    capacity = len(systems) / t_cap
    rate = 0.8 * capacity
    gaps = np.array([r["t"] for r in reqs])  # unit-rate Poisson arrivals
    arrivals = list(gaps / rate)
    lat, span = _replay(P, systems, arrivals, mixed, 4)
    lat64, span64 = _replay(P, systems, arrivals, plain, 1)
    pct = lambda v, q: 1e3 * float(np.percentile(v, q))
    return {"requests": len(systems), "cells": [int(min(s.n_cells for s in systems)),
                                                  int(max(s.n_cells for s in systems))],
            "slots": 4, "capacity_solves_per_s": capacity, "rate_per_s": rate,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "solves_per_s": len(lat) / span,
            "fp64_plain_one_at_a_time": {"p50_ms": pct(lat64, 50), "p99_ms": pct(lat64, 99),
                                         "solves_per_s": len(lat64) / span64},
            "what": "arrival-to-result latency through cptr_submit/cptr_poll (host buffers); "
                    "each request: create + setup + solve + destroy on its own stream"}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


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


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The FP64 CPU oracle on the host cores, same workload and metric."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from synth import config_system
    oracle.build()
    s = config_system("c2", pe=args.pe)
    times, its = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o = oracle.Oracle.from_system(s).setup()
        x, info = o.solve(s.rhs)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt); its.append(info["iters"])
    tot = sum(times)
    value = len(times) / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (FP64 CPU oracle)", "parallelism": "single core"},
        "iters": its[-1],
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(times)} full solves (setup + FGMRES) of the workload"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
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

    s = config_system("c2", pe=args.pe)
    prec = P.MIXED if args.precision == "mixed" else P.FP64
    stream = torch.cuda.Stream(device=dev)
    solver = P.Solver.from_system(s, precision=prec)
    P.cptr_set_stream(solver.h, stream.cuda_stream)
    b = torch.from_numpy(s.rhs).to(dev)
    x = torch.zeros_like(b)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step():
        x.zero_()
        P.cptr_setup(solver.h)
        st, info = P.cptr_solve(solver.h, b, x)
        return info

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    if rank == 0:
        clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = P.cptr_get_info(solver.h)["launches"]
    evs = []
    infos = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(step())
            e1.record(stream)
            evs.append((e0, e1))
    torch.cuda.synchronize()
    launches = P.cptr_get_info(solver.h)["launches"] - launches0
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(bb) for a, bb in evs]
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
        o = oracle.Oracle.from_system(s)
        rel = float(np.linalg.norm(s.rhs - o.spmv(x_host)) / np.linalg.norm(s.rhs))
        extras["true_rel_resid"] = rel
        # ---- roofline: every profiled kernel, dominant = largest time per solve
        peak, peak_kind = measured_peaks()
        its = last["iters"]
        per_solve = {P.KERNEL_SPMV: its + 1, P.KERNEL_ILU_FWD: its, P.KERNEL_ILU_BWD: its,
                     P.KERNEL_VC_PRE0: its, P.KERNEL_CORRECTION: its, P.KERNEL_MDOT: 2 * its}
        tri = {0: "k_ilu_{}", 1: "k_tri_cluster<{}>"}.get(last["tri_schedule"],
                                                           "k_tri_chunk<{}>")
        names = {P.KERNEL_SPMV: "k_bsr_spmv", P.KERNEL_ILU_FWD: tri.format("fwd"),
                 P.KERNEL_ILU_BWD: tri.format("bwd"), P.KERNEL_VC_PRE0: "k_vc_pre",
                 P.KERNEL_CORRECTION: "k_correction", P.KERNEL_MDOT: "k_cgs_dot"}
        kern = {}
        with torch.cuda.stream(stream):
            for k, cnt in per_solve.items():
                ms, nbytes = P.cptr_profile_kernel(solver.h, k, 10)
                kern[names[k]] = {"ms": ms, "bytes": nbytes, "GBps": nbytes / (ms * 1e6),
                                  "frac": nbytes / (ms * 1e6) / peak, "per_solve": cnt,
                                  "ms_per_solve": ms * cnt}
        dom = max(kern, key=lambda k: kern[k]["ms_per_solve"])
        d = kern[dom]
        traffic = ncu_traffic(dom)
        extras["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": d["GBps"], "peak": peak,
                              "unit": "GB/s", "frac": d["frac"], "traffic": traffic,
                              "algorithmic_bytes": d["bytes"], "avg_launch_ms": d["ms"],
                              "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"}
        extras["kernels"] = {k: {kk: (round(vv, 6) if isinstance(vv, float) else vv)
                                 for kk, vv in v.items()} for k, v in kern.items()}
        # ---- plain FP64 GPU form (no graphs): the comparison point of the target
        with P.Solver.from_system(s, precision=P.FP64, use_graphs=0) as g64:
            P.cptr_set_stream(g64.h, stream.cuda_stream)
            x64 = torch.zeros_like(b)
            t64 = []
            with torch.cuda.stream(stream):
                for k in range(4):
                    flush.fill_(1)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    x64.zero_()
                    e0.record(stream)
                    P.cptr_setup(g64.h)
                    _, i64 = P.cptr_solve(g64.h, b, x64)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    if k >= 1:
                        t64.append(e0.elapsed_time(e1))
            xd = x64.cpu().numpy()
        extras["fp64_plain"] = {"ms_per_step": statistics.mean(t64), "iters": i64["iters"],
                                "speedup_of_value": statistics.mean(t64) / (tot_ms / args.steps)}
        extras["mixed_vs_fp64_x_relerr"] = float(np.linalg.norm(x_host - xd) / np.linalg.norm(xd))
        # ---- end to end through the C ABI with host buffers (copies timed)
        # Newton-loop use: one context per system; every step uploads the new
        # Jacobian values and rhs from pinned host memory, rebuilds the
        # preconditioner, solves and reads x back (all inside the timed region)
        vals_h = torch.from_numpy(np.ascontiguousarray(s.vals)).pin_memory()
        rhs_h = torch.from_numpy(s.rhs).pin_memory()
        x_h = torch.zeros(4 * s.n_cells, dtype=torch.float64).pin_memory()
        e2e_t = []
        with P.Solver.from_system(s, precision=prec) as ge:
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
        cold = []
        for k in range(3):
            xh = np.zeros(4 * s.n_cells)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with P.Solver.from_system(s, precision=prec) as ge:
                ge.setup()
                ge.solve(s.rhs, xh)
            cold.append(time.perf_counter() - t0)
        extras["e2e_cold"] = {"value": 1.0 / statistics.median(cold), "unit": "solves/s",
                              "what": "cptr_create(host BSR) + cptr_setup + cptr_solve + "
                                      "cptr_destroy per system, wall clock, median of 3"}
        # ---- first MGR reduction (Section 3.4): the same grid with equation row 2
        # a cell-local volume constraint, solved reduced (mgr=1) and unreduced
        from synth import with_volume_constraint
        sm = with_volume_constraint(s, seed=7)
        bm = torch.from_numpy(sm.rhs).to(dev)
        rows_m = np.repeat(np.arange(sm.n_cells), np.diff(sm.rowptr))
        vm = sm.vals.reshape(-1, 4, 4)

        def full_resid(xv):
            ax = np.zeros((sm.n_cells, 4))
            np.add.at(ax, rows_m, np.einsum("bij,bj->bi", vm, xv.reshape(-1, 4)[sm.col]))
            return float(np.linalg.norm(sm.rhs - ax.ravel()) / np.linalg.norm(sm.rhs))

        mgr = {"workload": "c2 grid with a local volume-constraint row 2 "
                           "(synth.with_volume_constraint, seed 7)"}
        with torch.cuda.stream(stream):
            for label, mflag in (("reduced", 1), ("unreduced", 0)):
                with P.Solver.from_system(sm, precision=prec, mgr=mflag) as gm:
                    P.cptr_set_stream(gm.h, stream.cuda_stream)
                    xm = torch.zeros_like(bm)
                    tm = []
                    for k in range(4):
                        flush.fill_(1)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        xm.zero_()
                        e0.record(stream)
                        P.cptr_setup(gm.h)
                        _, im = P.cptr_solve(gm.h, bm, xm)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        if k >= 1:
                            tm.append(e0.elapsed_time(e1))
                    mgr[label] = {"ms_per_step": statistics.mean(tm), "iters": im["iters"],
                                  "status": im["status"],
                                  "true_rel_resid": full_resid(xm.cpu().numpy())}
        extras["mgr"] = mgr
        # ---- one aggregate level on the first AMG level (reading R8) vs the default
        agg = {}
        with torch.cuda.stream(stream):
            for aflag in (1, 0):
                with P.Solver.from_system(s, precision=prec, agg=aflag) as ga:
                    P.cptr_set_stream(ga.h, stream.cuda_stream)
                    xa = torch.zeros_like(b)
                    ta = []
                    for k in range(4):
                        flush.fill_(1)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        xa.zero_()
                        e0.record(stream)
                        P.cptr_setup(ga.h)
                        _, ia = P.cptr_solve(ga.h, b, xa)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        if k >= 1:
                            ta.append(e0.elapsed_time(e1))
                    agg["agg" if aflag else "default"] = {
                        "ms_per_step": statistics.mean(ta), "setup_ms": ia["setup_s"] * 1e3,
                        "iters": ia["iters"], "amg_levels": ia["amg_levels"],
                        "op_complexity": ia["op_complexity"], "status": ia["status"]}
        extras["aggressive_first_level"] = agg
        # ---- CPR (pressure-only first stage) vs CPTR over the Peclet sweep
        cmp = {}
        with torch.cuda.stream(stream):
            for pe in (0.01, 1.0, 100.0):
                sp = config_system("c2", pe=pe)
                xs = torch.zeros(4 * sp.n_cells, dtype=torch.float64, device=dev)
                bs = torch.from_numpy(sp.rhs).to(dev)
                for name, kw in (("cptr", {}), ("cpr", {"e0": 0, "e1": -1})):
                    with P.Solver.from_system(sp, precision=prec, **kw) as gs:
                        P.cptr_set_stream(gs.h, stream.cuda_stream)
                        for k in range(2):  # the first setup also tunes
                            xs.zero_()
                            torch.cuda.synchronize()
                            t0 = time.perf_counter()
                            P.cptr_setup(gs.h)
                            _, info = P.cptr_solve(gs.h, bs, xs)
                            torch.cuda.synchronize()
                            dt = time.perf_counter() - t0
                        cmp[f"{name}_pe{pe:g}"] = {"iters": info["iters"],
                                                   "ms_per_step": 1e3 * dt,
                                                   "setup_ms": 1e3 * info["setup_s"],
                                                   "solve_ms": 1e3 * info["solve_s"]}
        extras["cpr_vs_cptr"] = cmp
        # ---- serving: continuous batching vs one-at-a-time plain FP64
        if args.serve_requests > 0:
            extras["serving"] = serving_leg(P, args.serve_requests)
        # ---- CPU baseline: the oracle on one host core, one full solve
        t0 = time.perf_counter()
        o2 = oracle.Oracle.from_system(s).setup()
        o2.solve(s.rhs)
        tc = time.perf_counter() - t0
        extras["cpu_baseline"] = {"value": 1.0 / tc, "unit": "solves/s", "cores": 1,
                                  "kind": "oracle",
                                  "sample": "one full solve (setup + FGMRES) of the workload "
                                            "by the single-threaded FP64 C oracle"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == P.MIXED else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision, "pe": args.pe,
                       "l2": "flushed between steps (512 MiB device write)",
                       "parallelism": f"replicas x{world}"},
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


if __name__ == "__main__":
    sys.exit(main())
