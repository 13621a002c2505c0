"""Benchmark: emRKC node-timesteps/s on one GB300 (or N replicas).

Default workload: the 3-D slab of 201 x 71 x 31 nodes (442,401 nodes, 2.52 M
Kuhn tetrahedra, D = diag(1.33, 0.18, 0.18) mS/cm), TTP06 epicardial,
dt = 0.05 ms, stimulus 50 uA/cm^2 for 2 ms on the 0.15 cm corner cube.
One timed step = one emRKC step through the C ABI: the power iteration for
rho_F and rho_S (once, at t = 0, inside the timed region, as in the paper's
Sec. 5 setup; a run with the power iteration before every step is reported
beside it), the stage counts, the fused stage kernel and the inner SpMV
stages.  The headline path is the mixed-precision
form; the plain FP64 form is measured on the same workload beside it, and the
mixed result is compared with the FP64 result over a T = 50 ms horizon.

L2 (129 MB) is flushed before every timed step by writing a 512 MB buffer on
the same stream (outside the step's CUDA-event interval).

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (a slab with fewer z-layers), same metric.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# DRAM traffic of the dominant kernel from one ncu capture of the headline
# workload (dram__bytes_read.sum + dram__bytes_write.sum of one launch; the
# command is in profiles/stage_kernel_mixed_tma_pf_slab_ttp.md).  Reported only
# while the kernel sources hash to the captured state.
NCU_TRAFFIC = {"kernel": "stage_kernel_mixed_tma_pf<ModelTTP06<float>, false>", "workload": "slab_ttp",
               "bytes_per_launch": 55202816 + 1882880,
               "sources": ("paper_2401_01745_gb300/csrc/kernels.cuh", "paper_2401_01745_gb300/csrc/models.cuh",
                           "paper_2401_01745_gb300/csrc/kernels_mixed.cu"),
               "sha256": "285376c43bd783704d2d98124bd2f8a99c46226ae7667b8f479d918256ee1d31"}


def _sources_sha256(paths):
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


HH_RHO_S_MAX = 42.0
# largest rho(f_S) of TTP06 over an action potential (the upstroke value of
# the power iteration, 6.5 1/ms) times the safety factor 1.05, rounded up
TTP_RHO_S_MAX = 7.0  # Table 2 rho_max of HH (40) times the safety factor 1.05
METRIC = "node-timesteps/s (emRKC step, <=1e-3 rel. L2 error in V vs plain FP64)"
UNIT = "node-timesteps/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        time.sleep(0.25)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            return world, rank, local
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def step_bytes_mixed(N, s, m, offd):
    """Compulsory bytes per node of one mixed-precision emRKC step (neighbour
    gathers assumed to hit in cache): per outer stage j the stage item reads V
    hi, z, the stimulus mask and the row of L (FP32 value + int32 column) and
    writes z; with m = 1 it also reads V lo and writes V hi/lo, otherwise it
    writes delta_1 (and L V + F when m >= 4); j >= 2 adds g_{j-2} (z, V hi/lo);
    each inner item k reads delta_{k-1} (delta_{k-2} for k >= 3, L V + F for
    m >= 4) and the row of L and writes delta_k, the last one reading g_{j-1}
    (and g_{j-2}) V hi/lo and writing V hi/lo; the last stage of the step
    reads V_n hi for the activation test, and with s >= 3 stage 1 keeps a
    copy of it."""
    z = (N - 1) * 4
    L = offd * 8
    total = 0.0
    for j in range(1, s + 1):
        st = 4 + z + 1 + L + z
        st += (4 + 8) if m == 1 else (4 + (4 if m >= 4 else 0))
        if j >= 2:
            st += z + 8
        if j == 1 and s >= 3:
            st += 4
        total += st
        for k in range(2, m + 1):
            inn = 4 + (4 if k >= 3 else 0) + (4 if m >= 4 else 0) + L
            inn += (8 + (8 if j >= 2 else 0) + 8) if k == m else 4
            total += inn
    # V_n hi for the activation test (for s = 2 it is g_{j-2}, already read)
    return total + (0 if s == 2 else 4)


def _aggregate(units, ms, world, device):
    """Whole-job throughput of N replicas: the units all ranks processed over
    the slowest rank's time (weak scaling).  Returns (value, max ms)."""
    ms_max = _max_over_ranks(ms, world, device)
    total = _sum_over_ranks(units, world, device)
    return total / (ms_max / 1e3), ms_max


# ---------------------------------------------------------------------------
# CPU oracle leg (reference arm and cpu_baseline): bounded sample of the slab


def _oracle_sample(steps_budget_s, K, W=0):
    """Oracle emRKC on a slab with the workload's x-y extent and fewer z-layers,
    sized so that K steps take about ``steps_budget_s`` seconds."""
    from oracle.emrkc import Monodomain, OracleRun
    from workloads import make_workload

    per_node_step = 1.0 / 3.4e5  # s, measured oracle cost (calibrated below)
    n_target = steps_budget_s / (max(K, 1) * per_node_step)
    nz = int(max(2, min(31, round(n_target / (201 * 71)))))
    w = make_workload(f"slab201x71x{nz}_ttp", h=0.01)
    prob = Monodomain.from_workload(w)
    # the same rho policy as the GPU arm: once at t = 0, inside the timed
    # region, on a fresh run (warm-up steps on a separate one)
    warm = OracleRun(prob, rho_every=0)
    for _ in range(W):
        warm.step(w.dt)
    r = OracleRun(prob, rho_every=0)
    t0 = time.perf_counter()
    for _ in range(K):
        r.step(w.dt)
    el = time.perf_counter() - t0
    return w.n, K, el


def run_reference(args):
    world, rank, local = _dist_init()
    if rank != 0:
        return 0
    budget = 120.0
    n, K, el = _oracle_sample(budget, args.steps, args.warmup)
    value = n * K / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": K, "warmup": args.warmup, "ms_per_step": 1e3 * el / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"slab 201x71x{n // (201 * 71)} nodes (bounded sample of the 201x71x31 slab), "
                               "TTP06 epi, dt 0.05 ms; rho once at t = 0 (timed)",
                   "nodes": n, "precision": "fp64 CPU oracle (numpy, single thread)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{K} emRKC steps on {n} nodes"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# Batched form: 256 uneven instances, one persistent launch per step


def run_batched(args):
    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads.configs import batched_specs, batched_workload

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    hbm_peak, peak_kind = _peaks()
    specs = batched_specs(args.instances)
    stream = torch.cuda.Stream(device=dev)
    b = pkg.Batch(rho_every=pkg.RHO_ONCE, stream=stream.cuda_stream, device=local)
    t0 = time.perf_counter()
    bytes_step = 0.0
    total_n = 0
    for sp in specs:
        w = batched_workload(sp)
        # HH: rho(f_S) reaches ~40 in the upstroke (Table 2); a rho estimated
        # once at rest (~0.7) would keep s = 1 and the step unstable there
        b.add_workload(w, rho_S_min=HH_RHO_S_MAX if w.model == pkg.MODEL_HH else 0.0)
        total_n += w.n
    setup_s = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            b.step(0.05)
    b.sync()
    tile, block, tune_ms = b.autotune(0.05, reps=3)
    # algorithmic bytes per step (mixed path, per instance: s outer stages of
    # one stage item and m - 1 inner items each)
    for iid in b.ids():
        info = b.info(iid)
        offd = 6 if len(specs[iid - 1]["dims"]) == 3 else 4  # stored off-diagonals per row
        bytes_step += info["n"] * step_bytes_mixed(info["N"], info["s"], info["m"], offd)
    torch.cuda.synchronize()
    _barrier(world)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = b.stats()["launches"]
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(args.steps):
                b.step(0.05)
            ev1.record(stream)
        stream.synchronize()
    b.sync()
    ms = ev0.elapsed_time(ev1)
    ms_max = _max_over_ranks(ms, world, dev)
    units = _sum_over_ranks(float(total_n * args.steps), world, dev)
    value = units / (ms_max / 1e3)
    st = b.stats()
    achieved = bytes_step / (ms / args.steps / 1e3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: {len(specs)} instances, n log-uniform 8k-500k (sum {total_n}), "
                               "2-D squares / 3-D slabs, HH or TTP06, sigma_l U(0.8,2), anisotropy U(4,10), "
                               "dt 0.05 ms", "nodes": total_n, "instances": len(specs),
                   "persistent_launches_per_step": (st["launches"] - l0) / args.steps,
                   "tile": tile, "block": block, "grid": st["grid"], "items_per_step": st["items"],
                   "setup_s": setup_s, "device_gb": st["device_bytes"] / 1e9,
                   "l2": "working set (GBs) larger than L2; no flush"},
        "roofline": {"bound": "hbm", "kernel": "batch_step_kernel (persistent, all instances)",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "bytes_per_step": bytes_step, "traffic": None,
                     "peak_source": f"{peak_kind}: MEASURED_PEAKS.json hbm_gbs"},
        "gpu_launches": int(st["launches"] - l0),
        "clocks": clk.summary(),
    }
    b.close()
    if rank == 0:
        print(json.dumps(out))
    return 0


def run_served(args):
    """Served form: Poisson request stream, HBM-budget admission, continuous batching."""
    import torch

    import paper_2401_01745_gb300 as pkg
    from paper_2401_01745_gb300.serve import MeshCache, Server
    from workloads.configs import request_workload, served_requests

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    reqs = served_requests(count=args.requests, rate=20.0, seed=4)
    cache = MeshCache(request_workload)
    t0 = time.perf_counter()
    cache.prepare(reqs)
    prep_s = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=dev)
    budget = 150e9
    runs = {}
    with ClockSampler(local) as clk:
        srv = Server(cache, budget, stream=stream.cuda_stream, device=local, keep_V=False)
        srv.run(reqs)
        runs["offered_20_per_s"] = srv.summary()
        srv.close()
        cap = runs["offered_20_per_s"]["node_timesteps_per_s"]
        work = float(np.mean([r["n_target"] * r["steps"] for r in reqs]))
        rate = 0.7 * cap / work
        reqs2 = served_requests(count=args.requests, rate=rate, seed=4)
        srv = Server(cache, budget, stream=stream.cuda_stream, device=local, keep_V=False)
        srv.run(reqs2)
        runs["sustainable_70pct"] = dict(srv.summary(), arrival_rate_per_s=rate)
        srv.close()
    head = runs["offered_20_per_s"]
    out = {"metric": METRIC + "; p50/p99 solve latency", "value": head["node_timesteps_per_s"], "unit": UNIT,
           "n_gpus": 1, "steps": None, "warmup": 0, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "p50_latency_s": head["p50_latency_s"], "p99_latency_s": head["p99_latency_s"],
           "config": {"workload": f"served: {args.requests} requests, Poisson arrivals 20/s, n log-U(1e4, 2e6) "
                                  "in 8 size classes, slab or shell, HH or TTP06, horizon U(20, 400) ms, "
                                  "dt 0.05 ms, HBM budget 150 GB, continuous batching", "mesh_prep_s": prep_s,
                      "offered_node_timesteps_per_s": 20.0 * work},
           "runs": runs, "clocks": clk.summary()}
    print(json.dumps(out))
    return 0


def run_shell(args):
    """Ventricle-like shell (~4.2 M nodes): mixed vs plain FP64 over T = 100 ms."""
    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads import make_workload

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    t0 = time.perf_counter()
    w = make_workload("shell_ttp")
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=dev)
    H = int(round(w.T / w.dt))
    res = {}
    with ClockSampler(local) as clk:
        for name, prec in (("mixed", pkg.PREC_MIXED), ("fp64", pkg.PREC_FP64)):
            sol = pkg.Solver(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                             amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, precision=prec,
                             rho_every=0, stream=stream.cuda_stream, device=local)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(H):
                    sol.step(w.dt)
                e1.record(stream)
            sol.sync()
            ms = e0.elapsed_time(e1)
            st = sol.stats()
            res[name] = dict(V=sol.get_state(var=0), act=sol.activation_times(), ms=ms, s=st["s"], m=st["m"])
            sol.close()
    Va, Vb = res["fp64"]["V"], res["mixed"]["V"]
    ta, tb = res["fp64"]["act"], res["mixed"]["act"]
    both = np.isfinite(ta) & np.isfinite(tb)
    err = float(np.sqrt(np.sum(M * (Va - Vb) ** 2) / np.sum(M * Va * Va)))
    vm = w.n * H / (res["mixed"]["ms"] / 1e3)
    v64 = w.n * H / (res["fp64"]["ms"] / 1e3)
    out = {"metric": METRIC, "value": vm, "unit": UNIT, "n_gpus": 1, "steps": H, "warmup": 0,
           "ms_per_step": res["mixed"]["ms"] / H, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "shell: 32x362x362 structured box mapped onto a truncated prolate-"
                                  "ellipsoidal shell, interior jitter +-20%, fibres +60 -> -60 deg, TTP06, "
                                  "apical stimulus, dt 0.05 ms, T 100 ms, rho once at t = 0 (timed)",
                      "nodes": w.n, "cells": int(w.cells.shape[0]), "entries_per_row": col.size / w.n,
                      "s": res["mixed"]["s"], "m": res["mixed"]["m"], "setup_s": setup_s},
           "fp64": {"value": v64, "unit": UNIT, "ms_per_step": res["fp64"]["ms"] / H, "dtype": "f64"},
           "accuracy": {"rel_l2_err_V_vs_fp64": err, "T_ms": w.T,
                        "max_activation_diff_ms": float(np.max(np.abs(ta[both] - tb[both]))) if both.any() else None,
                        "activated_nodes": int(both.sum()),
                        "activation_pattern_equal": bool(np.array_equal(np.isfinite(ta), np.isfinite(tb)))},
           "headline_speedup_vs_fp64": vm / v64, "clocks": clk.summary()}
    print(json.dumps(out))
    return 0


def run_compare(args):
    """Work-precision comparison on the 3-D cuboid (Sec. 5.3 shape): emRKC
    (FP64 and mixed) and mRKC (Algorithm 2, FP64) against IMEX-RL (Algorithm
    4, FP64, CG to lin_rtol) at
    several dt, errors in V at T against a fine-step EXEX-RL reference (Sec. 5
    uses EXEX-RL at dt = 1e-4 ms; here dt_ref, stated in the output).  Each
    run is timed with CUDA events around all its steps (state resident, no L2
    flush: the 58k-node state fits in L2)."""
    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads import make_workload

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    w = make_workload("slab101x36x16_ttp", h=0.02, t_off=2.0)
    T, dt_ref = args.compare_T, args.compare_dt_ref
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    stream = torch.cuda.Stream(device=dev)

    def solve(method, prec, dt, profile=False, **kw):
        sol = pkg.Solver(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                         amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, precision=prec, rho_every=0,
                         stream=stream.cuda_stream, device=local, method=method, profile=profile, **kw)
        H = int(round(T / dt))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        V = None
        try:
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(H):
                    sol.step(dt)
                e1.record(stream)
            sol.sync()
            V = sol.get_state(var=0)
        except pkg.EmrkcError:  # the solution overflowed: the method is unstable at this dt
            stream.synchronize()
        ms = e0.elapsed_time(e1) if V is not None else float("nan")
        st = sol.stats()
        sol.close()
        return V, ms, H, st

    def rel(V, Vr):
        return float(np.sqrt(np.sum(M * (V - Vr) ** 2) / np.sum(M * Vr * Vr)))

    # warm-up (module load, clocks)
    solve(pkg.METHOD_EMRKC, pkg.PREC_MIXED, 0.1)
    with ClockSampler(local) as clk:
        Vref, ms_ref, H_ref, _ = solve(pkg.METHOD_EXEX_RL, pkg.PREC_FP64, dt_ref)
        rows = []
        for dt in args.compare_dts:
            for name, method, prec in (("emRKC-fp64", pkg.METHOD_EMRKC, pkg.PREC_FP64),
                                       ("emRKC-mixed", pkg.METHOD_EMRKC, pkg.PREC_MIXED),
                                       ("mRKC-fp64", pkg.METHOD_MRKC, pkg.PREC_FP64),
                                       ("IMEX-RL-fp64", pkg.METHOD_IMEX_RL, pkg.PREC_FP64)):
                kw = {"lin_rtol": args.lin_rtol} if method == pkg.METHOD_IMEX_RL else {}
                V, ms, H, st = solve(method, prec, dt, **kw)
                r = {"method": name, "dt": dt, "steps": H, "ms": ms, "ms_per_step": ms / H,
                     "rel_err_V": rel(V, Vref) if V is not None else None, "stable": V is not None}
                if method == pkg.METHOD_IMEX_RL:
                    r["cg_iters_per_step"] = st["total_lin_iters"] / H
                else:
                    r["s"], r["m"] = st["s"], st["m"]
                rows.append(r)
        # F wedge (Sec. 5.5): time in f_F work per step, FP64 on both sides, at
        # a dt where emRKC takes m >= 2 (its first f_F evaluation of every
        # outer stage is fused into the stage kernel with the ionic model; the
        # other s (m - 1) are the inner SpMV kernels)
        dtw = args.compare_wedge_dt
        _, _, He, se = solve(pkg.METHOD_EMRKC, pkg.PREC_FP64, dtw, profile=True)
        _, _, Hi, si = solve(pkg.METHOD_IMEX_RL, pkg.PREC_FP64, dtw, profile=True, lin_rtol=args.lin_rtol)
    n_inner = max(se["phase_launches"]["inner"], 1)
    spmv_ms = se["phase_ms"]["inner"] / n_inner
    fF_est = se["s"] * se["m"] * spmv_ms
    cg_ms = si["phase_ms"]["inner"] / Hi
    # CG iteration bytes per node (FP64): q = B p with p = z + beta p gathered
    # (z, p, M, the row of L with its diagonal: 12 B per stored entry; p, q
    # out), then x, r, z updated (p, x, r, q, P^-1, M in; x, r, z out)
    ell_entries = si["matrix_entries"] / w.n
    cg_bytes = 8 * 3 + 12 * ell_entries + 16 + 8 * 6 + 8 * 3
    iters = max(si["total_lin_iters"], 1)
    cg_gbs = cg_bytes * w.n * iters / (si["phase_ms"]["inner"] / 1e3) / 1e9
    wedge = {"dt": dtw, "emrkc_s_m": [se["s"], se["m"]],
             "emrkc_ms_per_inner_spmv_stage": spmv_ms,
             "emrkc_fF_ms_per_step_estimate": fF_est,
             "emrkc_stage_ms_per_step": se["phase_ms"]["stage"] / He,
             "imex_cg_solve_ms_per_step": cg_ms,
             "imex_cg_iters_per_step": si["total_lin_iters"] / Hi,
             "imex_ionic_setup_ms_per_step": si["phase_ms"]["stage"] / Hi,
             "ratio_imex_solve_to_emrkc_fF": cg_ms / fF_est if fF_est > 0 else None,
             "imex_cg_bytes_per_node_per_iteration": cg_bytes,
             "imex_cg_achieved_gbs": cg_gbs, "imex_cg_frac_of_hbm": cg_gbs / _peaks()[0],
             "note": ("emRKC f_F per step estimated as s * m inner-SpMV-stage times (the first evaluation of each "
                      "outer stage is fused into the stage kernel)")}
    best = {}
    for r in rows:
        if r["stable"] and r["rel_err_V"] <= args.compare_target:
            b = best.get(r["method"])
            if b is None or r["ms"] < b["ms"]:
                best[r["method"]] = r
    out = {"metric": "work-precision: wall ms to T vs rel. L2 error in V", "unit": "ms", "n_gpus": 1,
           "higher_is_better": False, "dtype": "mixed", "data": "synthetic",
           "config": {"workload": "slab 101x36x16 nodes (h = 0.02 cm, 2.0x0.7x0.3 cm, 58,176 nodes), D = "
                                  "diag(1.33, 0.18, 0.18), TTP06 epi, corner stimulus 2 ms", "T_ms": T,
                      "reference": f"EXEX-RL FP64 at dt = {dt_ref} ms ({H_ref} steps, {ms_ref:.0f} ms)",
                      "imex_lin_rtol": args.lin_rtol, "rho_policy": "once at t = 0"},
           "runs": rows, "fastest_within_target": {"target_rel_err": args.compare_target, **best},
           "f_wedge": wedge, "clocks": clk.summary()}
    print(json.dumps(out))
    return 0


def run_stability(args):
    """Practical stability (Sec. 5.1): the 1-D TTP06 cable at dx = 0.025 mm up
    to T = 100 ms with increasing dt; the relative norm ||V_N|| / ||V*|| (V*:
    emRKC FP64 at dt = 0.01 ms) and the stage counts, for emRKC (FP64 and
    mixed, rho once at t = 0); and the largest stable dt of EXEX-RL."""
    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads import make_workload

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    pkg.build()
    w = make_workload("cable_ttp")
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)

    def solve(dt, T, prec, method=0, rho_every=0, rho_S_min=0.0):
        sol = pkg.Solver(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                         amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, precision=prec, rho_every=rho_every,
                         device=local, method=method, rho_S_min=rho_S_min)
        ok = True
        try:
            for _ in range(int(round(T / dt))):
                sol.step(dt)
            sol.sync()
        except pkg.EmrkcError:
            ok = False
        st = sol.stats()
        V = sol.get_state(var=0) if ok else None
        sol.close()
        return V, st, ok

    Vref, _, _ = solve(0.01, 100.0, pkg.PREC_FP64)
    nref = float(np.sqrt(M @ (Vref * Vref)))
    rows = []
    policies = ((pkg.PREC_FP64, "fp64", 0, 0.0, "once"), (pkg.PREC_MIXED, "mixed", 0, 0.0, "once"),
                (pkg.PREC_FP64, "fp64", 1, 0.0, "every step"),
                (pkg.PREC_FP64, "fp64", 0, TTP_RHO_S_MAX, f"once, rho_S >= {TTP_RHO_S_MAX}"),
                (pkg.PREC_MIXED, "mixed", 0, TTP_RHO_S_MAX, f"once, rho_S >= {TTP_RHO_S_MAX}"))
    for prec, pname, rho_every, rho_min, label in policies:
        for dt in args.stability_dts:
            V, st, ok = solve(dt, 100.0, prec, rho_every=rho_every, rho_S_min=rho_min)
            fin = ok and bool(np.all(np.isfinite(V)))
            rows.append({"precision": pname, "rho": label, "dt": dt,
                         "s": st["s"], "m": st["m"],
                         "rel_norm": float(np.sqrt(M @ (V * V)) / nref) if fin else None,
                         "rel_err": float(np.sqrt(M @ ((V - Vref) ** 2)) / nref) if fin else None,
                         "finite": fin})
    exex = []
    for dt in (0.001, 0.002, 0.003, 0.0035, 0.004, 0.005):
        V, _, ok = solve(dt, 20.0, pkg.PREC_FP64, pkg.METHOD_EXEX_RL)
        exex.append({"dt": dt, "bounded": bool(ok and np.all(np.abs(V) < 200))})
    stable = [r["dt"] for r in rows if r["precision"] == "fp64" and r["rho"] == "once" and r["finite"]
              and 0.5 < r["rel_norm"] < 1.5]
    stable_every = [r["dt"] for r in rows if r["rho"] == "every step" and r["finite"] and 0.5 < r["rel_norm"] < 1.5]
    stable_bound = [r["dt"] for r in rows if r["rho"].startswith("once, rho_S") and r["precision"] == "fp64"
                    and r["finite"] and 0.5 < r["rel_norm"] < 1.5]
    out = {"metric": "practical stability: largest dt with a bounded solution", "unit": "ms",
           "value": max(stable) if stable else None, "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "cable: [0, 2] cm, dx = 0.0025 cm (801 nodes), sigma 1.33 mS/cm, TTP06 epi, "
                                  "stimulus x <= 0.15 cm for t <= 2 ms, T = 100 ms",
                      "reference": "emRKC FP64 at dt = 0.01 ms",
                      "rho_policy": "value: once at t = 0 (FP64); rows also for every step"},
           "largest_bounded_dt_rho_every_step": max(stable_every) if stable_every else None,
           "largest_bounded_dt_rho_S_bound": max(stable_bound) if stable_bound else None,
           "emrkc": rows,
           "exex_rl": {"T_ms": 20.0, "runs": exex,
                       "largest_bounded_dt": max([e["dt"] for e in exex if e["bounded"]], default=None)}}
    print(json.dumps(out))
    return 0


def run_latency(args):
    """The 65 x 65 HH square (4,225 nodes) with the power iteration before
    every step (Sec. 5.2 shape): too small to fill a GPU, so it is reported as
    microseconds per step, FP64 and mixed, timed from rest over 400 steps."""
    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads import make_workload

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    w = make_workload("square65_hh")
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    stream = torch.cuda.Stream(device=dev)
    H = int(round(w.T / w.dt))
    out = {"metric": "latency: microseconds per emRKC step (rho every step)", "unit": "us/step",
           "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "steps": H,
           "config": {"workload": "square65_hh: 65x65 nodes on [0,1]^2 cm (h = 1/64), sigma 1 mS/cm, HH, corner "
                                  "stimulus 1 ms, dt 0.05 ms, T 20 ms, rho every step (timed)", "nodes": w.n}}
    with ClockSampler(local) as clk:
        for name, prec in (("fp64", pkg.PREC_FP64), ("mixed", pkg.PREC_MIXED)):
            res = []
            for rep in range(args.warmup // 3 + 2):
                sol = pkg.Solver(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                                 amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, precision=prec, rho_every=1,
                                 stream=stream.cuda_stream, device=local)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    for _ in range(H):
                        sol.step(w.dt)
                    e1.record(stream)
                sol.sync()
                st = sol.stats()
                res.append((e0.elapsed_time(e1) * 1e3 / H, st["total_pow_iters"] / H))
                sol.close()
            us, its = res[-1]  # the first runs are warm-up
            out[name] = {"us_per_step": us, "power_iterations_per_step": its,
                         "node_timesteps_per_s": w.n / (us * 1e-6)}
    out["value"] = out["mixed"]["us_per_step"]
    out["clocks"] = clk.summary()
    print(json.dumps(out))
    return 0


def run_fibrosis(args):
    """Fibrosis robustness workload (Sec. 5.4 with fibrosis): the 201 x 71 x 31
    slab with sigma_t = 0 on the cells where a seeded smooth random field
    exceeds its median; mixed vs FP64 throughput and error over T = 20 ms."""
    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads import make_workload

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    w = make_workload("fibslab201x71x31_ttp", h=0.01)
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    stream = torch.cuda.Stream(device=dev)
    H = int(round(20.0 / w.dt))
    res = {}
    with ClockSampler(local) as clk:
        for name, prec in (("mixed", pkg.PREC_MIXED), ("fp64", pkg.PREC_FP64)):
            sol = pkg.Solver(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                             amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, precision=prec, rho_every=0,
                             stream=stream.cuda_stream, device=local)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(H):
                    sol.step(w.dt)
                e1.record(stream)
            sol.sync()
            st = sol.stats()
            res[name] = dict(ms=e0.elapsed_time(e1), V=sol.get_state(var=0), act=sol.activation_times(),
                             s=st["s"], m=st["m"], rho_F=st["rho_F"])
            sol.close()
    Va, Vb = res["fp64"]["V"], res["mixed"]["V"]
    ta, tb = res["fp64"]["act"], res["mixed"]["act"]
    both = np.isfinite(ta) & np.isfinite(tb)
    out = {"metric": METRIC, "value": w.n * H / (res["mixed"]["ms"] / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": H, "ms_per_step": res["mixed"]["ms"] / H, "higher_is_better": True, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "fibrosis slab: 201x71x31 Kuhn-tet slab, fibres along x (1.33/0.18 mS/cm), "
                                  "sigma_t = 0 above the median of a seeded smooth field (corr. length 0.05 cm), "
                                  "TTP06, dt 0.05 ms, T 20 ms, rho once at t = 0 (timed)", "nodes": w.n,
                      "fibrotic_cells": float(w.extra["fibrotic_cells"].mean()),
                      "s": res["mixed"]["s"], "m": res["mixed"]["m"], "rho_F": res["mixed"]["rho_F"]},
           "fp64": {"value": w.n * H / (res["fp64"]["ms"] / 1e3), "ms_per_step": res["fp64"]["ms"] / H},
           "accuracy": {"rel_l2_err_V_vs_fp64": float(np.sqrt(np.sum(M * (Va - Vb) ** 2) / np.sum(M * Va * Va))),
                        "max_activation_diff_ms": float(np.max(np.abs(ta[both] - tb[both]))) if both.any() else None,
                        "activated_nodes": int(both.sum())},
           "clocks": clk.summary()}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000, help="timed steps (1000 = T 50 ms at dt 0.05)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="slab_ttp")
    ap.add_argument("--rho-every", type=int, default=0, help="0: once at t = 0 (Sec. 5 setup); k: every k steps")
    ap.add_argument("--every-step-steps", type=int, default=200)
    ap.add_argument("--fp64-steps", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline only (for profiler runs)")
    ap.add_argument("--batched", action="store_true", help="batched form: many instances per launch")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--shell", action="store_true", help="ventricle-like shell, mixed vs FP64 over T = 100 ms")
    ap.add_argument("--served", action="store_true", help="served form: request stream, p50/p99 latency")
    ap.add_argument("--requests", type=int, default=100)
    ap.add_argument("--compare", action="store_true", help="work-precision: emRKC vs IMEX-RL vs EXEX-RL reference")
    ap.add_argument("--compare-T", type=float, default=10.0)
    ap.add_argument("--compare-dt-ref", type=float, default=2.5e-4)
    ap.add_argument("--compare-dts", type=float, nargs="+", default=[0.4, 0.2, 0.1, 0.05, 0.025])
    ap.add_argument("--compare-target", type=float, default=1e-2)
    ap.add_argument("--compare-wedge-dt", type=float, default=0.2)
    ap.add_argument("--lin-rtol", type=float, default=1e-8)
    ap.add_argument("--stability", action="store_true", help="Sec. 5.1 practical-stability sweep on the 1-D cable")
    ap.add_argument("--latency", action="store_true", help="65x65 HH square, rho every step, us/step")
    ap.add_argument("--fibrosis", action="store_true", help="fibrosis slab: mixed vs FP64 over T = 20 ms")
    ap.add_argument("--stability-dts", type=float, nargs="+",
                    default=[0.05, 0.1, 0.25, 0.5, 1.0, 2.0, 3.0, 4.0, 4.5, 5.0, 6.0, 8.0])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.shell:
        return run_shell(args)
    if args.compare:
        return run_compare(args)
    if args.stability:
        return run_stability(args)
    if args.latency:
        return run_latency(args)
    if args.fibrosis:
        return run_fibrosis(args)
    if args.served:
        return run_served(args)
    if args.batched:
        if args.steps == 1000:
            args.steps = 100
        return run_batched(args)

    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads import make_workload

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    w = make_workload(args.workload)
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    stream = torch.cuda.Stream(device=dev)
    prec = pkg.PREC_MIXED if args.precision == "mixed" else pkg.PREC_FP64
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    hbm_peak, peak_kind = _peaks()
    N = pkg.num_vars(w.model)

    def make(precision, profile=False, rho_every=None):
        return pkg.Solver(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                          amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, precision=precision,
                          rho_every=args.rho_every if rho_every is None else rho_every,
                          stream=stream.cuda_stream, device=local, profile=profile)

    def timed_steps(sol, K_, flush_l2=True):
        """K_ steps, each bracketed by CUDA events on the solver's stream, with
        L2 flushed before each step outside the bracket."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K_)]
        l0 = sol.stats()["launches"]
        with torch.cuda.stream(stream):
            for k in range(K_):
                if flush_l2:
                    flush.fill_(float(k))
                evs[k][0].record(stream)
                sol.step(w.dt)
                evs[k][1].record(stream)
        stream.synchronize()
        sol.sync()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, sol.stats()["launches"] - l0

    # ---- warm-up on a separate instance (module load, clocks, allocator) ----
    warm = make(prec)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            warm.step(w.dt)
    warm.sync()
    warm.close()

    # ---- headline: K steps from rest on a fresh solver (includes rho at t = 0) ----
    sol = make(prec)
    torch.cuda.synchronize()
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, launches = timed_steps(sol, args.steps)
    torch.cuda.synchronize()
    _barrier(world)
    st = sol.stats()
    total_ms = sum(ms)
    value, total_ms_max = _aggregate(float(w.n * args.steps), total_ms, world, dev)
    sol.close()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == pkg.PREC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": (f"{args.workload}: 201x71x31-node Kuhn-tet slab 2.0x0.7x0.3 cm, TTP06 epi, "
                                "dt 0.05 ms, 50 uA/cm^2 corner stimulus; timed from rest (t = 0)"
                                if args.workload == "slab_ttp" else
                                f"{args.workload}: {w.n}-node synthetic mesh, dt {w.dt} ms, corner stimulus; "
                                "timed from rest (t = 0)"),
                   "nodes": w.n, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "precision": ("mixed: FP32 z, ionic model, gating, SpMV, inner increments; FP64 V "
                                 "recurrence, stage coefficients, rho" if prec == pkg.PREC_MIXED else "fp64"),
                   "rho_policy": ("once at t = 0 (inside the timed region)" if args.rho_every == 0
                                  else f"every {args.rho_every} steps"),
                   "s": st["s"], "m": st["m"], "power_iterations": st["total_pow_iters"],
                   "l2": "flushed before every timed step (512 MB write, outside the step's events)"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if args.no_extras:
        if rank == 0:
            print(json.dumps(out))
        return 0

    # ---- per-kernel durations (CUDA events around every launch, same stream) ----
    solp = make(prec, profile=True)
    Kp = args.steps
    timed_steps(solp, Kp)
    p1 = solp.stats()
    solp.close()
    phase_ms, phase_n = p1["phase_ms"], p1["phase_launches"]
    zb = 4 if prec == pkg.PREC_MIXED else 8
    nnz_row = p1["matrix_entries"] / w.n  # stored entries of L per row (sliced ELL)
    if prec == pkg.PREC_MIXED:
        mat_b = nnz_row * (4 + 4)  # off-diagonal FP32 value + int32 column
        # stage: V hi, z, mask, L in; z, delta_1 out (and L V + F when m >= 4)
        m_inner = p1["m"]
        lf = 4 if m_inner >= 4 else 0
        bytes_stage = 4 + (N - 1) * zb + 1 + mat_b + (N - 1) * zb + 4 + lf
        # last inner stage: delta_1 (delta_2 when m >= 3), V hi + lo, L in; V hi + lo out
        bytes_inner = 4 + (4 if m_inner >= 3 else 0) + lf + 8 + mat_b + 8
    else:
        mat_b = nnz_row * (8 + 4)
        bytes_stage = 8 + (N - 1) * zb + 1 + mat_b + (N - 1) * zb + 8 + 8  # V, z, mask, L; z, u_1, F
        bytes_inner = 8 + 8 + 8 + mat_b + 8  # u_1, V, F, L; V
    per_launch = {"stage": bytes_stage, "inner": bytes_inner}
    step_kernels = {k: phase_ms[k] for k in ("stage", "inner")}
    dom_key = max(step_kernels, key=lambda k: step_kernels[k])
    avg_ms = phase_ms[dom_key] / max(phase_n[dom_key], 1)
    achieved = per_launch[dom_key] * w.n / (avg_ms / 1e3) / 1e9
    out["roofline"] = {
        "bound": "hbm", "kernel": "stage_kernel_mixed (fused RL + TTP06 + first SpMV + outer update)"
        if dom_key == "stage" else "inner_kernel_mixed (SpMV stage + FP64 V update)",
        "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
        "peak_source": f"{peak_kind}: MEASURED_PEAKS.json hbm_gbs (burst copy)",
        "bytes_per_node_per_launch": per_launch[dom_key], "avg_launch_us": avg_ms * 1e3,
        "matrix_entries_per_row": nnz_row,
        "traffic": None}
    if (dom_key == "stage" and prec == pkg.PREC_MIXED and args.workload == NCU_TRAFFIC["workload"]
            and _sources_sha256(NCU_TRAFFIC["sources"]) == NCU_TRAFFIC["sha256"]):
        out["roofline"]["traffic"] = NCU_TRAFFIC["bytes_per_launch"]
        out["roofline"]["traffic_note"] = ("ncu dram bytes read + write of one launch (cold cache); at this size "
                                           "the state fits in L2, so most writes are still in L2 at kernel end")
        out["roofline"]["algorithmic_bytes_per_launch"] = per_launch[dom_key] * w.n
    out["kernels"] = {k: {"ms_per_step": phase_ms[k] / Kp, "launches_per_step": phase_n[k] / Kp,
                          "avg_launch_us": 1e3 * phase_ms[k] / max(phase_n[k], 1)}
                      for k in phase_ms if phase_n[k] > 0}
    if "stage" in per_launch and "inner" in per_launch:
        out["kernels"]["stage"]["gbs"] = bytes_stage * w.n / (phase_ms["stage"] / max(phase_n["stage"], 1) / 1e3) / 1e9
        out["kernels"]["inner"]["gbs"] = bytes_inner * w.n / (phase_ms["inner"] / max(phase_n["inner"], 1) / 1e3) / 1e9

    # ---- rho every step (Algorithm 5 warm started before every step) ----
    sole = make(prec, rho_every=1)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            sole.step(w.dt)
    sole.sync()
    mse, _ = timed_steps(sole, args.every_step_steps)
    ste = sole.stats()
    sole.close()
    out["rho_every_step"] = {"value": w.n * args.every_step_steps / (sum(mse) / 1e3), "unit": UNIT,
                             "ms_per_step": sum(mse) / args.every_step_steps, "steps": args.every_step_steps,
                             "power_iterations_per_step": ste["total_pow_iters"] / (args.warmup + args.every_step_steps)}

    # ---- end to end through the C ABI with host buffers ----
    # (1) every step takes its input, the applied stimulus (node mask from
    # pinned host memory), and returns its result, V, to pinned host memory;
    # the state stays on the device, as a model's weights do in a training
    # step; the timed region starts from rest, power iteration included, and
    # ends when the last step's V is on the host.  Pipelined form (the e2e
    # line): emrkc_set_stimulus_async + emrkc_step + emrkc_get_state_async
    # into two pinned buffers in rotation, the copies overlapping the next
    # steps on the copy engines, one emrkc_sync at the end.  Synchronous form
    # beside it: emrkc_set_stimulus + emrkc_step + emrkc_get_state.
    Ke = min(args.steps, 1000)
    pinned_mask = torch.from_numpy(np.ascontiguousarray(w.stim_mask, dtype=np.uint8)).pin_memory()
    pinned_out = torch.empty((w.n,), dtype=torch.float64, pin_memory=True)
    pinned_ring = [torch.empty((w.n,), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    mask_np, out_np = pinned_mask.numpy(), pinned_out.numpy()
    ring_np = [b.numpy() for b in pinned_ring]

    def e2e_async(sol, K):
        for k in range(K):
            sol.set_stimulus_async(mask_np, w.stim_amp, w.t_on, w.t_off)
            sol.step(w.dt)
            sol.get_state_async(0, ring_np[k % 2])
        sol.sync()

    warm = make(prec)
    e2e_async(warm, args.warmup)
    warm.close()
    sol = make(prec)
    torch.cuda.synchronize()
    _barrier(world)
    t0 = time.perf_counter()
    e2e_async(sol, Ke)
    e2e_s = _max_over_ranks(time.perf_counter() - t0, world, dev)
    last_ok = bool(np.array_equal(ring_np[(Ke - 1) % 2], sol.get_state(var=0)))
    sol.close()
    out["e2e"] = {"value": _sum_over_ranks(float(w.n * Ke), world, dev) / e2e_s, "unit": UNIT,
                  "h2d_bytes_per_step": int(w.n), "d2h_bytes_per_step": int(w.n * 8), "steps": Ke,
                  "api": "per step: emrkc_set_stimulus_async(node mask, pinned host) + emrkc_step + "
                         "emrkc_get_state_async(V, two pinned host buffers in rotation); one emrkc_sync at "
                         "the end; from rest, power iteration at t = 0 included",
                  "last_result_matches_get_state": last_ok,
                  "l2": "not flushed between steps (the state stays resident, as in a running service; the "
                        "device-timed value flushes)"}
    warm = make(prec)
    for _ in range(args.warmup):
        warm.set_stimulus(mask_np, w.stim_amp, w.t_on, w.t_off)
        warm.step(w.dt)
        warm.get_state(var=0, out=out_np)
    warm.close()
    sol = make(prec)
    torch.cuda.synchronize()
    _barrier(world)
    parts = np.zeros(3)
    t0 = time.perf_counter()
    for _ in range(Ke):
        ta = time.perf_counter()
        sol.set_stimulus(mask_np, w.stim_amp, w.t_on, w.t_off)
        tb = time.perf_counter()
        sol.step(w.dt)
        tc = time.perf_counter()
        sol.get_state(var=0, out=out_np)
        parts += (tb - ta, tc - tb, time.perf_counter() - tc)
    sol.sync()
    es_s = _max_over_ranks(time.perf_counter() - t0, world, dev)
    sol.close()
    out["e2e_sync"] = {"value": _sum_over_ranks(float(w.n * Ke), world, dev) / es_s, "unit": UNIT,
                       "h2d_bytes_per_step": int(w.n), "d2h_bytes_per_step": int(w.n * 8), "steps": Ke,
                       "api": "per step: emrkc_set_stimulus(node mask, pinned host) + emrkc_step + "
                              "emrkc_get_state(V, pinned host), each call waiting for its copy",
                       "host_us_per_step": {"set_stimulus": 1e6 * parts[0] / Ke, "step": 1e6 * parts[1] / Ke,
                                            "get_state": 1e6 * parts[2] / Ke}}
    # (2) the whole state through the host every step (all variables in, V out)
    sol = make(prec)
    pinned_in = torch.empty((N, w.n), dtype=torch.float64, pin_memory=True)
    sol.get_state(out=pinned_in.numpy())
    Kf = min(args.steps, 100)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            sol.set_state(pinned_in.numpy())
            sol.step(w.dt)
            sol.get_state(var=0, out=pinned_out.numpy())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(Kf):
            sol.set_state(pinned_in.numpy())
            sol.step(w.dt)
            sol.get_state(var=0, out=pinned_out.numpy())
    sol.sync()
    ef_s = _max_over_ranks(time.perf_counter() - t0, world, dev)
    sol.close()
    out["e2e_full_state"] = {"value": _sum_over_ranks(float(w.n * Kf), world, dev) / ef_s, "unit": UNIT,
                             "h2d_bytes_per_step": int(N * w.n * 8), "d2h_bytes_per_step": int(w.n * 8),
                             "steps": Kf, "api": "per step: emrkc_set_state(all variables, pinned host) + "
                                                 "emrkc_step + emrkc_get_state(V, pinned host)"}

    # ---- plain FP64 form on the same workload, and accuracy of the mixed form ----
    if prec == pkg.PREC_MIXED and rank == 0:
        s64 = make(pkg.PREC_FP64)
        ms64, _ = timed_steps(s64, args.fp64_steps)
        s64.close()
        v64 = w.n * args.fp64_steps / (sum(ms64) / 1e3)
        out["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": sum(ms64) / args.fp64_steps,
                       "steps": args.fp64_steps, "dtype": "f64",
                       "note": "same workload and rho policy, timed from rest", "headline_speedup": value / v64}
        if not args.no_accuracy:
            H = int(round(w.T / w.dt))
            a = make(pkg.PREC_FP64)
            b = make(pkg.PREC_MIXED)
            with torch.cuda.stream(stream):
                for _ in range(H):
                    a.step(w.dt)
                    b.step(w.dt)
            a.sync()
            b.sync()
            Va, Vb = a.get_state(var=0), b.get_state(var=0)
            ta, tb = a.activation_times(), b.activation_times()
            a.close()
            b.close()
            err = float(np.sqrt(np.sum(M * (Va - Vb) ** 2) / np.sum(M * Va * Va)))
            both = np.isfinite(ta) & np.isfinite(tb)
            out["accuracy"] = {"rel_l2_err_V_vs_fp64": err, "T_ms": H * w.dt,
                               "max_activation_diff_ms": (float(np.max(np.abs(ta[both] - tb[both])))
                                                          if both.any() else None),
                               "activated_nodes": int(both.sum()),
                               "activation_pattern_equal": bool(np.array_equal(np.isfinite(ta), np.isfinite(tb)))}

    if rank == 0 and not args.no_cpu_baseline:
        n_s, K_s, el = _oracle_sample(15.0, 10)
        out["cpu_baseline"] = {"value": n_s * K_s / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"{K_s} FP64 oracle emRKC steps (numpy, 1 thread) on a "
                                         f"201x71x{n_s // (201 * 71)} slab ({n_s} nodes), same h, model, dt"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
