"""Benchmark: emRKC node-timesteps/s on one GB300 (or N replicas).

Default line: the batched form.  256 seeded instances (n log-uniform 8k-500k
nodes, 31.2 M in all; 2-D squares and 3-D slabs; HH or TTP06; sigma_l
U(0.8, 2.0) mS/cm, anisotropy U(4, 10)) advance one emRKC step each in ONE
persistent kernel launch per step, replayed as a CUDA graph, in the
mixed-precision form.  `value` = node-timesteps/s of the whole batch with the
state resident in HBM (far larger than L2, so no flush); `roofline` = the
persistent kernel's algorithmic bytes over its launch duration (CUDA events
around every launch); `e2e` = the same steps through the C ABI with every
instance's stimulus mask in from pinned host memory and every instance's V
out to pinned host memory each step; `fp64` = the plain FP64 form
(single-instance path) on the same instances; `accuracy` = the mixed batch
against FP64 per instance over T = 50 ms on a sample.  On one GPU the line
also carries the single-instance 442k-node TTP06 slab (`slab`), the 4.19 M
node ventricle-like shell, mixed vs FP64 over T = 100 ms (`shell`), the
served form with p50/p99 latency (`served`) and the 65 x 65 HH square with
rho every step (`latency`); `cpu_baseline` is the FP64 CPU oracle on all host
cores (one process per core) on instances of the same batched workload.

Modes: --batched (the batched line only), --single (single-instance line on
--workload with every end-to-end variant), --shell, --served, --latency,
--compare, --stability, --fibrosis.  --impl reference times the FP64 CPU
oracle on the host cores on a bounded sample of the batched workload.
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
               "bytes_per_launch": 55213824 + 1949184,
               "sources": ("paper_2401_01745_gb300/csrc/kernels.cuh", "paper_2401_01745_gb300/csrc/models.cuh",
                           "paper_2401_01745_gb300/csrc/kernels_mixed.cu"),
               "sha256": "da739140793334712781c681125641805b77b220066bda35e61cae750859dc9b"}


def _sources_sha256(paths):
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


HH_RHO_S_MAX = 42.0  # Table 2 rho_max of HH (40) times the safety factor 1.05
# largest rho(f_S) of TTP06 over an action potential (the upstroke value of
# the power iteration, 6.5 1/ms) times the safety factor 1.05, rounded up
TTP_RHO_S_MAX = 7.0
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
# CPU oracle legs (reference arm and cpu_baseline): the FP64 oracle as it
# stands, one process per host core, each on its own instance of the batched
# workload (the instances are independent, so the oracle's code is
# unchanged); processes are started with the spawn method (never forked from
# a process that has touched the GPU).


def _cpu_info():
    """Usable host cores and the CPU model from /proc/cpuinfo."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            info = fh.read()
        for key in ("model name", "Model", "CPU part"):
            for ln in info.splitlines():
                if ln.startswith(key):
                    model = f"{key}: {ln.split(':', 1)[1].strip()}"
                    break
            if model:
                break
    except OSError:
        pass
    return cores, model or "unknown"


def _oracle_worker(job):
    """One process: build instance ``index`` of the batched workload, run the
    FP64 oracle from rest (rho once at t = 0, as the GPU arm) after every
    process of the pool is ready, and time its steps.  With ``rounds`` set,
    the process takes that many rounds of k steps, k chosen from its warm-up
    step time so that a round lasts about ``round_s`` (at least one step), so
    that every core stays busy whatever its instance's size; otherwise steps
    are taken until ``budget_s`` has passed (at least one)."""
    index, count, rounds, warmup, budget_s, round_s, barrier = job
    from oracle.emrkc import Monodomain, OracleRun
    from workloads.configs import batched_specs, batched_workload

    sp = batched_specs(count)[index]
    w = batched_workload(sp)
    prob = Monodomain.from_workload(w)
    rho_min = HH_RHO_S_MAX if w.model == 2 else 0.0
    warm = OracleRun(prob, rho_every=0, rho_S_min=rho_min)
    tw = time.perf_counter()
    for _ in range(max(warmup, 2)):
        warm.step(w.dt)
    t_step = (time.perf_counter() - tw) / max(warmup, 2)
    per_round = max(1, int(round(round_s / max(t_step, 1e-9))))
    r = OracleRun(prob, rho_every=0, rho_S_min=rho_min)
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    k = 0
    if rounds is not None:
        for _ in range(rounds * per_round):
            r.step(w.dt)
            k += 1
    else:
        while k == 0 or time.perf_counter() - t0 < budget_s:
            r.step(w.dt)
            k += 1
    return {"index": index, "n": w.n, "model": int(w.model), "steps": k, "seconds": time.perf_counter() - t0,
            "steps_per_round": per_round}


def _sample_instances(count, k):
    """k instances of the batched workload with its mix: HH and TTP06 in
    equal numbers (the coin flip's expectation), each spread evenly over that
    model's instances sorted by size."""
    from workloads.configs import batched_specs

    specs = batched_specs(count)
    picks = []
    for model, share in ((2, k // 2), (3, k - k // 2)):
        lst = sorted((sp for sp in specs if sp["model"] == model), key=lambda sp: (int(np.prod(sp["dims"])), sp["index"]))
        picks += [lst[min(len(lst) - 1, int((j + 0.5) * len(lst) / share))]["index"] for j in range(share) if lst]
    return sorted(set(picks))


def _oracle_pool(count, rounds=None, warmup=0, budget_s=10.0, procs=None, round_s=1.0):
    """The oracle on ``procs`` instances of the batched workload at once, one
    process per host core (instances from _sample_instances).  Returns (node-steps/s of the whole pool, cores,
    per-process records)."""
    import multiprocessing as mp

    cores, _ = _cpu_info()
    procs = procs or cores
    idx = _sample_instances(count, procs)
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:  # one thread per process: the oracle as it stands, one core each
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Manager() as mgr:
            barrier = mgr.Barrier(len(idx))
            with ctx.Pool(len(idx)) as pool:
                recs = pool.map(_oracle_worker, [(i, count, rounds, warmup, budget_s, round_s, barrier) for i in idx])
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    wall = max(r["seconds"] for r in recs)
    units = sum(r["n"] * r["steps"] for r in recs)
    return units / wall, len(idx), recs


def _pool_sample_text(recs, count, rounds=None, round_s=1.0):
    n = sum(r["n"] for r in recs)
    text = (f"FP64 oracle (numpy, one process per core, one thread each) on {len(recs)} of the {count} "
            f"batched instances (half HH, half TTP06, each spread over that model's sizes; {n} nodes in all, "
            f"{sum(1 for r in recs if r['model'] == 2)} HH / {sum(1 for r in recs if r['model'] == 3)} TTP06), "
            f"from rest, rho once at t = 0; {min(r['steps'] for r in recs)}-{max(r['steps'] for r in recs)} "
            "steps per process, all processes started together")
    if rounds:
        text += (f"; one bench step = one round in which each process takes the steps that last about "
                 f"{round_s} s on its instance ({min(r['steps_per_round'] for r in recs)}-"
                 f"{max(r['steps_per_round'] for r in recs)})")
    return text + "; value = node-steps of all processes / the slowest process's time"


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, on a bounded
    sample of the batched workload (the GPU arm's config), same metric."""
    world, rank, local = _dist_init()
    if rank != 0:
        return 0
    cores, cpu = _cpu_info()
    value, used, recs = _oracle_pool(args.instances, rounds=args.steps, warmup=args.warmup)
    ms = 1e3 * max(r["seconds"] for r in recs) / args.steps
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": batched_workload_text(args.instances),
                   "sample": _pool_sample_text(recs, args.instances, rounds=args.steps), "cpu": cpu,
                   "host_cores": cores},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": _pool_sample_text(recs, args.instances, rounds=args.steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# Batched form (the default line): 256 uneven instances, one persistent launch
# per step


def batched_workload_text(count):
    return (f"batched: {count} instances (seed 3), n log-uniform 8k-500k, 2-D squares (h 1/64 cm) / 3-D "
            "slabs 20:7:3 (h 0.01 cm) by coin flip, HH or TTP06 by coin flip, sigma_l U(0.8, 2.0) mS/cm, "
            "anisotropy U(4, 10), stimulus patch at a uniform boundary node, dt 0.05 ms, FP32 bulk "
            "(mixed precision), rho once per instance at its first step (HH: rho_S >= 42)")


MIXED_PRECISION_TEXT = ("mixed: FP32 z, ionic model, gating, SpMV and inner increments; V as a float-float "
                        "pair (hi + lo, 48 significand bits); stage coefficients from FP64 recurrences on the "
                        "host, rounded to FP32 in the kernels; FP64 rho scalars of Algorithm 5")


def _batched_setup(pkg, specs, stream, local, fp64_for=()):
    """Mixed-precision batch of every spec; FP64 solvers (single-instance
    path) for the spec indices in ``fp64_for``."""
    from workloads.configs import batched_workload

    b = pkg.Batch(rho_every=pkg.RHO_ONCE, stream=stream.cuda_stream, device=local)
    fp64 = {}
    total_n = 0
    masks = []
    for sp in specs:
        w = batched_workload(sp)
        rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
        # HH: rho(f_S) reaches ~40 in the upstroke (Table 2); a rho estimated
        # once at rest (~0.7) would keep s = 1 and the step unstable there
        rho_min = HH_RHO_S_MAX if w.model == pkg.MODEL_HH else 0.0
        b.add(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask, amplitude=w.stim_amp,
              t_on=w.t_on, t_off=w.t_off, rho_S_min=rho_min)
        if sp["index"] in fp64_for:
            fp64[sp["index"]] = pkg.Solver(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                                           amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off,
                                           precision=pkg.PREC_FP64, rho_every=pkg.RHO_ONCE, rho_S_min=rho_min,
                                           stream=stream.cuda_stream, device=local)
        total_n += w.n
        masks.append(np.ascontiguousarray(w.stim_mask, dtype=np.uint8))
    return b, fp64, total_n, masks


def _batched_bytes(b, specs):
    """Algorithmic bytes of one batched step (mixed path, per instance: s
    outer stages of one stage item and m - 1 inner items each)."""
    total = 0.0
    for iid, sp in zip(b.ids(), specs):
        info = b.info(iid)
        offd = 6 if len(sp["dims"]) == 3 else 4  # stored off-diagonals per row
        total += info["n"] * step_bytes_mixed(info["N"], info["s"], info["m"], offd)
    return total


# DRAM traffic of batch_step_kernel from one ncu capture of the first 48
# instances (dram__bytes_read.sum + dram__bytes_write.sum of one launch and
# the algorithmic bytes of the same launch; profiles/batch_step_kernel_48_instances.md);
# scaled to the full batch by the algorithmic bytes (the traffic of a launch
# grows with the work it does).  Reported only while the kernel sources hash
# to the captured state.
NCU_BATCH_TRAFFIC = {"instances": 48, "threads_per_sm": 1536, "bytes_per_launch": 749352192 + 268642816,
                     "algorithmic_bytes_per_launch": 1040028606.0,
                     "sources": ("paper_2401_01745_gb300/csrc/kernels.cuh", "paper_2401_01745_gb300/csrc/models.cuh",
                                 "paper_2401_01745_gb300/csrc/batch.cu"),
                     "sha256": "b67c0704be81cca79d00aa3c31a6e33451f8814f8d9d3cfe2eeb0eb10e737d47"}


def batched_line(args, world, rank, local, dev):
    """The batched headline: node-timesteps/s of one persistent launch per
    step over the whole batch, its roofline, end-to-end through the C ABI,
    the FP64 form on the same instances, and accuracy against FP64."""
    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads.configs import batched_specs

    hbm_peak, peak_kind = _peaks()
    specs = batched_specs(args.instances)
    stream = torch.cuda.Stream(device=dev)
    acc_idx = [sp["index"] for sp in specs[::max(1, len(specs) // args.accuracy_instances)]][:args.accuracy_instances]
    t0 = time.perf_counter()
    b, fp64, total_n, masks = _batched_setup(pkg, specs, stream, local,
                                         fp64_for=set(range(len(specs))) if args.fp64_all else set())
    setup_s = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            b.step(0.05)
    b.sync()
    tile, block, tune_ms = b.autotune(0.05, reps=3)
    if args.threads_per_sm:
        # a fixed register budget (for a profiler capture of one build); the
        # autotuner's tile, block and schedule are kept
        b.set_occupancy(args.threads_per_sm)
    bytes_step = _batched_bytes(b, specs)
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
    launches = b.stats()["launches"] - l0
    ms = ev0.elapsed_time(ev1)
    value, ms_max = _aggregate(float(total_n * args.steps), ms, world, dev)
    st = b.stats()
    # the persistent kernel alone: CUDA events around every launch on the
    # batch's stream over K further steps (launched directly, not as a graph)
    b.set_profile(True)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            b.step(0.05)
    b.sync()
    kms, kn = b.kernel_time()
    b.set_profile(False)
    avg_launch_ms = kms / max(kn, 1)
    achieved = bytes_step / (avg_launch_ms / 1e3) / 1e9
    traffic = None
    if (NCU_BATCH_TRAFFIC["sha256"] == _sources_sha256(NCU_BATCH_TRAFFIC["sources"])
            and st["threads_per_sm"] == NCU_BATCH_TRAFFIC["threads_per_sm"]):
        traffic = NCU_BATCH_TRAFFIC["bytes_per_launch"] * bytes_step / NCU_BATCH_TRAFFIC["algorithmic_bytes_per_launch"]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": batched_workload_text(len(specs)), "nodes": total_n, "instances": len(specs),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "precision": MIXED_PRECISION_TEXT,
                   "persistent_launches_per_step": launches / args.steps,
                   "tile": tile, "block": block, "schedule": st["schedule"], "grid": st["grid"],
                   "threads_per_sm": st["threads_per_sm"],
                   "items_per_step": st["items"],
                   "stage_counts": _stage_count_summary(b, specs),
                   "setup_s": setup_s, "device_gb": st["device_bytes"] / 1e9,
                   "l2": "not flushed: the working set (state and matrices, GBs) is far larger than L2 (129 MB)"},
        "roofline": {"bound": "hbm", "kernel": "batch_step_kernel (persistent; every instance's stage and inner "
                                                "items in one launch)",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "peak_source": f"{peak_kind}: hbm_gbs (burst copy)" if peak_kind == "measured"
                     else "fallback: 6,800 GB/s (MEASURED_PEAKS.json absent)",
                     "algorithmic_bytes_per_launch": bytes_step, "avg_launch_us": avg_launch_ms * 1e3,
                     "launches_timed": kn, "traffic": traffic,
                     "traffic_note": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch over the "
                                      f"first {NCU_BATCH_TRAFFIC['instances']} instances at "
                                      f"{NCU_BATCH_TRAFFIC['threads_per_sm']} resident threads per SM, scaled to "
                                      "the full batch by algorithmic bytes") if traffic is not None else
                     "no ncu capture of the current kernel sources at this register budget"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    # ---- end to end through the C ABI with host buffers ----
    # per step: the node masks of every instance in from pinned host memory
    # (emrkc_batch_set_stimulus_async), one persistent launch, V of every
    # instance out to pinned host memory (emrkc_batch_get_V_async, two
    # buffers in rotation); one emrkc_batch_sync at the end
    pin_mask = torch.from_numpy(np.concatenate(masks)).pin_memory()
    del masks
    mask_np = pin_mask.numpy()

    def e2e_run(dtype):
        ring = [torch.empty((total_n,), dtype=dtype, pin_memory=True) for _ in range(2)]
        ring_np = [r.numpy() for r in ring]
        get = b.get_V32_async if dtype == torch.float32 else b.get_V_async
        for k in range(args.warmup):
            b.set_stimulus_async(mask_np)
            b.step(0.05)
            get(ring_np[k % 2])
        b.sync()
        torch.cuda.synchronize()
        _barrier(world)
        t0 = time.perf_counter()
        for k in range(args.steps):
            b.set_stimulus_async(mask_np)
            b.step(0.05)
            get(ring_np[k % 2])
        b.sync()
        e2e_s = _max_over_ranks(time.perf_counter() - t0, world, dev)
        last = ring_np[(args.steps - 1) % 2].astype(np.float64)
        direct = np.concatenate([b.get_state(iid, var=0) for iid in b.ids()])
        ok = (np.array_equal(last, direct) if dtype == torch.float64 else
              bool(np.all(np.abs(last - direct) <= np.spacing(np.abs(last.astype(np.float32))) * 0.5000001)))
        return _sum_over_ranks(float(total_n * args.steps), world, dev) / e2e_s, ok

    v32, ok32 = e2e_run(torch.float32)
    v64, ok64 = e2e_run(torch.float64)
    api = ("per step: emrkc_batch_set_stimulus_async(node masks of every instance, pinned host) + emrkc_batch_step "
           "+ emrkc_batch_get_V{}_async(V of every instance, two pinned host buffers in rotation); one "
           "emrkc_batch_sync at the end")
    out["e2e"] = {"value": v32, "unit": UNIT, "h2d_bytes_per_step": int(total_n), "d2h_bytes_per_step": int(4 * total_n),
                  "steps": args.steps, "result": "V of every instance rounded to FP32 (the nearest float of the "
                                                 "float-float V), 4 bytes per node",
                  "api": api.format("32"), "last_result_matches_get_state": ok32}
    out["e2e_V64"] = {"value": v64, "unit": UNIT, "h2d_bytes_per_step": int(total_n),
                      "d2h_bytes_per_step": int(8 * total_n), "steps": args.steps,
                      "result": "V of every instance in FP64 (hi + lo), 8 bytes per node", "api": api.format(""),
                      "last_result_matches_get_state": ok64}
    b.close()
    del pin_mask
    if world > 1 or args.no_extras:
        return out
    # ---- the plain FP64 form on the same instances (single-instance path) ----
    if fp64:
        evs = []
        for sol in fp64.values():  # the power iteration at t = 0, untimed (as in the mixed run)
            sol.step(0.05)
        for idx, sol in fp64.items():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(args.fp64_steps):
                    sol.step(0.05)
                e1.record(stream)
            evs.append((sol.n, e0, e1))
        stream.synchronize()
        ms64 = sum(a.elapsed_time(c) for _, a, c in evs)
        v64 = sum(n for n, _, _ in evs) * args.fp64_steps / (ms64 / 1e3)
        for sol in fp64.values():
            sol.close()
        fp64.clear()
        out["fp64"] = {"value": v64, "unit": UNIT, "dtype": "f64", "steps": args.fp64_steps,
                       "ms_total": ms64, "instances": len(evs),
                       "note": "plain FP64 emRKC (single-instance path, one solver per instance, run one after "
                               "another on one stream) on the same instances after their first step (rho at "
                               "t = 0), as the mixed batch is timed after its warm-up steps",
                       "multiple": value / v64}
    # ---- accuracy: mixed batch vs FP64 per instance on a sample, T = 50 ms ----
    if args.accuracy_instances > 0:
        out["accuracy"] = _batched_accuracy(pkg, specs, acc_idx, stream, local, args.accuracy_T)
    return out


def _stage_count_summary(b, specs):
    cnt = {}
    for iid in b.ids():
        info = b.info(iid)
        key = f"{'HH' if info['model'] == 2 else 'TTP06'} s={info['s']} m={info['m']}"
        cnt[key] = cnt.get(key, 0) + 1
    return cnt


def _batched_accuracy(pkg, specs, idx, stream, local, T):
    """Instances ``idx`` of the batch, mixed batch against the FP64 solver of
    the same instance over T ms: relative L2 error in V (lumped mass) and the
    activation times."""
    import torch

    from workloads.configs import batched_workload

    sub = [specs[i] for i in idx]
    b = pkg.Batch(rho_every=pkg.RHO_ONCE, stream=stream.cuda_stream, device=local)
    sols, Ms = [], []
    for sp in sub:
        w = batched_workload(sp)
        rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
        rho_min = HH_RHO_S_MAX if w.model == pkg.MODEL_HH else 0.0
        b.add(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask, amplitude=w.stim_amp,
              t_on=w.t_on, t_off=w.t_off, rho_S_min=rho_min)
        sols.append(pkg.Solver(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                               amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, precision=pkg.PREC_FP64,
                               rho_every=pkg.RHO_ONCE, rho_S_min=rho_min, stream=stream.cuda_stream,
                               device=local))
        Ms.append(M)
    H = int(round(T / 0.05))
    with torch.cuda.stream(stream):
        for _ in range(H):
            b.step(0.05)
            for s in sols:
                s.step(0.05)
    b.sync()
    rows = []
    for iid, sp, s, M in zip(b.ids(), sub, sols, Ms):
        s.sync()
        Va, Vb = s.get_state(var=0), b.get_state(iid, var=0)
        ta, tb = s.activation_times(), b.activation_times(iid)
        both = np.isfinite(ta) & np.isfinite(tb)
        info = b.info(iid)
        rows.append({"instance": sp["index"], "n": int(Va.size), "model": "HH" if sp["model"] == 2 else "TTP06",
                     "s": info["s"], "m": info["m"],
                     "rel_l2_err_V": float(np.sqrt(np.sum(M * (Va - Vb) ** 2) / np.sum(M * Va * Va))),
                     "max_activation_diff_ms": float(np.max(np.abs(ta[both] - tb[both]))) if both.any() else None,
                     "activated_nodes": int(both.sum()),
                     "activation_pattern_equal": bool(np.array_equal(np.isfinite(ta), np.isfinite(tb)))})
        s.close()
    b.close()
    act = [r["max_activation_diff_ms"] for r in rows if r["max_activation_diff_ms"] is not None]
    return {"T_ms": T, "instances": len(rows), "reference": "plain FP64 emRKC (GPU, single-instance path) of "
                                                           "the same instance, same rho policy",
            "max_rel_l2_err_V": max(r["rel_l2_err_V"] for r in rows),
            "max_activation_diff_ms": max(act) if act else None,
            "activation_patterns_equal": all(r["activation_pattern_equal"] for r in rows),
            "per_instance": rows}


def run_batched(args):
    import torch

    import paper_2401_01745_gb300 as pkg

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    out = batched_line(args, world, rank, local, dev)
    if rank == 0:
        print(json.dumps(out))
    return 0


def served_result(args, local, dev, requests):
    """Served form: Poisson request stream, HBM-budget admission, continuous batching."""
    import torch

    from paper_2401_01745_gb300.serve import MeshCache, Server
    from workloads.configs import request_workload, served_requests

    reqs = served_requests(count=requests, rate=20.0, seed=4)
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
        reqs2 = served_requests(count=requests, rate=rate, seed=4)
        srv = Server(cache, budget, stream=stream.cuda_stream, device=local, keep_V=False)
        srv.run(reqs2)
        runs["sustainable_70pct"] = dict(srv.summary(), arrival_rate_per_s=rate)
        srv.close()
    head = runs["offered_20_per_s"]
    return {"metric": METRIC + "; p50/p99 solve latency", "value": head["node_timesteps_per_s"], "unit": UNIT,
            "n_gpus": 1, "steps": None, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "p50_latency_s": head["p50_latency_s"], "p99_latency_s": head["p99_latency_s"],
            "config": {"workload": f"served: {requests} requests, Poisson arrivals 20/s (seed 4), n log-U(1e4, "
                                   "2e6) in 8 size classes, slab or shell, HH or TTP06, horizon U(20, 400) ms, "
                                   "dt 0.05 ms, HBM budget 150 GB, continuous batching; latency = arrival -> "
                                   "final V on the host", "mesh_prep_s": prep_s,
                       "offered_node_timesteps_per_s": 20.0 * work},
            "runs": runs, "clocks": clk.summary()}


def run_served(args):
    import torch

    import paper_2401_01745_gb300 as pkg

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    print(json.dumps(served_result(args, local, dev, args.requests)))
    return 0


def _activation_mismatch(ta, tb, Vb_T, Va_T, T, th):
    """Nodes activated by time T in exactly one of two runs (a: reference,
    b: compared): how close to T their crossing was and how far the other
    run's V was from the threshold at T."""
    only_a = np.isfinite(ta) & ~np.isfinite(tb)
    only_b = np.isfinite(tb) & ~np.isfinite(ta)
    rec = {"only_reference": int(only_a.sum()), "only_compared": int(only_b.sum())}
    if only_a.any() or only_b.any():
        t_act = np.concatenate([ta[only_a], tb[only_b]])
        v_other = np.concatenate([Vb_T[only_a], Va_T[only_b]])
        rec["max_T_minus_crossing_ms"] = float(np.max(T - t_act))
        rec["max_threshold_minus_other_V_mV"] = float(np.max(th - v_other))
    return rec


def shell_result(args, local, dev):
    """Ventricle-like shell (~4.2 M nodes): mixed vs plain FP64 over T = 100
    ms, and the nodes activated by T in only one of the two runs (followed
    one more step)."""
    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads import make_workload

    t0 = time.perf_counter()
    w = make_workload("shell_ttp")
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=dev)
    H = int(round(w.T / w.dt))
    sols, res = {}, {}
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
            st = sol.stats()
            res[name] = dict(V=sol.get_state(var=0), act=sol.activation_times(), ms=e0.elapsed_time(e1),
                             s=st["s"], m=st["m"])
            sols[name] = sol
    Va, Vb = res["fp64"]["V"], res["mixed"]["V"]
    ta, tb = res["fp64"]["act"], res["mixed"]["act"]
    both = np.isfinite(ta) & np.isfinite(tb)
    th = -20.0
    mism = _activation_mismatch(ta, tb, Vb, Va, w.T, th)
    # follow the nodes activated in one run only for one more step
    unmatched = np.isfinite(ta) != np.isfinite(tb)
    if unmatched.any():
        for sol in sols.values():
            sol.step(w.dt)
            sol.sync()
        ta2, tb2 = sols["fp64"].activation_times(), sols["mixed"].activation_times()
        ok2 = unmatched & np.isfinite(ta2) & np.isfinite(tb2)
        mism["after_one_more_step"] = {
            "still_unmatched": int((unmatched & ~ok2).sum()),
            "max_activation_diff_ms": float(np.max(np.abs(ta2[ok2] - tb2[ok2]))) if ok2.any() else None}
    for sol in sols.values():
        sol.close()
    err = float(np.sqrt(np.sum(M * (Va - Vb) ** 2) / np.sum(M * Va * Va)))
    vm = w.n * H / (res["mixed"]["ms"] / 1e3)
    v64 = w.n * H / (res["fp64"]["ms"] / 1e3)
    return {"metric": METRIC, "value": vm, "unit": UNIT, "n_gpus": 1, "steps": H, "warmup": 0,
            "ms_per_step": res["mixed"]["ms"] / H, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "shell: 32x362x362 structured box mapped onto a truncated prolate-"
                                   "ellipsoidal shell, interior jitter +-20%, fibres +60 -> -60 deg, TTP06, "
                                   "apical stimulus, dt 0.05 ms, T 100 ms, rho once at t = 0 (timed)",
                       "nodes": w.n, "cells": int(w.cells.shape[0]), "entries_per_row": col.size / w.n,
                       "s": res["mixed"]["s"], "m": res["mixed"]["m"], "setup_s": setup_s,
                       "precision": MIXED_PRECISION_TEXT},
            "fp64": {"value": v64, "unit": UNIT, "ms_per_step": res["fp64"]["ms"] / H, "dtype": "f64",
                     "multiple": vm / v64},
            "accuracy": {"rel_l2_err_V_vs_fp64": err, "T_ms": w.T,
                         "max_activation_diff_ms": float(np.max(np.abs(ta[both] - tb[both]))) if both.any()
                         else None,
                         "activated_nodes_both": int(both.sum()),
                         "activation_pattern_equal": not bool(unmatched.any()),
                         "activated_in_one_run_only": mism},
            "clocks": clk.summary()}


def run_shell(args):
    import torch

    import paper_2401_01745_gb300 as pkg

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    print(json.dumps(shell_result(args, local, dev)))
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


def latency_result(args, local, dev):
    """The 65 x 65 HH square (4,225 nodes) with the power iteration before
    every step (Sec. 5.2 shape): too small to fill a GPU, so it is reported
    as microseconds per step, FP64 and mixed, timed from rest over 400 steps.
    rho_S >= 42 (Table 2's rho_max of HH, 40, times 1.05): with rho_S from
    the power iteration alone this workload takes s = 1 through the upstroke
    and its trajectory is unstable (HH at dt = 0.05 ms is outside the
    stiffness separation emRKC assumes).  The mixed run's V at T = 20 ms is
    compared with the FP64 run's (the FP64 path matches the CPU oracle on this
    workload and setting to 1e-10 in the GPU parity tests)."""
    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads import make_workload

    w = make_workload("square65_hh")
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    stream = torch.cuda.Stream(device=dev)
    H = int(round(w.T / w.dt))
    out = {"metric": "latency: microseconds per emRKC step (rho every step)", "unit": "us/step",
           "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "steps": H,
           "config": {"workload": "square65_hh: 65x65 nodes on [0,1]^2 cm (h = 1/64), sigma 1 mS/cm, HH, corner "
                                  "stimulus 1 ms, dt 0.05 ms, T 20 ms, rho every step (timed), rho_S >= "
                                  f"{HH_RHO_S_MAX}", "nodes": w.n, "rho_S_min": HH_RHO_S_MAX}}
    finals = {}

    def timed(prec):
        res = []
        for rep in range(args.warmup // 3 + 2):
            sol = pkg.Solver(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                             amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, precision=prec, rho_every=1,
                             rho_S_min=HH_RHO_S_MAX, stream=stream.cuda_stream, device=local)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = sol.stats()["launches"]
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(H):
                    sol.step(w.dt)
                e1.record(stream)
            sol.sync()
            st = sol.stats()
            res.append((e0.elapsed_time(e1) * 1e3 / H, st["total_pow_iters"] / H, st["s"], st["m"],
                        (st["launches"] - l0) / H))
            final = (sol.get_state(var=0), sol.activation_times())
            sol.close()
        return res[-1], final  # the first runs are warm-up

    with ClockSampler(local) as clk:
        for name, prec in (("fp64", pkg.PREC_FP64), ("mixed", pkg.PREC_MIXED)):
            (us, its, s_, m_, lps), finals[name] = timed(prec)
            out[name] = {"us_per_step": us, "power_iterations_per_step": its, "s": s_, "m": m_,
                         "launches_per_step": lps, "node_timesteps_per_s": w.n / (us * 1e-6)}
        # the other step form of each precision: mixed runs the
        # device-resident step by default (one launch), FP64 the host-driven
        # one (a launch per phase, the stage counts read back after each
        # power iteration)
        for name, prec, alt, val in (("fp64", pkg.PREC_FP64, "device_resident_step", "1"),
                                     ("mixed", pkg.PREC_MIXED, "host_driven_step", "0")):
            os.environ["EMRKC_FUSED_STEP"] = val
            try:
                (us, _, _, _, lps), _ = timed(prec)
            finally:
                os.environ.pop("EMRKC_FUSED_STEP", None)
            out[name][alt] = {"us_per_step": us, "launches_per_step": lps}
    (Va, ta), (Vb, tb) = finals["fp64"], finals["mixed"]
    both = np.isfinite(ta) & np.isfinite(tb)
    out["accuracy"] = {"rel_l2_err_V_mixed_vs_fp64": float(np.sqrt(np.sum(M * (Va - Vb) ** 2) / np.sum(M * Va * Va))),
                       "T_ms": w.T,
                       "max_activation_diff_ms": float(np.max(np.abs(ta[both] - tb[both]))) if both.any() else None,
                       "activation_pattern_equal": bool(np.array_equal(np.isfinite(ta), np.isfinite(tb))),
                       "fp64_vs_oracle": "<= 1e-10 relative L2 in V over T = 20 ms "
                                         "(tests/test_gpu_parity.py, rho_S >= 42)"}
    out["value"] = out["mixed"]["us_per_step"]
    out["clocks"] = clk.summary()
    return out


def run_latency(args):
    import torch

    import paper_2401_01745_gb300 as pkg

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    print(json.dumps(latency_result(args, local, dev)))
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


def slab_result(args, world, rank, local, dev, full=False):
    """The single-instance form on one mesh (default: the 442,401-node TTP06
    slab): K steps from rest (rho once at t = 0 inside the timed region) with
    L2 flushed before every step, the per-kernel roofline, the plain FP64 form
    and the mixed result's accuracy against it, end to end through the C ABI.
    ``full`` adds the synchronous and whole-state end-to-end variants and the
    rho-every-step run."""
    import torch

    import paper_2401_01745_gb300 as pkg
    from workloads import make_workload

    w = make_workload(args.workload)
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    stream = torch.cuda.Stream(device=dev)
    prec = pkg.PREC_MIXED if args.precision == "mixed" else pkg.PREC_FP64
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    hbm_peak, peak_kind = _peaks()
    N = pkg.num_vars(w.model)
    K_steps = args.slab_steps

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

    # ---- K steps from rest on a fresh solver (includes rho at t = 0) ----
    sol = make(prec)
    torch.cuda.synchronize()
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, launches = timed_steps(sol, K_steps)
    torch.cuda.synchronize()
    _barrier(world)
    st = sol.stats()
    total_ms = sum(ms)
    value, total_ms_max = _aggregate(float(w.n * K_steps), total_ms, world, dev)
    sol.close()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K_steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / K_steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == pkg.PREC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": (f"{args.workload}: 201x71x31-node Kuhn-tet slab 2.0x0.7x0.3 cm, TTP06 epi, "
                                "dt 0.05 ms, 50 uA/cm^2 corner stimulus; timed from rest (t = 0)"
                                if args.workload == "slab_ttp" else
                                f"{args.workload}: {w.n}-node synthetic mesh, dt {w.dt} ms, corner stimulus; "
                                "timed from rest (t = 0)"),
                   "nodes": w.n, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "precision": MIXED_PRECISION_TEXT if prec == pkg.PREC_MIXED else "fp64",
                   "rho_policy": ("once at t = 0 (inside the timed region; its cost is spread over the "
                                  f"{K_steps} timed steps)" if args.rho_every == 0
                                  else f"every {args.rho_every} steps"),
                   "s": st["s"], "m": st["m"], "power_iterations": st["total_pow_iters"],
                   "l2": "flushed before every timed step (512 MB write, outside the step's events)"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if args.no_extras:
        return out

    # ---- per-kernel durations (CUDA events around every launch, same stream) ----
    solp = make(prec, profile=True)
    timed_steps(solp, K_steps)
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
        if dom_key == "stage" else "inner_kernel_mixed (SpMV stage + float-float V update)",
        "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
        "peak_source": f"{peak_kind}: hbm_gbs (burst copy)" if peak_kind == "measured"
        else "fallback: 6,800 GB/s (MEASURED_PEAKS.json absent)",
        "bytes_per_node_per_launch": per_launch[dom_key], "avg_launch_us": avg_ms * 1e3,
        "matrix_entries_per_row": nnz_row,
        "traffic": None}
    if (dom_key == "stage" and prec == pkg.PREC_MIXED and args.workload == NCU_TRAFFIC["workload"]
            and _sources_sha256(NCU_TRAFFIC["sources"]) == NCU_TRAFFIC["sha256"]):
        out["roofline"]["traffic"] = NCU_TRAFFIC["bytes_per_launch"]
        out["roofline"]["traffic_note"] = ("ncu dram bytes read + write of one launch (cold cache); at this size "
                                           "the state fits in L2, so most writes are still in L2 at kernel end")
        out["roofline"]["algorithmic_bytes_per_launch"] = per_launch[dom_key] * w.n
    out["kernels"] = {k: {"ms_per_step": phase_ms[k] / K_steps, "launches_per_step": phase_n[k] / K_steps,
                          "avg_launch_us": 1e3 * phase_ms[k] / max(phase_n[k], 1)}
                      for k in phase_ms if phase_n[k] > 0}
    if "stage" in per_launch and "inner" in per_launch:
        out["kernels"]["stage"]["gbs"] = bytes_stage * w.n / (phase_ms["stage"] / max(phase_n["stage"], 1) / 1e3) / 1e9
        out["kernels"]["inner"]["gbs"] = bytes_inner * w.n / (phase_ms["inner"] / max(phase_n["inner"], 1) / 1e3) / 1e9
    # whole step: algorithmic bytes of one step (stage + inner) over the
    # measured time of a step after the power iteration at t = 0
    steady = sorted(ms)[len(ms) // 2]
    out["step_bytes_per_node"] = bytes_stage + (p1["m"] - 1) * bytes_inner if prec == pkg.PREC_MIXED else None
    if prec == pkg.PREC_MIXED:
        out["step_frac_of_hbm"] = out["step_bytes_per_node"] * w.n / (steady / 1e3) / 1e9 / hbm_peak
        out["median_step_ms"] = steady

    # ---- end to end through the C ABI with host buffers (reading c24) ----
    Ke = min(K_steps, 1000)
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
    if full:
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
        # the whole state through the host every step (all variables in, V out)
        sol = make(prec)
        pinned_in = torch.empty((N, w.n), dtype=torch.float64, pin_memory=True)
        sol.get_state(out=pinned_in.numpy())
        Kf = min(K_steps, 100)
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
        # rho every step (Algorithm 5 warm started before every step)
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
                                 "power_iterations_per_step":
                                     ste["total_pow_iters"] / (args.warmup + args.every_step_steps)}

    # ---- plain FP64 form on the same workload, and accuracy of the mixed form ----
    if prec == pkg.PREC_MIXED and rank == 0:
        s64 = make(pkg.PREC_FP64)
        ms64, _ = timed_steps(s64, args.fp64_steps)
        s64.close()
        v64 = w.n * args.fp64_steps / (sum(ms64) / 1e3)
        out["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": sum(ms64) / args.fp64_steps,
                       "steps": args.fp64_steps, "dtype": "f64",
                       "note": "same workload and rho policy, timed from rest", "multiple": value / v64}
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
    del flush
    return out


def run_single(args):
    """The single-instance line on --workload (default the 442k-node slab)."""
    import torch

    import paper_2401_01745_gb300 as pkg

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    out = slab_result(args, world, rank, local, dev, full=True)
    if rank == 0:
        print(json.dumps(out))
    return 0


def _headline(args):
    """Default run: the batched line; on one GPU also the single-instance slab,
    the shell, the served form and the 65 x 65 latency line as extra keys,
    and the CPU oracle on all host cores as cpu_baseline."""
    import torch

    import paper_2401_01745_gb300 as pkg

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    t_start = time.perf_counter()
    out = batched_line(args, world, rank, local, dev)
    legs_s = {"batched": time.perf_counter() - t_start}
    if world == 1 and not args.no_extras:
        for key, fn, skip in (("slab", lambda: slab_result(args, world, rank, local, dev), args.no_slab),
                              ("shell", lambda: shell_result(args, local, dev), args.no_shell),
                              ("served", lambda: served_result(args, local, dev, args.served_requests),
                               args.no_served),
                              ("latency", lambda: latency_result(args, local, dev), args.no_latency)):
            if skip:
                continue
            t0 = time.perf_counter()
            out[key] = fn()
            torch.cuda.synchronize()
            legs_s[key] = time.perf_counter() - t0
    if rank == 0 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        cores, cpu = _cpu_info()
        value, used, recs = _oracle_pool(args.instances, budget_s=args.cpu_budget_s)
        one, _, recs1 = _oracle_pool(args.instances, budget_s=args.cpu_budget_s / 2, procs=1)
        out["cpu_baseline"] = {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                               "sample": _pool_sample_text(recs, args.instances), "cpu": cpu,
                               "host_cores": cores, "one_core_value": one,
                               "one_core_sample": _pool_sample_text(recs1, args.instances)}
        legs_s["cpu_baseline"] = time.perf_counter() - t0
    out["legs_wall_s"] = legs_s
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed steps of the batched line")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances", type=int, default=256, help="instances of the batched workload")
    ap.add_argument("--threads-per-sm", type=int, default=0, choices=[0, 1024, 1536, 2048],
                    help="batched line: resident threads per SM after autotuning (0: the autotuner's choice)")
    ap.add_argument("--accuracy-instances", type=int, default=16)
    ap.add_argument("--accuracy-T", type=float, default=50.0)
    ap.add_argument("--no-fp64-all", dest="fp64_all", action="store_false",
                    help="skip the FP64 form on the batched instances")
    ap.add_argument("--cpu-budget-s", type=float, default=10.0)
    ap.add_argument("--single", action="store_true", help="single-instance line on --workload")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="slab_ttp")
    ap.add_argument("--slab-steps", type=int, default=None, help="timed steps of the single-instance line")
    ap.add_argument("--rho-every", type=int, default=0, help="0: once at t = 0 (Sec. 5 setup); k: every k steps")
    ap.add_argument("--every-step-steps", type=int, default=200)
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--served-requests", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline only (for profiler runs)")
    ap.add_argument("--no-slab", action="store_true")
    ap.add_argument("--no-shell", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-latency", action="store_true")
    ap.add_argument("--batched", action="store_true", help="batched line only")
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
    if args.slab_steps is None:
        args.slab_steps = 1000 if args.single else args.steps
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
        return run_batched(args)
    if args.single:
        return run_single(args)
    return _headline(args)


if __name__ == "__main__":
    sys.exit(main())
