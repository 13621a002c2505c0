"""Served form: a continuous-batching request loop over the batched step.

Requests (monodomain solves of different sizes, geometries, ionic models and
horizons) arrive over time.  The server admits a waiting request as soon as
its device memory fits under the HBM budget (first come, first served),
keeps every admitted solve's state on the device, advances all admitted
solves together with one persistent launch per step (emrkc_batch_step), and
retires a solve when it reaches its horizon: its final V is copied to the
host, its latency (arrival -> V on the host) recorded, and its memory freed,
which may admit the next waiting request.

Meshes are prepared once per (geometry, size class) and reused, the way a
serving system keeps its models loaded; only the ionic model and horizon
differ between requests of the same class.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import MODEL_HH, Batch, assemble_p1, instance_bytes, num_vars


@dataclass
class Result:
    index: int
    arrival: float
    admitted: float
    finished: float
    n: int
    steps: int
    model: int
    V: np.ndarray = field(repr=False, default=None)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class MeshCache:
    """Assembled P1 matrices per (geometry, size class)."""

    def __init__(self, make_workload_fn):
        self._make = make_workload_fn
        self._cache = {}

    def get(self, req):
        key = (req["geometry"], req["size_class"])
        if key not in self._cache:
            w = self._make(req)
            rp, col, K, M = assemble_p1(w.coords, w.cells, w.D)
            self._cache[key] = (w, rp, col, K, M)
        return self._cache[key]

    def prepare(self, requests):
        for r in requests:
            self.get(r)


class Server:
    """Continuous batching of emRKC solves under an HBM budget."""

    def __init__(self, mesh_cache: MeshCache, budget_bytes: float, dt: float = 0.05, sync_every: int = 8,
                 hh_rho_S_min: float = 42.0, stream=None, device=0, keep_V: bool = True):
        self.cache = mesh_cache
        self.budget = float(budget_bytes)
        self.dt = dt
        self.sync_every = sync_every
        self.hh_rho_S_min = hh_rho_S_min
        self.keep_V = keep_V
        self.batch = Batch(stream=stream, device=device)
        self.active = {}  # instance id -> (req, admitted time, steps done, bytes)
        self.used = 0.0
        self.results = []
        self.node_steps = 0.0
        self.peak_active = 0
        self.peak_bytes = 0.0

    def request_bytes(self, req):
        w, rp, col, K, M = self.cache.get(req)
        # stored off-diagonal entries of L per row (near-zero entries dropped)
        return instance_bytes(w.n, col.size / w.n, req["model"])

    def _admit(self, req, now):
        w, rp, col, K, M = self.cache.get(req)
        rho_min = self.hh_rho_S_min if req["model"] == MODEL_HH else 0.0
        iid = self.batch.add(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=req["model"], mask=w.stim_mask,
                             amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, rho_S_min=rho_min)
        b = self.request_bytes(req)
        self.active[iid] = [req, now, 0, b, w.n]
        self.used += b
        self.peak_bytes = max(self.peak_bytes, self.used)

    def run(self, requests, clock=time.perf_counter):
        """Serve ``requests`` (arrival times in seconds from the start)."""
        pending = sorted(requests, key=lambda r: r["arrival"])
        waiting = []
        t0 = clock()
        k = 0
        step_count = 0
        while k < len(pending) or waiting or self.active:
            now = clock() - t0
            while k < len(pending) and pending[k]["arrival"] <= now:
                waiting.append(pending[k])
                k += 1
            while waiting and self.used + self.request_bytes(waiting[0]) <= self.budget:
                self._admit(waiting.pop(0), clock() - t0)
            if not self.active:
                if waiting:  # a single request larger than the budget can never run
                    raise RuntimeError("request larger than the HBM budget")
                if k < len(pending):
                    time.sleep(max(0.0, min(0.01, pending[k]["arrival"] - (clock() - t0))))
                continue
            self.peak_active = max(self.peak_active, len(self.active))
            self.batch.step(self.dt)
            step_count += 1
            done = []
            for iid, rec in self.active.items():
                rec[2] += 1
                self.node_steps += rec[4]
                if rec[2] >= rec[0]["steps"]:
                    done.append(iid)
            if done:
                self.batch.sync()
                for iid in done:
                    req, adm, steps, b, n = self.active.pop(iid)
                    V = self.batch.get_state(iid, var=0) if self.keep_V else None
                    fin = clock() - t0
                    self.results.append(Result(req["index"], req["arrival"], adm, fin, n, steps, req["model"], V))
                    self.batch.remove(iid)
                    self.used -= b
            elif step_count % self.sync_every == 0:
                self.batch.sync()
        self.batch.sync()
        self.wall = clock() - t0
        return self.results

    def summary(self):
        lat = np.array([r.latency for r in self.results])
        return {
            "requests": len(self.results),
            "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_latency_s": float(lat.mean()) if lat.size else None,
            "node_timesteps_per_s": self.node_steps / self.wall if self.wall > 0 else None,
            "wall_s": self.wall,
            "peak_active": self.peak_active,
            "peak_device_gb": self.peak_bytes / 1e9,
            "budget_gb": self.budget / 1e9,
        }

    def close(self):
        self.batch.close()
