"""Served form: continuous batching under an HBM budget.

A small seeded request stream (mixed sizes, geometries, ionic models and
horizons) is served with a budget that forces requests to wait for memory;
every request finishes, the budget is never exceeded, and each result equals
the same solve run alone (single-instance mixed-precision path, same rho
policy and step count).
"""

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from paper_2401_01745_gb300.serve import MeshCache, Server
from workloads.configs import request_workload, served_requests

pytestmark = pytest.mark.gpu


def test_served_results_equal_solo_runs():
    pkg.build()
    # arrivals 0.25 ms apart on average: the second request arrives while the
    # first (at least 20 steps) is still on the device, whatever the GPU's speed
    reqs = served_requests(count=8, rate=4000.0, seed=11, n_min=2e3, n_max=3e4, horizon=(1.0, 4.0),
                           size_classes=3)
    cache = MeshCache(request_workload)
    cache.prepare(reqs)
    srv = Server(cache, budget_bytes=1.0, dt=0.05)
    sizes = [srv.request_bytes(r) for r in reqs]
    srv.budget = 2.2 * max(sizes)  # at most about two solves resident at a time
    results = srv.run(reqs)
    summ = srv.summary()
    srv.close()
    assert len(results) == len(reqs)
    assert summ["peak_device_gb"] * 1e9 <= srv.budget + 1
    assert summ["peak_active"] >= 2  # solves overlapped on the device
    assert all(r.latency >= 0 for r in results)
    by_index = {r["index"]: r for r in reqs}
    for res in results:
        req = by_index[res.index]
        w, rp, col, K, M = cache.get(req)
        sol = pkg.Solver(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=req["model"], mask=w.stim_mask,
                         amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, precision=pkg.PREC_MIXED,
                         rho_every=pkg.RHO_ONCE, rho_S_min=42.0 if req["model"] == pkg.MODEL_HH else 0.0)
        for _ in range(req["steps"]):
            sol.step(0.05)
        sol.sync()
        V = sol.get_state(var=0)
        sol.close()
        assert res.steps == req["steps"]
        assert np.max(np.abs(res.V - V)) <= 1e-6 * np.max(np.abs(V))
