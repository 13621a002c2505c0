"""Batched and served results against the FP64 CPU oracle.

The batched persistent step and the serving loop run the mixed-precision
form; each instance's V after its steps is compared with the oracle's
Algorithm 3 run of the same instance (same seeded inputs, same rho policy,
same step count): relative L2 error in V (lumped mass) <= 1e-3, activation
times within 0.05 ms where both runs crossed the threshold, and the same set
of activated nodes.  Cases: HH with rho_S >= 42 (s = 2, m = 1), TTP06 with
rho estimated once (s = 1, m = 2), fixed rho giving s = 3 and m = 5 (buffers
rewritten within a launch: loads through L2), an instance that joins the
batch late and one that leaves early, and a served request stream.
"""

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from oracle.emrkc import Monodomain, OracleRun
from workloads import make_workload

pytestmark = pytest.mark.gpu

TOL_V = 1e-3
TOL_ACT_MS = 0.05


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _oracle(w, steps, dt, **kw):
    prob = Monodomain.from_workload(w)
    ref = OracleRun(prob, **kw)
    for _ in range(steps):
        ref.step(dt)
    return prob, ref


def _check(prob, ref, V, act, sm=None):
    err = prob.l2_norm(V - ref.Y[0]) / prob.l2_norm(ref.Y[0])
    assert err <= TOL_V, f"rel L2 error in V {err:.3e}"
    if sm is not None:
        assert {(l[0], l[1]) for l in ref.log} == {sm}
    if act is not None:
        assert np.array_equal(np.isfinite(act), np.isfinite(ref.act))
        fin = np.isfinite(ref.act)
        if fin.any():
            assert np.max(np.abs(act[fin] - ref.act[fin])) <= TOL_ACT_MS
    return err


def test_batch_matches_oracle_rho_once():
    """HH (rho_S >= 42: s = 2, m = 1) and TTP06 (s = 1, m = 2) instances of
    different sizes in one batch, rho estimated once per instance."""
    dt, steps = 0.05, 60
    cases = [("square33x29_hh", 1.0 / 64, 42.0), ("slab41x15x7_ttp", 0.01, 0.0),
             ("slab19x11x9_hh", 0.01, 42.0), ("slab23x9x5_ttp", 0.01, 0.0)]
    ws = [make_workload(n, h=h) for n, h, _ in cases]
    b = pkg.Batch(rho_every=pkg.RHO_ONCE)
    ids = [b.add_workload(w, rho_S_min=r) for w, (_, _, r) in zip(ws, cases)]
    for _ in range(steps):
        b.step(dt)
    b.sync()
    for iid, w, (name, _, rmin) in zip(ids, ws, cases):
        prob, ref = _oracle(w, steps, dt, rho_every=0, rho_S_min=rmin)
        info = b.info(iid)
        sm = (2, 1) if rmin > 0 else (1, 2)
        assert (info["s"], info["m"]) == sm, name
        act = b.activation_times(iid)
        assert np.isfinite(act).any(), name  # the wave started
        _check(prob, ref, b.get_state(iid, var=0), act, sm)
    b.close()


def test_batch_matches_oracle_three_outer_five_inner_stages():
    """Fixed rho giving s = 3 and m = 5: every state and increment buffer is
    rewritten within one launch, so the persistent kernel reads through L2."""
    dt, steps = 0.05, 40
    rF, rS = 7000.0, 300.0
    ws = [make_workload("slab41x15x7_ttp", h=0.01), make_workload("square33x29_hh", h=1.0 / 64)]
    b = pkg.Batch(rho_every=pkg.RHO_FIXED, rho_F=rF, rho_S=rS)
    ids = [b.add_workload(w) for w in ws]
    for _ in range(steps):
        b.step(dt)
    b.sync()
    for iid, w in zip(ids, ws):
        assert (b.info(iid)["s"], b.info(iid)["m"]) == (3, 5)
        prob, ref = _oracle(w, steps, dt, fixed_rho=(rF, rS))
        _check(prob, ref, b.get_state(iid, var=0), b.activation_times(iid), (3, 5))
    b.close()


def test_batch_join_and_leave_match_oracle():
    """An instance that joins after 10 steps and one that leaves after 20
    match the oracle for the steps they took."""
    dt = 0.05
    wa = make_workload("slab23x9x5_ttp", h=0.01)
    wb = make_workload("square33x29_hh", h=1.0 / 64)
    b = pkg.Batch()
    ia = b.add_workload(wa)
    for _ in range(10):
        b.step(dt)
    ib = b.add_workload(wb, rho_S_min=42.0)
    for _ in range(10):
        b.step(dt)
    b.sync()
    Va, acta = b.get_state(ia, var=0), b.activation_times(ia)
    b.remove(ia)
    for _ in range(30):
        b.step(dt)
    b.sync()
    Vb, actb = b.get_state(ib, var=0), b.activation_times(ib)
    b.close()
    prob, ref = _oracle(wa, 20, dt, rho_every=0)
    _check(prob, ref, Va, acta)
    prob, ref = _oracle(wb, 40, dt, rho_every=0, rho_S_min=42.0)
    _check(prob, ref, Vb, actb)


def test_served_results_match_oracle():
    """A served stream (slab and shell meshes, HH and TTP06, horizons of
    20-80 steps, at most about two solves resident): each final V against the
    oracle's run of the same request."""
    from paper_2401_01745_gb300.serve import MeshCache, Server
    from workloads.configs import request_workload, served_requests

    reqs = served_requests(count=6, rate=4000.0, seed=11, n_min=2e3, n_max=1.2e4, horizon=(1.0, 4.0),
                           size_classes=3)
    cache = MeshCache(request_workload)
    cache.prepare(reqs)
    srv = Server(cache, budget_bytes=1.0, dt=0.05)
    srv.budget = 2.2 * max(srv.request_bytes(r) for r in reqs)
    results = srv.run(reqs)
    assert srv.summary()["peak_active"] >= 2
    srv.close()
    by_index = {r["index"]: r for r in reqs}
    assert len(results) == len(reqs)
    for res in results:
        req = by_index[res.index]
        w = request_workload(req)
        prob, ref = _oracle(w, req["steps"], 0.05, rho_every=0,
                            rho_S_min=42.0 if req["model"] == pkg.MODEL_HH else 0.0)
        assert res.steps == req["steps"]
        _check(prob, ref, res.V, None)


def test_full_batch_sampled_instances_match_oracle():
    """The batched workload at full size (256 instances, 31.2M nodes) in the
    launch configuration the benchmark times (autotuned tile and block, graph
    replay), 40 steps from rest: the smallest 2-D and 3-D instances of each
    ionic model (TTP06 with s = 1 and m = 1 or 2, HH with s = 2, m = 1)
    against the oracle element by element; every instance finite, within the
    physiological range of its model, and with the same step count and time."""
    from workloads.configs import batched_specs, batched_workload

    dt, steps = 0.05, 40
    specs = batched_specs(256)
    b = pkg.Batch(rho_every=pkg.RHO_ONCE)
    for sp in specs:
        b.add_workload(batched_workload(sp), rho_S_min=42.0 if sp["model"] == pkg.MODEL_HH else 0.0)
    for _ in range(3):
        b.step(dt)
    b.sync()
    b.autotune(dt, reps=2)
    for _ in range(steps - 3):
        b.step(dt)
    b.sync()
    ids = b.ids()
    assert len(ids) == 256 and b.stats()["total_nodes"] == 31163705
    for iid in ids:
        info = b.info(iid)
        assert info["steps"] == steps and abs(info["t"] - steps * dt) < 1e-9
        V = b.get_state(iid, var=0)
        assert np.all(np.isfinite(V)) and V.min() > -100.0 and V.max() < 80.0
    # the sample: smallest 2-D and 3-D instances of each model
    sample = {}
    for sp in specs:
        key = (sp["model"], len(sp["dims"]))
        n = int(np.prod(sp["dims"]))
        if key not in sample or n < sample[key][0]:
            sample[key] = (n, sp)
    assert len(sample) == 4
    for (model, dim), (n, sp) in sorted(sample.items()):
        w = batched_workload(sp)
        iid = ids[sp["index"]]
        rmin = 42.0 if model == pkg.MODEL_HH else 0.0
        prob, ref = _oracle(w, steps, dt, rho_every=0, rho_S_min=rmin)
        info = b.info(iid)
        assert (info["s"], info["m"]) == (ref.log[-1][0], ref.log[-1][1])
        _check(prob, ref, b.get_state(iid, var=0), b.activation_times(iid))
    b.close()


def test_batch_tiny_and_empty():
    """Degenerate batches: no instance at all (steps are no-ops), and
    instances of 2, 3 and 4 nodes (one ragged sliced-ELL slice, a single
    tile) beside a larger one, each against the oracle."""
    b = pkg.Batch()
    b.step(0.05)
    b.sync()
    assert b.stats()["instances"] == 0 and b.stats()["launches"] == 0
    dt, steps = 0.05, 30
    names = ["line2_hh", "line3_ttp", "square2x2_hh", "slab23x9x5_ttp"]
    ws = [make_workload(n) if n != "slab23x9x5_ttp" else make_workload(n, h=0.01) for n in names]
    rmins = [42.0 if w.model == pkg.MODEL_HH else 0.0 for w in ws]
    ids = [b.add_workload(w, rho_S_min=r) for w, r in zip(ws, rmins)]
    for _ in range(steps):
        b.step(dt)
    b.sync()
    for iid, w, r in zip(ids, ws, rmins):
        prob, ref = _oracle(w, steps, dt, rho_every=0, rho_S_min=r)
        _check(prob, ref, b.get_state(iid, var=0), b.activation_times(iid))
    b.close()
