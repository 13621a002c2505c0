"""Batched persistent step: every instance's result equals its solo run.

Uneven instances (HH and TTP06, 2-D and 3-D, different sizes and stage
counts) share one persistent launch per step; each instance's state after K
steps is compared with the same instance run alone by the single-instance
mixed-precision path (same per-node arithmetic, so agreement is expected to
the last bit; the assertion allows 1e-6 of the variable's scale).
"""

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _solo(w, steps, dt, **kw):
    s = pkg.Solver.from_workload(w, precision=pkg.PREC_MIXED, **kw)
    for _ in range(steps):
        s.step(dt)
    s.sync()
    Y = s.get_state()
    act = s.activation_times()
    st = s.stats()
    s.close()
    return Y, act, (st["s"], st["m"])


def _close(Y, Yref):
    for k in range(Y.shape[0]):
        scale = max(np.max(np.abs(Yref[k])), 1e-12)
        assert np.max(np.abs(Y[k] - Yref[k])) <= 1e-6 * scale, f"variable {k}"


WORKLOADS = [("square33x29_hh", 1.0 / 64), ("slab23x9x5_ttp", 0.01), ("slab41x13x7_ttp", 0.01),
             ("slab19x11x9_hh", 0.01), ("square61x7_ttp", 0.005)]


def test_batch_equals_solo_rho_once():
    dt, steps = 0.02, 60
    ws = [make_workload(n, h=h) for n, h in WORKLOADS]
    b = pkg.Batch(rho_every=pkg.RHO_ONCE)
    ids = [b.add_workload(w) for w in ws]
    for _ in range(steps):
        b.step(dt)
    b.sync()
    exact = 0
    for iid, w in zip(ids, ws):
        Y = b.get_state(iid)
        Yref, aref, sm = _solo(w, steps, dt, rho_every=pkg.RHO_ONCE)
        info = b.info(iid)
        assert (info["s"], info["m"]) == sm
        assert info["steps"] == steps and abs(info["t"] - steps * dt) < 1e-12
        _close(Y, Yref)
        a = b.activation_times(iid)
        assert np.array_equal(np.isnan(a), np.isnan(aref))
        exact += int(np.array_equal(Y, Yref))
    st = b.stats()
    assert st["instances"] == len(ws) and st["launches"] == steps
    b.close()
    print(f"bitwise-equal instances: {exact}/{len(ws)}")


@pytest.mark.parametrize("rF,rS,sm_expected", [(3000.0, 60.0, (2, 5)), (1000.0, 60.0, (2, 3)),
                                                (1000.0, 300.0, (3, 2)), (250.0, 10.0, (1, 3))])
def test_batch_equals_solo_many_stages(rF, rS, sm_expected):
    """Fixed rho sets (s, m): the phase chain of the persistent kernel covers
    outer and inner three-term recurrences, with buffers written once per
    launch (s = 1, m = 3: loads through L1) and rewritten within a launch
    (s >= 2 with m >= 2, s = 3 or m = 5: loads through L2)."""
    dt, steps = 0.05, 30
    ws = [make_workload(n, h=h) for n, h in WORKLOADS[:3]]
    b = pkg.Batch(rho_every=pkg.RHO_FIXED, rho_F=rF, rho_S=rS)
    ids = [b.add_workload(w) for w in ws]
    for _ in range(steps):
        b.step(dt)
    b.sync()
    for iid, w in zip(ids, ws):
        Yref, _, sm = _solo(w, steps, dt, rho_every=pkg.RHO_FIXED, rho_F=rF, rho_S=rS)
        assert sm == sm_expected
        assert (b.info(iid)["s"], b.info(iid)["m"]) == sm
        _close(b.get_state(iid), Yref)
    b.close()


def test_continuous_batching_join_and_leave():
    """An instance that joins after 10 steps and one that leaves after 20 both
    match their solo runs for the steps they took."""
    dt = 0.02
    wa = make_workload("slab23x9x5_ttp", h=0.01)
    wb = make_workload("square33x29_hh", h=1.0 / 64)
    b = pkg.Batch()
    ia = b.add_workload(wa)
    for _ in range(10):
        b.step(dt)
    ib = b.add_workload(wb)
    for _ in range(10):
        b.step(dt)
    b.sync()
    Ya = b.get_state(ia)
    b.remove(ia)
    for _ in range(15):
        b.step(dt)
    b.sync()
    Yb = b.get_state(ib)
    _close(Ya, _solo(wa, 20, dt, rho_every=pkg.RHO_ONCE)[0])
    _close(Yb, _solo(wb, 25, dt, rho_every=pkg.RHO_ONCE)[0])
    assert b.info(ib)["steps"] == 25
    with pytest.raises(pkg.EmrkcError):
        b.info(ia)
    b.close()


def test_autotune_keeps_state():
    dt = 0.05
    b = pkg.Batch()
    ids = [b.add_workload(make_workload(n, h=h)) for n, h in WORKLOADS[1:3]]
    for _ in range(3):
        b.step(dt)
    b.sync()
    before = [b.get_state(i) for i in ids]
    tile, block, ms = b.autotune(dt, reps=2)
    assert tile in (512, 1024, 2048, 4096, 8192) and block in (128, 256) and ms > 0
    after = [b.get_state(i) for i in ids]
    for x, y in zip(before, after):
        np.testing.assert_array_equal(x, y)
    st = b.stats()
    b.step(dt)
    b.sync()
    assert b.stats()["tile"] == tile
    b.close()


def test_dependency_wait_timeout_is_reported():
    """With a wait limit of 0 polls, an item whose dependency is not yet done
    gives up at once: the kernel records the failure, every CTA returns, and
    emrkc_batch_sync reports EMRKC_ERR_TIMEOUT (no device hang, no trap)."""
    b = pkg.Batch()
    b.add_workload(make_workload("slab101x41x21_ttp", h=0.01))  # s = 1, m = 2: two phases
    b.set_config(256, 128)
    b.set_spin_limit(0)
    code = None
    for _ in range(5):
        try:
            b.step(0.05)
            b.sync()
        except pkg.EmrkcError as e:
            code = e.code
            break
    assert code == 5
    b.close()


def test_non_finite_instance_is_reported_by_id():
    """An instance whose fixed rho_F is far below rho(f_F) (m = 1 with
    dt rho(f_F) ~ 6, so the highest diffusion modes grow every step) overflows.
    emrkc_batch_sync, which reads every instance's flag word with one copy,
    names that instance by its id; once it leaves, the batch steps on cleanly
    and the other instance equals its solo run."""
    good = make_workload("slab23x9x5_ttp", h=0.01)
    bad = make_workload("slab19x11x9_hh", h=0.01)
    b = pkg.Batch()
    ig = b.add_workload(good)
    ib = b.add_workload(bad, rho_every=pkg.RHO_FIXED, rho_F=1.0, rho_S=1.0)
    for _ in range(40):
        b.step(0.05)
    with pytest.raises(pkg.EmrkcError) as ei:
        b.sync()
    assert ei.value.code == 4 and f"instance {ib}:" in str(ei.value)
    b.remove(ib)
    for _ in range(10):
        b.step(0.05)
    b.sync()
    Y = b.get_state(ig)
    b.close()
    Yref, _, _ = _solo(good, 50, 0.05)
    _close(Y, Yref)


def test_batch_pipelined_io_matches_waiting_calls():
    """emrkc_batch_set_stimulus_async / emrkc_batch_get_V_async (every
    instance's mask in, every instance's V out, two host buffers in rotation)
    give exactly the V that emrkc_batch_get_state returns, after each step,
    and a mask set this way acts like the mask given at creation."""
    dt, steps = 0.05, 12
    ws = [make_workload(n, h=h) for n, h in WORKLOADS[:3]]
    a, b = pkg.Batch(), pkg.Batch()
    ia = [a.add_workload(w) for w in ws]
    for w in ws:  # b: created without a stimulus; masks only through the async call
        rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
        b.add(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=None, amplitude=w.stim_amp,
              t_on=w.t_on, t_off=w.t_off)
    assert b.ids() == sorted(b.ids()) and a.ids() == ia
    masks = np.concatenate([np.ascontiguousarray(w.stim_mask, dtype=np.uint8) for w in ws])
    total = sum(w.n for w in ws)
    assert a.total_nodes() == total
    ring = [np.empty(total), np.empty(total)]
    got = []
    for k in range(steps):
        a.step(dt)
        b.set_stimulus_async(masks)
        b.step(dt)
        b.get_V_async(ring[k % 2])
        if k % 2 == 1:
            b.sync()
            a.sync()
            ref = np.concatenate([a.get_state(i, var=0) for i in ia])
            got.append(np.array_equal(ring[k % 2], ref))
    assert all(got)
    # V rounded to FP32: the nearest float of the V that get_state returns
    v32 = np.empty(total, dtype=np.float32)
    b.get_V32_async(v32)
    b.sync()
    ref = np.concatenate([b.get_state(i, var=0) for i in b.ids()])
    assert np.all(np.abs(v32.astype(np.float64) - ref) <= np.spacing(np.abs(v32)) * 0.5000001)
    with pytest.raises(pkg.EmrkcError):
        b.get_V_async(np.empty(total - 1))
    a.close()
    b.close()


def test_batch_kernel_timing():
    b = pkg.Batch()
    b.add_workload(make_workload("slab23x9x5_ttp", h=0.01))
    b.step(0.05)
    b.set_profile(True)
    for _ in range(4):
        b.step(0.05)
    b.sync()
    ms, n = b.kernel_time()
    assert n == 4 and ms > 0
    b.set_profile(False)
    b.step(0.05)
    b.sync()
    assert b.kernel_time()[1] == 4
    b.close()


@pytest.mark.parametrize("schedule", [1, 2])
def test_work_list_orders_give_identical_states(schedule):
    """The persistent kernel's work-list order (whole phases, or at most 16 or
    4 tiles of an instance in turn) changes only when each node is computed:
    every instance's state is bit for bit the same."""
    dt, steps = 0.05, 12
    ws = [make_workload(n, h=h) for n, h in WORKLOADS]
    out = []
    for sched in (0, schedule):
        b = pkg.Batch()
        ids = [b.add_workload(w) for w in ws]
        b.set_config(256, 128)
        b.set_schedule(sched)
        for _ in range(steps):
            b.step(dt)
        b.sync()
        assert b.stats()["schedule"] == sched
        out.append([b.get_state(i) for i in ids])
        b.close()
    for x, y in zip(*out):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("tps", [1024, 2048])
def test_register_budgets_give_identical_states(tps):
    """The persistent kernel compiled for 1024, 1536 (default) or 2048
    resident threads per SM (64, 40 or 32 registers per thread; the heavier
    models spill at the smaller budgets) computes the same per-node
    arithmetic: every instance's state is bit for bit the same.  Instances
    with s = 2, m = 1 (HH), s = 1 and m = 2 (TTP06) and the inner-stage
    recurrences of a fixed rho (s = 2, m = 3) are covered."""
    dt, steps = 0.05, 12
    ws = [make_workload(n, h=h) for n, h in WORKLOADS]
    out = []
    for t in (1536, tps):
        b = pkg.Batch()
        ids = [b.add_workload(w) for w in ws]
        ids.append(b.add_workload(ws[1], rho_every=pkg.RHO_FIXED, rho_F=1000.0, rho_S=60.0))
        b.set_occupancy(t)
        for _ in range(steps):
            b.step(dt)
        b.sync()
        assert b.stats()["threads_per_sm"] == t
        out.append([b.get_state(i) for i in ids])
        b.close()
    for x, y in zip(*out):
        np.testing.assert_array_equal(x, y)
    with pytest.raises(pkg.EmrkcError):
        b = pkg.Batch()
        try:
            b.set_occupancy(1000)
        finally:
            b.close()
