"""The device-resident emRKC step against the host-driven step and the oracle.

Problems that one thread-block cluster holds (at most 4 nodes per thread)
take one launch per step: Algorithm 5 when the rho policy makes it due,
Algorithm 1 (stage counts and coefficients) from the estimates, and every
outer and inner stage of Algorithm 3, separated by cluster barriers, with no
host round trip (the default for mixed precision; EMRKC_FUSED_STEP=1 here
for FP64 too).  The same solver with EMRKC_FUSED_STEP=0 drives the step
from the host (a launch per phase, the stage counts read back after each
power iteration).  Both evaluate the same per-node arithmetic and the same
Algorithm 1 expressions; compiled into two kernels they may still round
differently in the last bit.  FP64 states agree to 1e-10 and mixed states
to 1e-6 (relative, every variable), the per-step stage counts are equal,
and the FP64 path matches the oracle to 1e-10.  Cases: both precisions, rho every step, every
third step, once and fixed; s = 1, 2, 3 and 5 (the three buffer routings)
and m = 1 to 5, with loads through L1 (s <= 2 and m = 1, s = 1 and m <= 3)
and through L2 (the other stage counts).
"""

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from oracle.emrkc import Monodomain, OracleRun
from workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _run(w, steps, monkeypatch, fused, **kw):
    monkeypatch.setenv("EMRKC_FUSED_STEP", "1" if fused else "0")
    sol = pkg.Solver.from_workload(w, **kw)
    log = []
    l0 = sol.stats()["launches"]
    for _ in range(steps):
        sol.step(w.dt)
        st = sol.stats()
        log.append((st["s"], st["m"], st["pow_iters_F"], st["pow_iters_S"]))
    launches = sol.stats()["launches"] - l0
    Y = sol.get_state()
    act = sol.activation_times()
    st = sol.stats()
    sol.close()
    monkeypatch.delenv("EMRKC_FUSED_STEP", raising=False)
    return Y, act, log, launches, st


def _close(Y, Yref, rel):
    for k in range(Y.shape[0]):
        scale = max(np.max(np.abs(Yref[k])), 1e-12)
        assert np.max(np.abs(Y[k] - Yref[k])) <= rel * scale, f"variable {k}"


CASES = [
    # name, h, precision, policy kwargs, expected (s, m) of the last step (None: not fixed)
    ("square33x29_hh", 1.0 / 64, pkg.PREC_FP64, dict(rho_every=1, rho_S_min=42.0), (2, 1)),
    ("square33x29_hh", 1.0 / 64, pkg.PREC_MIXED, dict(rho_every=1, rho_S_min=42.0), (2, 1)),
    ("slab23x9x5_ttp", 0.01, pkg.PREC_MIXED, dict(rho_every=pkg.RHO_ONCE), (1, 2)),
    ("slab23x9x5_ttp", 0.01, pkg.PREC_FP64, dict(rho_every=3), None),
    ("slab23x9x5_ttp", 0.01, pkg.PREC_FP64, dict(rho_every=pkg.RHO_FIXED, rho_F=7000.0, rho_S=300.0), (3, 5)),
    ("slab23x9x5_ttp", 0.01, pkg.PREC_MIXED, dict(rho_every=pkg.RHO_FIXED, rho_F=7000.0, rho_S=300.0), (3, 5)),
    ("square33x29_hh", 1.0 / 64, pkg.PREC_FP64, dict(rho_every=pkg.RHO_FIXED, rho_F=12000.0, rho_S=800.0), (5, 4)),
    ("square33x29_hh", 1.0 / 64, pkg.PREC_MIXED, dict(rho_every=pkg.RHO_FIXED, rho_F=12000.0, rho_S=800.0), (5, 4)),
    # L1 loads with inner stages (s = 1, m = 3); L2 loads for s = 2, m = 2
    ("slab23x9x5_ttp", 0.01, pkg.PREC_MIXED, dict(rho_every=pkg.RHO_FIXED, rho_F=250.0, rho_S=10.0), (1, 3)),
    ("slab23x9x5_ttp", 0.01, pkg.PREC_MIXED, dict(rho_every=pkg.RHO_FIXED, rho_F=400.0, rho_S=60.0), (2, 2)),
]


@pytest.mark.parametrize("name,h,prec,kw,sm", CASES)
def test_fused_step_equals_host_driven_step(monkeypatch, name, h, prec, kw, sm):
    w = make_workload(name, h=h)
    steps = 30
    Yf, actf, logf, lf, stf = _run(w, steps, monkeypatch, True, precision=prec, **kw)
    Yh, acth, logh, lh, sth = _run(w, steps, monkeypatch, False, precision=prec, **kw)
    assert lf == steps  # one launch per step
    assert lh > steps
    # the same stage counts every step; the power iteration's iteration
    # counts may differ: the same per-node code compiled into two kernels can
    # round differently in the last bit, and the FP64 differences
    # f(y + q v) - f(y) of Algorithm 5 amplify that in the stopping test
    assert [l[:2] for l in logf] == [l[:2] for l in logh]
    if sm is not None:
        assert (stf["s"], stf["m"]) == sm
    assert stf["rho_F"] == pytest.approx(sth["rho_F"], rel=1e-9 if prec == pkg.PREC_FP64 else 1e-6)
    # FP64: the oracle parity bar (the upstroke amplifies the last-bit
    # differences over the 30 steps to about 1e-11)
    _close(Yf, Yh, 1e-10 if prec == pkg.PREC_FP64 else 1e-6)
    fin = np.isfinite(acth)
    assert np.array_equal(np.isfinite(actf), fin)
    if fin.any():
        assert np.max(np.abs(actf[fin] - acth[fin])) <= (1e-8 if prec == pkg.PREC_FP64 else 1e-3)


@pytest.mark.parametrize("name,h,kw", [("square33x29_hh", 1.0 / 64, dict(rho_every=1, rho_S_min=42.0)),
                                       ("slab23x9x5_ttp", 0.01, dict(rho_every=2))])
def test_fused_step_fp64_matches_oracle(monkeypatch, name, h, kw):
    w = make_workload(name, h=h)
    steps = 40
    Y, act, log, launches, _ = _run(w, steps, monkeypatch, True, precision=pkg.PREC_FP64, **kw)
    assert launches == steps
    prob = Monodomain.from_workload(w)
    ref = OracleRun(prob, **kw)
    for _ in range(steps):
        ref.step(w.dt)
    assert [(s, m) for s, m, _, _ in log] == [(l[0], l[1]) for l in ref.log]
    err = prob.l2_norm(Y[0] - ref.Y[0]) / prob.l2_norm(ref.Y[0])
    assert err <= 1e-10
    for k in range(1, Y.shape[0]):
        scale = max(np.max(np.abs(ref.Y[k])), 1e-12)
        assert np.max(np.abs(Y[k] - ref.Y[k])) <= 1e-9 * scale
    fin = np.isfinite(ref.act)
    assert np.array_equal(np.isfinite(act), fin)
    if fin.any():
        assert np.max(np.abs(act[fin] - ref.act[fin])) <= 1e-8


def test_fused_step_then_host_estimate_and_back(monkeypatch):
    """An explicit estimate between device-resident steps (emrkc_estimate_rho)
    continues from the device's last iterate: it converges in a few warm
    iterations, and the following steps equal those of a host-driven solver
    that made the same calls."""
    w = make_workload("slab23x9x5_ttp", h=0.01)
    out = {}
    for fused in (True, False):
        monkeypatch.setenv("EMRKC_FUSED_STEP", "1" if fused else "0")
        sol = pkg.Solver.from_workload(w, precision=pkg.PREC_FP64, rho_every=2)
        for _ in range(5):
            sol.step(w.dt)
        r = sol.estimate_rho()
        for _ in range(5):
            sol.step(w.dt)
        out[fused] = (r, sol.get_state(), sol.stats()["total_pow_iters"])
        sol.close()
    monkeypatch.delenv("EMRKC_FUSED_STEP", raising=False)
    (rf, Yf, itf), (rh, Yh, ith) = out[True], out[False]
    assert rf[2] <= 3 and rf[3] <= 3  # warm
    assert rf[0] == pytest.approx(rh[0], rel=1e-9) and rf[1] == pytest.approx(rh[1], rel=1e-6)
    _close(Yf, Yh, 1e-10)
