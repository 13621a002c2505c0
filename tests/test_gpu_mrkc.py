"""GPU parity of mRKC (Algorithm 2 with the stiffest-gate split of Sec. 3.3)
against the FP64 oracle: relative L2 error in V <= 1e-10, other variables
<= 1e-9 of their scale, activation times <= 1e-8 ms, identical (s, m) per
step."""

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from oracle.emrkc import Monodomain, OracleRun
from workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _pair(w, dt, steps, Y0=None, **kw):
    rho_every = kw.pop("rho_every", 1)
    fixed = kw.pop("fixed", None)
    opts = dict(precision=pkg.PREC_FP64, method=pkg.METHOD_MRKC, rho_every=rho_every)
    if fixed is not None:
        opts.update(rho_every=pkg.RHO_FIXED, rho_F=fixed[0], rho_S=fixed[1])
    sol = pkg.Solver.from_workload(w, **opts)
    if Y0 is not None:
        sol.set_state(Y0)
    prob = Monodomain.from_workload(w)
    ref = OracleRun(prob, Y0=Y0, rho_every=rho_every if fixed is None else 1, fixed_rho=fixed, method="mrkc")
    log = []
    for _ in range(steps):
        sol.step(dt)
        ref.step(dt)
        st = sol.stats()
        log.append((st["s"], st["m"]))
    sol.sync()
    Y = sol.get_state()
    act = sol.activation_times()
    st = sol.stats()
    sol.close()
    assert log == [(l[0], l[1]) for l in ref.log]
    err = prob.l2_norm(Y[0] - ref.Y[0]) / prob.l2_norm(ref.Y[0])
    assert err <= 1e-10, f"rel L2 error in V {err:.3e}"
    for k in range(1, prob.N):
        scale = max(np.max(np.abs(ref.Y[k])), 1e-12)
        d = np.max(np.abs(Y[k] - ref.Y[k])) / scale
        assert d <= 1e-9, f"variable {k}: max rel diff {d:.3e}"
    assert np.array_equal(np.isnan(act), np.isnan(ref.act))
    fin = np.isfinite(ref.act)
    if fin.any():
        assert np.max(np.abs(act[fin] - ref.act[fin])) <= 1e-8
    return st, ref, log


@pytest.mark.parametrize("fixed", [(5000.0, 300.0), (900.0, 40.0)])
def test_mrkc_parity_fixed_rho_many_stages(fixed):
    w = make_workload("slab13x7x5_ttp", h=0.01)
    st, ref, log = _pair(w, 0.1, 25, fixed=fixed)
    if fixed[0] > 1000:
        assert st["s"] >= 3 and st["m"] >= 3


def test_mrkc_parity_rho_every_step_hh():
    w = make_workload("square17x13_hh", h=1.0 / 32)
    st, ref, log = _pair(w, 0.02, 120, rho_every=1)
    assert np.isfinite(ref.act).any()
    # rho~_F includes the fast m gate: above rho(L) = 8 sigma / (h^2 chi Cm)
    assert st["rho_F"] > 1.05 * 8.0 / ((1.0 / 32) ** 2 * 1400.0)


def test_mrkc_parity_rho_once_ttp():
    w = make_workload("slab21x9x5_ttp", h=0.01)
    st, ref, log = _pair(w, 0.05, 60, rho_every=0)
    # the estimates of Algorithm 5 agree to rounding amplified by the iteration
    assert abs(st["rho_F"] - ref.log[-1][2]) <= 1e-8 * ref.log[-1][2]
    assert abs(st["rho_S"] - ref.log[-1][3]) <= 1e-8 * ref.log[-1][3]


def test_mrkc_parity_passive_eigenvector():
    w = make_workload("line30_passive", length=0.29, stim_amp=0.0)
    x = w.coords[:, 0]
    Y0 = np.empty((3, w.n))
    Y0[0] = np.cos(4 * np.pi * x / 0.29)
    Y0[1] = 0.9
    Y0[2] = -0.5
    _pair(w, 0.3, 10, Y0=Y0, fixed=(3000.0, 50.0))


def test_mrkc_equals_emrkc_without_ionic_model():
    w = make_workload("square17x13_none", h=1.0 / 32, stim_amp=0.0)
    rng = np.random.default_rng(7)
    V0 = rng.normal(size=w.n)
    out = []
    for method in (pkg.METHOD_EMRKC, pkg.METHOD_MRKC):
        sol = pkg.Solver.from_workload(w, precision=pkg.PREC_FP64, method=method, rho_every=pkg.RHO_FIXED,
                                       rho_F=500.0, rho_S=3.0)
        sol.set_state(V0, var=0)
        for _ in range(20):
            sol.step(0.2)
        sol.sync()
        out.append(sol.get_state(var=0))
        sol.close()
    np.testing.assert_allclose(out[0], out[1], rtol=0, atol=1e-13 * np.max(np.abs(V0)))
