"""Robustness workloads of Sec. 5.1 and Sec. 5.4 on the GPU.

* Practical stability (Sec. 5.1): the 1-D TTP06 cable at dx = 0.025 mm.
  EXEX-RL is bounded only up to dt = 0.003 ms (dt rho_F <= 2, as in the
  paper).  emRKC with rho estimated once at rest is bounded up to dt = 1 ms;
  with the known bound rho(f_S) <= 7 1/ms it stays bounded to dt = 3 ms (the
  paper reports 4.5 ms).
* Fibrosis (Sec. 5.4): sigma_t = 0 on the cells where a seeded smooth random
  field exceeds its median; FP64 parity with the oracle and mixed vs FP64.
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


def _run(w, dt, T, **kw):
    sol = pkg.Solver.from_workload(w, **kw)
    steps = int(round(T / dt))
    for _ in range(steps):
        sol.step(dt)
    sol.sync()
    V = sol.get_state(var=0)
    st = sol.stats()
    sol.close()
    return V, st


@pytest.fixture(scope="module")
def cable_reference():
    w = make_workload("cable_ttp")
    V, _ = _run(w, 0.01, 100.0, precision=pkg.PREC_FP64, rho_every=0)
    return w, V


def _norm_ratio(w, V, Vref):
    M = Monodomain.from_workload(w).M
    return np.sqrt(M @ (V * V)) / np.sqrt(M @ (Vref * Vref))


@pytest.mark.parametrize("dt", [0.5, 1.0])
@pytest.mark.parametrize("prec", [pkg.PREC_FP64, pkg.PREC_MIXED])
def test_practical_stability_cable_rho_once(cable_reference, dt, prec):
    w, Vref = cable_reference
    V, st = _run(w, dt, 100.0, precision=prec, rho_every=0)
    assert np.all(np.isfinite(V))
    assert 0.95 <= _norm_ratio(w, V, Vref) <= 1.05
    assert st["m"] >= 2  # diffusion needs inner stages already at moderate dt (Sec. 5.1)


def test_rho_once_at_rest_is_unstable_at_2ms():
    """rho(f_S) estimated once at rest (0.2 1/ms) keeps s = 1; the explicit
    outer step then cannot follow the upstroke (rho(f_S) about 6.5 1/ms) at
    dt = 2 ms and the solution overflows (reported, not a device fault)."""
    w = make_workload("cable_ttp")
    with pytest.raises(pkg.EmrkcError) as ei:
        _run(w, 2.0, 100.0, precision=pkg.PREC_FP64, rho_every=0)
    assert ei.value.code == 4


@pytest.mark.parametrize("dt", [2.0, 3.0])
@pytest.mark.parametrize("prec", [pkg.PREC_FP64, pkg.PREC_MIXED])
def test_practical_stability_cable_known_rho_bound(cable_reference, dt, prec):
    """With the known bound rho(f_S) <= 7 1/ms over the action potential the
    outer iteration takes s >= 3 and the solution stays bounded."""
    w, Vref = cable_reference
    V, st = _run(w, dt, 100.0, precision=prec, rho_every=0, rho_S_min=7.0)
    assert np.all(np.isfinite(V))
    assert 0.9 <= _norm_ratio(w, V, Vref) <= 1.1
    assert st["s"] >= 3


def test_exex_rl_stability_limit_cable():
    w = make_workload("cable_ttp")
    # dt rho_F = 0.003 * 608 = 1.8 < 2: bounded
    V, _ = _run(w, 0.003, 6.0, precision=pkg.PREC_FP64, method=pkg.METHOD_EXEX_RL)
    assert np.all(np.isfinite(V)) and np.all(np.abs(V) < 200)
    # dt rho_F = 3.6: the highest diffusion mode grows by 2.6 per step and overflows
    with pytest.raises(pkg.EmrkcError) as ei:
        _run(w, 0.006, 12.0, precision=pkg.PREC_FP64, method=pkg.METHOD_EXEX_RL)
    assert ei.value.code == 4  # EMRKC_ERR_NONFINITE


def test_fibrosis_fp64_parity_many_stages():
    w = make_workload("fibslab13x7x5_ttp", h=0.01)
    fixed = (5000.0, 300.0)
    sol = pkg.Solver.from_workload(w, precision=pkg.PREC_FP64, rho_every=pkg.RHO_FIXED, rho_F=fixed[0],
                                   rho_S=fixed[1])
    prob = Monodomain.from_workload(w)
    ref = OracleRun(prob, fixed_rho=fixed)
    for _ in range(25):
        sol.step(0.1)
        ref.step(0.1)
    sol.sync()
    Y = sol.get_state()
    st = sol.stats()
    sol.close()
    assert st["s"] >= 3 and st["m"] >= 3
    err = prob.l2_norm(Y[0] - ref.Y[0]) / prob.l2_norm(ref.Y[0])
    assert err <= 1e-10
    for k in range(1, prob.N):
        scale = max(np.max(np.abs(ref.Y[k])), 1e-12)
        assert np.max(np.abs(Y[k] - ref.Y[k])) / scale <= 1e-9


def test_fibrosis_mixed_vs_fp64():
    w = make_workload("fibslab41x15x7_ttp", h=0.01)
    V64, _ = _run(w, 0.05, 15.0, precision=pkg.PREC_FP64, rho_every=0)
    V32, _ = _run(w, 0.05, 15.0, precision=pkg.PREC_MIXED, rho_every=0)
    M = Monodomain.from_workload(w).M
    err = np.sqrt(M @ (V32 - V64) ** 2) / np.sqrt(M @ (V64 * V64))
    assert err <= 1e-3
    assert np.max(V64) > 0.0  # the wave is under way
