"""GPU parity of the comparison integrators of Sec. 5 (EXEX-RL, IMEX-RL,
Algorithm 4) against the FP64 oracle (oracle/reference.py).

The oracle solves the implicit diffusion system of IMEX-RL by a direct sparse
LU factorisation; the GPU solves it by Jacobi-preconditioned CG to a relative
residual of 1e-13 in the lumped-mass norm.  Tolerances as for emRKC: relative
L2 error in V <= 1e-10, other variables <= 1e-9 of their scale, activation
times <= 1e-8 ms.
"""

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from oracle.emrkc import Monodomain
from oracle.reference import RLRun
from workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _gpu_run(w, method, dt, steps, **kw):
    sol = pkg.Solver.from_workload(w, precision=pkg.PREC_FP64, method=method, **kw)
    for _ in range(steps):
        sol.step(dt)
    sol.sync()
    Y = sol.get_state()
    act = sol.activation_times()
    st = sol.stats()
    sol.close()
    return Y, act, st


def _compare(w, Y, act, ref, tol_v=1e-10):
    prob = ref.p
    err = prob.l2_norm(Y[0] - ref.Y[0]) / prob.l2_norm(ref.Y[0])
    assert err <= tol_v, f"rel L2 error in V {err:.3e}"
    for k in range(1, prob.N):
        scale = max(np.max(np.abs(ref.Y[k])), 1e-12)
        d = np.max(np.abs(Y[k] - ref.Y[k])) / scale
        assert d <= 1e-9, f"variable {k}: max rel diff {d:.3e}"
    assert np.array_equal(np.isnan(act), np.isnan(ref.act))
    fin = np.isfinite(ref.act)
    if fin.any():
        assert np.max(np.abs(act[fin] - ref.act[fin])) <= 1e-8
    return err


@pytest.mark.parametrize("name,kw,dt,steps", [
    ("square17x13_hh", {"h": 1.0 / 32}, 0.01, 300),
    ("slab21x9x5_ttp", {"h": 0.01}, 0.01, 200),
    ("line40_hh", {"length": 0.39}, 0.005, 400),
])
def test_exex_rl_parity(name, kw, dt, steps):
    w = make_workload(name, **kw)
    Y, act, st = _gpu_run(w, pkg.METHOD_EXEX_RL, dt, steps)
    ref = RLRun(Monodomain.from_workload(w), "exex", dt)
    for _ in range(steps):
        ref.step()
    _compare(w, Y, act, ref)
    assert st["s"] == 0 and st["m"] == 0 and st["steps"] == steps


@pytest.mark.parametrize("name,h,dt,steps", [
    ("square33x33_hh", 1.0 / 64, 0.05, 120),
    ("slab21x9x5_ttp", 0.01, 0.1, 60),
    ("slab17x7x5_hh", 0.02, 0.25, 40),
])
def test_imex_rl_parity(name, h, dt, steps):
    w = make_workload(name, h=h)
    Y, act, st = _gpu_run(w, pkg.METHOD_IMEX_RL, dt, steps, lin_rtol=1e-13, lin_max_iter=2000)
    ref = RLRun(Monodomain.from_workload(w), "imex", dt)
    for _ in range(steps):
        ref.step()
    _compare(w, Y, act, ref)
    assert st["lin_iters"] >= 1 and st["lin_residual"] <= 1e-13
    assert st["total_lin_iters"] >= steps


def test_imex_rl_iteration_cap_and_conservation():
    w = make_workload("square17x13_none", h=1.0 / 32, stim_amp=0.0)
    rng = np.random.default_rng(5)
    V0 = rng.normal(size=w.n)
    sol = pkg.Solver.from_workload(w, precision=pkg.PREC_FP64, method=pkg.METHOD_IMEX_RL, lin_rtol=1e-14,
                                   lin_max_iter=3)
    sol.set_state(V0, var=0)
    sol.step(0.5)
    sol.sync()
    st = sol.stats()
    assert st["lin_iters"] == 3 and st["lin_residual"] > 1e-14
    sol.close()
    # a converged implicit diffusion step conserves sum_i M_i V_i (1^T K = 0)
    sol = pkg.Solver.from_workload(w, precision=pkg.PREC_FP64, method=pkg.METHOD_IMEX_RL, lin_rtol=1e-14,
                                   lin_max_iter=5000)
    sol.set_state(V0, var=0)
    for _ in range(20):
        sol.step(0.5)
    sol.sync()
    V = sol.get_state(var=0)
    sol.close()
    M = Monodomain.from_workload(w).M
    assert abs(M @ V - M @ V0) <= 1e-11 * (np.abs(M) @ np.abs(V0))
    assert np.std(V) < 0.5 * np.std(V0)


def test_rl_methods_reject_mixed_precision():
    w = make_workload("square5x5_hh")
    for method in (pkg.METHOD_EXEX_RL, pkg.METHOD_IMEX_RL):
        with pytest.raises(pkg.EmrkcError) as ei:
            pkg.Solver.from_workload(w, precision=pkg.PREC_MIXED, method=method)
        assert ei.value.code == 1
