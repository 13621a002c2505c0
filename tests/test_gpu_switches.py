"""The launch-shape switches of the mixed path give the same results.

`EMRKC_NO_TMA=1` selects the register-loaded stage kernel instead of the
persistent bulk-copy one; by default the bulk-copy kernel prefetches the next
tile into one state region and a second ELL buffer, `EMRKC_TMA_NBUF=1` or `2`
give it one or two whole-tile stage buffers instead, `EMRKC_TMA_ELL=0` has it read the ELL
rows from global memory instead of staging them; `EMRKC_NO_PDL=1` drops
programmatic dependent launch.  All are read at solver creation.  The
per-node arithmetic of the stage (Rush-Larsen step, ionic currents, first
inner stage, Algorithm 3) is the same in every variant, so V after a wave has started must agree to FP32
rounding, and each variant must match the FP64 oracle within the mixed
tolerance.
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


def _run(w, steps):
    sol = pkg.Solver.from_workload(w, precision=pkg.PREC_MIXED, rho_every=0)
    for _ in range(steps):
        sol.step(w.dt)
    sol.sync()
    V = sol.get_state(var=0)
    st = sol.stats()
    sol.close()
    return V, st


@pytest.fixture(scope="module")
def case():
    # 41 x 15 x 7 slab: 4,305 nodes (33 full 128-node tiles and a ragged tail);
    # after 2 ms about half of it is activated.
    w = make_workload("slab41x15x7_ttp")
    steps = 40
    orc = OracleRun(Monodomain.from_workload(w), rho_every=0)
    for _ in range(steps):
        orc.step(w.dt)
    return w, steps, orc.Y[0].copy()


@pytest.mark.parametrize("env", [{}, {"EMRKC_NO_TMA": "1"}, {"EMRKC_NO_PDL": "1"},
                                 {"EMRKC_NO_TMA": "1", "EMRKC_NO_PDL": "1"},
                                 {"EMRKC_TMA_NBUF": "1"}, {"EMRKC_TMA_NBUF": "2"}, {"EMRKC_TMA_ELL": "0"},
                                 {"EMRKC_TMA_NBUF": "2", "EMRKC_TMA_ELL": "0"}])
def test_switches_same_result(case, monkeypatch, env):
    w, steps, Vo = case
    V0, st0 = _run(w, steps)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    V1, st1 = _run(w, steps)
    assert (st1["s"], st1["m"]) == (st0["s"], st0["m"])
    assert np.linalg.norm(V1 - V0) <= 1e-6 * np.linalg.norm(V0)
    assert np.linalg.norm(V1 - Vo) <= 1e-3 * np.linalg.norm(Vo)


@pytest.mark.parametrize("prec", [pkg.PREC_MIXED, pkg.PREC_FP64])
def test_power_iteration_cluster_matches_grid(monkeypatch, prec):
    """Problems of at most 16k nodes run Algorithm 5 in one thread-block
    cluster (hardware cluster barrier); EMRKC_NO_CLUSTER=1 forces the
    cooperative grid.  The two differ only in how partial sums are grouped."""
    w = make_workload("slab41x15x7_ttp")
    out = []
    for env in ({}, {"EMRKC_NO_CLUSTER": "1"}):
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        sol = pkg.Solver.from_workload(w, precision=prec, rho_every=1, seed=5)
        for _ in range(10):
            sol.step(w.dt)
        rF, rS, itF, itS = sol.estimate_rho()
        V = sol.get_state(var=0)
        sol.close()
        out.append((rF, rS, itF, itS, V))
    (a, b) = out
    # FP64 path: FP64 sums, grouping changes the last bits; mixed path: FP32
    # per-thread and per-CTA sums, grouping changes ~1e-7 of each sum
    tol = 1e-9 if prec == pkg.PREC_FP64 else 1e-4
    assert abs(a[2] - b[2]) <= 1 and abs(a[3] - b[3]) <= 1
    assert a[0] == pytest.approx(b[0], rel=tol)
    assert a[1] == pytest.approx(b[1], rel=tol)
    assert np.linalg.norm(a[4] - b[4]) <= 1e-12 * np.linalg.norm(b[4])


def test_wide_rows_fall_back_to_unstaged_stage_kernel(monkeypatch):
    """Rows wider than the staging width (the jittered shell has up to ~27
    entries per row) cannot use the prefetching kernel; the bulk-copy kernel
    then runs with one stage buffer and the rows read from global memory.
    Every launch shape must agree with the others and with the FP64 path."""
    from paper_2401_01745_gb300 import assemble_p1
    w = make_workload("shell_ttp", nr=6, nuv=24)
    w.stim_amp = 100.0
    rp, col, K, M = assemble_p1(w.coords, w.cells, w.D)
    assert np.max(np.diff(rp)) > 9  # diagonal + more than 8 off-diagonal entries
    steps = 40
    out = {}
    for name, env in (("default", {}), ("one_buffer", {"EMRKC_TMA_NBUF": "1"}), ("no_tma", {"EMRKC_NO_TMA": "1"})):
        for k in ("EMRKC_TMA_NBUF", "EMRKC_NO_TMA"):
            monkeypatch.delenv(k, raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        out[name] = _run(w, steps)[0]
    monkeypatch.delenv("EMRKC_TMA_NBUF", raising=False)
    monkeypatch.delenv("EMRKC_NO_TMA", raising=False)
    sol = pkg.Solver.from_workload(w, precision=pkg.PREC_FP64, rho_every=0)
    for _ in range(steps):
        sol.step(w.dt)
    sol.sync()
    V64 = sol.get_state(var=0)
    sol.close()
    for name in ("one_buffer", "no_tma"):
        assert np.linalg.norm(out[name] - out["default"]) <= 1e-6 * np.linalg.norm(out["default"])
    assert np.linalg.norm(out["default"] - V64) <= 1e-3 * np.linalg.norm(V64)
