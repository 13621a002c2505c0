"""Pipelined host I/O: emrkc_set_stimulus_async / emrkc_get_state_async.

The asynchronous calls must give exactly what the synchronous ones give: the
same kernels run in the same order on the solver's stream, only the copies
move to a second stream ordered by events.  Checked bit for bit against a
twin solver driven through emrkc_set_stimulus / emrkc_get_state, with two
host buffers in rotation and a stimulus that changes between steps.
"""

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _masks(w):
    m0 = np.ascontiguousarray(w.stim_mask, dtype=np.uint8)
    m1 = np.zeros(w.n, dtype=np.uint8)
    m1[w.n // 2: w.n // 2 + 64] = 1  # a second site in the middle of the node range
    return m0, m1


@pytest.mark.parametrize("prec", [pkg.PREC_MIXED, pkg.PREC_FP64])
def test_async_matches_sync(prec):
    w = make_workload("slab41x15x7_ttp")
    m0, m1 = _masks(w)
    a = pkg.Solver.from_workload(w, precision=prec, rho_every=0)
    b = pkg.Solver.from_workload(w, precision=prec, rho_every=0)
    ring = [np.empty(w.n), np.empty(w.n)]
    gates = [np.empty(w.n), np.empty(w.n)]
    for k in range(24):
        mask = m0 if (k // 5) % 2 == 0 else m1
        a.set_stimulus_async(mask, 50.0, 0.0, 0.6 + 0.05 * k)
        b.set_stimulus(mask, 50.0, 0.0, 0.6 + 0.05 * k)
        a.step(w.dt)
        b.step(w.dt)
        a.get_state_async(0, ring[k % 2])
        a.get_state_async(5, gates[k % 2])
        if k % 2 == 1:
            a.sync()
            Vb = b.get_state(var=0)
            gb = b.get_state(var=5)
            assert np.array_equal(ring[k % 2], Vb)
            assert np.array_equal(gates[k % 2], gb)
    a.sync()
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(a.activation_times(), b.activation_times(), equal_nan=True)
    a.close()
    b.close()


def test_async_every_step_values():
    # each of two rotating buffers holds the V of its own step
    w = make_workload("slab41x15x7_ttp")
    a = pkg.Solver.from_workload(w, precision=pkg.PREC_MIXED, rho_every=0)
    b = pkg.Solver.from_workload(w, precision=pkg.PREC_MIXED, rho_every=0)
    ring = [np.empty(w.n), np.empty(w.n)]
    ref = []
    for k in range(2):
        a.step(w.dt)
        a.get_state_async(0, ring[k])
        b.step(w.dt)
        ref.append(b.get_state(var=0))
    a.sync()
    assert np.array_equal(ring[0], ref[0])
    assert np.array_equal(ring[1], ref[1])
    assert not np.array_equal(ring[0], ring[1])
    a.close()
    b.close()


def test_async_argument_errors():
    w = make_workload("slab41x15x7_ttp")
    a = pkg.Solver.from_workload(w, precision=pkg.PREC_MIXED, rho_every=0)
    buf = np.empty(w.n)
    with pytest.raises(pkg.EmrkcError):
        a.get_state_async(-1, buf)  # whole state is not offered asynchronously
    with pytest.raises(pkg.EmrkcError):
        a.get_state_async(a.N, buf)
    with pytest.raises(ValueError):
        a.get_state_async(0, np.empty(w.n - 1))
    with pytest.raises(ValueError):
        a.set_stimulus_async(np.zeros(w.n, dtype=np.int32))
    a.sync()
    a.close()
