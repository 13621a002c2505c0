"""Rounding sensitivity of the literal emRKC step for HH on the 65 x 65 square.

With dt = 0.05 ms the outer stage count s comes from rho_S alone, m = 1,
and rho_F ~ 25 is comparable to rho_S ~ 40, outside hypothesis B of Lemma
4.2 (rho_F >> rho_S).  The step then oscillates after the upstroke and
amplifies perturbations at the level of one rounding error: this test shows
it on the oracle itself, which is why GPU/oracle parity for this workload is
checked before the instability and at a stable dt (tests/test_gpu_parity.py).
"""

import numpy as np

from oracle.emrkc import Monodomain, OracleRun
from workloads import make_workload


def _divergence(prob, dt, steps):
    a = OracleRun(prob, rho_every=1)
    b = OracleRun(prob, rho_every=1)
    b.Y[0] *= 1.0 + 1e-15
    for _ in range(steps):
        a.step(dt)
        b.step(dt)
    return prob.l2_norm(a.Y[0] - b.Y[0]) / prob.l2_norm(a.Y[0]), a


def test_hh_square65_dt005_amplifies_rounding():
    w = make_workload("square65_hh")
    prob = Monodomain.from_workload(w)
    d35, _ = _divergence(prob, 0.05, 35)
    assert d35 < 1e-13  # before the instability: rounding level
    d200, a = _divergence(prob, 0.05, 200)
    assert d200 > 1e-8  # a 1e-15 perturbation has grown by > 7 orders
    assert a.Y[0].max() > 60.0  # V overshoots E_Na = 40 mV: the unstable regime


def test_hh_square65_dt002_is_stable():
    w = make_workload("square65_hh")
    prob = Monodomain.from_workload(w)
    d, a = _divergence(prob, 0.02, 400)
    assert d < 1e-13
    assert a.Y[0].max() < 45.0
