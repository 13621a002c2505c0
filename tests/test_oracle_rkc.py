"""Pins of the oracle's RKC coefficients and recurrence (Algorithm 1, Sec. 3.1, 4.5).

Each check compares the oracle with an independent fact: Chebyshev
polynomials evaluated by numpy / scipy library routines, or identities the
paper states (nu_j + kappa_j = 1 and the b_s/b_j U_{s-j} sum in Sec. 4.5).
"""

import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as C
from scipy.special import eval_chebyu

from oracle.rkc import EPS_DAMP, get_coeffs, get_stages, rkc_iteration

BETA = 2.0 - 4.0 * EPS_DAMP / 3.0


def cheb_T(s, x):
    return C.chebval(x, [0] * s + [1])


def cheb_dT(s, x):
    return C.chebval(x, C.chebder([0] * s + [1]))


@pytest.mark.parametrize("s", [1, 2, 3, 5, 8, 13, 40, 200])
def test_c_s_equals_one(s):
    mu, nu, kappa, c, w0, w1 = get_coeffs(s)
    assert abs(c[s] - 1.0) <= 1e-13


@pytest.mark.parametrize("s", [2, 3, 7, 50])
def test_nu_plus_kappa_is_one(s):
    # Sec. 4.5: nu_j + kappa_j = 1
    mu, nu, kappa, c, w0, w1 = get_coeffs(s)
    for j in range(2, s + 1):
        assert abs(nu[j] + kappa[j] - 1.0) <= 1e-14


@pytest.mark.parametrize("s", [1, 2, 4, 9, 30])
def test_omega_definitions_against_numpy(s):
    mu, nu, kappa, c, w0, w1 = get_coeffs(s)
    assert w0 == pytest.approx(1.0 + EPS_DAMP / s ** 2, rel=1e-15)
    assert w1 == pytest.approx(cheb_T(s, w0) / cheb_dT(s, w0), rel=1e-12)
    assert mu[1] == pytest.approx(w1 / w0, rel=1e-14)


@pytest.mark.parametrize("s", [1, 2, 3, 6, 11, 25])
def test_sum_identity_sec45(s):
    # sum_j (b_s / b_j) U_{s-j}(omega_0) mu_j = 1, b_j = 1/T_j(omega_0)
    mu, nu, kappa, c, w0, w1 = get_coeffs(s)
    b = np.array([1.0 / cheb_T(j, w0) for j in range(s + 1)])
    total = sum(b[s] / b[j] * eval_chebyu(s - j, w0) * mu[j] for j in range(1, s + 1))
    assert total == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("s", [1, 2, 3, 5, 10, 20])
def test_recurrence_equals_chebyshev_stability_polynomial(s):
    # Applied to y' = lambda y, one RKC iteration multiplies y by
    # R_s(z) = T_s(w0 + w1 z) / T_s(w0) with z = dt lambda (Sec. 3.1).
    mu, nu, kappa, c, w0, w1 = get_coeffs(s)
    zs = np.linspace(-BETA * s * s, 0.0, 37)
    for z in zs:
        out = rkc_iteration(0.0, np.array([1.0]), 1.0, lambda t, y: z * y, s)[0]
        ref = cheb_T(s, w0 + w1 * z) / cheb_T(s, w0)
        assert out == pytest.approx(ref, abs=1e-12)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 8, 16, 32])
def test_stability_interval(s):
    # |R_s(z)| <= 1 on [-beta s^2, 0] (Sec. 3.1).
    mu, nu, kappa, c, w0, w1 = get_coeffs(s)
    zs = np.linspace(-BETA * s * s, 0.0, 4001)
    R = cheb_T(s, w0 + w1 * zs) / cheb_T(s, w0)
    assert np.max(np.abs(R)) <= 1.0 + 1e-12
    # and the damping keeps it below 1 - eps/ something away from 0: |R| <= 1/T_s(w0)
    inner = zs[zs <= -(w0 - 1.0) / w1 - 1e-9]
    R_in = cheb_T(s, w0 + w1 * inner) / cheb_T(s, w0)
    assert np.max(np.abs(R_in)) <= 1.0 / cheb_T(s, w0) + 1e-12


def test_stage_times_are_chebyshev_ratios():
    # c_j = T_s(w0) T_j'(w0) / (T_s'(w0) T_j(w0)): the internal stage times
    s = 9
    mu, nu, kappa, c, w0, w1 = get_coeffs(s)
    for j in range(1, s + 1):
        ref = cheb_T(s, w0) * cheb_dT(j, w0) / (cheb_dT(s, w0) * cheb_T(j, w0))
        assert c[j] == pytest.approx(ref, rel=1e-12)


def test_get_stages_is_smallest_stable_count():
    # s is the smallest positive integer with beta s^2 >= dt rho (Algorithm 1)
    rng = np.random.default_rng(7)
    for _ in range(2000):
        dt = 10 ** rng.uniform(-4, 1)
        rho = 10 ** rng.uniform(-2, 4)
        s, ls = get_stages(dt, rho)
        assert s >= 1
        assert ls == pytest.approx(BETA * s * s)
        assert BETA * s * s >= dt * rho * (1 - 1e-12)
        if s > 1:
            assert BETA * (s - 1) ** 2 < dt * rho
    assert get_stages(0.05, 0.0) == (1, BETA)


def test_first_order_on_scalar_problem():
    # error of one RKC step on y' = -y is O(dt^2) (first order method)
    errs = []
    for dt in [0.1, 0.05, 0.025]:
        y = rkc_iteration(0.0, np.array([1.0]), dt, lambda t, y: -y, 4)[0]
        errs.append(abs(y - math.exp(-dt)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8)
