"""First-order damped Runge-Kutta-Chebyshev method (Algorithm 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""

from __future__ import annotations

import math

import numpy as np

EPS_DAMP = 0.05  # damping epsilon of Algorithm 1 (Sec. 3.1)


def get_stages(dt, rho, eps=EPS_DAMP):
    """s = ceil(sqrt(dt rho / beta)), beta = 2 - 4 eps / 3, l_s = beta s^2.

    Reading: s is at least 1 (the printed formula gives 0 when rho = 0).
    """
    beta = 2.0 - 4.0 * eps / 3.0
    s = int(math.ceil(math.sqrt(dt * rho / beta)))
    s = max(1, s)
    return s, beta * s * s


def chebyshev_T(j, x):
    """T_0..T_j at x and T_0'..T_j' at x by the three-term recurrences."""
    T = np.zeros(j + 1)
    dT = np.zeros(j + 1)
    T[0] = 1.0
    dT[0] = 0.0
    if j >= 1:
        T[1] = x
        dT[1] = 1.0
    for k in range(1, j):
        T[k + 1] = 2.0 * x * T[k] - T[k - 1]
        dT[k + 1] = 2.0 * T[k] + 2.0 * x * dT[k] - dT[k - 1]
    return T, dT


def get_coeffs(s, eps=EPS_DAMP):
    """mu_j, nu_j, kappa_j (j = 1..s, index 0 unused) and c_j (j = 0..s).

    omega_0 = 1 + eps/s^2, omega_1 = T_s(omega_0)/T_s'(omega_0),
    b_j = 1/T_j(omega_0), mu_1 = omega_1/omega_0, c_1 = mu_1, and for j >= 2
    mu_j = 2 omega_1 b_j/b_{j-1}, nu_j = 2 omega_0 b_j/b_{j-1},
    kappa_j = -b_j/b_{j-2}, c_j = nu_j c_{j-1} + kappa_j c_{j-2} + mu_j.
    """
    w0 = 1.0 + eps / (s * s)
    T, dT = chebyshev_T(s, w0)
    w1 = T[s] / dT[s]
    b = 1.0 / T
    mu = np.zeros(s + 1)
    nu = np.zeros(s + 1)
    kappa = np.zeros(s + 1)
    c = np.zeros(s + 1)
    mu[1] = w1 / w0
    c[1] = mu[1]
    for j in range(2, s + 1):
        mu[j] = 2.0 * w1 * b[j] / b[j - 1]
        nu[j] = 2.0 * w0 * b[j] / b[j - 1]
        kappa[j] = -b[j] / b[j - 2]
        c[j] = nu[j] * c[j - 1] + kappa[j] * c[j - 2] + mu[j]
    return mu, nu, kappa, c, w0, w1


def rkc_iteration(t, y, dt, f, s, eps=EPS_DAMP):
    """g_0 = y, g_1 = g_0 + mu_1 dt f(t, g_0),
    g_j = nu_j g_{j-1} + kappa_j g_{j-2} + mu_j dt f(t + c_{j-1} dt, g_{j-1})."""
    mu, nu, kappa, c, _, _ = get_coeffs(s, eps)
    g_prev2 = y
    g_prev = y + mu[1] * dt * f(t, y)
    for j in range(2, s + 1):
        g = nu[j] * g_prev + kappa[j] * g_prev2 + mu[j] * dt * f(t + c[j - 1] * dt, g_prev)
        g_prev2, g_prev = g_prev, g
    return g_prev
