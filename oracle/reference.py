"""Reference integrators for the same semi-discrete system (float64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  rk4_run      classical RK4 on y' = f_F + f_S + f_E (monolithic); a brute-
               force fine-step reference for convergence tests, in the role
               of the paper's small-step reference solution (Sec. 5).
  imex_rl_step IMEX Rush-Larsen step (Algorithm 4): exponential Euler for
               z_E, explicit Euler for z_S, implicit in the diffusion.
  exex_rl_step the same with the V update done explicitly (EXEX-RL, Sec. 5).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def full_rhs(prob, t, Y):
    return prob.f_F(t, Y) + prob.f_S(t, Y) + prob.f_E(t, Y)


def rk4_run(prob, Y0, T, dt):
    n_steps = int(round(T / dt))
    Y = np.array(Y0, dtype=np.float64)
    t = 0.0
    for _ in range(n_steps):
        k1 = full_rhs(prob, t, Y)
        k2 = full_rhs(prob, t + 0.5 * dt, Y + 0.5 * dt * k1)
        k3 = full_rhs(prob, t + 0.5 * dt, Y + 0.5 * dt * k2)
        k4 = full_rhs(prob, t + dt, Y + dt * k3)
        Y = Y + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        t += dt
    return Y


def _ionic_split_update(prob, t, Y, dt):
    V, zE, zS = prob.parts(Y)
    out = Y.copy()
    if prob.nE:
        lam, zinf = prob.model.gating(V, zE, zS)
        out[1:1 + prob.nE] = zE + np.expm1(dt * lam) * (zE - zinf)
    if prob.nS:
        out[1 + prob.nE:] = zS + dt * prob.model.g_S(V, out[1:1 + prob.nE], zS)
    return out


def exex_rl_step(prob, t, Y, dt):
    out = _ionic_split_update(prob, t, Y, dt)
    V = Y[0]
    _, zE1, zS1 = prob.parts(out)
    I_ion = prob.model.I_ion(V, zE1, zS1)
    out[0] = V + dt * (prob.diffusion(V) + (prob.I_stim(t) - I_ion) / prob.Cm)
    return out


class ImexRL:
    """IMEX-RL with a direct sparse solve of (Cm M + dt/chi K) V = rhs."""

    def __init__(self, prob, dt):
        self.prob = prob
        self.dt = dt
        A = sp.diags(prob.Cm * prob.M) + (dt / prob.chi) * prob.K
        self.lu = spla.splu(A.tocsc())

    def step(self, t, Y):
        p = self.prob
        dt = self.dt
        out = _ionic_split_update(p, t, Y, dt)
        V = Y[0]
        _, zE1, zS1 = p.parts(out)
        I_ion = p.model.I_ion(V, zE1, zS1)
        rhs = p.Cm * p.M * V + dt * p.M * (p.I_stim(t) - I_ion)
        out[0] = self.lu.solve(rhs)
        return out


class RLRun:
    """Time-stepping driver for EXEX-RL / IMEX-RL (Sec. 5, Algorithm 4) with
    activation times: first upward crossing of the threshold, linearly
    interpolated within the step (the same definition as OracleRun)."""

    def __init__(self, prob, method, dt, act_threshold=-20.0):
        if method not in ("exex", "imex"):
            raise ValueError("method must be 'exex' or 'imex'")
        self.p = prob
        self.method = method
        self.dt = dt
        self.imex = ImexRL(prob, dt) if method == "imex" else None
        self.Y = prob.initial_state()
        self.t = 0.0
        self.steps = 0
        self.th = act_threshold
        self.act = np.full(prob.n, np.nan)

    def step(self):
        V_old = self.Y[0].copy()
        if self.method == "imex":
            Y = self.imex.step(self.t, self.Y)
        else:
            Y = exex_rl_step(self.p, self.t, self.Y, self.dt)
        V_new = Y[0]
        cross = np.isnan(self.act) & (V_old < self.th) & (V_new >= self.th)
        if np.any(cross):
            self.act[cross] = self.t + self.dt * (self.th - V_old[cross]) / (V_new[cross] - V_old[cross])
        self.Y = Y
        self.t += self.dt
        self.steps += 1
        return Y
