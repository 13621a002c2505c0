"""The emRKC time step for the P1 monodomain system (Algorithm 3), float64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The state is a (N, n) array: row 0 is V, rows 1..nE the gating variables
z_E, the remaining rows z_S.  The split follows Eq. (mono_in_FSE):
  f_F(y) = ((chi Cm M)^-1 A V, 0, 0)          with A = -K (reading of Sec. 2.1)
  f_S(t, y) = (Cm^-1 (I_stim(t) - I_ion(y)), 0, g_S(y))
  f_E(y) = (0, Lambda_E (z_E - z_inf), 0)
Algorithm 3 is followed literally, including the inner RKC iteration over
the full state (no closed form for the constant z-components).  mRKC
(Algorithm 2) with the stiffest-gate split of Sec. 3.3 is here too.
"""

from __future__ import annotations

import numpy as np

from .fem import assemble_p1
from .ionic import make_model
from .power import compute_rho, start_vector
from .rkc import EPS_DAMP, get_stages, rkc_iteration

SAFETY = 1.05  # safety factor on power-iteration estimates (App. A)


class Monodomain:
    """Semi-discrete monodomain system (Eq. sd_sys) with lumped mass."""

    def __init__(self, K, M, chi, Cm, model, stim_mask, stim_amp=50.0, t_on=0.0, t_off=1.0):
        self.K = K.tocsr()
        self.M = np.asarray(M, dtype=np.float64)
        self.chi = float(chi)
        self.Cm = float(Cm)
        self.model = model
        self.nE = model.nE
        self.nS = model.nS
        self.N = 1 + model.nE + model.nS
        self.n = self.M.size
        self.stim_mask = np.asarray(stim_mask, dtype=np.float64)
        self.stim_amp = float(stim_amp)
        self.t_on = float(t_on)
        self.t_off = float(t_off)

    @classmethod
    def from_workload(cls, w):
        K, M = assemble_p1(w.coords, w.cells, w.D)
        return cls(K, M, w.chi, w.Cm, make_model(w.model), w.stim_mask, w.stim_amp, w.t_on, w.t_off)

    # -- pieces of the state ------------------------------------------------
    def parts(self, Y):
        return Y[0], Y[1:1 + self.nE], Y[1 + self.nE:]

    def initial_state(self):
        y0 = self.model.y0()
        return np.repeat(y0[:, None], self.n, axis=1).astype(np.float64)

    def I_stim(self, t):
        """Nodal stimulus: amplitude on the masked nodes for t_on <= t <= t_off."""
        if self.t_on <= t <= self.t_off:
            return self.stim_amp * self.stim_mask
        return np.zeros(self.n)

    # -- the three right-hand sides (Eq. mono_in_FSE) ------------------------
    def diffusion(self, V):
        """(chi Cm M)^-1 A V with A = -K."""
        return -(self.K @ V) / (self.chi * self.Cm * self.M)

    def f_F(self, t, Y):
        out = np.zeros_like(Y)
        out[0] = self.diffusion(Y[0])
        return out

    def f_S(self, t, Y):
        V, zE, zS = self.parts(Y)
        out = np.zeros_like(Y)
        out[0] = (self.I_stim(t) - self.model.I_ion(V, zE, zS)) / self.Cm
        if self.nS:
            out[1 + self.nE:] = self.model.g_S(V, zE, zS)
        return out

    def f_E(self, t, Y):
        V, zE, zS = self.parts(Y)
        out = np.zeros_like(Y)
        if self.nE:
            lam, zinf = self.model.gating(V, zE, zS)
            out[1:1 + self.nE] = lam * (zE - zinf)
        return out

    # -- Algorithm 3 ----------------------------------------------------------
    def exponential_euler(self, Y, eta):
        """y + (e^{eta Lambda} - I)(y - y_inf), the identity of Algorithm 3."""
        out = Y.copy()
        if self.nE:
            V, zE, zS = self.parts(Y)
            lam, zinf = self.model.gating(V, zE, zS)
            out[1:1 + self.nE] = zE + np.expm1(eta * lam) * (zE - zinf)
        return out

    def averaged_force(self, t, Y, eta, m):
        yE = self.exponential_euler(Y, eta)
        fS = self.f_S(t, yE)  # frozen during the inner iteration

        def f_u(r, u):
            return self.f_F(r, u) + fS

        u_eta = rkc_iteration(t, yE, eta, f_u, m, EPS_DAMP)
        return (u_eta - Y) / eta

    def averaged_force_progressive(self, t, Y, eta, m):
        """The alternative split of the auxiliary problem (Sec. 4.2, remark on
        adding the exponential part progressively): u(0) = y and
        u' = f_F(u) + f_S(y_E) + phi(eta Lambda(y)) f_E(y), where
        phi(eta Lambda) f_E(y) = (y_E - y) / eta by the definition of y_E."""
        yE = self.exponential_euler(Y, eta)
        g = self.f_S(t, yE) + (yE - Y) / eta  # frozen during the inner iteration

        def f_u(r, u):
            return self.f_F(r, u) + g

        u_eta = rkc_iteration(t, Y, eta, f_u, m, EPS_DAMP)
        return (u_eta - Y) / eta

    def stage_counts(self, dt, rho_F, rho_S):
        s, l_s = get_stages(dt, rho_S, EPS_DAMP)
        eta = 2.0 * dt / l_s
        m, _ = get_stages(eta, rho_F, EPS_DAMP)
        return s, m, eta

    def emrkc_step(self, t, Y, dt, rho_F, rho_S, progressive=False):
        """One emRKC step; returns (y_{n+1}, s, m, eta).  progressive=True
        uses the alternative split of the auxiliary problem."""
        s, m, eta = self.stage_counts(dt, rho_F, rho_S)
        af = self.averaged_force_progressive if progressive else self.averaged_force

        def fbar(tt, yy):
            return af(tt, yy, eta, m)

        return rkc_iteration(t, Y, dt, fbar, s, EPS_DAMP), s, m, eta

    # -- mRKC (Algorithm 2) with the stiffest-gate split (Sec. 3.3) ----------
    # f~_F = f_F + f_E^1 and f~_S = f_S + f_E^2 (Eq. mRCK_fFfS_monodomain),
    # where f_E^1 holds the exponential-type term of the single stiffest gating
    # variable (index k of z_E) and f_E^2 those of all other gates.
    def f_E1(self, t, Y, k):
        out = np.zeros_like(Y)
        if self.nE:
            V, zE, zS = self.parts(Y)
            lam, zinf = self.model.gating(V, zE, zS)
            out[1 + k] = lam[k] * (zE[k] - zinf[k])
        return out

    def f_E2(self, t, Y, k):
        out = self.f_E(t, Y)
        if self.nE:
            out[1 + k] = 0.0
        return out

    def fF_tilde(self, t, Y, k):
        return self.f_F(t, Y) + self.f_E1(t, Y, k)

    def fS_tilde(self, t, Y, k):
        return self.f_S(t, Y) + self.f_E2(t, Y, k)

    def mrkc_averaged_force(self, t, Y, eta, m, k):
        """Averaged_Force of Algorithm 2: m RKC stages over
        u' = f~_F(u) + f~_S(t, y) (f~_S frozen) on [0, eta], u(0) = y."""
        fS = self.fS_tilde(t, Y, k)

        def f_u(r, u):
            return self.fF_tilde(r, u, k) + fS

        u_eta = rkc_iteration(t, Y, eta, f_u, m, EPS_DAMP)
        return (u_eta - Y) / eta

    def mrkc_step(self, t, Y, dt, rho_F, rho_S, k):
        """One mRKC step (Algorithm 2); returns (y_{n+1}, s, m, eta)."""
        s, m, eta = self.stage_counts(dt, rho_F, rho_S)

        def fbar(tt, yy):
            return self.mrkc_averaged_force(tt, yy, eta, m, k)

        return rkc_iteration(t, Y, dt, fbar, s, EPS_DAMP), s, m, eta

    def rho_Ft_fn(self, Y, k):
        """f~_F restricted to its nonzero block (V, z_E[k]), as a function of
        that block (the other components are held at Y)."""
        n = self.n

        def f(t, x):
            Z = Y.copy()
            Z[0] = x[:n]
            Z[1 + k] = x[n:]
            out = self.fF_tilde(t, Z, k)
            return np.concatenate([out[0], out[1 + k]])

        return f

    def rho_St_fn(self, k):
        def f(t, y):
            return self.fS_tilde(t, y.reshape(self.N, self.n), k).ravel()

        return f

    # -- spectral radii (Algorithm 5) ----------------------------------------
    def rho_F_fn(self, t, V):
        return self.diffusion(V)

    def rho_S_fn(self, t, y):
        return self.f_S(t, y.reshape(self.N, self.n)).ravel()

    def l2_norm(self, V):
        """Discrete L2(Omega) norm with the lumped mass: sqrt(V^T M V)."""
        return float(np.sqrt(np.sum(self.M * V * V)))


class OracleRun:
    """Time-stepping driver: rho policy, emRKC steps, activation times.

    rho_every = k >= 1 recomputes rho_F and rho_S every k-th step (warm
    started), rho_every = 0 only before the first step; fixed_rho =
    (rho_F, rho_S) bypasses the power iteration and uses the values as given.
    rho_S_min is a known bound on the stiffness of f_S (Sec. 3.1: rho is
    "known or estimated"); the step uses max(safety * estimate, rho_S_min).

    Cold start (reading of App. A): an estimate with no initial guess (its
    rho still 0, the start vector arbitrary) runs Algorithm 5 to the relative
    tolerance pow_tol_cold = 1e-4 (at most pow_max_iter_cold iterations); the
    warm-started calls that follow use the App. A tolerance 1e-2.  From an
    arbitrary start the 1e-2 test can stop on an early plateau: on 3-D slabs
    of the batched workload it returned 0.80-0.97 of the largest eigenvalue
    of L, which the safety factor 1.05 does not cover.
    """

    def __init__(self, prob: Monodomain, Y0=None, rho_every=1, fixed_rho=None, seed=0,
                 safety=SAFETY, act_threshold=-20.0, pow_tol=1e-2, pow_eps=1e-8, pow_max_iter=50,
                 rho_S_min=0.0, progressive=False, method="emrkc", stiff_gate=0, pow_tol_cold=1e-4,
                 pow_max_iter_cold=1000):
        self.p = prob
        self.progressive = progressive
        if method not in ("emrkc", "mrkc"):
            raise ValueError("method must be 'emrkc' or 'mrkc'")
        self.method = method
        self.stiff_gate = stiff_gate
        self.Y = prob.initial_state() if Y0 is None else np.array(Y0, dtype=np.float64)
        self.t = 0.0
        self.steps = 0
        self.rho_every = rho_every
        self.fixed_rho = fixed_rho
        self.safety = safety
        self.pow = dict(eps=pow_eps, tol=pow_tol, max_iter=pow_max_iter)
        self.pow_cold = dict(eps=pow_eps, tol=pow_tol_cold, max_iter=pow_max_iter_cold)
        # mRKC: f~_F acts on (V, z_E[k]), so its iterate has 2n entries
        self.vF = start_vector(seed & 0xFFFFFFFFFFFFFFFF, prob.n * (2 if method == "mrkc" else 1))
        self.vS = start_vector(~seed & 0xFFFFFFFFFFFFFFFF, prob.N * prob.n)
        self.rhoF_raw = 0.0
        self.rhoS_raw = 0.0
        self.act_threshold = act_threshold
        self.rho_S_min = rho_S_min  # known lower bound on rho(f_S) (the rho of Alg. 1 may be known)
        self.act = np.full(prob.n, np.nan)
        self.log = []  # (s, m, rho_F, rho_S, itF, itS) per step

    def update_rho(self):
        itF = itS = 0
        # cold start (no initial guess yet): the tighter tolerance
        powF = self.pow_cold if self.rhoF_raw == 0.0 else self.pow
        powS = self.pow_cold if self.rhoS_raw == 0.0 else self.pow
        if self.method == "mrkc":
            k = self.stiff_gate
            x = np.concatenate([self.Y[0], self.Y[1 + k]])
            self.vF, self.rhoF_raw, itF = compute_rho(self.t, x, self.p.rho_Ft_fn(self.Y, k), self.vF,
                                                      self.rhoF_raw, **powF)
            self.vS, self.rhoS_raw, itS = compute_rho(self.t, self.Y.ravel(), self.p.rho_St_fn(k), self.vS,
                                                      self.rhoS_raw, **powS)
            return itF, itS
        self.vF, self.rhoF_raw, itF = compute_rho(self.t, self.Y[0], self.p.rho_F_fn, self.vF,
                                                  self.rhoF_raw, **powF)
        self.vS, self.rhoS_raw, itS = compute_rho(self.t, self.Y.ravel(), self.p.rho_S_fn, self.vS,
                                                  self.rhoS_raw, **powS)
        return itF, itS

    def step(self, dt):
        itF = itS = 0
        if self.fixed_rho is not None:
            rho_F, rho_S = self.fixed_rho
        else:
            due = (self.steps == 0) if self.rho_every == 0 else (self.steps % self.rho_every == 0)
            if due:
                itF, itS = self.update_rho()
            rho_F = self.safety * self.rhoF_raw
            rho_S = max(self.safety * self.rhoS_raw, self.rho_S_min)
        V_old = self.Y[0].copy()
        if self.method == "mrkc":
            Y, s, m, eta = self.p.mrkc_step(self.t, self.Y, dt, rho_F, rho_S, self.stiff_gate)
        else:
            Y, s, m, eta = self.p.emrkc_step(self.t, self.Y, dt, rho_F, rho_S, self.progressive)
        V_new = Y[0]
        th = self.act_threshold
        cross = np.isnan(self.act) & (V_old < th) & (V_new >= th)
        if np.any(cross):
            self.act[cross] = self.t + dt * (th - V_old[cross]) / (V_new[cross] - V_old[cross])
        self.Y = Y
        self.t += dt
        self.steps += 1
        self.log.append((s, m, rho_F, rho_S, itF, itS))
        return s, m

    def run(self, T, dt):
        n_steps = int(round(T / dt))
        if abs(n_steps * dt - T) > 1e-9 * max(1.0, abs(T)):
            raise ValueError("T is not an integer multiple of dt")
        for _ in range(n_steps):
            self.step(dt)
        return self.Y


def run_workload(w, steps=None, **kw):
    """Convenience: build the oracle problem of a workload and run it."""
    prob = Monodomain.from_workload(w)
    r = OracleRun(prob, rho_every=kw.pop("rho_every", w.rho_every), **kw)
    n_steps = w.steps if steps is None else steps
    for _ in range(n_steps):
        r.step(w.dt)
    return prob, r
