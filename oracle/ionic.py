"""Ionic models in Hodgkin-Huxley form (Sec. 2, Eq. monodomain), float64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Each model splits its state into V, the gating variables z_E (integrated by
the exponential step, Eq. def_fE) and the remaining variables z_S (part of
f_S, Eq. mono_in_FSE).  The interface, vectorised over nodes:

  gating(V, zE, zS) -> (Lam, zinf): Lambda_E (diagonal, <= 0) and z_inf, so
                       that g_E = Lam * (zE - zinf).  Reading of Sec. 2:
                       Lambda = -(alpha + beta), z_inf = alpha/(alpha+beta)
                       (the printed minus sign on z_inf contradicts Eq.
                       monodomain_gate); tau-form gates use Lambda = -1/tau.
  I_ion(V, zE, zS)  -> total ionic current (uA/cm^2 with 1 uF/cm^2, i.e. the
                       models' native per-capacitance normalisation).
  g_S(V, zE, zS)    -> right-hand side of the z_S variables.
"""

from __future__ import annotations

import numpy as np


def _x_over_expm1(x):
    """x / (e^x - 1), with the removable singularity at 0 (value 1 - x/2 for |x| < 1e-7)."""
    x = np.asarray(x, dtype=np.float64)
    small = np.abs(x) < 1e-7
    safe = np.where(small, 1.0, x)
    return np.where(small, 1.0 - 0.5 * x, safe / np.expm1(safe))


class NoModel:
    """Pure diffusion: N = 1 (V only), I_ion = 0."""

    name = "none"
    nE = 0
    nS = 0
    names = ("V",)

    def y0(self):
        return np.array([0.0])

    def gating(self, V, zE, zS):
        return np.zeros((0, V.size)), np.zeros((0, V.size))

    def I_ion(self, V, zE, zS):
        return np.zeros_like(V)

    def g_S(self, V, zE, zS):
        return np.zeros((0, V.size))


class PassiveModel:
    """Linear test model with closed-form emRKC amplification factors.

    I_ion = g_p V; one gate w with constant rates (Lambda = -(a_w + b_w),
    w_inf = a_w/(a_w + b_w)); one auxiliary variable c with g_S = -k_c c.
    The three components are decoupled, so each evolves under the scalar
    test equation of Sec. 4.4.
    """

    name = "passive"
    nE = 1
    nS = 1
    names = ("V", "w", "c")
    g_p = 0.5
    a_w = 20.0
    b_w = 30.0
    k_c = 2.0

    def y0(self):
        return np.array([0.0, 1.0, 1.0])

    def gating(self, V, zE, zS):
        lam = np.full((1, V.size), -(self.a_w + self.b_w))
        zinf = np.full((1, V.size), self.a_w / (self.a_w + self.b_w))
        return lam, zinf

    def I_ion(self, V, zE, zS):
        return self.g_p * V

    def g_S(self, V, zE, zS):
        return -self.k_c * zS


class HHModel:
    """Hodgkin-Huxley (1952) squid axon, modern sign convention.

    V_rest = -75 mV, E_Na = V_rest + 115, E_K = V_rest - 12,
    E_L = V_rest + 10.613; g_Na, g_K, g_L = 120, 36, 0.3 mS/cm^2; rates in
    v = V - V_rest (mV, 1/ms).  z_E = (m, h, n); no z_S (Sec. 2).
    """

    name = "hh"
    nE = 3
    nS = 0
    names = ("V", "m", "h", "n")
    V_rest = -75.0
    E_Na = -75.0 + 115.0
    E_K = -75.0 - 12.0
    E_L = -75.0 + 10.613
    g_Na = 120.0
    g_K = 36.0
    g_L = 0.3

    def rates(self, V):
        v = V - self.V_rest
        a_m = _x_over_expm1((25.0 - v) / 10.0)  # 0.1 (25 - v) / (exp((25 - v)/10) - 1)
        b_m = 4.0 * np.exp(-v / 18.0)
        a_h = 0.07 * np.exp(-v / 20.0)
        b_h = 1.0 / (np.exp((30.0 - v) / 10.0) + 1.0)
        a_n = 0.1 * _x_over_expm1((10.0 - v) / 10.0)  # 0.01 (10 - v) / (exp((10 - v)/10) - 1)
        b_n = 0.125 * np.exp(-v / 80.0)
        return np.stack([a_m, a_h, a_n]), np.stack([b_m, b_h, b_n])

    def y0(self):
        a, b = self.rates(np.array([self.V_rest]))
        zinf = (a / (a + b))[:, 0]
        return np.concatenate([[self.V_rest], zinf])

    def gating(self, V, zE, zS):
        a, b = self.rates(V)
        return -(a + b), a / (a + b)

    def I_ion(self, V, zE, zS):
        m, h, n = zE
        return (self.g_Na * m ** 3 * h * (V - self.E_Na)
                + self.g_K * n ** 4 * (V - self.E_K)
                + self.g_L * (V - self.E_L))

    def g_S(self, V, zE, zS):
        return np.zeros((0, V.size))


class TTP06Model:
    """ten Tusscher & Panfilov (2006) human ventricular model, epicardial cell.

    State order: V; gates z_E = (m, h, j, xr1, xr2, xs, r, s, d, f, f2, fCass);
    z_S = (Rbar, Ki, Nai, Cai, CaSR, CaSS).  Currents in pA/pF, time in ms,
    concentrations in mM.  Free calcium concentrations are states; fast
    buffering enters through the derivative factors beta = 1/(1 + B K/(c+K)^2).
    """

    name = "ttp06_epi"
    nE = 12
    nS = 6
    names = ("V", "m", "h", "j", "xr1", "xr2", "xs", "r", "s", "d", "f", "f2", "fCass",
             "Rbar", "Ki", "Nai", "Cai", "CaSR", "CaSS")

    # physical constants and cell geometry
    R = 8314.472
    Temp = 310.0
    F = 96485.3415
    Cap = 0.185
    Vc = 0.016404
    Vsr = 0.001094
    Vss = 0.00005468
    Ko = 5.4
    Nao = 140.0
    Cao = 2.0
    # conductances and pump/exchanger parameters (epicardium)
    GNa = 14.838
    GK1 = 5.405
    Gto = 0.294
    GKr = 0.153
    GKs = 0.392
    pKNa = 0.03
    GCaL = 3.980e-5
    kNaCa = 1000.0
    gamma = 0.35
    KmCa = 1.38
    KmNai = 87.5
    ksat = 0.1
    alpha_ncx = 2.5
    PNaK = 2.724
    KmK = 1.0
    KmNa = 40.0
    GpK = 0.0146
    GpCa = 0.1238
    KpCa = 0.0005
    GbNa = 0.00029
    GbCa = 0.000592
    # calcium handling
    Vmaxup = 0.006375
    Kup = 0.00025
    Vrel = 0.102
    k1p = 0.15
    k2p = 0.045
    k3 = 0.060
    k4 = 0.005
    EC = 1.5
    maxsr = 2.5
    minsr = 1.0
    Vleak = 0.00036
    Vxfer = 0.0038
    Bufc = 0.2
    Kbufc = 0.001
    Bufsr = 10.0
    Kbufsr = 0.3
    Bufss = 0.4
    Kbufss = 0.00025

    def y0(self):
        return np.array([-85.23,
                         0.00172, 0.7444, 0.7045, 0.00621, 0.4712, 0.0095, 2.42e-8, 0.999998,
                         3.373e-5, 0.7888, 0.9755, 0.9953,
                         0.9073, 136.89, 8.604, 0.000126, 3.64, 0.00036])

    @property
    def RTF(self):
        return self.R * self.Temp / self.F

    def gating(self, V, zE, zS):
        CaSS = zS[5]
        ex = np.exp
        # fast sodium: m, h, j
        m_inf = 1.0 / (1.0 + ex((-56.86 - V) / 9.03)) ** 2
        a_m = 1.0 / (1.0 + ex((-60.0 - V) / 5.0))
        b_m = 0.1 / (1.0 + ex((V + 35.0) / 5.0)) + 0.10 / (1.0 + ex((V - 50.0) / 200.0))
        tau_m = a_m * b_m
        h_inf = 1.0 / (1.0 + ex((V + 71.55) / 7.43)) ** 2
        hi = V >= -40.0
        a_h = np.where(hi, 0.0, 0.057 * ex(-(V + 80.0) / 6.8))
        b_h = np.where(hi, 0.77 / (0.13 * (1.0 + ex(-(V + 10.66) / 11.1))),
                       2.7 * ex(0.079 * V) + 3.1e5 * ex(0.3485 * V))
        tau_h = 1.0 / (a_h + b_h)
        j_inf = h_inf
        a_j = np.where(hi, 0.0,
                       (-2.5428e4 * ex(0.2444 * V) - 6.948e-6 * ex(-0.04391 * V)) * (V + 37.78)
                       / (1.0 + ex(0.311 * (V + 79.23))))
        b_j = np.where(hi, 0.6 * ex(0.057 * V) / (1.0 + ex(-0.1 * (V + 32.0))),
                       0.02424 * ex(-0.01052 * V) / (1.0 + ex(-0.1378 * (V + 40.14))))
        tau_j = 1.0 / (a_j + b_j)
        # rapid delayed rectifier: xr1, xr2
        xr1_inf = 1.0 / (1.0 + ex((-26.0 - V) / 7.0))
        tau_xr1 = (450.0 / (1.0 + ex((-45.0 - V) / 10.0))) * (6.0 / (1.0 + ex((V + 30.0) / 11.5)))
        xr2_inf = 1.0 / (1.0 + ex((V + 88.0) / 24.0))
        tau_xr2 = (3.0 / (1.0 + ex((-60.0 - V) / 20.0))) * (1.12 / (1.0 + ex((V - 60.0) / 20.0)))
        # slow delayed rectifier: xs
        xs_inf = 1.0 / (1.0 + ex((-5.0 - V) / 14.0))
        tau_xs = (1400.0 / np.sqrt(1.0 + ex((5.0 - V) / 6.0))) * (1.0 / (1.0 + ex((V - 35.0) / 15.0))) + 80.0
        # transient outward (epicardial): r, s
        r_inf = 1.0 / (1.0 + ex((20.0 - V) / 6.0))
        tau_r = 9.5 * ex(-(V + 40.0) ** 2 / 1800.0) + 0.8
        s_inf = 1.0 / (1.0 + ex((V + 20.0) / 5.0))
        tau_s = 85.0 * ex(-(V + 45.0) ** 2 / 320.0) + 5.0 / (1.0 + ex((V - 20.0) / 5.0)) + 3.0
        # L-type calcium: d, f, f2, fCass
        d_inf = 1.0 / (1.0 + ex((-8.0 - V) / 7.5))
        tau_d = ((1.4 / (1.0 + ex((-35.0 - V) / 13.0)) + 0.25) * (1.4 / (1.0 + ex((V + 5.0) / 5.0)))
                 + 1.0 / (1.0 + ex((50.0 - V) / 20.0)))
        f_inf = 1.0 / (1.0 + ex((V + 20.0) / 7.0))
        tau_f = (1102.5 * ex(-(V + 27.0) ** 2 / 225.0) + 200.0 / (1.0 + ex((13.0 - V) / 10.0))
                 + 180.0 / (1.0 + ex((V + 30.0) / 10.0)) + 20.0)
        f2_inf = 0.67 / (1.0 + ex((V + 35.0) / 7.0)) + 0.33
        tau_f2 = (600.0 * ex(-(V + 25.0) ** 2 / 170.0) + 31.0 / (1.0 + ex((25.0 - V) / 10.0))
                  + 16.0 / (1.0 + ex((V + 30.0) / 10.0)))
        q = (CaSS / 0.05) ** 2
        fcass_inf = 0.6 / (1.0 + q) + 0.4
        tau_fcass = 80.0 / (1.0 + q) + 2.0
        zinf = np.stack([m_inf, h_inf, j_inf, xr1_inf, xr2_inf, xs_inf, r_inf, s_inf,
                         d_inf, f_inf, f2_inf, fcass_inf])
        tau = np.stack([tau_m, tau_h, tau_j, tau_xr1, tau_xr2, tau_xs, tau_r, tau_s,
                        tau_d, tau_f, tau_f2, tau_fcass])
        return -1.0 / tau, zinf

    def currents(self, V, zE, zS):
        m, h, j, xr1, xr2, xs, r, s, d, f, f2, fcass = zE
        Rbar, Ki, Nai, Cai, CaSR, CaSS = zS
        ex = np.exp
        RTF = self.RTF
        E_K = RTF * np.log(self.Ko / Ki)
        E_Na = RTF * np.log(self.Nao / Nai)
        E_Ks = RTF * np.log((self.Ko + self.pKNa * self.Nao) / (Ki + self.pKNa * Nai))
        E_Ca = 0.5 * RTF * np.log(self.Cao / Cai)
        a_K1 = 0.1 / (1.0 + ex(0.06 * (V - E_K - 200.0)))
        b_K1 = ((3.0 * ex(0.0002 * (V - E_K + 100.0)) + ex(0.1 * (V - E_K - 10.0)))
                / (1.0 + ex(-0.5 * (V - E_K))))
        xK1 = a_K1 / (a_K1 + b_K1)
        sqko = np.sqrt(self.Ko / 5.4)
        I_K1 = self.GK1 * sqko * xK1 * (V - E_K)
        I_to = self.Gto * r * s * (V - E_K)
        I_Kr = self.GKr * sqko * xr1 * xr2 * (V - E_K)
        I_Ks = self.GKs * xs * xs * (V - E_Ks)
        I_Na = self.GNa * m ** 3 * h * j * (V - E_Na)
        I_bNa = self.GbNa * (V - E_Na)
        u = 2.0 * (V - 15.0) / RTF
        I_CaL = (self.GCaL * d * f * f2 * fcass * 2.0 * self.F * _x_over_expm1(u)
                 * (0.25 * CaSS * ex(u) - self.Cao))
        I_bCa = self.GbCa * (V - E_Ca)
        e1 = ex(self.gamma * V / RTF)
        e2 = ex((self.gamma - 1.0) * V / RTF)
        I_NaCa = (self.kNaCa * (e1 * Nai ** 3 * self.Cao - e2 * self.Nao ** 3 * Cai * self.alpha_ncx)
                  / ((self.KmNai ** 3 + self.Nao ** 3) * (self.KmCa + self.Cao) * (1.0 + self.ksat * e2)))
        I_NaK = (self.PNaK * self.Ko / (self.Ko + self.KmK) * Nai / (Nai + self.KmNa)
                 / (1.0 + 0.1245 * ex(-0.1 * V / RTF) + 0.0353 * ex(-V / RTF)))
        I_pCa = self.GpCa * Cai / (self.KpCa + Cai)
        I_pK = self.GpK * (V - E_K) / (1.0 + ex((25.0 - V) / 5.98))
        return dict(I_K1=I_K1, I_to=I_to, I_Kr=I_Kr, I_Ks=I_Ks, I_Na=I_Na, I_bNa=I_bNa,
                    I_CaL=I_CaL, I_bCa=I_bCa, I_NaCa=I_NaCa, I_NaK=I_NaK, I_pCa=I_pCa, I_pK=I_pK)

    def I_ion(self, V, zE, zS):
        c = self.currents(V, zE, zS)
        return sum(c.values())

    def g_S(self, V, zE, zS):
        c = self.currents(V, zE, zS)
        Rbar, Ki, Nai, Cai, CaSR, CaSS = zS
        kcasr = self.maxsr - (self.maxsr - self.minsr) / (1.0 + (self.EC / CaSR) ** 2)
        k1 = self.k1p / kcasr
        k2 = self.k2p * kcasr
        dRbar = -k2 * CaSS * Rbar + self.k4 * (1.0 - Rbar)
        O = k1 * CaSS ** 2 * Rbar / (self.k3 + k1 * CaSS ** 2)
        I_rel = self.Vrel * O * (CaSR - CaSS)
        I_up = self.Vmaxup / (1.0 + self.Kup ** 2 / Cai ** 2)
        I_leak = self.Vleak * (CaSR - Cai)
        I_xfer = self.Vxfer * (CaSS - Cai)
        b_c = 1.0 / (1.0 + self.Bufc * self.Kbufc / (Cai + self.Kbufc) ** 2)
        b_sr = 1.0 / (1.0 + self.Bufsr * self.Kbufsr / (CaSR + self.Kbufsr) ** 2)
        b_ss = 1.0 / (1.0 + self.Bufss * self.Kbufss / (CaSS + self.Kbufss) ** 2)
        capF = self.Cap / (self.Vc * self.F)
        dCai = b_c * ((I_leak - I_up) * self.Vsr / self.Vc + I_xfer
                      - (c["I_bCa"] + c["I_pCa"] - 2.0 * c["I_NaCa"]) * 0.5 * capF)
        dCaSR = b_sr * (I_up - I_rel - I_leak)
        dCaSS = b_ss * (-c["I_CaL"] * self.Cap / (2.0 * self.Vss * self.F)
                        + I_rel * self.Vsr / self.Vss - I_xfer * self.Vc / self.Vss)
        dNai = -(c["I_Na"] + c["I_bNa"] + 3.0 * c["I_NaK"] + 3.0 * c["I_NaCa"]) * capF
        dKi = -(c["I_K1"] + c["I_to"] + c["I_Kr"] + c["I_Ks"] - 2.0 * c["I_NaK"] + c["I_pK"]) * capF
        return np.stack([dRbar, dKi, dNai, dCai, dCaSR, dCaSS])


MODELS = {0: NoModel, 1: PassiveModel, 2: HHModel, 3: TTP06Model}


def make_model(model_id: int):
    return MODELS[model_id]()
