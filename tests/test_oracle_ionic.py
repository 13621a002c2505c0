"""Pins of the oracle's ionic models and exponential Euler step (Sec. 2, 4.1, Table 2)."""

import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle.emrkc import Monodomain, OracleRun
from oracle.ionic import HHModel, PassiveModel, TTP06Model, _x_over_expm1
from oracle.power import compute_rho, start_vector
from workloads import make_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.split())
    return rows


def test_hh_rest_gates_golden():
    y0 = HHModel().y0()
    vals = dict(zip(HHModel.names, y0))
    for name, value, tol in _read("hh_rest_gates.txt"):
        assert vals[name] == pytest.approx(float(value), abs=float(tol))


def test_hh_rest_current_vanishes():
    hh = HHModel()
    y0 = hh.y0()
    I = hh.I_ion(np.array([y0[0]]), y0[1:, None], np.zeros((0, 1)))
    # E_L = V_rest + 10.613 is quoted to 3 decimals: |I| is a few 1e-3 uA/cm^2
    assert abs(I[0]) < 1e-2


def test_hh_removable_singularities():
    hh = HHModel()
    # alpha_m at v = 25 and alpha_n at v = 10 are 0/0 with limits 1.0 and 0.1
    for v, k, lim in [(25.0, 0, 1.0), (10.0, 2, 0.1)]:
        a, _ = hh.rates(np.array([hh.V_rest + v, hh.V_rest + v + 1e-6, hh.V_rest + v - 1e-6]))
        assert a[k, 0] == pytest.approx(lim, rel=1e-12)
        assert a[k, 1] == pytest.approx(lim, rel=1e-6)
        assert a[k, 2] == pytest.approx(lim, rel=1e-6)
    x = np.array([0.0, 1e-9, -1e-9, 1e-3, -2.0, 30.0])
    ref = np.array([1.0, 1 - 5e-10, 1 + 5e-10, 1e-3 / np.expm1(1e-3), -2.0 / np.expm1(-2.0),
                    30.0 / np.expm1(30.0)])
    np.testing.assert_allclose(_x_over_expm1(x), ref, rtol=1e-14)


@pytest.mark.parametrize("model_id,V", [(2, -75.0), (2, -20.0), (2, 30.0), (3, -85.0), (3, -10.0), (3, 25.0)])
def test_rush_larsen_exact_for_frozen_V(model_id, V):
    """Exponential Euler with V frozen equals the exact solution of the gate ODE
    dz/dt = Lambda (z - z_inf), here integrated independently by a high-accuracy
    ODE solver in the alpha/beta (or tau) form of Eq. (monodomain_gate)."""
    w = make_workload(f"line2_{'hh' if model_id == 2 else 'ttp'}", length=0.001)
    prob = Monodomain.from_workload(w)
    Y = prob.initial_state()
    Y[0] = V
    eta = 0.37
    YE = prob.exponential_euler(Y, eta)
    Vv, zE, zS = prob.parts(Y)
    lam, zinf = prob.model.gating(Vv, zE, zS)
    if model_id == 2:
        a, b = prob.model.rates(Vv)

        def rhs(t, z):  # Eq. (monodomain_gate): alpha (1 - z) - beta z
            return a[:, 0] * (1 - z) - b[:, 0] * z
    else:
        tau = -1.0 / lam[:, 0]

        def rhs(t, z):
            return (zinf[:, 0] - z) / tau
    sol = solve_ivp(rhs, (0.0, eta), zE[:, 0], method="Radau", rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(YE[1:1 + prob.nE, 0], sol.y[:, -1], rtol=2e-9, atol=1e-12)
    # V and z_S are untouched by the exponential step
    assert YE[0, 0] == Y[0, 0]
    np.testing.assert_array_equal(YE[1 + prob.nE:], Y[1 + prob.nE:])


def test_hh_single_cell_action_potential():
    """Textbook features of the 1952 Hodgkin-Huxley membrane action potential
    (6.3 C, rest at V_rest): an overshooting spike of about 100 mV amplitude,
    about 1-2 ms wide at half amplitude, followed by an after-hyperpolarisation
    that approaches but never crosses the potassium reversal potential
    E_K = V_rest - 12 mV, then recovery toward rest."""
    hh = HHModel()
    w = make_workload("line2_hh", length=0.001)
    w.stim_mask[:] = 1
    w.stim_amp = 20.0
    w.t_on, w.t_off = 0.0, 0.5
    prob = Monodomain.from_workload(w)
    r = OracleRun(prob, rho_every=1)
    dt = 0.01
    V = []
    for _ in range(2000):
        r.step(dt)
        V.append(r.Y[0, 0])
    V = np.array(V)
    t = dt * np.arange(1, V.size + 1)
    rest, E_K = hh.V_rest, hh.V_rest - 12.0
    amp = V.max() - rest
    assert 90.0 < amp < 115.0
    assert V.max() > 0.0  # overshoot
    above = t[V > rest + 0.5 * amp]
    assert 0.8 < above.max() - above.min() < 2.5
    undershoot = V[t > t[V.argmax()]].min()
    assert E_K < undershoot < rest - 5.0
    assert abs(V[-1] - rest) < 2.0


def test_table2_hh_stiffness():
    """rho_S of HH over an action potential peaks near Table 2's rho_max = 40."""
    rows = {r[0]: (int(r[1]), float(r[2])) for r in _read("table2_stiffness.txt")}
    N, rho_max = rows["hh"]
    assert HHModel.nE + HHModel.nS == N
    w = make_workload("line2_hh", length=0.001)
    w.stim_mask[:] = 1
    prob = Monodomain.from_workload(w)
    r = OracleRun(prob, rho_every=1, safety=1.0)
    for _ in range(300):
        r.step(0.02)
    peak = max(l[3] for l in r.log)
    assert 0.85 * rho_max <= peak <= 1.2 * rho_max


def test_table2_ttp_stiffness():
    """The full right-hand side Jacobian of TTP06 at rest has spectral radius
    near Table 2's rho_max = 1000 (set by the fast m gate)."""
    rows = {r[0]: (int(r[1]), float(r[2])) for r in _read("table2_stiffness.txt")}
    N, rho_max = rows["ttp06_epi"]
    assert TTP06Model.nE + TTP06Model.nS == N
    w = make_workload("line2_ttp", length=0.001)
    prob = Monodomain.from_workload(w)
    Y = prob.initial_state()

    def f(t, y):
        YY = y.reshape(prob.N, -1)
        return (prob.f_S(t, YY) + prob.f_E(t, YY)).ravel()

    _, rho, _ = compute_rho(0.0, Y.ravel(), f, start_vector(11, Y.size), 0.0, tol=1e-6, max_iter=500)
    assert 0.8 * rho_max <= rho <= 1.2 * rho_max


def test_ttp_rest_state_nearly_stationary():
    m = TTP06Model()
    y0 = m.y0()
    V = np.array([y0[0]])
    zE = y0[1:13, None]
    zS = y0[13:, None]
    assert abs(m.I_ion(V, zE, zS)[0]) < 0.01  # pA/pF, vs ~ -50 at the upstroke
    gS = m.g_S(V, zE, zS)[:, 0]
    assert np.all(np.abs(gS) < 1e-3)
    lam, zinf = m.gating(V, zE, zS)
    assert np.all(np.abs(lam[:, 0] * (zE[:, 0] - zinf[:, 0])) < 0.01)


def _ttp_random_states(rng, k):
    """Random TTP06 states within physiological ranges."""
    V = rng.uniform(-95.0, 50.0, k)
    zE = rng.uniform(0.0, 1.0, (12, k))
    zS = np.stack([rng.uniform(0.3, 1.0, k),        # Rbar
                   rng.uniform(125.0, 145.0, k),    # Ki (mM)
                   rng.uniform(6.0, 14.0, k),       # Nai
                   rng.uniform(5e-5, 2e-3, k),      # Cai
                   rng.uniform(0.5, 4.5, k),        # CaSR
                   rng.uniform(5e-5, 2e-2, k)])     # CaSS
    return V, zE, zS


def test_ttp_charge_balance():
    """Every ionic current of TTP06 moves charge between the membrane and the
    tracked ion pools, so (without stimulus) the membrane's dV/dt = -I_ion
    equals the rate of change of the cell's total ion charge per unit
    capacitance: (V_c F / C) [dNa_i + dK_i + 2 (dCa_c + (V_sr/V_c) dCa_sr +
    (V_ss/V_c) dCa_ss)], where the calcium terms count free plus buffered
    calcium (d(total)/dt = d(free)/dt / beta).  The fluxes between the
    compartments (release, uptake, leak, transfer) cancel.  Checked pointwise
    at random states; it fails if any current is missing from, or enters with
    a wrong sign or stoichiometry into, either I_ion or the concentration
    equations."""
    m = TTP06Model()
    rng = np.random.default_rng(6)
    V, zE, zS = _ttp_random_states(rng, 500)
    Rbar, Ki, Nai, Cai, CaSR, CaSS = zS
    dV = -m.I_ion(V, zE, zS)
    g = m.g_S(V, zE, zS)
    dKi, dNai, dCai, dCaSR, dCaSS = g[1], g[2], g[3], g[4], g[5]

    def total_rate(dc, c, buf, kbuf):  # free -> free + buffered
        return dc * (1.0 + buf * kbuf / (c + kbuf) ** 2)

    dCa_tot = (total_rate(dCai, Cai, m.Bufc, m.Kbufc)
               + m.Vsr / m.Vc * total_rate(dCaSR, CaSR, m.Bufsr, m.Kbufsr)
               + m.Vss / m.Vc * total_rate(dCaSS, CaSS, m.Bufss, m.Kbufss))
    charge_rate = m.Vc * m.F / m.Cap * (dNai + dKi + 2.0 * dCa_tot)
    scale = np.abs(np.stack(list(m.currents(V, zE, zS).values()))).sum(axis=0)
    assert np.all(np.abs(charge_rate - dV) <= 1e-9 * scale + 1e-12)
    # the check is sensitive: a Na/Ca exchanger with 2 instead of 3 Na per
    # cycle in dNa_i shifts the charge rate by I_NaCa
    c = m.currents(V, zE, zS)
    slip = charge_rate - c["I_NaCa"]
    assert np.max(np.abs(slip - dV)) > 1e-3 * np.max(np.abs(c["I_NaCa"]))


def test_ttp_gates_bounded_and_monotone_rates():
    """TTP06 gating: z_inf in [0, 1] and time constants positive over the
    whole voltage range (the Rush-Larsen step then keeps every gate in
    [0, 1]); the activation gates' z_inf (m, xr1, xs, r, d) rise and the
    inactivation gates' (h, j, xr2, s, f, f2) fall with V."""
    m = TTP06Model()
    V = np.linspace(-120.0, 80.0, 2001)
    zE = np.full((12, V.size), 0.5)
    zS = np.tile(m.y0()[13:, None], (1, V.size))
    lam, zinf = m.gating(V, zE, zS)
    assert np.all((zinf >= 0.0) & (zinf <= 1.0)) and np.all(lam < 0.0)
    for k in (0, 3, 5, 6, 8):  # m, xr1, xs, r, d
        assert np.all(np.diff(zinf[k]) >= -1e-15), k
    for k in (1, 2, 4, 7, 9, 10):  # h, j, xr2, s, f, f2
        assert np.all(np.diff(zinf[k]) <= 1e-15), k


@pytest.mark.slow
def test_ttp_single_cell_action_potential():
    """Published TTP06 epicardial characteristics: rest near -85 mV, upstroke
    velocity of a few hundred mV/ms, APD90 near 300 ms, the epicardial
    spike-and-dome shape and a calcium transient peaking near 1 uM (parity of
    the model beyond these features is unpinned)."""
    w = make_workload("line2_ttp", length=0.001)
    w.stim_mask[:] = 1
    w.stim_amp = 52.0
    w.t_off = 1.0
    prob = Monodomain.from_workload(w)
    r = OracleRun(prob, rho_every=1)
    dt = 0.1
    V, Cai = [], []
    for _ in range(4000):
        r.step(dt)
        V.append(r.Y[0, 0])
        Cai.append(r.Y[1 + 12 + 3, 0])  # z_S = (Rbar, Ki, Nai, Cai, CaSR, CaSS)
    V, Cai = np.array(V), np.array(Cai)
    t = dt * np.arange(1, V.size + 1)
    assert -87.0 < V[-1] < -83.0
    assert 10.0 < V.max() < 80.0
    dVdt = np.diff(np.concatenate([[-85.23], V])) / dt
    assert 150.0 < dVdt.max() < 600.0
    amp = V.max() + 85.23
    after = (t > t[V.argmax()]) & (V < -85.23 + 0.1 * amp)
    apd90 = t[np.nonzero(after)[0][0]]
    assert 240.0 < apd90 < 360.0
    # epicardial spike-and-dome (transient outward current I_to): a notch
    # within 30 ms of the peak, then a dome several mV above it
    ip = int(V.argmax())
    early = V[ip:ip + int(30 / dt)]
    notch = int(early.argmin())
    dome = V[ip + notch:ip + int(150 / dt)].max()
    assert early.min() < V.max() - 10.0
    assert dome > early.min() + 3.0
    # calcium transient: from ~0.1 uM at rest to a peak near 1 uM tens of ms
    # after the upstroke, back toward rest by the end of the beat
    assert 0.05e-3 < Cai[0] < 0.3e-3
    assert 0.4e-3 < Cai.max() < 2.0e-3
    assert 5.0 < t[Cai.argmax()] - t[ip] < 80.0
    assert Cai[-1] < 0.3e-3


def test_passive_model_linear():
    m = PassiveModel()
    V = np.array([1.0, -2.0])
    assert np.allclose(m.I_ion(V, None, None), m.g_p * V)
    lam, zinf = m.gating(V, None, None)
    assert np.allclose(lam, -(m.a_w + m.b_w))
    assert np.allclose(zinf, m.a_w / (m.a_w + m.b_w))
