"""Pins of the oracle's mRKC step (Algorithm 2 with the stiffest-gate split
of Sec. 3.3).

Independent facts used:
  * for the linear decoupled passive model on a 1-D cosine eigenvector, one
    mRKC step multiplies V by R_s(dt Phi_m(eta lF)(lF + lS)), the stiff gate's
    deviation by R_s(dt Phi_m(eta lE) lE) (it is integrated in the inner
    loop) and z_S by R_s(-dt k_c), with Phi_m(z) = (P_m(z) - 1) / z; the RKC
    polynomials are evaluated with numpy's Chebyshev routines;
  * the stiffest gate: over the physiological range of V the largest |Lambda|
    of HH and TTP06 belongs to the sodium activation m (z_E[0]), the variable
    the split moves into f~_F (Remark 3.1 picks it empirically);
  * rho(f~_F) on (V, z_E[k]) is max(rho(L), |lambda_E|) for the passive model;
  * with no ionic model (pure diffusion) mRKC coincides with emRKC;
  * first-order convergence against fine-step RK4.
"""

import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from numpy.polynomial import chebyshev as C

from oracle.emrkc import Monodomain, OracleRun
from oracle.fem import assemble_p1
from oracle.ionic import HHModel, PassiveModel, TTP06Model
from oracle.power import compute_rho, start_vector
from oracle.reference import rk4_run
from oracle.rkc import EPS_DAMP, get_stages
from workloads import isotropic_D, line_mesh, make_workload


def _P(m, z):
    w0 = 1.0 + EPS_DAMP / m ** 2
    T = [0] * m + [1]
    w1 = C.chebval(w0, T) / C.chebval(w0, C.chebder(T))
    return C.chebval(w0 + w1 * z, T) / C.chebval(w0, T)


def _Phi(m, z):
    return (_P(m, z) - 1.0) / z


def _line_problem(n, length, model, chi=1400.0, Cm=1.0, sigma=1.0):
    coords, cells = line_mesh(n, length)
    K, M = assemble_p1(coords, cells, isotropic_D(cells.shape[0], 1, sigma))
    return coords, Monodomain(K, M, chi, Cm, model, np.zeros(n), 0.0, 0.0, -1.0)


@pytest.mark.parametrize("dt,rhoF,rhoS", [(0.05, 80.0, 5.0), (0.5, 400.0, 40.0), (0.2, 3000.0, 120.0)])
@pytest.mark.parametrize("k", [2, 7])
def test_mrkc_scalar_amplification(dt, rhoF, rhoS, k):
    n, L = 22, 0.21
    h = L / (n - 1)
    chi, Cm, sigma = 1400.0, 1.0, 1.2
    coords, prob = _line_problem(n, L, PassiveModel(), chi, Cm, sigma)
    x = coords[:, 0]
    Y = prob.initial_state()
    Y[0] = np.cos(k * np.pi * x / L)
    Y[1] = 0.85
    Y[2] = -0.4
    Y1, s, m, eta = prob.mrkc_step(0.0, Y, dt, rhoF, rhoS, 0)
    s_ref, ls = get_stages(dt, rhoS)
    m_ref, _ = get_stages(2 * dt / ls, rhoF)
    assert (s, m) == (s_ref, m_ref)
    pm = PassiveModel()
    lamF = -(4 * sigma / (h * h * chi * Cm)) * np.sin(k * np.pi / (2 * (n - 1))) ** 2
    lamS = -pm.g_p / Cm
    lamE = -(pm.a_w + pm.b_w)
    winf = pm.a_w / (pm.a_w + pm.b_w)
    np.testing.assert_allclose(Y1[0], _P(s, dt * _Phi(m, eta * lamF) * (lamF + lamS)) * Y[0], rtol=1e-11,
                               atol=1e-13)
    np.testing.assert_allclose(Y1[1] - winf, _P(s, dt * _Phi(m, eta * lamE) * lamE) * (Y[1] - winf),
                               rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(Y1[2], _P(s, -dt * pm.k_c) * Y[2], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("model", [HHModel(), TTP06Model()])
def test_stiffest_gate_is_sodium_activation(model):
    V = np.linspace(-100.0, 60.0, 1601)
    y0 = model.y0()
    zE = np.repeat(y0[1:1 + model.nE, None], V.size, axis=1)
    zS = np.repeat(y0[1 + model.nE:, None], V.size, axis=1)
    lam, _ = model.gating(V, zE, zS)
    peak = np.max(np.abs(lam), axis=1)
    assert np.argmax(peak) == 0
    assert peak[0] > 1.5 * np.max(peak[1:])


def test_rho_F_tilde_closed_form():
    n, L = 30, 0.29
    coords, prob = _line_problem(n, L, PassiveModel(), sigma=0.02)
    Y = prob.initial_state()
    A = sp.diags(1.0 / (prob.chi * prob.Cm * prob.M)) @ prob.K
    lam_L = abs(spla.eigs(A.tocsc(), k=1, which="LM", return_eigenvectors=False)[0])
    pm = PassiveModel()
    assert lam_L < pm.a_w + pm.b_w  # the gate sets the radius here
    x = np.concatenate([Y[0], Y[1]])
    _, rho, _ = compute_rho(0.0, x, prob.rho_Ft_fn(Y, 0), start_vector(3, 2 * n), 0.0, tol=1e-10, max_iter=500)
    assert abs(rho - (pm.a_w + pm.b_w)) <= 1e-6 * rho
    coords, prob = _line_problem(n, L, PassiveModel(), sigma=3.0)
    Y = prob.initial_state()
    A = sp.diags(1.0 / (prob.chi * prob.Cm * prob.M)) @ prob.K
    lam_L = abs(spla.eigs(A.tocsc(), k=1, which="LM", return_eigenvectors=False)[0])
    assert lam_L > pm.a_w + pm.b_w  # now the diffusion does
    x = np.concatenate([Y[0], Y[1]])
    _, rho, _ = compute_rho(0.0, x, prob.rho_Ft_fn(Y, 0), start_vector(3, 2 * n), 0.0, tol=1e-10, max_iter=2000)
    assert abs(rho - lam_L) <= 1e-6 * lam_L


def test_mrkc_equals_emrkc_without_ionic_model():
    w = make_workload("square9x7_none", h=1.0 / 16)
    prob = Monodomain.from_workload(w)
    rng = np.random.default_rng(1)
    Y0 = rng.normal(size=(1, w.n))
    a = OracleRun(prob, Y0=Y0, fixed_rho=(300.0, 2.0))
    b = OracleRun(prob, Y0=Y0, fixed_rho=(300.0, 2.0), method="mrkc")
    for _ in range(10):
        assert a.step(0.2) == b.step(0.2)
    np.testing.assert_allclose(a.Y, b.Y, rtol=0, atol=1e-14 * np.max(np.abs(Y0)))


def test_mrkc_first_order_convergence_against_rk4():
    w = make_workload("square9x9_hh", h=0.5 / 8)
    prob = Monodomain.from_workload(w)
    T = 4.0
    Yref = rk4_run(prob, prob.initial_state(), T, 1e-3)
    dts = [2.0 ** -i for i in range(5, 9)]
    errs = []
    for dt in dts:
        r = OracleRun(prob, rho_every=1, method="mrkc")
        r.run(T, dt)
        errs.append(prob.l2_norm(r.Y[0] - Yref[0]) / prob.l2_norm(Yref[0]))
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 0.8 <= slope <= 1.25, (errs, slope)
    # the split moves the fast m gate into f~_F: at rest on this coarse mesh
    # rho~_F is the m gate's |Lambda| = alpha_m + beta_m, not rho(L)
    r = OracleRun(prob, rho_every=1, method="mrkc")
    r.step(0.01)
    Y0 = prob.initial_state()
    lam, _ = HHModel().gating(Y0[0], Y0[1:4], Y0[4:])
    rho_L = 8.0 * 1.0 / ((0.5 / 8) ** 2 * 1400.0)
    assert abs(lam[0, 0]) > rho_L
    assert abs(r.log[0][2] / 1.05 - abs(lam[0, 0])) <= 0.03 * abs(lam[0, 0])
