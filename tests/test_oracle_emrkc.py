"""Pins of the oracle's emRKC step, driver and power iteration.

Independent facts used:
  * Sec. 4.4: for a linear decoupled problem one emRKC step multiplies each
    eigencomponent by R_s(dt (Phi_m(eta lF)(lF + lS) e^{eta lE} + phi(eta lE) lE)),
    evaluated here with numpy's Chebyshev routines on the closed-form
    eigenvalue of the 1-D P1 Laplacian with lumped mass.
  * conservation of sum_i M_ii V_i under pure diffusion with Neumann BC;
  * x <-> y mirror symmetry of the right-diagonal mesh with a corner stimulus;
  * first-order convergence against fine-step RK4 (Thm. 4.5, Sec. 5.2);
  * closed-form largest eigenvalue for the power iteration (Algorithm 5),
    and scipy's Lanczos eigenvalue (eigsh) of the symmetric form of L for the
    cold-start estimate of the driver;
  * the progressive split of the auxiliary problem (Sec. 4.2 remark) equals
    the split of Algorithm 3 up to rounding when f_F acts on V alone and f_E
    on z_E alone: the inner RKC integrates the constant gate forcing exactly
    (c_m = 1), so u_z(eta) = y_E;
  * Algorithm 4 on the same eigenvector: explicit Euler multiplies V by
    1 + dt (lF + lS), the implicit diffusion step by (1 + dt lS) / (1 - dt lF),
    the gate relaxes exactly and z_S takes one explicit Euler step.
"""

import math

import numpy as np
import pytest
import scipy.sparse as sp
from numpy.polynomial import chebyshev as C

from oracle.emrkc import Monodomain, OracleRun
from oracle.fem import assemble_p1
from oracle.ionic import NoModel, PassiveModel, make_model
from oracle.power import compute_rho, start_vector
from oracle.reference import ImexRL, RLRun, exex_rl_step, rk4_run
from oracle.rkc import EPS_DAMP, get_stages
from workloads import isotropic_D, line_mesh, make_workload, square_tri_mesh


def _P(m, z):
    """Stability polynomial of m-stage damped RKC via numpy Chebyshev routines."""
    w0 = 1.0 + EPS_DAMP / m ** 2
    T = [0] * m + [1]
    w1 = C.chebval(w0, T) / C.chebval(w0, C.chebder(T))
    return C.chebval(w0 + w1 * z, T) / C.chebval(w0, T)


def _line_problem(n, length, model, chi=1400.0, Cm=1.0, sigma=1.0):
    coords, cells = line_mesh(n, length)
    K, M = assemble_p1(coords, cells, isotropic_D(cells.shape[0], 1, sigma))
    return coords, Monodomain(K, M, chi, Cm, model, np.zeros(n), 0.0, 0.0, -1.0)


@pytest.mark.parametrize("dt,rhoF,rhoS", [(0.05, 30.0, 5.0), (0.5, 400.0, 40.0), (0.2, 2000.0, 120.0)])
@pytest.mark.parametrize("k", [3, 11])
def test_scalar_amplification_sec44(dt, rhoF, rhoS, k):
    n, L = 24, 0.23
    h = L / (n - 1)
    chi, Cm, sigma = 1400.0, 1.0, 1.3
    coords, prob = _line_problem(n, L, PassiveModel(), chi, Cm, sigma)
    x = coords[:, 0]
    Y = prob.initial_state()
    Y[0] = np.cos(k * np.pi * x / L)
    Y[1] = 0.9
    Y[2] = -0.7
    Y1, s, m, eta = prob.emrkc_step(0.0, Y, dt, rhoF, rhoS)
    s_ref, ls = get_stages(dt, rhoS)
    m_ref, _ = get_stages(2 * dt / ls, rhoF)
    assert (s, m) == (s_ref, m_ref)
    lamF = -(4 * sigma / (h * h * chi * Cm)) * np.sin(k * np.pi / (2 * (n - 1))) ** 2
    pm = PassiveModel()
    lamS = -pm.g_p / Cm
    lamE = -(pm.a_w + pm.b_w)
    winf = pm.a_w / (pm.a_w + pm.b_w)
    zF = eta * lamF
    Phi = (_P(m, zF) - 1.0) / zF
    ampV = _P(s, dt * Phi * (lamF + lamS))
    np.testing.assert_allclose(Y1[0], ampV * Y[0], rtol=1e-12, atol=1e-13)
    phiE = math.expm1(eta * lamE) / (eta * lamE)
    ampW = _P(s, dt * phiE * lamE)
    np.testing.assert_allclose(Y1[1] - winf, ampW * (Y[1] - winf), rtol=1e-12, atol=1e-14)
    ampC = _P(s, -dt * pm.k_c)
    np.testing.assert_allclose(Y1[2], ampC * Y[2], rtol=1e-12, atol=1e-14)


def test_conservation_pure_diffusion():
    coords, cells = square_tri_mesh(17, 13, 1.0, 0.75)
    K, M = assemble_p1(coords, cells, isotropic_D(cells.shape[0], 2, 2.0))
    prob = Monodomain(K, M, 1400.0, 1.0, NoModel(), np.zeros(coords.shape[0]), 0.0, 0.0, -1.0)
    rng = np.random.default_rng(1)
    Y0 = rng.normal(size=(1, coords.shape[0]))
    r = OracleRun(prob, Y0=Y0, fixed_rho=(4000.0, 1.0))
    tot0 = np.sum(M * Y0[0])
    for _ in range(300):
        s, m = r.step(0.5)
    assert m > 1
    # rounding bound: 300 steps x s*m stage updates x eps x sqrt(n) ~ 1e-11
    assert abs(np.sum(M * r.Y[0]) - tot0) <= 1e-11 * np.sum(M * np.abs(Y0[0]))
    # the field itself has changed a lot (smoothing), so the check is not vacuous
    assert np.linalg.norm(r.Y[0] - Y0[0]) > 0.5 * np.linalg.norm(Y0[0] - Y0[0].mean())


def test_mirror_symmetry_square():
    w = make_workload("square17x17_hh", h=1.0 / 32)
    prob = Monodomain.from_workload(w)
    r = OracleRun(prob, rho_every=1)
    for _ in range(150):
        r.step(0.02)
    V = r.Y[0].reshape(17, 17)
    assert np.max(np.abs(V - V.T)) <= 1e-11 * np.max(np.abs(V))
    assert np.nanmax(r.act) > 0.5  # the wave has left the stimulus region


def _rel_l2(prob, V, Vref):
    return prob.l2_norm(V - Vref) / prob.l2_norm(Vref)


@pytest.mark.parametrize("nx", [9, 17])
def test_first_order_convergence_against_rk4(nx):
    w = make_workload(f"square{nx}x{nx}_hh", h=0.5 / (nx - 1))
    w.t_off = 1.0
    prob = Monodomain.from_workload(w)
    T = 4.0
    Yref = rk4_run(prob, prob.initial_state(), T, 1e-3)
    # asymptotic range: for HH, emRKC loses stability at large dt (Sec. 5.2
    # reports missing HH points there), so the rate is fitted for dt <= 2^-5
    dts = [2.0 ** -i for i in range(5, 9)]
    errs = []
    for dt in dts:
        r = OracleRun(prob, rho_every=1)
        r.run(T, dt)
        errs.append(_rel_l2(prob, r.Y[0], Yref[0]))
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 0.8 <= slope <= 1.2, (errs, slope)
    assert errs[-1] < 5e-3


def test_single_cell_brute_force():
    w = make_workload("line2_hh", length=1e-3)
    w.stim_mask[:] = 1
    prob = Monodomain.from_workload(w)
    T = 3.0
    Yref = rk4_run(prob, prob.initial_state(), T, 5e-4)
    dts = [2.0 ** -i for i in range(3, 9)]
    errs = []
    for dt in dts:
        r = OracleRun(prob, rho_every=1)
        r.run(T, dt)
        errs.append(np.max(np.abs(r.Y - Yref) / (np.abs(Yref) + 1e-3)))
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 0.8 <= slope <= 1.25, (errs, slope)


def test_power_iteration_line_closed_form():
    n, L, chi, Cm, sigma = 10, 0.9, 1400.0, 1.0, 1.1
    coords, prob = _line_problem(n, L, NoModel(), chi, Cm, sigma)
    h = L / (n - 1)
    rho_max = 4 * sigma / (h * h * chi * Cm)
    V = np.cos(np.pi * coords[:, 0] / L) + 2.0
    v0 = start_vector(0, n)
    _, rho, it = compute_rho(0.0, V, prob.rho_F_fn, v0, 0.0, tol=1e-12, max_iter=20000)
    assert rho == pytest.approx(rho_max, rel=1e-6)
    _, rho2, it2 = compute_rho(0.0, V, prob.rho_F_fn, v0, 0.0)
    assert 0.8 * rho_max <= rho2 <= rho_max * (1 + 1e-9)
    assert it2 >= 1


def test_power_iteration_square_kronecker_mass():
    nx, h, sigma, chi, Cm = 9, 1.0 / 8, 1.0, 1400.0, 1.0
    coords, cells = square_tri_mesh(nx, nx, 1.0, 1.0)
    K, M = assemble_p1(coords, cells, isotropic_D(cells.shape[0], 2, sigma))
    m1 = np.full(nx, h)
    m1[0] = m1[-1] = h / 2
    Mk = np.kron(m1, m1)
    prob = Monodomain(K, Mk, chi, Cm, NoModel(), np.zeros(nx * nx), 0.0, 0.0, -1.0)
    V = np.linspace(-80, 20, nx * nx)
    _, rho, _ = compute_rho(0.0, V, prob.rho_F_fn, start_vector(5, nx * nx), 0.0, tol=1e-13,
                            max_iter=50000)
    assert rho == pytest.approx(8 * sigma / (h * h * chi * Cm), rel=1e-6)


@pytest.mark.parametrize("name,h", [("slab23x9x5_ttp", 0.01), ("square33x29_hh", 1.0 / 64)])
def test_cold_start_estimate_reaches_largest_eigenvalue(name, h):
    """The driver's first estimate (no initial guess) iterates Algorithm 5 to
    the cold-start tolerance 1e-4: rho_F is within 2e-3 below the largest
    eigenvalue of L = -(chi Cm M)^-1 K, which scipy's eigsh gives from the
    symmetric form M^-1/2 K M^-1/2 / (chi Cm).  From the same start vector the
    App. A tolerance 1e-2 stops on an early plateau, more than 3 % low, which
    the safety factor 1.05 does not make up."""
    import scipy.sparse.linalg as sla
    w = make_workload(name, h=h)
    prob = Monodomain.from_workload(w)
    d = 1.0 / np.sqrt(prob.chi * prob.Cm * prob.M)
    S = sp.diags(d) @ prob.K @ sp.diags(d)
    lam = sla.eigsh(S.tocsc(), k=1, which="LA", return_eigenvectors=False, tol=1e-12)[0]
    r = OracleRun(prob, rho_every=0)
    r.update_rho()
    assert lam * (1 - 2e-3) <= r.rhoF_raw <= lam * (1 + 1e-9)
    _, rho_warm_tol, _ = compute_rho(0.0, prob.initial_state()[0], prob.rho_F_fn, start_vector(0, prob.n), 0.0)
    assert rho_warm_tol < 0.97 * lam
    # later calls are warm started: the App. A tolerance, a few iterations
    itF, _ = r.update_rho()
    assert itF <= 3


def test_power_iteration_zero_state_and_vector():
    coords, prob = _line_problem(5, 1.0, NoModel())
    _, rho, it = compute_rho(0.0, np.zeros(5), prob.rho_F_fn, np.zeros(5), 3.0)
    assert rho == 0.0 and it == 0
    _, rho, it = compute_rho(0.0, np.zeros(5), prob.rho_F_fn, start_vector(1, 5), 0.0)
    assert rho > 0.0 and np.isfinite(rho)


def test_start_vector_definition():
    # the scalar and the vectorised branches implement the same definition
    a = start_vector(12345, 4096)
    b = start_vector(12345, 5000)[:4096]
    np.testing.assert_array_equal(a, b)
    assert np.all(a >= -0.5) and np.all(a < 0.5)
    assert abs(a.mean()) < 0.02


def test_activation_times_monotone_on_cable():
    coords, cells = line_mesh(60, 1.5)
    K, M = assemble_p1(coords, cells, isotropic_D(cells.shape[0], 1, 1.0))
    mask = (coords[:, 0] <= 0.1).astype(float)
    prob = Monodomain(K, M, 1400.0, 1.0, make_model(2), mask, 50.0, 0.0, 1.0)
    r = OracleRun(prob, rho_every=1)
    r.run(15.0, 0.02)
    act = r.act
    far = coords[:, 0] > 0.2
    assert np.all(np.isfinite(act[coords[:, 0] < 0.8]))
    a = act[far & np.isfinite(act)]
    assert np.all(np.diff(a) > 0)


def test_imex_rl_first_order_and_exex_agreement():
    w = make_workload("square9x9_hh", h=0.5 / 8)
    prob = Monodomain.from_workload(w)
    T = 3.0
    Yref = rk4_run(prob, prob.initial_state(), T, 1e-3)
    dts = [2.0 ** -i for i in range(4, 9)]
    errs = []
    for dt in dts:
        im = ImexRL(prob, dt)
        Y = prob.initial_state()
        t = 0.0
        for _ in range(int(round(T / dt))):
            Y = im.step(t, Y)
            t += dt
        errs.append(_rel_l2(prob, Y[0], Yref[0]))
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 0.8 <= slope <= 1.25, (errs, slope)
    Y = prob.initial_state()
    t = 0.0
    dt = 1e-3
    for _ in range(int(round(T / dt))):
        Y = exex_rl_step(prob, t, Y, dt)
        t += dt
    assert _rel_l2(prob, Y[0], Yref[0]) < 5e-3


@pytest.mark.parametrize("dt", [0.01, 0.2])
@pytest.mark.parametrize("k", [2, 9])
def test_rl_methods_closed_form_eigenvector(dt, k):
    n, L = 20, 0.19
    h = L / (n - 1)
    chi, Cm, sigma = 1400.0, 1.0, 1.1
    coords, prob = _line_problem(n, L, PassiveModel(), chi, Cm, sigma)
    x = coords[:, 0]
    Y = prob.initial_state()
    Y[0] = np.cos(k * np.pi * x / L)
    Y[1] = 0.8
    Y[2] = -0.6
    pm = PassiveModel()
    lamF = -(4 * sigma / (h * h * chi * Cm)) * np.sin(k * np.pi / (2 * (n - 1))) ** 2
    lamS = -pm.g_p / Cm
    lamE = -(pm.a_w + pm.b_w)
    winf = pm.a_w / (pm.a_w + pm.b_w)
    Ye = exex_rl_step(prob, 0.0, Y, dt)
    Yi = ImexRL(prob, dt).step(0.0, Y)
    np.testing.assert_allclose(Ye[0], (1 + dt * (lamF + lamS)) * Y[0], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Yi[0], (1 + dt * lamS) / (1 - dt * lamF) * Y[0], rtol=1e-12, atol=1e-13)
    for Y1 in (Ye, Yi):
        np.testing.assert_allclose(Y1[1] - winf, math.exp(dt * lamE) * (Y[1] - winf), rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(Y1[2], (1 - dt * pm.k_c) * Y[2], rtol=1e-13, atol=1e-15)


def test_rl_driver_activation_times():
    w = make_workload("square9x9_hh", h=0.5 / 8)
    prob = Monodomain.from_workload(w)
    r = RLRun(prob, "imex", 0.05)
    for _ in range(400):
        r.step()
    a = r.act
    assert np.isfinite(a).all()
    # the stimulated corner activates first, the far corner last, and the
    # activation time grows along the first row and along the diagonal
    d = np.hypot(w.coords[:, 0], w.coords[:, 1])
    assert a[np.argmin(d)] == a.min() and a[np.argmax(d)] == a.max()
    A = a.reshape(9, 9)
    assert np.all(np.diff(A[0, 1:]) > 0) and np.all(np.diff(np.diag(A)) > 0)


@pytest.mark.parametrize("name,h,dt,fixed", [
    ("square9x9_hh", 1.0 / 16, 0.05, (400.0, 60.0)),
    ("slab7x5x4_ttp", 0.01, 0.1, (900.0, 30.0)),
])
def test_progressive_split_equals_algorithm3(name, h, dt, fixed):
    w = make_workload(name, h=h)
    prob = Monodomain.from_workload(w)
    a = OracleRun(prob, fixed_rho=fixed)
    b = OracleRun(prob, fixed_rho=fixed, progressive=True)
    for _ in range(30):
        sa, ma = a.step(dt)
        sb, mb = b.step(dt)
        assert (sa, ma) == (sb, mb)
    assert sa >= 2 and ma >= 2
    scale = np.max(np.abs(a.Y), axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(a.Y - b.Y) / scale) <= 1e-11
    # not vacuous: the exponential step moves the gates of the current state
    yE = prob.exponential_euler(a.Y, 0.01)
    assert np.max(np.abs(yE[1:1 + prob.nE] - a.Y[1:1 + prob.nE])) > 1e-4
