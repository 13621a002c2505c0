"""Pins of the oracle's P1 assembly and lumped mass (Sec. 2.1, Eq. sd_sys)."""

import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.fem import assemble_p1
from workloads import (axis_D, fibre_D, isotropic_D, line_mesh, shell_tet_mesh,
                       slab_tet_mesh, square_tri_mesh)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_elements():
    out = {}
    with open(os.path.join(GOLDEN, "p1_reference_elements.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            v = np.array([float(x) for x in vals])
            k = int(round(np.sqrt(v.size)))
            out[name] = v.reshape(k, k)
    return out


def test_reference_elements():
    g = _golden_elements()
    K, M = assemble_p1(np.array([[0.0, 0], [1, 0], [0, 1]]), np.array([[0, 1, 2]]), isotropic_D(1, 2, 1.0))
    np.testing.assert_allclose(K.toarray(), g["tri"], atol=1e-15)
    np.testing.assert_allclose(M, np.full(3, 0.5 / 3), rtol=1e-15)
    X = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    K, M = assemble_p1(X, np.array([[0, 1, 2, 3]]), isotropic_D(1, 3, 1.0))
    np.testing.assert_allclose(K.toarray(), g["tet"], atol=1e-15)
    np.testing.assert_allclose(M, np.full(4, 1.0 / 24), rtol=1e-15)


def _k1_m1(n, h):
    """1-D P1 stiffness (1/h) tridiag(-1, 2, -1) with Neumann ends and lumped mass."""
    main = np.full(n, 2.0)
    main[0] = main[-1] = 1.0
    K1 = sp.diags([main, -np.ones(n - 1), -np.ones(n - 1)], [0, 1, -1]) / h
    m = np.full(n, h)
    m[0] = m[-1] = h / 2
    return K1.tocsr(), sp.diags(m)


def test_square_right_diagonal_is_kronecker_five_point():
    nx, ny, h = 9, 7, 0.125
    coords, cells = square_tri_mesh(nx, ny, (nx - 1) * h, (ny - 1) * h)
    K, M = assemble_p1(coords, cells, isotropic_D(cells.shape[0], 2, 1.7))
    Kx, Mx = _k1_m1(nx, h)
    Ky, My = _k1_m1(ny, h)
    # x is the fastest index: kron(y-part, x-part)
    Kref = 1.7 * (sp.kron(My, Kx) + sp.kron(Ky, Mx))
    np.testing.assert_allclose(K.toarray(), Kref.toarray(), atol=1e-13)
    assert M.sum() == pytest.approx((nx - 1) * (ny - 1) * h * h, rel=1e-14)
    # true lumped P1 mass differs from the Kronecker mass only at corners
    Mk = sp.kron(My, Mx).diagonal()
    diff = np.nonzero(np.abs(M - Mk) > 1e-15)[0]
    corners = {0, nx - 1, nx * (ny - 1), nx * ny - 1}
    assert set(diff.tolist()) <= corners


def test_slab_kuhn_with_diagonal_D_is_seven_point():
    """Kuhn tets are path simplices with orthogonal edges, so with diagonal D
    only axis neighbours couple (7-point).  Interior rows equal the
    Kronecker 7-point stencil; boundary weights depend on how many Kuhn tets
    share an edge, so they are pinned by the energy of linear functions."""
    nx, ny, nz, h = 6, 5, 4, 0.5
    coords, cells = slab_tet_mesh(nx, ny, nz, (nx - 1) * h, (ny - 1) * h, (nz - 1) * h)
    sig = (1.33, 0.18, 0.11)
    K, M = assemble_p1(coords, cells, axis_D(cells.shape[0], sig))
    Kx, Mx = _k1_m1(nx, h)
    Ky, My = _k1_m1(ny, h)
    Kz, Mz = _k1_m1(nz, h)
    Kref = (sig[0] * sp.kron(Mz, sp.kron(My, Kx)) + sig[1] * sp.kron(Mz, sp.kron(Ky, Mx))
            + sig[2] * sp.kron(Kz, sp.kron(My, Mx))).toarray()
    Kd = K.toarray()
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    idx = (k * ny + j) * nx + i
    interior = ((i > 0) & (i < nx - 1) & (j > 0) & (j < ny - 1) & (k > 0) & (k < nz - 1))
    rows = idx[interior]
    np.testing.assert_allclose(Kd[rows], Kref[rows], atol=1e-14)
    # sparsity: nonzeros only on axis neighbours
    nb = np.abs(Kref) > 0
    assert np.all(np.abs(Kd[~nb]) <= 1e-14)
    assert np.max(np.abs(Kd.sum(axis=1))) <= 1e-14
    assert M.sum() == pytest.approx((nx - 1) * (ny - 1) * (nz - 1) * h ** 3, rel=1e-13)
    vol = (nx - 1) * (ny - 1) * (nz - 1) * h ** 3
    for a in range(3):
        V = coords[:, a]
        assert V @ (K @ V) == pytest.approx(sig[a] * vol, rel=1e-12)


def test_line_mesh():
    coords, cells = line_mesh(6, 1.0)
    K, M = assemble_p1(coords, cells, isotropic_D(cells.shape[0], 1, 2.0))
    Kref, Mref = _k1_m1(6, 0.2)
    np.testing.assert_allclose(K.toarray(), 2.0 * Kref.toarray(), atol=1e-13)
    np.testing.assert_allclose(M, Mref.diagonal(), rtol=1e-14)


@pytest.fixture(scope="module")
def small_shell():
    coords, cells = shell_tet_mesh(4, 9, seed=5)
    rng = np.random.default_rng(3)
    a = rng.normal(size=(cells.shape[0], 3))
    D = fibre_D(a, 1.33, 0.18)
    K, M = assemble_p1(coords, cells, D)
    return coords, cells, D, K, M


def test_shell_symmetric_and_row_sums_zero(small_shell):
    coords, cells, D, K, M = small_shell
    assert abs(K - K.T).max() <= 1e-14 * abs(K).max()
    assert np.max(np.abs(K @ np.ones(K.shape[0]))) <= 1e-13 * abs(K).max()
    assert np.all(M > 0)


def test_shell_energy_of_linear_functions(small_shell):
    # P1 reproduces linear functions exactly: V = x gives V^T K V = sum_T |T| D_xx(T)
    coords, cells, D, K, M = small_shell
    P = coords[cells]
    vol = np.abs(np.einsum("ij,ij->i", P[:, 1] - P[:, 0],
                           np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6.0
    for a in range(3):
        V = coords[:, a]
        assert V @ (K @ V) == pytest.approx(np.sum(vol * D[:, a, a]), rel=1e-11)
    assert M.sum() == pytest.approx(vol.sum(), rel=1e-13)
    # mixed direction: V = x + 2y gives sum |T| (D_xx + 4 D_xy + 4 D_yy)
    V = coords[:, 0] + 2.0 * coords[:, 1]
    ref = np.sum(vol * (D[:, 0, 0] + 4 * D[:, 0, 1] + 4 * D[:, 1, 1]))
    assert V @ (K @ V) == pytest.approx(ref, rel=1e-11)
