"""P1 finite elements with mass lumping (Sec. 2.1, Eq. sd_sys).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

K_ij = sum_T int_T D grad(phi_j) . grad(phi_i)   (so the paper's A = -K,
       which makes f_F = (chi Cm M)^-1 A V dissipative)
M_ii = sum_T |T| / (dim + 1)                       (row-sum lumped mass)
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def assemble_p1(coords, cells, D):
    """Return (K as scipy CSR, lumped mass diagonal) for simplices of any dim.

    coords: (n, d) float64; cells: (nc, d+1) int; D: (nc, d, d) per-cell tensor.
    """
    coords = np.asarray(coords, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    n, d = coords.shape
    nc = cells.shape[0]
    P = coords[cells]  # (nc, d+1, d)
    J = np.transpose(P[:, 1:, :] - P[:, :1, :], (0, 2, 1))  # columns = edge vectors
    det = np.linalg.det(J)
    vol = np.abs(det) / math.factorial(d)
    Jinv = np.linalg.inv(J)  # row k = grad of barycentric coordinate k+1
    G = np.empty((nc, d + 1, d))
    G[:, 1:, :] = Jinv
    G[:, 0, :] = -Jinv.sum(axis=1)
    # element stiffness: vol * G D G^T
    Kloc = vol[:, None, None] * np.einsum("cad,cde,cbe->cab", G, D, G)
    rows = np.repeat(cells, d + 1, axis=1).ravel()
    cols = np.tile(cells, (1, d + 1)).ravel()
    K = sp.coo_matrix((Kloc.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    K.sum_duplicates()
    M = np.zeros(n)
    np.add.at(M, cells.ravel(), np.repeat(vol / (d + 1), d + 1))
    return K, M
