"""Conductivity tensors, stimulus masks and the counter-based generator.

``splitmix64`` is the SplitMix64 output function of Steele, Lea and Flood
(OOPSLA 2014): add the golden-ratio increment 0x9E3779B97F4A7C15, then two
xor-shift-multiply rounds with 0xBF58476D1CE4E5B9 and 0x94D049BB133111EB
and a final xor-shift.  ``u01`` maps the top 53 bits to [0, 1).
"""

from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(key, counter):
    """SplitMix64 of (key xor counter); vectorised over ``counter``."""
    with np.errstate(over="ignore"):
        z = (np.asarray(counter, dtype=np.uint64) ^ np.uint64(key)) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def u01(bits):
    """Top 53 bits of a uint64 as a double in [0, 1)."""
    return (np.asarray(bits, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def harmonic_sigma(sig_i: float, sig_e: float) -> float:
    """Bulk conductivity sigma = sigma_i sigma_e / (sigma_i + sigma_e) (Eq. def_D)."""
    return sig_i * sig_e / (sig_i + sig_e)


def isotropic_D(n_cells: int, dim: int, sigma: float):
    """Per-cell D = sigma I, shape (n_cells, dim, dim)."""
    D = np.zeros((n_cells, dim, dim))
    for a in range(dim):
        D[:, a, a] = sigma
    return D


def axis_D(n_cells: int, sigmas):
    """Per-cell diagonal D = diag(sigmas): fibres along x (Eq. def_D with a_l = e_x)."""
    sigmas = np.asarray(sigmas, dtype=np.float64)
    dim = sigmas.size
    D = np.zeros((n_cells, dim, dim))
    for a in range(dim):
        D[:, a, a] = sigmas[a]
    return D


def fibre_D(a_l, sigma_l: float, sigma_t: float):
    """Transversely isotropic D = sigma_t I + (sigma_l - sigma_t) a_l a_l^T.

    This is Eq. (def_D) with sigma_n = sigma_t, for unit fibre vectors a_l of
    shape (n_cells, dim).
    """
    a_l = np.asarray(a_l, dtype=np.float64)
    a_l = a_l / np.linalg.norm(a_l, axis=1, keepdims=True)
    dim = a_l.shape[1]
    return sigma_t * np.eye(dim)[None] + (sigma_l - sigma_t) * a_l[:, :, None] * a_l[:, None, :]


def corner_mask(coords, size: float, tol: float = 1e-9):
    """Nodes with every coordinate <= size (inclusive): the corner stimulus region."""
    return np.all(coords <= size + tol, axis=1).astype(np.uint8)


def radius_mask(coords, centre, radius: float, tol: float = 1e-9):
    """Nodes within ``radius`` of ``centre`` (inclusive)."""
    d = np.linalg.norm(coords - np.asarray(centre)[None, :], axis=1)
    return (d <= radius + tol).astype(np.uint8)
