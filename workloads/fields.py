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


def smooth_random_field(points, seed: int, corr_len: float, n_modes: int = 64):
    """Seeded, spatially correlated random field on ``points`` (n, dim),
    mapped to [0, 1] by its empirical quantile (rank / (n - 1)).

    The field is a random Fourier series: sum over n_modes of
    cos(2 pi k_j . x + phase_j) with wave vectors k_j drawn from a normal
    distribution of standard deviation 1 / (2 pi corr_len) per axis (a
    Gaussian spectral density, so the covariance decays like
    exp(-|x - y|^2 / (2 corr_len^2))) and phases uniform in [0, 2 pi).  Draws
    come from SplitMix64 on (seed, mode, component); normal variates by the
    Box-Muller transform.  (The paper generates its fibrosis field by solving
    a stochastic PDE; this field has the same role: a smooth, seeded pattern
    whose median splits the tissue in two.)
    """
    pts = np.asarray(points, dtype=np.float64)
    if pts.ndim == 1:
        pts = pts[:, None]
    n, dim = pts.shape
    j = np.arange(n_modes, dtype=np.uint64)
    acc = np.zeros(n)
    ks = np.zeros((n_modes, dim))
    for a in range(dim):
        u1 = u01(splitmix64(np.uint64(seed), j * np.uint64(16) + np.uint64(2 * a)))
        u2 = u01(splitmix64(np.uint64(seed), j * np.uint64(16) + np.uint64(2 * a + 1)))
        ks[:, a] = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2) / (2.0 * np.pi * corr_len)
    phase = 2.0 * np.pi * u01(splitmix64(np.uint64(seed), j * np.uint64(16) + np.uint64(15)))
    for m in range(n_modes):
        acc += np.cos(2.0 * np.pi * (pts @ ks[m]) + phase[m])
    order = np.argsort(acc, kind="stable")
    rank = np.empty(n)
    rank[order] = np.arange(n)
    return rank / max(n - 1, 1)


def fibrosis_D(coords, cells, a_l, sigma_l: float, sigma_t: float, seed: int, corr_len: float,
               quantile: float = 0.5):
    """Transversely isotropic D with fibrosis (Sec. 5.4 with fibrosis): sigma_t
    = 0 in every cell whose centroid value of the random field exceeds the
    given quantile (the median by default), decoupling cells across fibres.
    Returns (D, fibrotic cell mask)."""
    cent = np.asarray(coords)[np.asarray(cells)].mean(axis=1)
    u = smooth_random_field(cent, seed, corr_len)
    fib = u > quantile
    D_h = fibre_D(a_l, sigma_l, sigma_t)
    D_f = fibre_D(a_l, sigma_l, 0.0)
    D = np.where(fib[:, None, None], D_f, D_h)
    return D, fib
