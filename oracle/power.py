"""Nonlinear power iteration for spectral radii (Algorithm 5, App. A).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings where App. A is silent: Euclidean 2-norm; the loop runs at least
once (rho_old starts at 0); at most ``max_iter`` iterations; delta = eps
when ||y|| = 0; rho = 0 when ||v|| = 0.  The safety factor 1.05 is applied
by the caller.  The arbitrary start vector is drawn from SplitMix64 (Steele,
Lea, Flood 2014), written here independently of the CUDA path:
v_i = u01(splitmix64(key xor i)) - 0.5 with u01 = top 53 bits / 2^53.
"""

from __future__ import annotations

import numpy as np

_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def _splitmix64_int(x: int) -> int:
    z = (x + _GOLDEN) & _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def start_vector(key: int, length: int) -> np.ndarray:
    """v_i = u01(splitmix64(key ^ i)) - 0.5 (plain integer arithmetic for small
    lengths, uint64 arrays otherwise; both implement the same definition)."""
    if length <= 4096:
        out = np.empty(length)
        for i in range(length):
            out[i] = (_splitmix64_int((key ^ i) & _MASK) >> 11) * (2.0 ** -53) - 0.5
        return out
    with np.errstate(over="ignore"):
        z = (np.arange(length, dtype=np.uint64) ^ np.uint64(key & _MASK)) + np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 0.5


def compute_rho(t, y, f, v, rho, eps=1e-8, tol=1e-2, max_iter=50):
    """Return (v, rho, iterations) following Algorithm 5 step by step."""
    y = np.asarray(y, dtype=np.float64).ravel()
    v = np.asarray(v, dtype=np.float64).ravel().copy()
    n_y = np.linalg.norm(y)
    n_v = np.linalg.norm(v)
    delta = n_y * eps if n_y > 0.0 else eps
    if n_v == 0.0:
        return v, 0.0, 0
    q = delta / n_v
    rho_old = 0.0
    fy = f(t, y)  # f(t, y) is the same in every iteration
    it = 0
    # rho_old = 0 makes the condition true on entry, so at least one pass
    while abs(rho - rho_old) >= tol * rho and it < max_iter:
        rho_old = rho
        v_old = v
        z = y + q * v_old  # ||z - y|| = delta
        v = f(t, z) - fy
        n_v = np.linalg.norm(v)
        it += 1
        if n_v == 0.0:
            return v, 0.0, it
        q = delta / n_v
        rho = n_v / delta
    return v, rho, it
