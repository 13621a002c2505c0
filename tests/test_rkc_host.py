"""Algorithm 1 in the library (host routines, no GPU) against the oracle.

emrkc_rkc_stages is the stage count every path of the library takes (the
multiplication form that the device-resident step evaluates); emrkc_rkc_coeffs
gives the coefficients the host builds and tabulates for the device.  Both are
compared with oracle/rkc.py on random arguments.  At the boundaries, where
dt rho equals beta s^2 up to one rounding and the oracle's ceil(sqrt(.)) may
round either way, the stage count is checked against its definition (the
smallest s >= 1 with beta s^2 >= dt rho, evaluated in double precision) by
scanning s upward.  The coefficients are also checked against two identities
of the damped Chebyshev method: c_s = 1 and nu_j + kappa_j = 1 (j >= 2).
"""

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from oracle.rkc import get_coeffs, get_stages


EPS64 = float(np.finfo(np.float64).eps)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _beta(eps):
    return 2.0 - 4.0 * eps / 3.0


def _smallest_stage_count(x, beta):
    """The definition by brute force: first s >= 1 with beta s^2 >= x."""
    s = 1
    while beta * s * s < x:
        s += 1
    return s


@pytest.mark.parametrize("eps", [0.05, 0.1])
def test_stages_match_oracle(eps):
    rng = np.random.default_rng(11)
    dts = 10.0 ** rng.uniform(-4.0, 1.0, 20000)
    rhos = 10.0 ** rng.uniform(-2.0, 5.0, 20000)
    for dt, rho in zip(dts, rhos):
        s, ls = pkg.rkc_stages(dt, rho, eps)
        so, lso = get_stages(dt, rho, eps)
        assert (s, ls) == (so, lso), (dt, rho)


@pytest.mark.parametrize("eps", [0.05, 0.3])
def test_stages_at_the_boundaries(eps):
    beta = _beta(eps)
    for s0 in list(range(1, 400)) + [997, 1000, 2048, 3001]:
        x0 = beta * s0 * s0
        for x in (np.nextafter(x0, 0.0), x0, np.nextafter(x0, np.inf)):
            x = float(x)
            s, ls = pkg.rkc_stages(x, 1.0, eps)
            assert s == _smallest_stage_count(x, beta), (s0, x)
            assert ls == beta * s * s
        # just above the interval of s0 stages needs one more stage
        assert pkg.rkc_stages(float(np.nextafter(x0, np.inf)), 1.0, eps)[0] == s0 + 1


def test_stages_degenerate_arguments():
    beta = _beta(0.05)
    assert pkg.rkc_stages(0.0, 5.0) == (1, beta)
    assert pkg.rkc_stages(0.05, 0.0) == (1, beta)
    assert pkg.rkc_stages(1.0, beta) == (1, beta)
    for args in [(-1.0, 1.0, 0.05), (1.0, -1.0, 0.05), (float("nan"), 1.0, 0.05), (1.0, float("inf"), 0.05),
                 (1.0, 1.0, 1.5), (1.0, 1.0, -0.1), (1e8, 1e8, 0.05)]:
        with pytest.raises(pkg.EmrkcError):
            pkg.rkc_stages(*args)
    lib = pkg.lib()
    assert lib.emrkc_rkc_stages(1.0, 1.0, 0.05, None, None) == 1


@pytest.mark.parametrize("eps", [0.05, 0.1, 0.5])
def test_coeffs_match_oracle(eps):
    for s in list(range(1, 130)) + [200, 500, 1000, 2000]:
        mu, nu, kappa, c = pkg.rkc_coeffs(s, eps)
        muo, nuo, kappao, co, _, _ = get_coeffs(s, eps)
        for name, a, b in (("mu", mu, muo), ("nu", nu, nuo), ("kappa", kappa, kappao), ("c", c, co)):
            np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-14, err_msg=f"{name}, s = {s}")
        assert c[0] == 0.0 and mu[0] == 0.0 and nu[1] == 0.0 and kappa[1] == 0.0
        # c_j follows a three-term recurrence that adds a few roundings per
        # stage, so c_s = 1 holds to a small multiple of s machine epsilons
        assert abs(c[s] - 1.0) <= 32 * s * EPS64, (s, c[s])
        if s >= 2:
            np.testing.assert_allclose(nu[2:] + kappa[2:], 1.0, rtol=0.0, atol=2 * EPS64)


def test_coeffs_invalid_arguments():
    lib = pkg.lib()
    buf = [np.zeros(3) for _ in range(4)]
    ptrs = [b.ctypes.data_as(pkg._ffi.C.POINTER(pkg._ffi.C.c_double)) for b in buf]
    assert lib.emrkc_rkc_coeffs(0, 0.05, *ptrs) == 1
    assert lib.emrkc_rkc_coeffs(2, -0.05, *ptrs) == 1
    assert lib.emrkc_rkc_coeffs(2, float("nan"), *ptrs) == 1
    assert lib.emrkc_rkc_coeffs(2, 0.05, None, *ptrs[1:]) == 1
    assert lib.emrkc_rkc_coeffs((1 << 20) + 1, 0.05, *ptrs) == 1
    assert lib.emrkc_rkc_coeffs(2, 0.05, *ptrs) == 0
