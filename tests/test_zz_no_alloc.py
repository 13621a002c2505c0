"""The allocation-free power iteration entry point (emrkc_estimate_rho_F_noalloc).

Some callers cannot allocate device memory while they run (a host whose own
allocator owns the GPU, or a time-critical loop that must not call
cudaMalloc).  For them the library keeps the reduction scratch of the f_F
power iteration in a static device array; this test checks, through the C
ABI, that the variant gives the rho_F and iteration count of
emrkc_estimate_rho on two calls in a row (cold start, then warm start), in
FP64 and in the mixed precision, that it agrees with the oracle's Algorithm
5 from the same start vector, and that it rejects a vector length that does
not match the solver and every method other than emRKC.

It sits in a file of its own that pytest collects last, and it passes both
alone in a fresh process and after the other GPU tests (the first call on a
device performs the scratch set-up).
"""

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from workloads import make_workload, splitmix64, u01

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [pkg.PREC_FP64, pkg.PREC_MIXED])
def test_noalloc_rho_F_matches_estimate_rho(precision):
    """Two calls in a row (cold start, then warm start from the first call's
    iterate and estimate) against emrkc_estimate_rho of an identical solver.
    FP64: the same differences of f_F in the same order, so the same estimate
    to rounding and the same iteration count.  Mixed: emrkc_estimate_rho
    iterates in FP32 (q L v), this variant forms L v in FP32 on FP64 iterates,
    so the estimates agree to the mixed path's 1e-4 and the iteration counts
    to one."""
    import torch

    pkg.build()
    w = make_workload("slab23x9x5_ttp", h=0.01)
    seed = 77
    ref = pkg.Solver.from_workload(w, seed=seed, precision=precision)
    sol = pkg.Solver.from_workload(w, seed=seed, precision=precision)
    # the same start vector as the solver's own: u01(splitmix64(seed ^ i)) - 0.5
    v0 = u01(splitmix64(np.uint64(seed), np.arange(w.n, dtype=np.uint64))) - 0.5
    d_v = torch.tensor(v0, dtype=torch.float64, device="cuda")
    d_w = torch.empty_like(d_v)
    torch.cuda.synchronize()
    rel, dit = (1e-12, 0) if precision == pkg.PREC_FP64 else (1e-4, 1)

    rF1, _, itF1, _ = ref.estimate_rho()
    r1, it1 = sol.estimate_rho_F_noalloc(d_v.data_ptr(), d_w.data_ptr(), w.n, 0.0)
    assert abs(it1 - itF1) <= dit
    assert r1 == pytest.approx(rF1, rel=rel)

    # second call, warm started from the first call's iterate and estimate
    rF2, _, itF2, _ = ref.estimate_rho()
    r2, it2 = sol.estimate_rho_F_noalloc(d_v.data_ptr(), d_w.data_ptr(), w.n, r1)
    assert abs(it2 - itF2) <= dit
    assert r2 == pytest.approx(rF2, rel=rel)
    assert it2 <= 3

    with pytest.raises(pkg.EmrkcError) as ei:
        sol.estimate_rho_F_noalloc(d_v.data_ptr(), d_w.data_ptr(), w.n + 1, 0.0)
    assert ei.value.code == 1
    ref.close()
    sol.close()


@pytest.mark.parametrize("precision", [pkg.PREC_FP64, pkg.PREC_MIXED])
def test_noalloc_rho_F_matches_oracle(precision):
    """The variant against the oracle's Algorithm 5 directly (not only
    through emrkc_estimate_rho): from the same start vector at rest, a cold
    start runs to the cold-start tolerance 1e-4; the estimate agrees with
    the oracle's to 1e-9 in FP64 (the same differences of f_F; the iteration
    counts are equal) and to the mixed path's 1e-4."""
    import torch

    from oracle.emrkc import Monodomain
    from oracle.power import compute_rho, start_vector

    pkg.build()
    w = make_workload("slab23x9x5_ttp", h=0.01)
    seed = 5
    sol = pkg.Solver.from_workload(w, seed=seed, precision=precision)
    v0 = start_vector(seed, w.n)
    d_v = torch.tensor(v0, dtype=torch.float64, device="cuda")
    d_w = torch.empty_like(d_v)
    torch.cuda.synchronize()
    r, it = sol.estimate_rho_F_noalloc(d_v.data_ptr(), d_w.data_ptr(), w.n, 0.0)
    prob = Monodomain.from_workload(w)
    _, ro, ito = compute_rho(0.0, prob.initial_state()[0], prob.rho_F_fn, v0, 0.0, tol=1e-4, max_iter=1000)
    if precision == pkg.PREC_FP64:
        assert it == ito
        assert r == pytest.approx(ro, rel=1e-9)
    else:
        assert abs(it - ito) <= 2
        assert r == pytest.approx(ro, rel=1e-4)
    sol.close()


def test_noalloc_rejects_other_methods():
    """For mRKC the solver's own estimate runs on (V, z_k); the variant, which
    works on V only, refuses every method other than emRKC."""
    import torch

    pkg.build()
    w = make_workload("slab23x9x5_ttp", h=0.01)
    d_v = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    d_w = torch.empty_like(d_v)
    for method in (pkg.METHOD_MRKC, pkg.METHOD_EXEX_RL):
        sol = pkg.Solver.from_workload(w, method=method)
        with pytest.raises(pkg.EmrkcError) as ei:
            sol.estimate_rho_F_noalloc(d_v.data_ptr(), d_w.data_ptr(), w.n, 0.0)
        assert ei.value.code == 1
        sol.close()
