"""The allocation-free power iteration entry point (emrkc_estimate_rho_F_noalloc).

Some callers cannot allocate device memory while they run (a host whose own
allocator owns the GPU, or a time-critical loop that must not call
cudaMalloc).  For them the library keeps the reduction scratch of the f_F
power iteration in a static device array; this test checks, through the C
ABI, that the variant gives the same rho_F and iteration count as
emrkc_estimate_rho on two calls in a row (cold start, then warm start), and
that it rejects a vector length that does not match the solver.

It sits in a file of its own that pytest collects last, and it passes both
alone in a fresh process and after the other GPU tests (the first call on a
device performs the scratch set-up).
"""

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from workloads import make_workload, splitmix64, u01

pytestmark = pytest.mark.gpu


def test_noalloc_rho_F_matches_estimate_rho():
    import torch

    pkg.build()
    w = make_workload("slab23x9x5_ttp", h=0.01)
    seed = 77
    ref = pkg.Solver.from_workload(w, seed=seed)
    sol = pkg.Solver.from_workload(w, seed=seed)
    # the same start vector as the solver's own: u01(splitmix64(seed ^ i)) - 0.5
    v0 = u01(splitmix64(np.uint64(seed), np.arange(w.n, dtype=np.uint64))) - 0.5
    d_v = torch.tensor(v0, dtype=torch.float64, device="cuda")
    d_w = torch.empty_like(d_v)
    torch.cuda.synchronize()

    rF1, _, itF1, _ = ref.estimate_rho()
    r1, it1 = sol.estimate_rho_F_noalloc(d_v.data_ptr(), d_w.data_ptr(), w.n, 0.0)
    assert it1 == itF1
    assert r1 == pytest.approx(rF1, rel=1e-12)

    # second call, warm started from the first call's iterate and estimate
    rF2, _, itF2, _ = ref.estimate_rho()
    r2, it2 = sol.estimate_rho_F_noalloc(d_v.data_ptr(), d_w.data_ptr(), w.n, r1)
    assert it2 == itF2
    assert r2 == pytest.approx(rF2, rel=1e-12)
    assert it2 <= 3

    with pytest.raises(pkg.EmrkcError) as ei:
        sol.estimate_rho_F_noalloc(d_v.data_ptr(), d_w.data_ptr(), w.n + 1, 0.0)
    assert ei.value.code == 1
    ref.close()
    sol.close()
