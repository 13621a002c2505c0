"""Host-side checks of the C-ABI library (no GPU needed).

* the library builds and exports every function include/emrkc.h declares;
* the host P1 assembler agrees with the oracle's independent assembly;
* creating a solver without a CUDA device fails loudly (no CPU fallback).
"""

import os
import re

import numpy as np
import pytest

import paper_2401_01745_gb300 as pkg
from oracle.fem import assemble_p1 as oracle_assemble
from workloads import fibre_D, make_workload, shell_tet_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.lib()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(emrkc_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_model_sizes(lib):
    assert [pkg.num_vars(m) for m in range(4)] == [1, 3, 4, 19]
    assert [pkg.num_gates(m) for m in range(4)] == [0, 1, 3, 12]
    assert pkg.num_vars(7) == -1


def test_default_options(lib):
    o = pkg.default_options()
    assert o.eps == 0.05 and o.safety == 1.05 and o.pow_tol == 1e-2 and o.pow_eps == 1e-8
    assert o.rho_every == 1 and o.precision == 0 and o.act_threshold == -20.0
    assert o.method == 0 and o.lin_rtol == 1e-10 and o.lin_max_iter == 1000


def _csr_dense(rp, col, K, n):
    A = np.zeros((n, n))
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            A[i, col[p]] += K[p]
    return A


@pytest.mark.parametrize("name", ["square9x7_hh", "slab6x5x4_ttp", "line12_hh"])
def test_assembly_matches_oracle_structured(lib, name):
    w = make_workload(name)
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    Ko, Mo = oracle_assemble(w.coords, w.cells, w.D)
    np.testing.assert_allclose(_csr_dense(rp, col, K, w.n), Ko.toarray(), rtol=0, atol=1e-13 * abs(Ko).max())
    np.testing.assert_allclose(M, Mo, rtol=1e-14)
    for i in range(w.n):  # sorted, unique columns per row
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_assembly_matches_oracle_shell(lib):
    coords, cells = shell_tet_mesh(4, 8, seed=9)
    rng = np.random.default_rng(2)
    D = fibre_D(rng.normal(size=(cells.shape[0], 3)), 1.33, 0.18)
    rp, col, K, M = pkg.assemble_p1(coords, cells, D)
    Ko, Mo = oracle_assemble(coords, cells, D)
    n = coords.shape[0]
    np.testing.assert_allclose(_csr_dense(rp, col, K, n), Ko.toarray(), rtol=0, atol=1e-13 * abs(Ko).max())
    np.testing.assert_allclose(M, Mo, rtol=1e-13)


def test_assembly_rejects_bad_input(lib):
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]])
    with pytest.raises(pkg.EmrkcError):  # zero-area triangle
        pkg.assemble_p1(coords, np.array([[0, 1, 2]]), np.tile(np.eye(2), (1, 1, 1)))
    with pytest.raises(pkg.EmrkcError):  # index out of range
        pkg.assemble_p1(coords, np.array([[0, 1, 5]]), np.tile(np.eye(2), (1, 1, 1)))


def test_create_without_gpu_fails_loudly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    w = make_workload("square5x5_hh")
    with pytest.raises(pkg.EmrkcError) as ei:
        pkg.Solver.from_workload(w)
    assert ei.value.code == 2  # EMRKC_ERR_CUDA


def test_create_validates_arguments(lib):
    w = make_workload("square5x5_hh")
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    bad = col.copy()
    bad[3] = w.n + 7
    with pytest.raises(pkg.EmrkcError) as ei:
        pkg.Solver(rp, bad, K, M)
    assert ei.value.code == 1
    with pytest.raises(pkg.EmrkcError) as ei:
        pkg.Solver(rp, col, K, -M)
    assert ei.value.code == 1
    with pytest.raises(pkg.EmrkcError) as ei:
        pkg.Solver(rp, col, K, M, model=9)
    assert ei.value.code == 1
    with pytest.raises(pkg.EmrkcError) as ei:  # unknown time integrator
        pkg.Solver(rp, col, K, M, method=7)
    assert ei.value.code == 1
    for method in (pkg.METHOD_EXEX_RL, pkg.METHOD_IMEX_RL, pkg.METHOD_MRKC):  # FP64 only
        with pytest.raises(pkg.EmrkcError) as ei:
            pkg.Solver(rp, col, K, M, method=method, precision=pkg.PREC_MIXED)
        assert ei.value.code == 1
    with pytest.raises(pkg.EmrkcError) as ei:
        pkg.Solver(rp, col, K, M, method=pkg.METHOD_IMEX_RL, lin_max_iter=-1)
    assert ei.value.code == 1


def _raw_create(lib, n, rp, col, K, M):
    import ctypes as C

    from paper_2401_01745_gb300._ffi import Matrix, Tissue

    mat = Matrix(n, K.size, rp.ctypes.data_as(C.POINTER(C.c_int64)), col.ctypes.data_as(C.POINTER(C.c_int32)),
                 K.ctypes.data_as(C.POINTER(C.c_double)), M.ctypes.data_as(C.POINTER(C.c_double)))
    h = C.c_void_p()
    rc = lib.emrkc_create(C.byref(mat), C.byref(Tissue(1400.0, 1.0)), 2, None, None, C.byref(h))
    return rc, lib.emrkc_last_error(None).decode()


def test_create_edge_cases_rejected_on_host(lib):
    """Degenerate and out-of-range matrices are rejected before any device
    work: no nodes, a row pointer that does not end at nnz or is not
    monotone, a non-finite entry, and more rows than int32 columns address
    (checked before the row pointer is read)."""
    w = make_workload("square5x5_hh")
    rp, col, K, M = pkg.assemble_p1(w.coords, w.cells, w.D)
    rc, msg = _raw_create(lib, 0, rp, col, K, M)
    assert rc == 1 and "size" in msg
    bad = rp.copy()
    bad[-1] += 1
    rc, msg = _raw_create(lib, w.n, bad, col, K, M)
    assert rc == 1 and "row_ptr" in msg
    bad = rp.copy()
    bad[3], bad[4] = bad[4], bad[3]
    rc, msg = _raw_create(lib, w.n, bad, col, K, M)
    assert rc == 1
    Kn = K.copy()
    Kn[5] = np.nan
    rc, msg = _raw_create(lib, w.n, rp, col, Kn, M)
    assert rc == 1 and "non-finite" in msg
    rc, msg = _raw_create(lib, 2 ** 31, rp, col, K, M)
    assert rc == 1 and "rows" in msg
