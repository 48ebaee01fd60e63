"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every entry point ``include/spvar.h`` declares, and its host-side
calls (edge list -> CSR, schedule, acceptance table, input validation) agree
with the oracle or return the documented error codes before any device work.
"""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spvar.h")


@pytest.fixture(scope="module")
def L():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_1706_07826_gb300 import build as B
    B.build()
    from paper_1706_07826_gb300 import spvar
    return spvar.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spvar_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("spvar_problem_create", "spvar_sample", "spvar_persistence", "spvar_reduce", "spvar_solve",
                 "spvar_plan_create", "spvar_plan_run", "spvar_thresholds"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_strerror(L):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.spvar_strerror(code)
    assert L.spvar_strerror(-99) == b"unknown error"


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@pytest.mark.parametrize("inst", [I.cubic3d(5, 1), I.chimera(3, 2), I.weak_strong(2, 3), I.random_graph(9, 20, 4)],
                         ids=lambda x: x.name)
def test_csr_from_edges_matches_oracle(L, inst):
    from paper_1706_07826_gb300 import spvar
    rp, col, val = spvar.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J)
    ref = O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h)
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col) and np.array_equal(val, ref.val)


def test_csr_from_edges_rejects_bad_input(L):
    from paper_1706_07826_gb300 import spvar
    with pytest.raises(spvar.SpvarError):
        spvar.csr_from_edges(3, [0], [0], [1])
    with pytest.raises(spvar.SpvarError):
        spvar.csr_from_edges(3, [0, 1], [1, 0], [1, 1])


@pytest.mark.parametrize("T,b0,b1,dmax,scale", [(1000, 0.1, 3.0, 12, 1), (5000, 0.1, 3.0, 24, 1),
                                                (1000, 0.1, 3.0, 1400, 100), (7, 0.5, 0.5, 4, 1)])
def test_schedule_and_table_bit_identical_to_oracle(L, T, b0, b1, dmax, scale):
    from paper_1706_07826_gb300 import spvar
    beta = spvar.beta_geometric(T, b0, b1)
    assert np.array_equal(beta, O.beta_geometric(T, b0, b1))
    assert np.array_equal(spvar.thresholds(beta, dmax, scale), O.thresholds(beta, dmax, scale))


@pytest.mark.parametrize("T,P,beta,g0,g1,dmax,scale", [(200, 8, 3.0, 3.0, 0.01, 12, 1), (100, 16, 5.0, 2.0, 1e-4, 24, 1),
                                                      (50, 2, 1.0, 0.5, 0.5, 1400, 100), (30, 1, 2.0, 1.0, 1.0, 12, 1)])
def test_sqa_table_bit_identical_to_oracle(L, T, P, beta, g0, g1, dmax, scale):
    from paper_1706_07826_gb300 import spvar
    gamma = spvar.gamma_linear(T, g0, g1)
    assert np.array_equal(gamma, O.gamma_linear(T, g0, g1))
    b = np.full(T, beta)
    assert np.array_equal(spvar.sqa_table(T, P, b, gamma, dmax, scale), O.sqa_table(T, P, b, gamma, dmax, scale))


def test_sqa_table_rejects_bad_input(L):
    from paper_1706_07826_gb300 import spvar
    for args in ((10, 3, 1.0, 1.0, 12), (10, 0, 1.0, 1.0, 12), (10, 4, 1.0, 0.0, 12), (10, 4, 1.0, 1.0, -2)):
        with pytest.raises(spvar.SpvarError):
            spvar.sqa_table(*args)


def _create(L, n, rp, col, val, h, offset=0, scale=1):
    out = ctypes.c_void_p()
    rp, col, val, h = (np.ascontiguousarray(x, np.int32) for x in (rp, col, val, h))
    rc = L.spvar_problem_create(n, _ptr(rp), _ptr(col) if col.size else None, _ptr(val) if val.size else None,
                                _ptr(h) if h.size else None, offset, scale, None, ctypes.byref(out))
    return rc


def test_problem_create_validation_errors(L):
    # asymmetric value
    assert _create(L, 2, [0, 1, 2], [1, 0], [1, 2], [0, 0]) == -1
    # missing partner
    assert _create(L, 3, [0, 1, 1, 1], [1], [1], [0, 0, 0]) == -1
    # diagonal entry
    assert _create(L, 2, [0, 1, 1], [0], [1], [0, 0]) == -1
    # columns not ascending
    assert _create(L, 3, [0, 2, 3, 4], [2, 1, 0, 0], [1, 1, 1, 1], [0, 0, 0]) == -1
    # zero-valued coupler
    assert _create(L, 2, [0, 1, 2], [1, 0], [0, 0], [0, 0]) == -1
    # coupler beyond int16
    assert _create(L, 2, [0, 1, 2], [1, 0], [40000, 40000], [0, 0]) == -7
    # energy range beyond the 32-bit arithmetic
    n = 40000
    assert _create(L, n, np.zeros(n + 1), [], [], np.full(n, 30000)) in (-2, -7)
    # bad scale / negative n
    assert _create(L, 2, [0, 1, 2], [1, 0], [1, 1], [0, 0], scale=0) == -1
    assert _create(L, -1, [0], [], [], []) == -1


def test_problem_create_without_device_reports_enomem(L):
    """A valid problem passes host validation; with no CUDA device the device
    allocation fails and the call returns SPVAR_ENOMEM with no handle (the
    allocation-failure path, reached without a GPU)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    inst = I.cubic3d(3, 1)
    from paper_1706_07826_gb300 import spvar
    rp, col, val = spvar.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J)
    out = ctypes.c_void_p(1234)
    h = np.zeros(inst.n, np.int32)
    rc = L.spvar_problem_create(inst.n, _ptr(np.ascontiguousarray(rp, np.int32)),
                                _ptr(np.ascontiguousarray(col, np.int32)), _ptr(np.ascontiguousarray(val, np.int32)),
                                _ptr(h), 0, 1, None, ctypes.byref(out))
    assert rc == -3 and not out.value
