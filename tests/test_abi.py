"""The C-ABI library loads (no GPU needed) and exports every symbol that
include/lsq.h declares; host-only entry points answer without a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def liblsq():
    from paper_2603_16644_gb300 import _build

    path = _build.build()
    return C.CDLL(path)


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "lsq.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lsq_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for need in ["lsq_sketch", "lsq_precond_qr", "lsq_condest", "lsq_pne_solve", "lsq_hpne_solve",
                 "lsq_workspace_size", "lsq_trsm_gram", "lsq_factor_solve", "lsq_pne_solve_host"]:
        assert need in syms


def test_every_declared_symbol_is_exported(liblsq):
    missing = [s for s in declared_symbols() if not hasattr(liblsq, s)]
    assert not missing, missing


def test_host_only_calls(liblsq):
    liblsq.lsq_precision_from_kappa0.restype = C.c_int32
    liblsq.lsq_precision_from_kappa0.argtypes = [C.c_double]
    f = liblsq.lsq_precision_from_kappa0
    assert [f(1.0), f(2.5), f(3.5), f(6.0), f(8.0), f(9.0), f(float("inf")), f(float("nan"))] == [0, 1, 2, 3, 3, 4, 4, 4]
    liblsq.lsq_status_string.restype = C.c_char_p
    assert liblsq.lsq_status_string(0) == b"LSQ_OK"
    assert liblsq.lsq_version() >= 100
    # test-only wait bound of the triangular solves: host state only
    liblsq.lsq_test_set_solve_wait_ns.restype = C.c_int64
    liblsq.lsq_test_set_solve_wait_ns.argtypes = [C.c_int64]
    s = liblsq.lsq_test_set_solve_wait_ns
    assert s(0) == -1 and s(-5) == -1
    old = s(1000)
    assert old == 2_000_000_000
    assert s(old) == 1000


def test_binding_matches_oracle_precision_table(liblsq):
    import oracle as O
    import paper_2603_16644_gb300 as lsq

    for k in [-1.0, 0.0, 1.99, 2.0, 2.99, 3.0, 3.99, 4.0, 7.5, 8.0, 8.0000001, 12.0, float("inf")]:
        assert lsq.precision_from_kappa0(k) == O.precision_from_kappa0(k)


def test_calls_fail_loudly_without_cuda_tensors(liblsq):
    import torch

    import paper_2603_16644_gb300 as lsq

    A = torch.zeros((10, 3), dtype=torch.float64)
    with pytest.raises(lsq.LsqError):
        lsq.pne(A, torch.zeros(10, dtype=torch.float64))
