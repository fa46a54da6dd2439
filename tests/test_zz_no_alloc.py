"""lsq_trsm_gram_noalloc: the preconditioning + Gram step for callers that
cannot allocate device memory where they call it (allocator callbacks,
frameworks that own every allocation, loops that must not synchronise on
cudaMalloc).  Its scratch is a fixed per-device array inside the library.

Checked through the C ABI against the oracle (A_p elementwise within the
perturbation bound of two backward-stable substitutions; G and c against the
oracle's sequential sums of the same A_p, elementwise within both sums'
error bounds) and against the workspace entry point lsq_trsm_gram on the same
inputs, on two calls in a row with different shapes and modes (the second
call must not see anything the first left in the shared array), including a
shape whose split-K count has to be cut to fit the fixed array.
This file sorts last so a stop-at-first-failure run has done every other
test first; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
import problems as P
from tests.gpu_util import substitution_perturbation_bound

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")
U64 = 2.0 ** -53


def _noalloc(A, Rs, b, hpne):
    L = lsq.lib()
    f = L.lsq_trsm_gram_noalloc
    f.restype = C.c_int32
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                  C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    m, n = A.shape
    Ap = torch.full((n, m), float("nan"), dtype=torch.float64, device="cuda").t()
    G = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda").t()
    c = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    rc = f(A.data_ptr(), m, n, A.stride(1), Rs.data_ptr(), Rs.stride(1), b.data_ptr(), int(hpne), Ap.data_ptr(), m,
           G.data_ptr(), n, c.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, lsq.status_string(rc)
    torch.cuda.synchronize()
    return Ap.cpu().numpy(), G.cpu().numpy(), c.cpu().numpy()


def _case(m, n, kap, seed):
    pr = P.make_problem(m, n, kap, 1e-6, seed)
    rng = np.random.default_rng(seed)
    R = np.triu(rng.standard_normal((n, n))) * 0.1 + np.diag(1.0 + rng.random(n))
    return (lsq.colmajor(torch.from_numpy(pr.A).cuda()), lsq.colmajor(torch.from_numpy(R).cuda()),
            torch.from_numpy(pr.b).cuda())


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _check_against_oracle(A, R, b, hpne, Ap, G, c, sample_rows=None):
    """A_p: the oracle's substitution on (a sample of) the rows, elementwise
    within the perturbation bound of two backward-stable solves.  G, c: the
    oracle's dot products of the same A_p (and A), elementwise within
    2 gamma_m (|X|^T |Y|): both are FP64 sums of the same m products, in
    different orders."""
    A_np, R_np, b_np = A.cpu().numpy(), R.cpu().numpy(), b.cpu().numpy()
    m = A_np.shape[0]
    rows = np.arange(m) if sample_rows is None else sample_rows
    Ap_or = O.trsm_right_upper(np.asfortranarray(A_np[rows]), R_np)
    tol = substitution_perturbation_bound(Ap_or, R_np)
    bad = np.abs(Ap[rows] - Ap_or) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], (np.abs(Ap[rows] - Ap_or) / tol).max())
    Y = A_np if hpne else Ap
    Go, co = O.gram(np.asfortranarray(Ap), np.asfortranarray(Y), b_np)
    gamma = m * U64 / (1 - m * U64)
    assert np.all(np.abs(G - Go) <= 2 * gamma * (np.abs(Ap).T @ np.abs(Y)))
    assert np.all(np.abs(c - co) <= 2 * gamma * (np.abs(Ap).T @ np.abs(b_np)))


# (m, n, hpne).  120000 x 512 HPNE plans 19 K splits of its Gram, but only 7
# partial 512 x 512 matrices fit beside the GEMV partials in the fixed array:
# the call runs with the K range cut into 7 chunks.
@pytest.mark.parametrize("order", [((5000, 300, False), (70000, 1100, True)), ((70000, 1100, False), (3000, 64, True)),
                                   ((120000, 512, True), (4000, 100, False))])
def test_noalloc_matches_oracle_and_workspace_entry_point(order):
    for (m, n, hpne) in order:
        A, R, b = _case(m, n, 1e3, m + n)
        Ap, G, c = _noalloc(A, R, b, hpne)
        rows = None
        if m > 20000:
            rng = np.random.default_rng(m)
            rows = np.concatenate([np.arange(3), rng.choice(m, 200, replace=False), np.arange(m - 3, m)])
        _check_against_oracle(A, R, b, hpne, Ap, G, c, rows)
        # the workspace entry point with the tensor-core FP64 products switched
        # off runs the same CUDA-core TRSM kernel; the Gram may use fewer K
        # splits (summation order only)
        prev = lsq.set_fp64_emulation(False)
        try:
            Ap_ref, G_ref, c_ref = (t.cpu().numpy() for t in lsq.trsm_gram(A, R, b, hpne=hpne))
        finally:
            lsq.set_fp64_emulation(prev)
        np.testing.assert_array_equal(Ap, Ap_ref)
        assert _rel(G, G_ref) <= 4 * m * U64
        assert _rel(c, c_ref) <= 4 * m * U64
        if not hpne:
            np.testing.assert_array_equal(G, G.T)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = lsq.lib()
    f = L.lsq_trsm_gram_noalloc
    f.restype = C.c_int32
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                  C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    # 8 * ceil(m / 16384) * n bytes of GEMV partials > 16 MiB: rejected before any launch
    m, n = 16384 * 1024, 4096
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    rc = f(p, m, n, m, p, n, p, 0, p, m, p, n, p, torch.cuda.current_stream().cuda_stream)
    assert rc == 1  # LSQ_ERR_ARG
