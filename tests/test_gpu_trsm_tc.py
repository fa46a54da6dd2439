"""A_p = A R^{-1} with tensor-core updates (lsq_trsm_tc): exact where every
value has an exact digit representation, within the perturbation bound of
two backward-stable solves against the oracle's substitution otherwise, in
place, deterministic, and on sampled rows of the full-size workload."""
import numpy as np
import pytest
import torch

import oracle as O
import problems as P
from tests.gpu_util import dev_colmajor, substitution_perturbation_bound, to_np

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")

U = 2.0 ** -53


def solve_tc(A, R):
    Ap, info = lsq.trsm_tc(dev_colmajor(A), dev_colmajor(R))
    assert int(to_np(info)[0]) == 0
    return to_np(Ap)


def integer_case(m, n, seed):
    """Ap_true integer, R upper with integer off-diagonal entries and a
    power-of-two diagonal, A = Ap_true R exactly: every quantity of the
    recursive solve is a small multiple of 1/2 and exact in FP64."""
    rng = np.random.default_rng(seed)
    Apt = rng.integers(-50, 51, size=(m, n)).astype(np.float64)
    R = np.triu(rng.integers(-3, 4, size=(n, n)).astype(np.float64), 1)
    R[np.arange(n), np.arange(n)] = rng.choice([1.0, -1.0, 2.0, -2.0], size=n)
    A = Apt @ R  # exact: integers far below 2^53
    return A, R, Apt


@pytest.mark.parametrize("m,n", [(1000, 200), (300, 33), (129, 64), (5000, 512), (2000, 700)])
def test_exact_on_exactly_representable_data(m, n):
    A, R, Apt = integer_case(m, n, m + n)
    Ap = solve_tc(A, R)
    np.testing.assert_array_equal(Ap, Apt)


def perturbation_bound(Ap_ref, R, K):
    """Both solves are backward stable: Ap_x R = A + E_x.  The substitution has
    |E| <= n u |Ap| |R|; a digit-sliced update adds per entry at most
    K 2^-50.6 max_k |Ap[i, k]| max_k |R[k, j]|.  So |Ap_tc - Ap_ref| <=
    (|E_tc| + |E_ref|) |R^{-1}|."""
    return substitution_perturbation_bound(Ap_ref, R, K)


@pytest.mark.parametrize("m,n,kappa", [(3000, 200, 1e2), (3000, 200, 1e10), (2500, 600, 1e8)])
def test_within_perturbation_bound_of_oracle(m, n, kappa):
    pr = P.make_problem(m, n, kappa, 0.0, P.seed_for(1, 70 + int(np.log10(kappa))))
    ref = O.solve(pr.A, pr.b, kind=O.SPARSE_SIGN, s=4 * n, zeta=8, seed=4, sketch_prec=O.FP32, qr_prec=O.FP32)
    Rs = ref["Rs"]
    Ap_or = O.trsm_right_upper(pr.A, Rs)
    Ap = solve_tc(pr.A, Rs)
    tol = perturbation_bound(Ap_or, Rs, min(n, 512))
    bad = np.abs(Ap - Ap_or) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], np.abs(Ap - Ap_or).max())
    # and as close to the oracle as the FP64 CUDA-core substitution is
    Ap_cc = fp64_cuda_core_ap(dev_colmajor(pr.A), dev_colmajor(Rs))
    e_tc = np.linalg.norm(Ap - Ap_or)
    e_cc = np.linalg.norm(Ap_cc - Ap_or)
    assert e_tc <= 4 * e_cc + 1e-15 * np.linalg.norm(Ap_or), (e_tc, e_cc)


def fp64_cuda_core_ap(Ad, Rd):
    prev = lsq.set_fp64_emulation(False)
    try:
        b = torch.zeros(Ad.shape[0], dtype=torch.float64, device="cuda")
        Ap, _, _ = lsq.trsm_gram(Ad, Rd, b)
    finally:
        lsq.set_fp64_emulation(prev)
    return to_np(Ap)


def test_in_place_and_deterministic():
    A, R, _ = integer_case(700, 150, 3)
    rng = np.random.default_rng(5)
    A = A + rng.standard_normal(A.shape)  # not exactly representable any more
    Ad = dev_colmajor(A)
    Rd = dev_colmajor(R)
    Ap1, _ = lsq.trsm_tc(Ad, Rd)
    Ap2, _ = lsq.trsm_tc(Ad, Rd)
    B = Ad.clone()
    Ap3, info = lsq.trsm_tc(B, Rd, out=B)
    assert int(to_np(info)[0]) == 0
    a1, a2, a3 = to_np(Ap1), to_np(Ap2), to_np(Ap3)
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(a1, a3)


def test_full_size_sampled_rows():
    # the bench shape (65536 x 1024) plus a ragged tail; rows are independent,
    # so the oracle solves a sample of them
    m, n = 65536 + 77, 1024
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.randn((n, m), dtype=torch.float64, device="cuda", generator=g).t()
    rng = np.random.default_rng(2)
    # an R like a preconditioner's: triangular factor of a random tall matrix
    # with graded columns (kappa ~ 1e6)
    R = np.linalg.qr(rng.standard_normal((2 * n, n)) * np.logspace(0, -6, n)[None, :], mode="r")
    Rd = dev_colmajor(R)
    Ap, info = lsq.trsm_tc(A, Rd)
    assert int(to_np(info)[0]) == 0
    Ap_cc = fp64_cuda_core_ap(A, Rd)
    rows = np.concatenate([np.arange(5), rng.choice(m, 59, replace=False), np.arange(m - 5, m)])
    idx = torch.from_numpy(rows).cuda()
    A_s = to_np(A[idx])
    Ap_s = to_np(Ap[idx])
    Ap_or = O.trsm_right_upper(A_s, R)
    tol = perturbation_bound(Ap_or, R, 512)
    assert np.all(np.abs(Ap_s - Ap_or) <= tol)
    e_tc = np.linalg.norm(Ap_s - Ap_or)
    e_cc = np.linalg.norm(Ap_cc[rows] - Ap_or)
    assert e_tc <= 4 * e_cc + 1e-15 * np.linalg.norm(Ap_or), (e_tc, e_cc)


def test_nonfinite_rows_propagate():
    A, R, _ = integer_case(400, 100, 9)
    A[17, 3] = np.nan
    A[200, 90] = np.inf
    Ap = solve_tc(A, R)
    assert not np.isfinite(Ap[17, 3:]).any()
    assert not np.isfinite(Ap[200, 90:]).any()
    ok = np.ones(400, bool)
    ok[[17, 200]] = False
    assert np.isfinite(Ap[ok]).all()
