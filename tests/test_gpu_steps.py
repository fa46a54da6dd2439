"""Step-by-step parity of the CUDA path with the oracle (Alg. 1 steps).

Integer and index work is compared bit for bit (sparse-sign operator,
sparse-sign sketches, column exponents, pivots, breakdown indices); floating
point within tolerances derived from the arithmetic of each step.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import oracle as O
import problems as P
from tests.gpu_util import dev_colmajor, to_np

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")
U32 = 2.0 ** -24
U64 = 2.0 ** -53


@pytest.mark.parametrize("m,s,zeta,seed", [(1000, 200, 8, 5), (777, 31, 5, 3), (50, 8, 8, 1), (65536, 4096, 8, 2603),
                                           (3, 1, 1, 9)])
def test_sparse_sign_operator_bit_exact(m, s, zeta, seed):
    idx, sgn = lsq.sparse_sign_operator(seed, m, s, zeta)
    oi, os_ = O.sparse_sign_indices(seed, m, s, zeta)
    np.testing.assert_array_equal(to_np(idx), oi)
    np.testing.assert_array_equal(to_np(sgn), os_)


@pytest.mark.parametrize("prec", [O.FP8_E4M3, O.BF16, O.FP16, O.FP32, O.FP64])
def test_gaussian_operator(prec):
    """The ziggurat's proposals and its wedge test are IEEE products, sums and
    comparisons against the same tables, the grid rounding is exact: bit-exact.
    Only the tail (|z| > r, 0.026 % of the entries) goes through log, which
    differs by an ulp between libm and CUDA and can move an entry by one grid
    step (2^-17) next to a grid tie."""
    s, m, seed = 64, 3001, 77
    g = to_np(lsq.gaussian_operator(seed, s, m, prec))
    o = O.gaussian_operator(seed, s, m, prec)
    x, _ = O.zig_tables()
    tail = np.abs(O.gaussian_operator(seed, s, m, O.FP64)) > x[1]
    assert 10 < tail.sum() < 120, tail.sum()
    np.testing.assert_array_equal(g[~tail], o[~tail])
    gt, ot = g[tail], o[tail]
    neq = gt != ot
    assert neq.sum() <= 2
    if neq.any():
        p = {O.FP8_E4M3: 4, O.BF16: 8, O.FP16: 11, O.FP32: 24, O.FP64: 53}[prec]
        # a last-bit FP64 difference moves the grid value by one step, or
        # flips a rounding to the format, only next to a tie: neighbours
        step = np.maximum(2.0 ** -17, 2.0 ** (1 - p) * np.abs(ot[neq]))
        assert np.all(np.abs(gt[neq] - ot[neq]) <= 1.01 * step)


@pytest.mark.parametrize("prec", [O.FP8_E4M3, O.BF16, O.FP16, O.FP32, O.FP64])
@pytest.mark.parametrize("m,n,s,zeta", [(1037, 113, 300, 8), (2048, 64, 128, 4), (129, 65, 65, 3)])
def test_sparse_sketch_bit_exact(prec, m, n, s, zeta):
    rng = np.random.default_rng(m + n)
    A = np.asfortranarray(rng.standard_normal((m, n)) * np.exp2(rng.integers(-20, 20, n))[None, :])
    opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=s, zeta=zeta, seed=42, sketch_prec=prec)
    As, ce, info = lsq.sketch(dev_colmajor(A), opts)
    oAs, oce = O.sketch(A, O.SPARSE_SIGN, s, zeta, 42, prec)
    assert int(to_np(info)[0]) == 0
    np.testing.assert_array_equal(to_np(ce), oce)
    np.testing.assert_array_equal(to_np(As).astype(np.float64), oAs)


def test_sparse_sketch_full_size_bit_exact():
    # the 65536 x 1024, s = 4096, zeta = 8, BF16 sketch of the tall-skinny workload
    m, n, s = 65536, 1024, 4096
    rng = np.random.default_rng(7)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=s, zeta=8, seed=P.seed_for(1, 0), sketch_prec=lsq.BF16)
    As, ce, info = lsq.sketch(dev_colmajor(A), opts)
    oAs, oce = O.sketch(A, O.SPARSE_SIGN, s, 8, P.seed_for(1, 0), O.BF16)
    assert int(to_np(info)[0]) == 0
    np.testing.assert_array_equal(to_np(ce), oce)
    np.testing.assert_array_equal(to_np(As).astype(np.float64), oAs)


@pytest.mark.parametrize("prec", [O.FP8_E4M3, O.BF16, O.FP16, O.FP32, O.FP64])
@pytest.mark.parametrize("m,n,s", [(1037, 113, 300), (4096, 64, 192), (20011, 40, 120), (3, 2, 2)])
def test_srft_sketch_bit_exact(prec, m, n, s):
    # the butterflies of F are evaluated as in the oracle's sequential sweep
    # (levels in order, every pair the same sum and difference), the signs and
    # the sampled rows come from the same Philox words: bit for bit
    rng = np.random.default_rng(m + 3 * n)
    A = np.asfortranarray(rng.standard_normal((m, n)) * np.exp2(rng.integers(-20, 20, n))[None, :])
    opts = lsq.make_opts(kind=lsq.SRFT, s=s, zeta=0, seed=77, sketch_prec=prec)
    As, ce, info = lsq.sketch(dev_colmajor(A), opts)
    oAs, oce = O.sketch(A, O.SRFT, s, 0, 77, prec)
    assert int(to_np(info)[0]) == 0
    np.testing.assert_array_equal(to_np(ce), oce)
    np.testing.assert_array_equal(to_np(As).astype(np.float64), oAs)


@pytest.mark.parametrize("prec", [O.FP8_E4M3, O.BF16, O.FP16, O.FP32, O.FP64])
def test_gaussian_sketch_within_rounding(prec):
    m, n, s = 1037, 113, 250
    rng = np.random.default_rng(3)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    opts = lsq.make_opts(kind=lsq.GAUSSIAN, s=s, seed=9, sketch_prec=prec)
    As, ce, _ = lsq.sketch(dev_colmajor(A), opts)
    oAs, oce = O.sketch(A, O.GAUSSIAN, s, 0, 9, prec)
    np.testing.assert_array_equal(to_np(ce), oce)
    Om = O.gaussian_operator(9, s, m, prec)
    Ah = O.quantize(A, prec, oce)
    scale = np.abs(Om) @ np.abs(Ah)
    u = U64 if prec == O.FP64 else U32
    # both sums carry at most (m-1) u sum|terms|; operator entries may differ next to ties
    tol = 2 * m * u * scale + 2 ** -7 * np.abs(Ah).max() * 4
    if prec == O.FP64:
        # the FP64 sketch is a sum of K chunks of 1024 digit-sliced products,
        # each accurate to 1024 2^-50.6 2^3 max|A_chunk,c| (Omega sliced with
        # the fixed exponent 2^3 > |Omega|)
        dig = sum(1024 * 2.0 ** -50.6 * 8.0 * np.outer(np.ones(s), np.abs(Ah[k:k + 1024, :]).max(axis=0))
                  for k in range(0, m, 1024))
        tol = tol + dig
    assert np.all(np.abs(to_np(As) - oAs) <= tol)


@pytest.mark.parametrize("qr_prec", [O.FP32, O.FP64])
@pytest.mark.parametrize("s,n", [(300, 113), (256, 256), (4096, 200), (65, 1), (1000, 300), (1500, 600),
                                 (3000, 1030)])
def test_precond_qr(qr_prec, s, n):
    # FP64 with n > 256: blocks of 256 columns whose reflectors update the
    # later columns by digit-sliced tensor-core products (ragged last block)
    rng = np.random.default_rng(s + n)
    As = np.asfortranarray(rng.standard_normal((s, n)) @ np.diag(np.logspace(0, -2, n)))
    if qr_prec == O.FP32:
        As = O.round_to(As, O.FP32).reshape(As.shape, order="F")
    dt = torch.float32 if qr_prec == O.FP32 else torch.float64
    Ast = torch.from_numpy(np.ascontiguousarray(As.T)).cuda().to(dt).t()
    e = np.arange(n, dtype=np.int32) % 5 - 2
    R, info = lsq.precond_qr(Ast, torch.from_numpy(e).cuda(), qr_prec)
    R = to_np(R)
    assert int(to_np(info)[0]) == 0
    Ro = O.unscale_r(O.qr_r(As, qr_prec), e)
    assert np.all(np.diag(R) > 0) and np.all(np.tril(R, -1) == 0)
    u = U32 if qr_prec == O.FP32 else U64
    kap = O.kappa(As)
    # unique R with positive diagonal: both are backward-stable approximations of it
    Rc = np.linalg.cholesky(As.T @ As).T * np.exp2(-e)[None, :]
    dg = np.linalg.norm(R - Rc) / np.linalg.norm(Rc)
    do = np.linalg.norm(Ro - Rc) / np.linalg.norm(Rc)
    assert dg <= max(4 * do, 20 * n * u * kap), (dg, do)
    Ru = R * np.exp2(e)[None, :]
    assert np.linalg.norm(Ru.T @ Ru - As.T @ As) / np.linalg.norm(As) ** 2 <= 20 * s * u


def test_precond_qr_zero_column_reports_breakdown():
    s, n = 100, 10
    rng = np.random.default_rng(1)
    As = rng.standard_normal((s, n))
    As[:, 4] = 0.0
    Ast = torch.from_numpy(np.ascontiguousarray(As.T)).cuda().float().t()
    R, info = lsq.precond_qr(Ast, None, O.FP32)
    assert int(to_np(info)[0]) == 5


@pytest.mark.parametrize("hpne", [False, True])
@pytest.mark.parametrize("m,n,kap", [(1037, 113, 1e6), (3000, 200, 1e3), (500, 64, 1e8), (70, 1, 1.0)])
def test_trsm_gram(hpne, m, n, kap):
    pr = P.make_problem(m, n, kap, 1e-6, 1234)
    As, e = O.sketch(pr.A, O.SPARSE_SIGN, max(2 * n, 2), min(8, max(2 * n, 2)), 5, O.FP32)
    Rs = O.unscale_r(O.qr_r(As, O.FP32), e)
    Ap_o = O.trsm_right_upper(pr.A, Rs)
    G_o, c_o = O.gram(Ap_o, pr.A if hpne else Ap_o, pr.b)
    Ap, G, c = lsq.trsm_gram(dev_colmajor(pr.A), dev_colmajor(Rs), torch.from_numpy(pr.b).cuda(), hpne=hpne)
    Ap, G, c = to_np(Ap), to_np(G), to_np(c)
    kR = O.kappa(Rs)
    dAp = np.linalg.norm(Ap - Ap_o) / np.linalg.norm(Ap_o)
    assert dAp <= 4 * n * U64 * kR, dAp
    dG = np.linalg.norm(G - G_o) / np.linalg.norm(G_o)
    assert dG <= 2 * dAp * (np.linalg.norm(pr.A if hpne else Ap_o) * np.linalg.norm(Ap_o) / np.linalg.norm(G_o)) \
        + 4 * m * U64 * np.linalg.norm(Ap_o) ** 2 / np.linalg.norm(G_o), dG
    if not hpne:
        np.testing.assert_array_equal(G, G.T)
    dc = np.linalg.norm(c - c_o) / np.linalg.norm(c_o)
    assert dc <= 2 * dAp * np.linalg.norm(Ap_o) * np.linalg.norm(pr.b) / np.linalg.norm(c_o) + 4 * m * U64 * \
        np.linalg.norm(Ap_o) * np.linalg.norm(pr.b) / np.linalg.norm(c_o)


@pytest.mark.parametrize("n", [1, 7, 64, 65, 200, 1024, 1500])
def test_cholesky_solve(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((3 * n + 5, n))
    G = X.T @ X
    c = rng.standard_normal(n)
    R = np.triu(rng.standard_normal((n, n))) + 5 * np.eye(n)
    L_o, info_o = O.cholesky(G)
    y_o = O.solve_upper(R, O.solve_lower_t(L_o, O.solve_lower(L_o, c)))
    x, F, _, info = lsq.factor_solve(dev_colmajor(G), torch.from_numpy(c).cuda(), Rs=dev_colmajor(R))
    assert int(to_np(info)[0]) == 0 == info_o
    kG = O.kappa(G)
    assert np.linalg.norm(to_np(F) - L_o) / np.linalg.norm(L_o) <= 8 * n * U64 * kG
    assert np.linalg.norm(to_np(x) - y_o) / np.linalg.norm(y_o) <= 8 * n * U64 * kG * O.kappa(R)


@pytest.mark.parametrize("n", [1, 5, 33, 64, 200, 1024])
def test_lu_solve(n):
    rng = np.random.default_rng(100 + n)
    H = rng.standard_normal((n, n)) + np.diag(np.full(n, 0.5))
    c = rng.standard_normal(n)
    LU_o, piv_o, info_o = O.lu(H)
    x_o = O.lu_solve(LU_o, piv_o, c)
    x, F, piv, info = lsq.factor_solve(dev_colmajor(H), torch.from_numpy(c).cuda(), hpne=True)
    assert int(to_np(info)[0]) == 0 == info_o
    np.testing.assert_array_equal(to_np(piv), piv_o)
    kH = O.kappa(H)
    assert np.linalg.norm(to_np(F) - LU_o) / np.linalg.norm(LU_o) <= 8 * n * U64 * kH
    assert np.linalg.norm(to_np(x) - x_o) / np.linalg.norm(x_o) <= 8 * n * U64 * kH


def test_solve_wait_timeout_reports_and_recovers():
    """Fault injected on the host side (no GPU fault): with the test-only wait
    bound of the triangular solves cut to 1 ns, the blocks that find their
    predecessor's solution unpublished give up, record -2 in info and pass
    NaN on; the kernels return, and the next solve on the same context with
    the default bound is correct."""
    n = 1024
    rng = np.random.default_rng(11)
    X = rng.standard_normal((3 * n, n))
    G = X.T @ X
    c = rng.standard_normal(n)
    old = lsq.test_set_solve_wait_ns(1)
    try:
        _, _, _, info = lsq.factor_solve(dev_colmajor(G), torch.from_numpy(c).cuda())
        torch.cuda.synchronize()
        assert int(to_np(info)[0]) == -2
    finally:
        assert lsq.test_set_solve_wait_ns(old) == 1
    x, _, _, info = lsq.factor_solve(dev_colmajor(G), torch.from_numpy(c).cuda())
    assert int(to_np(info)[0]) == 0
    L_o, _ = O.cholesky(G)
    y_o = O.solve_lower_t(L_o, O.solve_lower(L_o, c))
    assert np.linalg.norm(to_np(x) - y_o) / np.linalg.norm(y_o) <= 8 * n * U64 * O.kappa(G)


def test_factor_breakdown_indices():
    G = np.diag([4.0, 1.0, -1.0, 2.0])
    _, _, _, info = lsq.factor_solve(dev_colmajor(G), torch.ones(4, dtype=torch.float64).cuda())
    assert int(to_np(info)[0]) == O.cholesky(G)[1] == 3
    H = np.array([[0.0, 1.0], [0.0, 2.0]])
    _, _, _, info = lsq.factor_solve(dev_colmajor(H), torch.ones(2, dtype=torch.float64).cuda(), hpne=True)
    assert int(to_np(info)[0]) == O.lu(H)[2] == 1


@pytest.mark.parametrize("kap", [1e1, 1e2, 1e3, 1e10])
def test_condest(kap):
    pr = P.make_problem(2000, 64, kap, 0.0, 91)
    k0, ch = lsq.condest(dev_colmajor(pr.A))
    k0, ch = float(to_np(k0)[0]), int(to_np(ch)[0])
    ok0, och, _, _, _ = O.condest(pr.A)
    if np.isinf(ok0):
        assert np.isinf(k0) and ch == och == O.FP64
    else:
        assert abs(k0 - ok0) <= 0.02, (k0, ok0)
        thresholds = np.array([2.0, 3.0, 4.0, 8.0])
        if np.min(np.abs(thresholds - ok0)) > 0.05:
            assert ch == och
