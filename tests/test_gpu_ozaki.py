"""FP64 products on the FP8 tensor cores by digit slicing (lsq_gram_tc for
X^T X, lsq_gemm_tn_tc for X^T Y): exact on integer data, within the FP64
error order on general data (also with K split into several exact chunks and
with badly scaled columns), and PNE / HPNE solves that use them meet the
solution tolerance against the oracle."""
import ctypes as C
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle as O
import problems as P
from tests.gpu_util import assert_solution_parity, dev_colmajor, to_np

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")


def gram_tc(X):
    L = lsq.lib()
    L.lsq_gram_tc.restype = C.c_int32
    L.lsq_gram_tc.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                              C.c_void_p, C.c_size_t, C.c_void_p]
    L.lsq_gram_tc_workspace_size.restype = C.c_size_t
    L.lsq_gram_tc_workspace_size.argtypes = [C.c_int64, C.c_int64]
    m, n = X.shape
    Xd = dev_colmajor(X)
    G = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(int(L.lsq_gram_tc_workspace_size(m, n)), dtype=torch.uint8, device="cuda")
    rc = L.lsq_gram_tc(Xd.data_ptr(), m, n, m, G.data_ptr(), n, info.data_ptr(), ws.data_ptr(), ws.numel(),
                       torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    assert int(to_np(info)[0]) == 0
    return to_np(G).T.copy()  # stored column-major in an (n, n) row-major tensor


def set_emulation(on):
    f = lsq.lib().lsq_set_fp64_emulation
    f.restype = C.c_int32
    f.argtypes = [C.c_int32]
    return f(int(on))


@pytest.mark.parametrize("m,n", [(3000, 200), (1000, 1), (70000, 130)])
def test_exact_on_integer_data(m, n):
    rng = np.random.default_rng(m + n)
    Xi = rng.integers(-8, 9, size=(m, n))
    G = gram_tc(Xi.astype(np.float64))
    np.testing.assert_array_equal(G, (Xi.T @ Xi).astype(np.float64))


def test_correctly_rounded_on_wide_integer_data():
    # |x| < 2^26: every value has an exact digit representation, and the exact
    # Gram entries (up to ~2^68, two K-chunks) exceed FP64: the combined digit
    # products are summed exactly and rounded once, so every entry is the
    # correctly rounded exact integer (Python's int -> float rounds to nearest even)
    m, n = 70000, 24
    rng = np.random.default_rng(3)
    Xi = rng.integers(-(2 ** 26), 2 ** 26, size=(m, n))
    G = gram_tc(Xi.astype(np.float64))
    Xo = Xi.astype(object)
    exact = Xo.T.dot(Xo)
    want = np.array([[float(exact[p, q]) for q in range(n)] for p in range(n)])
    np.testing.assert_array_equal(G, want)
    Yi = rng.integers(-(2 ** 26), 2 ** 26, size=(m, n))
    Gxy, info = lsq.gemm_tn_tc(dev_colmajor(Xi.astype(np.float64)), dev_colmajor(Yi.astype(np.float64)))
    assert int(to_np(info)[0]) == 0
    exy = Xo.T.dot(Yi.astype(object))
    np.testing.assert_array_equal(to_np(Gxy), np.array([[float(exy[p, q]) for q in range(n)] for p in range(n)]))


def test_nonfinite_columns_give_nan_rows_and_columns():
    m, n = 3000, 150
    rng = np.random.default_rng(4)
    Xi = rng.integers(-8, 9, size=(m, n)).astype(np.float64)
    X = Xi.copy()
    X[5, 3] = np.nan
    X[70, 140] = -np.inf
    G = gram_tc(X)
    bad = np.zeros(n, bool)
    bad[[3, 140]] = True
    assert np.isnan(G[bad, :]).all() and np.isnan(G[:, bad]).all()
    ok = ~bad
    np.testing.assert_array_equal(G[np.ix_(ok, ok)], (Xi.T @ Xi)[np.ix_(ok, ok)])


@pytest.mark.parametrize("m,n,spread", [(5000, 257, 0), (70000, 130, 0), (4000, 64, 30)])
def test_within_fp64_error_order(m, n, spread):
    rng = np.random.default_rng(7 + n)
    X = rng.standard_normal((m, n)) * np.exp2(rng.integers(-spread, spread + 1, n))[None, :]
    X = np.asfortranarray(X)
    G = gram_tc(X)
    Go, _ = O.gram(X, X)
    cm = np.abs(X).max(axis=0)
    # the scheme's own bound: truncation below 2^(e_p - 56) per entry, pairs
    # t + u > 13 dropped: per product below 2^-53 * 2^(e_p + e_q) <= 2^-51 cm_p cm_q
    tol_scheme = 2 * m * 2.0 ** -53 * np.outer(cm, cm)
    # against the exact rational value on sampled entries
    for (p, q) in [(0, 0), (n - 1, n - 1), (n // 2, n // 2), (3, 1), (n - 1, 0), (n // 3, n // 5)]:
        ex = sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(X[:, p], X[:, q])), Fraction(0))
        assert abs(G[p, q] - float(ex)) <= tol_scheme[p, q], (p, q)
    # against the oracle everywhere, allowing the oracle's sequential-sum bound gamma_m (|X|^T |X|)
    gamma = m * 2.0 ** -53 / (1 - m * 2.0 ** -53)
    assert np.all(np.abs(G - Go) <= tol_scheme + gamma * (np.abs(X).T @ np.abs(X)))
    np.testing.assert_array_equal(G, G.T)


@pytest.mark.parametrize("m,n", [(3000, 200), (70000, 130), (1000, 1)])
def test_gemm_tn_exact_on_integer_data(m, n):
    rng = np.random.default_rng(m + 3 * n)
    Xi = rng.integers(-8, 9, size=(m, n))
    Yi = rng.integers(-8, 9, size=(m, n))
    G, info = lsq.gemm_tn_tc(dev_colmajor(Xi.astype(np.float64)), dev_colmajor(Yi.astype(np.float64)))
    assert int(to_np(info)[0]) == 0
    np.testing.assert_array_equal(to_np(G), (Xi.T @ Yi).astype(np.float64))


@pytest.mark.parametrize("m,n,spread", [(5000, 257, 0), (4000, 64, 30)])
def test_gemm_tn_within_fp64_error_order(m, n, spread):
    rng = np.random.default_rng(11 + n)
    X = np.asfortranarray(rng.standard_normal((m, n)) * np.exp2(rng.integers(-spread, spread + 1, n))[None, :])
    Y = np.asfortranarray(rng.standard_normal((m, n)) * np.exp2(rng.integers(-spread, spread + 1, n))[None, :])
    Gd, info = lsq.gemm_tn_tc(dev_colmajor(X), dev_colmajor(Y))
    assert int(to_np(info)[0]) == 0
    G = to_np(Gd)
    Go, _ = O.gram(X, Y)
    tol_scheme = 2 * m * 2.0 ** -53 * np.outer(np.abs(X).max(axis=0), np.abs(Y).max(axis=0))
    for (p, q) in [(0, 0), (n - 1, n - 1), (3, 1), (1, 3), (n - 1, 0), (0, n - 1), (n // 3, n // 5)]:
        ex = sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(X[:, p], Y[:, q])), Fraction(0))
        assert abs(G[p, q] - float(ex)) <= tol_scheme[p, q], (p, q)
    gamma = m * 2.0 ** -53 / (1 - m * 2.0 ** -53)
    assert np.all(np.abs(G - Go) <= tol_scheme + gamma * (np.abs(X).T @ np.abs(Y)))


@pytest.mark.parametrize("hpne", [False, True])
def test_pne_with_emulated_gram_matches_oracle(hpne):
    m, n = 20000, 300
    for kap, rho in [(1e2, 0.0), (1e6, 1e-8), (1e10, 1e-3)]:
        pr = P.make_problem(m, n, kap, rho, P.seed_for(1, 50 + int(np.log10(kap))))
        opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=4 * n, zeta=8, seed=3, sketch_prec=lsq.FP32,
                             refine_steps=1)
        A = dev_colmajor(pr.A)
        b = torch.from_numpy(pr.b).cuda()
        solve = lsq.hpne if hpne else lsq.pne
        prev = set_emulation(True)
        try:
            x_em, info = solve(A, b, opts=opts)
            assert int(to_np(info)[0]) == 0
            set_emulation(False)
            x_64, _ = solve(A, b, opts=opts)
        finally:
            set_emulation(prev)
        ref = O.solve(pr.A, pr.b, hpne=hpne, kind=O.SPARSE_SIGN, s=4 * n, zeta=8, seed=3, sketch_prec=O.FP32,
                      qr_prec=O.FP32, refine_steps=1)
        assert_solution_parity(to_np(x_em), ref["x"], pr.x_star, kap, rho, f"kappa={kap}")
        e_em = P.rel_error(to_np(x_em), pr.x_star)
        e_64 = P.rel_error(to_np(x_64), pr.x_star)
        assert e_em <= 2 * e_64 + 1e-15, (kap, e_em, e_64)
