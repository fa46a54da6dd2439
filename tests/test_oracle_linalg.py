"""Pins of the oracle's dense linear-algebra steps against exact arithmetic
(Python ``fractions``), closed forms and independent library routines."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import problems as P


def frac_matrix(M):
    return [[Fraction(float(v)) for v in row] for row in np.asarray(M)]


def frac_solve(Mat, rhs):
    """Gauss-Jordan in exact rationals."""
    n = len(Mat)
    a = [row[:] + [rhs[i]] for i, row in enumerate(Mat)]
    for k in range(n):
        p = next(i for i in range(k, n) if a[i][k] != 0)
        a[k], a[p] = a[p], a[k]
        for i in range(n):
            if i != k and a[i][k] != 0:
                f = a[i][k] / a[k][k]
                a[i] = [x - f * y for x, y in zip(a[i], a[k])]
    return [a[i][n] / a[i][i] for i in range(n)]


def exact_lstsq(A, b):
    """Exact least-squares solution of the FP64 inputs: A^T A x = A^T b in rationals."""
    Af = frac_matrix(A)
    bf = [Fraction(float(v)) for v in b]
    m, n = len(Af), len(Af[0])
    AtA = [[sum(Af[i][p] * Af[i][q] for i in range(m)) for q in range(n)] for p in range(n)]
    Atb = [sum(Af[i][p] * bf[i] for i in range(m)) for p in range(n)]
    return np.array([float(v) for v in frac_solve(AtA, Atb)])


@pytest.mark.parametrize("m,n,seed", [(6, 3, 1), (12, 5, 2), (16, 8, 3), (9, 1, 4)])
def test_lstsq_qr_matches_exact_rational(m, n, seed):
    rng = np.random.default_rng(seed)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    b = rng.standard_normal(m)
    xe = exact_lstsq(A, b)
    x = O.lstsq_qr(A, b)
    kap = O.kappa(A)
    r = b - A @ xe
    bound = 64 * 2.0 ** -53 * kap * (1 + kap * np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(xe)))
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= bound
    np.testing.assert_allclose(x, np.linalg.lstsq(A, b, rcond=None)[0], rtol=1e-10, atol=1e-12)


def test_lstsq_consistent_integer_system():
    pr = P.make_problem(40, 7, 0, 0, 11, integer=True)
    x = O.lstsq_qr(pr.A, pr.b)
    assert np.linalg.norm(x - pr.x_star) / np.linalg.norm(pr.x_star) <= 64 * pr.kappa * 2.0 ** -53


@pytest.mark.parametrize("kappa,rho", [(1e2, 0.0), (1e6, 1e-8), (1e8, 1e-3)])
def test_lstsq_generated_problem_within_lemma_ls(kappa, rho):
    # Lemma l_ls: error <= kappa eps_A (1 + kappa * relres), with eps_A ~ c u for a
    # backward-stable solver.
    pr = P.make_problem(600, 40, kappa, rho, 5)
    x = O.lstsq_qr(pr.A, pr.b)
    eps = 40 * 600 * 2.0 ** -53
    relres = np.linalg.norm(pr.b - pr.A @ x) / np.linalg.norm(x)
    assert P.rel_error(x, pr.x_star) <= kappa * eps * (1 + kappa * relres)


def test_trsm_exact_on_unit_integer_r():
    rng = np.random.default_rng(6)
    m, n = 9, 6
    A = np.asfortranarray(rng.integers(-5, 6, size=(m, n)).astype(np.float64))
    R = np.triu(rng.integers(-3, 4, size=(n, n)).astype(np.float64), 1) + np.diag(rng.choice([1.0, -2.0, 4.0], n))
    Ap = O.trsm_right_upper(A, R)
    # exact rational A R^{-1}
    Af, Rf = frac_matrix(A), frac_matrix(R)
    for i in range(m):
        y = []
        for j in range(n):
            t = Af[i][j] - sum(y[k] * Rf[k][j] for k in range(j))
            y.append(t / Rf[j][j])
        assert [float(v) for v in y] == list(Ap[i])
    np.testing.assert_allclose(Ap @ R, A, atol=1e-12)


def test_gram_exact_on_integers():
    rng = np.random.default_rng(7)
    X = np.asfortranarray(rng.integers(-9, 10, size=(50, 6)).astype(np.float64))
    Y = np.asfortranarray(rng.integers(-9, 10, size=(50, 6)).astype(np.float64))
    b = rng.integers(-9, 10, size=50).astype(np.float64)
    G, c = O.gram(X, Y, b)
    np.testing.assert_array_equal(G, X.T @ Y)
    np.testing.assert_array_equal(c, X.T @ b)
    G2, _ = O.gram(X, X)
    np.testing.assert_array_equal(G2, G2.T)


def test_cholesky_exact_on_integer_factor():
    rng = np.random.default_rng(8)
    n = 7
    L = np.tril(rng.integers(-4, 5, size=(n, n)).astype(np.float64), -1) + np.diag(rng.integers(1, 6, n).astype(np.float64))
    G = L @ L.T
    Lc, info = O.cholesky(G)
    assert info == 0
    np.testing.assert_array_equal(Lc, L)


def test_cholesky_breakdown_index():
    G = np.diag([4.0, 1.0, -1.0, 2.0])
    _, info = O.cholesky(G)
    assert info == 3
    G = np.ones((3, 3))  # rank one: second pivot is exactly zero
    _, info = O.cholesky(G)
    assert info == 2


def test_lu_matches_lapack_pivots_and_factors():
    rng = np.random.default_rng(9)
    for n in (1, 5, 33):
        H = rng.standard_normal((n, n))
        LU, piv, info = O.lu(H)
        assert info == 0
        lu_ref, piv_ref = sla.lu_factor(H)
        np.testing.assert_array_equal(piv, piv_ref)
        np.testing.assert_allclose(LU, lu_ref, rtol=1e-11, atol=1e-12)
        L = np.tril(LU, -1) + np.eye(n)
        U = np.triu(LU)
        assert np.all(np.abs(L) <= 1.0)
        PH = H.copy()
        for k in range(n):
            PH[[k, piv[k]]] = PH[[piv[k], k]]
        np.testing.assert_allclose(L @ U, PH, atol=1e-12 * n)


def test_lu_first_max_tie_and_zero_pivot():
    H = np.array([[1.0, 2.0], [-1.0, 3.0]])  # |1| == |-1|: first row stays
    _, piv, info = O.lu(H)
    assert list(piv) == [0, 1] and info == 0
    _, _, info = O.lu(np.array([[0.0, 1.0], [0.0, 2.0]]))
    assert info == 1


def test_triangular_solves_and_lu_solve():
    rng = np.random.default_rng(10)
    n = 20
    L = np.tril(rng.standard_normal((n, n))) + 4 * np.eye(n)
    y = rng.standard_normal(n)
    np.testing.assert_allclose(O.solve_lower(L, y), sla.solve_triangular(L, y, lower=True), rtol=1e-12)
    np.testing.assert_allclose(O.solve_lower_t(L, y), sla.solve_triangular(L.T, y, lower=False), rtol=1e-12)
    np.testing.assert_allclose(O.solve_upper(L.T, y), sla.solve_triangular(L.T, y, lower=False), rtol=1e-12)
    np.testing.assert_allclose(O.solve_lower(L, y, unit=True),
                               sla.solve_triangular(L, y, lower=True, unit_diagonal=True), rtol=1e-12)
    H = rng.standard_normal((n, n))
    LU, piv, _ = O.lu(H)
    np.testing.assert_allclose(O.lu_solve(LU, piv, y), np.linalg.solve(H, y), rtol=1e-10)


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_qr_r_is_cholesky_factor_of_gram(prec):
    rng = np.random.default_rng(11)
    s, n = 120, 30
    As = np.asfortranarray(rng.standard_normal((s, n)) * np.exp2(rng.integers(-3, 3, n))[None, :])
    if prec == O.FP32:
        As = O.round_to(As, O.FP32).reshape(As.shape, order="F")
    R = O.qr_r(As, prec)
    assert np.all(np.diag(R) > 0) and np.all(np.tril(R, -1) == 0)
    Rc = np.linalg.cholesky(As.T @ As).T  # unique upper factor with positive diagonal
    u = 2.0 ** -53 if prec == O.FP64 else 2.0 ** -24
    assert np.linalg.norm(R - Rc) / np.linalg.norm(Rc) <= 200 * u * O.kappa(As)
    assert np.linalg.norm(R.T @ R - As.T @ As) / np.linalg.norm(As) ** 2 <= 50 * s * u
    Rq = np.linalg.qr(As, mode="r")
    Rq = Rq * np.sign(np.diag(Rq))[:, None]
    assert np.linalg.norm(R - Rq) / np.linalg.norm(Rq) <= 200 * u * O.kappa(As)


def test_qr_negative_and_zero_columns():
    As = np.asfortranarray(np.array([[-3.0, 1.0], [0.0, 2.0], [0.0, 0.0]]))
    R = O.qr_r(As, O.FP64)
    np.testing.assert_allclose(R, [[3.0, -1.0], [0.0, 2.0]], atol=1e-15)


def test_unscale_r_exact():
    R = np.triu(np.arange(1.0, 17.0).reshape(4, 4))
    e = np.array([3, -2, 0, 5], dtype=np.int32)
    Ru = O.unscale_r(R, e)
    np.testing.assert_array_equal(Ru, np.triu(R * np.exp2(-e)[None, :]))
