"""Pins of the oracle's alternative solution methods (Sec. 5 and Sec. 1):
HPNE through a QR factorization of A_p^T A, the seminormal equations
(Eq. e_sne, Thm. l_semi) with R = L^T R_s from the preconditioner, and the
not-normal equations (Eq. e_nne, Thm. l_notnorm) with B = A U_s^{-1}, U_s
from the LU of the sketch.

What fixes the answer is the mathematics:
  * in exact arithmetic each method returns the least-squares solution, so on
    consistent integer systems (b = A x_* exactly) the error sits at rounding
    level, and exact rational arithmetic on tiny problems gives x_* itself;
  * the measured error sits under the paper's bound for the method
    (Thm. l_semi for SNE, Thm. l_notnorm for the not-normal equations, Eq. eq32
    for HPNE whatever the n x n factorization), with exact condition numbers;
  * the two factorizations of the HPNE matrix solve the same system, so their
    solutions differ by at most the perturbation bound of two backward-stable
    solves;
  * the LU of the sketch matches LAPACK's getrf (same pivot rule);
  * the seminormal equations lose a factor kappa(A) against PNE (Thm. l_semi
    against Thm. t_55), and one refinement step (corrected seminormal
    equations) recovers it.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import problems as P

U2 = 2.0 ** -52
U = 2.0 ** -53


def test_lu_tall_matches_lapack():
    rng = np.random.default_rng(3)
    for (s, n) in [(40, 12), (200, 64), (33, 33)]:
        As = np.asfortranarray(rng.standard_normal((s, n)))
        U64, info = O.lu_tall_u(As, O.FP64)
        assert info == 0
        lu, piv = sla.lu_factor(As)
        Ul = np.triu(lu[:n, :n])
        np.testing.assert_allclose(U64, Ul, rtol=0, atol=64 * n * U * np.abs(Ul).max())
        # FP32 arithmetic: the same factor to FP32 rounding
        U32, info = O.lu_tall_u(As.astype(np.float32).astype(np.float64), O.FP32)
        assert info == 0
        assert np.abs(U32 - Ul).max() <= 64 * n * 2.0 ** -24 * np.abs(Ul).max()


def test_lu_tall_zero_pivot():
    As = np.zeros((10, 4))
    As[:, 0] = 1.0
    As[:, 2] = np.arange(10)
    _, info = O.lu_tall_u(As, O.FP64)
    assert info == 2


def test_solve_upper_t_matches_lapack():
    rng = np.random.default_rng(4)
    Um = np.triu(rng.standard_normal((50, 50))) + 5 * np.eye(50)
    y = rng.standard_normal(50)
    np.testing.assert_allclose(O.solve_upper_t(Um, y), sla.solve_triangular(Um, y, trans="T"), rtol=1e-12)


METHODS = [O.HPNE_QR, O.SNE, O.NNE_LU]


@pytest.mark.parametrize("method", METHODS)
def test_consistent_integer_systems_are_solved(method):
    pr = P.make_problem(200, 10, 0, 0, 23, integer=True)
    r = O.solve(pr.A, pr.b, method=method, kind=O.GAUSSIAN, s=30, seed=5, sketch_prec=O.FP64, qr_prec=O.FP64)
    assert r["info"] == 0
    kA = O.kappa(pr.A)
    lim = 1e3 * U2 * (kA ** 2 if method == O.SNE else kA * O.kappa(r["Rs"]))
    assert P.rel_error(r["x"], pr.x_star) <= lim


def _exact_ls(A, b):
    """Exact least-squares solution of the FP64 data by rational normal equations."""
    m, n = A.shape
    Af = [[Fraction(float(A[i, j])) for j in range(n)] for i in range(m)]
    bf = [Fraction(float(v)) for v in b]
    G = [[sum(Af[k][i] * Af[k][j] for k in range(m)) for j in range(n)] for i in range(n)]
    c = [sum(Af[k][i] * bf[k] for k in range(m)) for i in range(n)]
    for k in range(n):  # Gauss-Jordan, exact
        p = next(i for i in range(k, n) if G[i][k] != 0)
        G[k], G[p], c[k], c[p] = G[p], G[k], c[p], c[k]
        for i in range(n):
            if i != k and G[i][k] != 0:
                f = G[i][k] / G[k][k]
                G[i] = [a - f * bb for a, bb in zip(G[i], G[k])]
                c[i] -= f * c[k]
    return np.array([float(c[i] / G[i][i]) for i in range(n)])


@pytest.mark.parametrize("method", METHODS)
def test_tiny_problem_against_exact_rational_solution(method):
    pr = P.make_problem(14, 5, 1e3, 1e-3, 29)
    xe = _exact_ls(pr.A, pr.b)
    r = O.solve(pr.A, pr.b, method=method, kind=O.GAUSSIAN, s=10, seed=2, sketch_prec=O.FP64, qr_prec=O.FP64)
    assert r["info"] == 0
    kA = O.kappa(pr.A)
    lim = 1e2 * U2 * (kA ** 2 if method == O.SNE else kA * O.kappa(r["Rs"]))
    assert P.rel_error(r["x"], xe) <= lim


CASES = [
    (1000, 100, 1e8, 1e-6, O.GAUSSIAN, 200, O.FP32),
    (1500, 100, 1e4, 1e-3, O.SPARSE_SIGN, 300, O.FP64),
    (1500, 100, 1e6, 1e-8, O.SPARSE_SIGN, 300, O.BF16),
    (1200, 60, 1e3, 0.0, O.GAUSSIAN, 180, O.FP8_E4M3),
]


def _res(A, b, x):
    return np.linalg.norm(A @ x - b) / (np.linalg.norm(A, 2) * np.linalg.norm(x))


@pytest.mark.parametrize("case", CASES)
def test_hpne_qr_under_eq32_and_agrees_with_lu(case):
    m, n, kap, rho, kind, s, prec = case
    pr = P.make_problem(m, n, kap, rho, P.seed_for(0, 9))
    kw = dict(kind=kind, s=s, seed=4, sketch_prec=prec, qr_prec=O.FP32)
    rq = O.solve(pr.A, pr.b, method=O.HPNE_QR, **kw)
    rl = O.solve(pr.A, pr.b, method=O.HPNE, **kw)
    assert rq["info"] == 0 == rl["info"]
    np.testing.assert_array_equal(rq["Rs"], rl["Rs"])
    Rs = rq["Rs"]
    Ap = sla.solve_triangular(Rs, pr.A.T, trans="T", lower=False).T
    H = Ap.T @ pr.A
    nu = np.linalg.norm(Ap, 2) * np.linalg.norm(pr.A, 2) / np.linalg.norm(H, 2)
    bnd = O.kappa(H) * nu * U2 * (O.kappa(Rs) * _res(pr.A, pr.b, rq["x"]) + 1 + kap * U2)
    err = P.rel_error(rq["x"], pr.x_star)
    assert err <= n * bnd, (err, bnd)
    # the same n x n system, two backward-stable factorizations
    d = np.linalg.norm(rq["x"] - rl["x"]) / np.linalg.norm(rl["x"])
    assert d <= 4 * n * U * O.kappa(H) * 10, d


@pytest.mark.parametrize("case", CASES)
def test_sne_under_theorem_semi(case):
    m, n, kap, rho, kind, s, prec = case
    pr = P.make_problem(m, n, kap, rho, P.seed_for(0, 10))
    r = O.solve(pr.A, pr.b, method=O.SNE, kind=kind, s=s, seed=6, sketch_prec=prec, qr_prec=O.FP32)
    assert r["info"] == 0
    # Thm. l_semi with eps = gamma_n of a backward-stable FP64 evaluation
    eps = n * U2
    bnd = kap ** 2 * eps * (_res(pr.A, pr.b, r["x"]) + 1 + eps)
    err = P.rel_error(r["x"], pr.x_star)
    assert err <= bnd, (err, bnd)


@pytest.mark.parametrize("case", CASES)
def test_nne_under_theorem_notnorm(case):
    m, n, kap, rho, kind, s, prec = case
    pr = P.make_problem(m, n, kap, rho, P.seed_for(0, 11))
    r = O.solve(pr.A, pr.b, method=O.NNE_LU, kind=kind, s=s, seed=7, sketch_prec=prec, qr_prec=O.FP32)
    assert r["info"] == 0
    Us = r["Rs"]
    B = sla.solve_triangular(Us, pr.A.T, trans="T", lower=False).T  # A = B U_s
    BA = B.T @ pr.A
    nu = np.linalg.norm(B, 2) * np.linalg.norm(pr.A, 2) / np.linalg.norm(BA, 2)
    # eps_A = gamma_n; B = A U_s^{-1} is formed by substitution: eps_B <= gamma_n kappa(U_s)
    eA = n * U2
    eB = n * U2 * O.kappa(Us)
    bnd = O.kappa(BA) * nu * (eB * _res(pr.A, pr.b, r["x"]) + (1 + eB) * eA)
    err = P.rel_error(r["x"], pr.x_star)
    assert err <= n * bnd, (err, bnd)
    # the sketch's LU makes B well conditioned when u_p kappa(A) << 1
    if {O.FP64: 2.0 ** -53, O.FP32: 2.0 ** -24, O.BF16: 2.0 ** -8, O.FP8_E4M3: 2.0 ** -4}[prec] * kap < 1e-2:
        assert O.kappa(B) <= 1e3


def test_sne_loses_kappa_and_refinement_recovers_it():
    pr = P.make_problem(3000, 80, 1e6, 1e-8, 77)
    kw = dict(kind=O.SPARSE_SIGN, s=320, zeta=8, seed=5, sketch_prec=O.FP64, qr_prec=O.FP64)
    e_pne = P.rel_error(O.solve(pr.A, pr.b, method=O.PNE, **kw)["x"], pr.x_star)
    e_sne = P.rel_error(O.solve(pr.A, pr.b, method=O.SNE, **kw)["x"], pr.x_star)
    e_csne = P.rel_error(O.solve(pr.A, pr.b, method=O.SNE, refine_steps=1, **kw)["x"], pr.x_star)
    assert e_sne >= 100 * e_pne, (e_sne, e_pne)
    assert e_csne <= 10 * e_pne + 1e-14, (e_csne, e_pne)


@pytest.mark.parametrize("method", METHODS)
def test_refinement_does_not_hurt(method):
    pr = P.make_problem(4000, 120, 1e5, 1e-7, 78)
    kw = dict(method=method, kind=O.GAUSSIAN, s=360, seed=5, sketch_prec=O.FP32, qr_prec=O.FP32)
    e0 = P.rel_error(O.solve(pr.A, pr.b, refine_steps=0, **kw)["x"], pr.x_star)
    e1 = P.rel_error(O.solve(pr.A, pr.b, refine_steps=1, **kw)["x"], pr.x_star)
    assert e1 <= 2 * e0 + 1e-15


# --- condition estimate on a sketch -------------------------------------------
def test_kappa1_upper32_is_a_lower_bound_and_close():
    rng = np.random.default_rng(12)
    for kap in (1e1, 1e3, 1e5):
        n = 80
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        R = np.linalg.qr(Q @ np.diag(np.logspace(0, -np.log10(kap), n)) @ Q.T, mode="r")
        R = R * np.sign(np.diag(R))[:, None]
        R32 = R.astype(np.float32).astype(np.float64)
        exact = np.abs(R32).sum(0).max() * np.abs(np.linalg.inv(R32)).sum(0).max()
        k1 = O.kappa1_upper32(R)
        assert exact / 3 <= k1 <= exact * (1 + 1e-3), (kap, k1, exact)


@pytest.mark.parametrize("m,n", [(4000, 64), (6000, 300)])
def test_condest_sketch_tracks_kappa(m, n):
    for kap in (1e1, 1e2, 1e3, 1e4, 1e5):
        pr = P.make_problem(m, n, kap, 0.0, 17)
        k0, ch, k1, rc = O.condest_sketch(pr.A, 4)
        assert rc == 0
        if np.isinf(k0):
            # only where the FP32 factor itself does not resolve A
            assert 2.0 ** -24 * k1 > 1.0
            continue
        # like the estimate on A^T A (Sec. 6.1): kappa(A)^2 <= n ||G||_1 ||G^{-1}||_1
        # <= n^2 kappa(A)^2, up to the sketch's distortion of kappa(A) (a
        # factor ~2 for s = 2n) and Hager's underestimate (at most 3x)
        assert np.log10(kap) - 0.3 - 0.5 * np.log10(3) <= k0 <= np.log10(kap) + np.log10(n) + 0.3, (kap, k0)
        assert ch == O.precision_from_kappa0(k0)
        kl = O.condest(pr.A)[0]
        if np.isfinite(kl):
            assert abs(k0 - kl) <= 0.5, (kap, k0, kl)


def test_condest_sketch_saturates_to_double():
    pr = P.make_problem(4000, 64, 1e10, 0.0, 18)
    k0, ch, k1, rc = O.condest_sketch(pr.A, 4)
    assert rc == 0 and np.isinf(k0) and ch == O.FP64 and 2.0 ** -24 * k1 > 1.0
