"""Pins of the oracle's end-to-end method (Alg. 1, PNE Eq. e_pne, HPNE
Eq. e_hpne) and of its condition estimate (Sec. 6.1).

What fixes the answer here is the mathematics, not the oracle itself:
  * in exact arithmetic PNE and HPNE return the least-squares solution for
    ANY nonsingular R_s, so on consistent integer systems the error must be
    at rounding level;
  * the measured error must sit under the paper's bounds Eq. (eq41) (PNE,
    Thm. t_55) and Eq. (eq32) (HPNE, Thm. t_22), evaluated with exact
    condition numbers from an SVD;
  * kappa(A_p) <~ 10 for an effective preconditioner (Sec. 6.2);
  * the qualitative claims of Figs. 2-5 and 7;
  * the condition estimate is a lower bound of ||G^{-1}||_1 (Hager) and the
    kappa^2 inequality of Sec. 6.1 holds.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import problems as P

U2 = 2.0 ** -52  # the paper evaluates its bounds with u2 = 2^-52


def pne_with_r(A, b, R):
    Ap = O.trsm_right_upper(A, R)
    G, c = O.gram(Ap, Ap, b)
    L, info = O.cholesky(G)
    assert info == 0
    y = O.solve_lower_t(L, O.solve_lower(L, c))
    return O.solve_upper(R, y)


def hpne_with_r(A, b, R):
    Ap = O.trsm_right_upper(A, R)
    H, c = O.gram(Ap, A, b)
    LU, piv, info = O.lu(H)
    assert info == 0
    return O.lu_solve(LU, piv, c)


@pytest.mark.parametrize("solver", [pne_with_r, hpne_with_r])
def test_any_nonsingular_r_gives_ls_solution(solver):
    pr = P.make_problem(30, 6, 0, 0, 21, integer=True)
    rng = np.random.default_rng(0)
    for _ in range(3):
        R = np.triu(rng.standard_normal((6, 6))) + 3 * np.diag(np.sign(rng.standard_normal(6)))
        x = solver(pr.A, pr.b, R)
        kR = O.kappa(R)
        assert P.rel_error(x, pr.x_star) <= 1e3 * U2 * pr.kappa * kR * O.kappa(pr.A @ np.linalg.inv(R))


def bound_eq41(A, b, x, Rs, kA):
    Ap = sla.solve_triangular(Rs, A.T, trans="T", lower=False).T
    kR, kAp = O.kappa(Rs), O.kappa(Ap)
    res = np.linalg.norm(A @ x - b) / (np.linalg.norm(A, 2) * np.linalg.norm(x))
    return kR * kAp * U2 * (kAp * kR * res + 1 + kA * U2), kAp


def bound_eq32(A, b, x, Rs, kA):
    Ap = sla.solve_triangular(Rs, A.T, trans="T", lower=False).T
    H = Ap.T @ A
    nu = np.linalg.norm(Ap, 2) * np.linalg.norm(A, 2) / np.linalg.norm(H, 2)
    kR = O.kappa(Rs)
    res = np.linalg.norm(A @ x - b) / (np.linalg.norm(A, 2) * np.linalg.norm(x))
    return O.kappa(H) * nu * U2 * (kR * res + 1 + kA * U2), O.kappa(Ap)


CASES = [
    # (m, n, kappa, rho, kind, s, sketch precision)  -- Fig. 1 / 2 / 4 shapes
    (1000, 100, 1e8, 1e-6, O.GAUSSIAN, 200, O.FP32),
    (1000, 100, 1e8, 1e-12, O.GAUSSIAN, 200, O.FP32),
    (1000, 100, 1e8, 1e-2, O.GAUSSIAN, 200, O.FP32),
    (1500, 100, 1e4, 1e-3, O.SPARSE_SIGN, 300, O.FP64),
    (1500, 100, 1e6, 1e-8, O.SPARSE_SIGN, 300, O.BF16),
]


@pytest.mark.parametrize("case", CASES)
def test_pne_error_under_eq41(case):
    m, n, kap, rho, kind, s, prec = case
    pr = P.make_problem(m, n, kap, rho, P.seed_for(0, 7))
    r = O.solve(pr.A, pr.b, kind=kind, s=s, seed=3, sketch_prec=prec, qr_prec=O.FP32)
    assert r["info"] == 0
    bnd, kAp = bound_eq41(pr.A, pr.b, r["x"], r["Rs"], kap)
    err = P.rel_error(r["x"], pr.x_star)
    # eps_A of a backward-stable FP64 evaluation is gamma_n = n u, not u: factor n
    assert err <= n * bnd, (err, bnd)


@pytest.mark.parametrize("case", CASES)
def test_hpne_error_under_eq32(case):
    m, n, kap, rho, kind, s, prec = case
    pr = P.make_problem(m, n, kap, rho, P.seed_for(0, 8))
    r = O.solve(pr.A, pr.b, hpne=True, kind=kind, s=s, seed=4, sketch_prec=prec, qr_prec=O.FP32)
    assert r["info"] == 0
    bnd, _ = bound_eq32(pr.A, pr.b, r["x"], r["Rs"], kap)
    err = P.rel_error(r["x"], pr.x_star)
    assert err <= n * bnd, (err, bnd)


@pytest.mark.parametrize("kind,prec,kap", [(O.GAUSSIAN, O.FP64, 1e8), (O.SPARSE_SIGN, O.FP64, 1e10),
                                           (O.GAUSSIAN, O.FP32, 1e4), (O.SPARSE_SIGN, O.BF16, 1e1)])
def test_preconditioned_matrix_well_conditioned(kind, prec, kap):
    # kappa(A_p) <~ 10 when u_p * kappa(A) << 1 (Lemma rscond, Sec. 6.2, s = 3n)
    pr = P.make_problem(3000, 60, kap, 0.0, 31)
    r = O.solve(pr.A, pr.b, kind=kind, s=180, seed=9, sketch_prec=prec, qr_prec=O.FP64 if prec == O.FP64 else O.FP32)
    Ap = sla.solve_triangular(r["Rs"], pr.A.T, trans="T").T
    assert O.kappa(Ap) <= 10.0


def test_normal_equations_residual_orthogonality():
    pr = P.make_problem(2000, 80, 1e6, 1e-3, 41)
    r = O.solve(pr.A, pr.b, kind=O.SPARSE_SIGN, s=320, seed=1, sketch_prec=O.FP32)
    res = pr.b - pr.A @ r["x"]
    val = np.linalg.norm(pr.A.T @ res) / (np.linalg.norm(pr.A, 2) * np.linalg.norm(res)
                                         + np.linalg.norm(pr.A, 2) ** 2 * np.linalg.norm(r["x"]))
    assert val <= 1e3 * U2 * 10 ** 2


@pytest.mark.parametrize("hpne", [False, True])
def test_fig2_fig3_double_precision_matches_qr_for_large_residual(hpne):
    # Figs. 2-3: kappa = 1e4, everything in FP64; for residual > 1e-4 the
    # PNE/HPNE error is that of a QR solver.
    for rho in (1e-3, 1e-1):
        pr = P.make_problem(3000, 100, 1e4, rho, 51)
        r = O.solve(pr.A, pr.b, hpne=hpne, kind=O.GAUSSIAN, s=300, seed=2, sketch_prec=O.FP64, qr_prec=O.FP64)
        eq = P.rel_error(O.lstsq_qr(pr.A, pr.b), pr.x_star)
        assert P.rel_error(r["x"], pr.x_star) <= 3 * eq


@pytest.mark.parametrize("hpne", [False, True])
def test_fig4_fig5_single_preconditioner(hpne):
    # Figs. 4-5: kappa = 1e8 with an FP32 preconditioner: about 100x the QR error
    # for small residuals, about equal for large ones.
    pr = P.make_problem(3000, 100, 1e8, 1e-10, 61)
    r = O.solve(pr.A, pr.b, hpne=hpne, kind=O.GAUSSIAN, s=300, seed=3, sketch_prec=O.FP32, qr_prec=O.FP32)
    eq = P.rel_error(O.lstsq_qr(pr.A, pr.b), pr.x_star)
    assert P.rel_error(r["x"], pr.x_star) <= 1e3 * eq
    pr = P.make_problem(3000, 100, 1e8, 1e-2, 62)
    r = O.solve(pr.A, pr.b, hpne=hpne, kind=O.GAUSSIAN, s=300, seed=3, sketch_prec=O.FP32, qr_prec=O.FP32)
    eq = P.rel_error(O.lstsq_qr(pr.A, pr.b), pr.x_star)
    assert P.rel_error(r["x"], pr.x_star) <= 5 * eq


@pytest.mark.parametrize("hpne", [False, True])
def test_refinement_does_not_hurt(hpne):
    pr = P.make_problem(4000, 120, 1e6, 1e-8, 71)
    kw = dict(hpne=hpne, kind=O.SPARSE_SIGN, s=480, zeta=8, seed=5, sketch_prec=O.BF16, qr_prec=O.FP32)
    r0 = O.solve(pr.A, pr.b, refine_steps=0, **kw)
    r1 = O.solve(pr.A, pr.b, refine_steps=1, **kw)
    e0, e1 = P.rel_error(r0["x"], pr.x_star), P.rel_error(r1["x"], pr.x_star)
    assert e1 <= 2 * e0 + 1e-15
    np.testing.assert_array_equal(r0["Rs"], r1["Rs"])


def test_breakdown_reported_for_rank_deficient():
    pr = P.make_problem(500, 20, 1e2, 0.0, 81)
    A = pr.A.copy(order="F")
    A[:, 5] = A[:, 4]  # duplicated column: rank n-1
    r = O.solve(A, pr.b, kind=O.SPARSE_SIGN, s=40, seed=1, sketch_prec=O.FP64, qr_prec=O.FP64)
    assert r["info"] != 0 or not np.all(np.isfinite(r["x"])) or np.linalg.norm(r["x"]) > 1e8


# --- condition estimate (Sec. 6.1) -----------------------------------------------------
@pytest.mark.parametrize("kap", [1e1, 1e2, 1e3])
def test_condest_hager_is_lower_bound_and_close(kap):
    pr = P.make_problem(2000, 64, kap, 0.0, 91)
    k0, ch, nrm, gam, info = O.condest(pr.A)
    assert info == 0
    A32 = pr.A.astype(np.float32).astype(np.float64)
    G = A32.T @ A32
    inv1 = np.abs(np.linalg.inv(G)).sum(axis=0).max()
    assert gam <= inv1 * (1 + 1e-3)
    assert gam >= inv1 / 3
    assert abs(nrm - np.abs(G).sum(axis=0).max()) <= 1e-5 * nrm
    # kappa(A)^2 = kappa(A^T A) <= n ||A^T A||_1 ||(A^T A)^{-1}||_1  (exact values)
    kA = O.kappa(pr.A)
    assert kA ** 2 <= 64 * np.abs(G).sum(axis=0).max() * inv1 * (1 + 1e-6)
    assert np.log10(kA) - 0.25 <= k0 <= np.log10(kA) + np.log10(64) + 0.01


def test_condest_overflow_goes_to_double():
    pr = P.make_problem(1000, 50, 1e10, 0.0, 92)
    k0, ch, _, _, info = O.condest(pr.A)
    assert np.isinf(k0) and ch == O.FP64 and info > 0


def test_precision_table():
    f = O.precision_from_kappa0
    assert f(1.99) == O.FP8_E4M3 and f(2.0) == O.BF16 and f(2.99) == O.BF16
    assert f(3.0) == O.FP16 and f(3.99) == O.FP16 and f(4.0) == O.FP32
    assert f(8.0) == O.FP32 and f(8.01) == O.FP64 and f(float("inf")) == O.FP64 and f(float("nan")) == O.FP64


def test_fig7_auto_precision():
    # Fig. 7: kappa = 1e2 selects half precision and is nearly as accurate as QR;
    # kappa = 1e10 selects double and is as accurate as QR.
    for kap, want, factor in ((1e2, O.FP16, 10), (1e10, O.FP64, 3)):
        pr = P.make_problem(4096, 64, kap, 1e-6, 93)
        r = O.solve(pr.A, pr.b, kind=O.GAUSSIAN, s=192, seed=8, sketch_prec=O.AUTO, qr_prec=O.FP32)
        assert r["prec"] == want
        eq = P.rel_error(O.lstsq_qr(pr.A, pr.b), pr.x_star)
        assert P.rel_error(r["x"], pr.x_star) <= factor * eq
