"""Pins of the oracle's subsampled randomized Walsh-Hadamard sketch
Omega = S F D (Eq. e_sketch, Sec. 6.2, with F the real Sylvester-Hadamard
transform of order m' = 2^ceil(log2 m)):
  * on integer data the sketch equals (H D A)[rows] computed exactly with the
    explicit Hadamard matrix (scipy.linalg.hadamard), in FP64 and FP32;
  * the butterflies compute H: applied twice they give m' x exactly;
  * the signs are balanced, the sampled rows uniform over [0, m') and drawn
    with replacement;
  * d = 3n sampled rows embed range(A): kappa of the sketched orthonormal
    basis stays below 10, and PNE with this sketch meets Eq. (eq41) with
    kappa(A_p) <= 10 (Sec. 6.2).
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy import stats

import oracle as O
import problems as P


@pytest.mark.parametrize("m,n,s", [(1000, 7, 30), (64, 5, 20), (4097, 3, 50)])
@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_sketch_equals_explicit_hadamard_on_integers(m, n, s, prec):
    rng = np.random.default_rng(m + n)
    A = np.asfortranarray(rng.integers(-6, 7, size=(m, n)).astype(np.float64))
    sg, rows, mp = O.srft_operator(11, m, s)
    As, e = O.sketch(A, O.SRFT, s, 0, 11, prec)
    H = sla.hadamard(mp).astype(np.int64)
    Ahat = A * np.exp2(e)[None, :]  # the power-of-two column scaling (none for FP64) is exact
    Apad = np.zeros((mp, n))
    Apad[:m] = sg[:, None] * Ahat
    ref = (H @ Apad)[rows]
    np.testing.assert_array_equal(As, ref)


def test_butterflies_apply_hadamard_twice_to_identity():
    rng = np.random.default_rng(3)
    for mp in (1, 2, 8, 1024):
        x = rng.integers(-1000, 1000, mp).astype(np.float64)
        np.testing.assert_array_equal(O.fwht(O.fwht(x)), mp * x)
        np.testing.assert_array_equal(O.fwht(x), sla.hadamard(mp) @ x)


def test_signs_balanced_rows_uniform_with_replacement():
    sg, rows, mp = O.srft_operator(2603, 50000, 20000)
    assert mp == 65536
    assert set(np.unique(sg)) == {-1, 1}
    assert stats.binomtest(int((sg > 0).sum()), len(sg)).pvalue > 1e-3
    counts = np.bincount(rows // 4096, minlength=16)
    assert stats.chisquare(counts).pvalue > 1e-3
    # with replacement: repeats at the birthday rate, s^2 / (2 m') ~ 3050
    dup = len(rows) - len(np.unique(rows))
    assert 2500 < dup < 3600, dup


def test_three_n_rows_embed_the_column_space():
    m, n = 4000, 60
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    As, _ = O.sketch(np.asfortranarray(Q), O.SRFT, 3 * n, 0, 19, O.FP64)
    assert O.kappa(As) <= 10.0


@pytest.mark.parametrize("hpne", [False, True])
def test_pne_hpne_with_srft(hpne):
    pr = P.make_problem(3000, 100, 1e6, 1e-8, 111)
    r = O.solve(pr.A, pr.b, hpne=hpne, kind=O.SRFT, s=300, seed=5, sketch_prec=O.FP32, qr_prec=O.FP32)
    assert r["info"] == 0
    Ap = sla.solve_triangular(r["Rs"], pr.A.T, trans="T", lower=False).T
    assert O.kappa(Ap) <= 10.0
    # Figs. 2-5 shape: close to the QR solver's error at this residual
    eq = P.rel_error(O.lstsq_qr(pr.A, pr.b), pr.x_star)
    assert P.rel_error(r["x"], pr.x_star) <= 100 * eq
