"""FP64-accurate tensor-core products on graded data, elementwise against
the oracle.

Every digit-sliced product is accurate relative to the largest magnitude of
the row (of A_p) or column (of R, of X in X^T Y) its operands come from, the
order of FP64 rounding of that row or column; an entry that is small within
its row or column gets that absolute accuracy, not a relative one.  Graded
data (each row and each column spanning 2^-30 .. 2^30) is where this
normwise-per-row (per-column) accuracy and the componentwise accuracy of a
sequential FP64 sum differ most, so every bound below is checked entry by
entry:
  * A_p = A R^{-1} (lsq_trsm_tc, and inside lsq_trsm_gram): both A_p's are
    backward stable, A_p R = A + E, with |E| <= 2 n u |A_p| |R| for the
    substitutions plus K 2^-50.6 max_k |A_p[i, k]| max_k |R[k, j]| for the
    digit products, so |A_p - A_p^oracle| <= (|E_gpu| + |E_oracle|) |R^{-1}|;
  * X^T Y (lsq_gram_tc, lsq_gemm_tn_tc, and the Gram of lsq_trsm_gram):
    per entry at most 2 m 2^-53 max|x_p| max|y_q| for the digit slicing plus
    gamma_m (|X|^T |Y|) for the oracle's sequential sum.
"""
import numpy as np
import pytest
import torch

import oracle as O
from tests.gpu_util import dev_colmajor, substitution_perturbation_bound, to_np

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")

U = 2.0 ** -53


def graded(m, n, seed, span=30):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, n))
    X *= np.exp2(rng.uniform(-span, span, m))[:, None]
    X *= np.exp2(rng.uniform(-span, span, n))[None, :]
    return np.asfortranarray(X)


def graded_r(n, seed, kappa_span=4):
    """Upper triangular R with graded columns and moderate conditioning."""
    rng = np.random.default_rng(seed)
    R = np.triu(rng.standard_normal((n, n))) * 0.3
    R[np.arange(n), np.arange(n)] = np.sign(rng.standard_normal(n)) * (1.0 + rng.random(n))
    R *= np.exp2(rng.uniform(-kappa_span, kappa_span, n))[None, :]
    return R


def gram_bound(X, Y):
    m = X.shape[0]
    gamma = m * U / (1 - m * U)
    return 2 * m * U * np.outer(np.abs(X).max(axis=0), np.abs(Y).max(axis=0)) + gamma * (np.abs(X).T @ np.abs(Y))


@pytest.mark.parametrize("m,n", [(3000, 200), (1100, 600), (4096, 33)])
def test_trsm_tc_graded_rows_elementwise(m, n):
    A = graded(m, n, m + n)
    R = graded_r(n, n)
    Ap_d, info = lsq.trsm_tc(dev_colmajor(A), dev_colmajor(R))
    assert int(to_np(info)[0]) == 0
    Ap = to_np(Ap_d)
    Ap_or = O.trsm_right_upper(A, R)
    tol = substitution_perturbation_bound(Ap_or, R, min(n, 512))
    bad = np.abs(Ap - Ap_or) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], (np.abs(Ap - Ap_or) / tol).max())
    # rows scale exactly: the per-row digit exponents make the relative result
    # of a row independent of its scale
    rows = np.isfinite(Ap).all(axis=1)
    assert rows.all()


@pytest.mark.parametrize("m,n", [(3000, 200), (70000, 96)])
def test_gram_tc_graded_elementwise(m, n):
    X = graded(m, n, 3 * m + n)
    G_d, info = lsq.gram_tc(dev_colmajor(X))
    assert int(to_np(info)[0]) == 0
    G = to_np(G_d)
    Go, _ = O.gram(X, X)
    tol = gram_bound(X, X)
    bad = np.abs(G - Go) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], (np.abs(G - Go) / tol).max())
    np.testing.assert_array_equal(G, G.T)


@pytest.mark.parametrize("m,n", [(3000, 200), (70000, 96)])
def test_gemm_tn_tc_graded_elementwise(m, n):
    X = graded(m, n, 5 * m + n)
    Y = graded(m, n, 7 * m + n)
    G_d, info = lsq.gemm_tn_tc(dev_colmajor(X), dev_colmajor(Y))
    assert int(to_np(info)[0]) == 0
    G = to_np(G_d)
    Go, _ = O.gram(X, Y)
    tol = gram_bound(X, Y)
    bad = np.abs(G - Go) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], (np.abs(G - Go) / tol).max())


@pytest.mark.parametrize("hpne", [False, True])
def test_trsm_gram_graded_elementwise(hpne):
    m, n = 6000, 300
    A = graded(m, n, 11 + hpne)
    R = graded_r(n, 13)
    rng = np.random.default_rng(17)
    b = rng.standard_normal(m) * np.exp2(rng.uniform(-30, 30, m))
    Ap_d, G_d, c_d = lsq.trsm_gram(dev_colmajor(A), dev_colmajor(R), torch.from_numpy(b).cuda(), hpne=hpne)
    Ap, G, c = to_np(Ap_d), to_np(G_d), to_np(c_d)
    Ap_or = O.trsm_right_upper(A, R)
    tol = substitution_perturbation_bound(Ap_or, R, min(n, 512))
    bad = np.abs(Ap - Ap_or) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], (np.abs(Ap - Ap_or) / tol).max())
    # the Gram and right-hand side against the oracle's sums of the same A_p
    Y = A if hpne else Ap
    Go, co = O.gram(Ap, Y, b)
    tol_g = gram_bound(Ap, Y)
    bad = np.abs(G - Go) > tol_g
    assert not bad.any(), (np.argwhere(bad)[:5], (np.abs(G - Go) / tol_g).max())
    gamma = m * U / (1 - m * U)
    assert np.all(np.abs(c - co) <= 2 * gamma * (np.abs(Ap).T @ np.abs(b)))
