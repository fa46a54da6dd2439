"""Pins of the oracle's random sketch operators.

Philox4x32-10 against the published known-answer vectors; the sparse-sign
operator against its defining invariants (zeta distinct rows per column,
uniform rows, balanced signs, and the sketch it produces equals the explicit
dense Omega times A exactly on integer data); the Gaussian operator against
N(0, 1) (moments and a Kolmogorov-Smirnov test) and its exact entry values
against Box-Muller evaluated in 50-digit decimal arithmetic.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


@pytest.mark.parametrize("s,zeta", [(64, 8), (4096, 8), (37, 5), (8, 8)])
def test_sparse_sign_columns_distinct_in_range(s, zeta):
    m = 3000
    idx, sgn = O.sparse_sign_indices(12345, m, s, zeta)
    assert idx.min() >= 0 and idx.max() < s
    for j in range(m):
        assert len(set(idx[j].tolist())) == zeta
    assert set(np.unique(sgn).tolist()) <= {-1, 1}


def test_sparse_sign_uniform_and_balanced():
    m, s, zeta = 40000, 64, 8
    idx, sgn = O.sparse_sign_indices(7, m, s, zeta)
    counts = np.bincount(idx.ravel(), minlength=s)
    chi2 = stats.chisquare(counts)
    assert chi2.pvalue > 1e-4
    frac_neg = np.mean(sgn == -1)
    assert abs(frac_neg - 0.5) < 4 * 0.5 / np.sqrt(sgn.size)
    # different seeds give different streams, the same seed the same stream
    idx2, _ = O.sparse_sign_indices(8, 100, s, zeta)
    idx3, _ = O.sparse_sign_indices(7, 100, s, zeta)
    assert not np.array_equal(idx2, idx[:100])
    assert np.array_equal(idx3, idx[:100])


def test_sparse_sign_bad_args():
    with pytest.raises(ValueError):
        O.sparse_sign_indices(1, 10, 4, 8)  # zeta > s


def dense_sparse_sign(seed, m, s, zeta):
    idx, sgn = O.sparse_sign_indices(seed, m, s, zeta)
    Om = np.zeros((s, m))
    for j in range(m):
        Om[idx[j], j] = sgn[j]
    return Om


@pytest.mark.parametrize("prec", [O.BF16, O.FP32, O.FP64, O.FP8_E4M3])
def test_sparse_sketch_equals_dense_product_on_integers(prec):
    rng = np.random.default_rng(3)
    m, n, s, zeta = 700, 13, 48, 4
    A = np.asfortranarray(rng.integers(-7, 8, size=(m, n)).astype(np.float64))
    As, e = O.sketch(A, O.SPARSE_SIGN, s, zeta, 99, prec)
    Om = dense_sparse_sign(99, m, s, zeta)
    expect = Om @ (A * np.exp2(e)[None, :])  # exact: small integers times powers of two
    np.testing.assert_array_equal(As, expect)


def test_colexp_targets():
    rng = np.random.default_rng(4)
    A = np.asfortranarray(rng.standard_normal((50, 9)) * np.exp2(rng.integers(-30, 30, 9))[None, :])
    for prec, t in [(O.FP8_E4M3, 8), (O.FP16, 15), (O.BF16, 0), (O.FP32, 0)]:
        e = O.colexp(A, prec)
        mx = np.abs(A).max(axis=0) * np.exp2(e)
        assert np.all(mx >= 2.0 ** (t - 1)) and np.all(mx < 2.0 ** t)
    assert np.all(O.colexp(A, O.FP64) == 0)


def test_gaussian_entries_are_standard_normal():
    Om = O.gaussian_operator(2024, 64, 4000, O.FP64)
    z = Om.ravel()
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # rows and columns are not correlated
    c = np.corrcoef(Om[:, :2000])
    off = c[~np.eye(c.shape[0], dtype=bool)]
    assert np.abs(off).max() < 6 / np.sqrt(2000)
    # rounding to the sketch precision is the oracle's RNE rounding
    Om8 = O.gaussian_operator(2024, 64, 100, O.FP8_E4M3)
    np.testing.assert_array_equal(Om8, O.round_to(Om[:, :100], O.FP8_E4M3))


@pytest.mark.parametrize("prec", [O.FP64, O.FP32, O.BF16, O.FP8_E4M3])
def test_gaussian_sketch_matches_dense_product(prec):
    rng = np.random.default_rng(5)
    m, n, s = 300, 11, 30
    A = np.asfortranarray(rng.standard_normal((m, n)))
    As, e = O.sketch(A, O.GAUSSIAN, s, 0, 77, prec)
    Om = O.gaussian_operator(77, s, m, prec)
    Ahat = O.quantize(A, prec, e)
    expect = Om @ Ahat
    tol = 1e-13 if prec == O.FP64 else 4 * m * 2.0 ** -24
    scale = np.abs(Om) @ np.abs(Ahat)
    assert np.all(np.abs(As - expect) <= tol * scale + 1e-300)


# --- exact Gaussian entries, independently of libm ----------------------------
_PI50 = "3.14159265358979323846264338327950288419716939937510"


def _dec_cos(x, D):
    """cos(x) for a Decimal x in [0, 2 pi), by reduction to [-pi, pi] and its
    Taylor series (terms until they fall below 1e-55)."""
    pi = D(_PI50)
    if x > pi:
        x -= 2 * pi
    x2, term, total, k = x * x, D(1), D(1), 0
    while abs(term) > D("1e-55"):
        k += 2
        term = -term * x2 / (k * (k - 1))
        total += term
    return total


def _box_muller_exact(seed, i, j):
    """Box & Muller (1958), z = sqrt(-2 ln u1) cos(2 pi u2), in 50-digit
    decimal arithmetic from the uniforms of the Philox stream: counter
    (i, j_lo, j_hi, 2), u1 = (2^26 (w0 >> 5) + (w1 >> 6) + 1) / 2^53 in (0, 1],
    u2 = (2^26 (w2 >> 5) + (w3 >> 6)) / 2^53 in [0, 1)."""
    import decimal

    D = decimal.Decimal
    ctx = decimal.Context(prec=50)
    w = [int(v) for v in O.philox4x32_10([i, j & 0xFFFFFFFF, j >> 32, 2], [seed & 0xFFFFFFFF, seed >> 32])]
    n1 = (w[0] >> 5) * 2**26 + (w[1] >> 6) + 1
    n2 = (w[2] >> 5) * 2**26 + (w[3] >> 6)
    with decimal.localcontext(ctx):
        u1 = D(n1) / D(2**53)
        u2 = D(n2) / D(2**53)
        rad = (-2 * u1.ln()).sqrt()
        return float(rad * _dec_cos(2 * D(_PI50) * u2, D)), float(rad)


def test_gaussian_entries_match_box_muller_in_high_precision():
    """Pin of the exact Gaussian entry values: sampled entries recomputed with
    Box-Muller in 50-digit decimal arithmetic (no libm), from the Philox
    stream pinned above.  The FP64 entry can differ from the exact value only
    by the errors of log, sqrt, cos and the products, and by the rounded
    2 pi, a few units of 2^-52 scaled by the radius.  Swapped uniforms, sin for
    cos or a wrong shift in forming the uniforms give O(1) differences (the
    +1 that keeps u1 away from 0 moves an entry by less than the FP64 error
    and is not resolved here)."""
    rng = np.random.default_rng(3)
    worst = 0.0
    for seed in (0, 2024, 0xDEADBEEFCAFE):
        for _ in range(150):
            i, j = int(rng.integers(0, 1 << 20)), int(rng.integers(0, 1 << 34))
            z, rad = _box_muller_exact(seed, i, j)
            got = O.gaussian_entry(seed, i, j)
            err = abs(got - z)
            assert err <= 4e-15 * rad + 1e-300, (seed, i, j, got, z)
            worst = max(worst, err / max(rad, 1e-300))
    assert worst < 4e-15


@pytest.mark.parametrize("prec", [O.FP8_E4M3, O.BF16, O.FP16, O.FP32])
def test_rounded_gaussian_operator_matches_exact_values(prec):
    """The low-precision operator holds the exact Box-Muller value rounded
    once to the target format.  Entries whose FP64 value lies within the
    FP64 error bound of a rounding boundary of the target are skipped:
    there, the FP64 and the exact value may round apart."""
    seed, s, m = 99, 24, 40
    Om = O.gaussian_operator(seed, s, m, prec)
    skipped = 0
    for j in range(m):
        for i in range(s):
            z, rad = _box_muller_exact(seed, i, j)
            lo, hi = O.round_to(np.array([z - 4e-15 * rad]), prec)[0], O.round_to(np.array([z + 4e-15 * rad]), prec)[0]
            if lo != hi:
                skipped += 1
                continue
            assert Om[i, j] == lo, (prec, i, j, Om[i, j], z)
    assert skipped <= 2
