"""Pins of the oracle's learned-proposal pieces (not in the paper): the MLP
gradient against central finite differences of its own loss, the forward
pass on closed-form cases, and the features against independent numpy
evaluations."""
import numpy as np
import pytest

import oracle as O
import problems as P


def rand_params(d, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(O.mlp_param_count(d)) * scale


def test_param_count():
    d = 10
    assert O.mlp_param_count(d) == 64 * d + 64 + 2 * (64 * 64 + 64) + 4 * 64 + 4


def test_forward_closed_forms():
    d = 10
    p = np.zeros(O.mlp_param_count(d))
    p[-4:] = [0.5, -1.0, 2.0, 0.0]  # only the output bias: logits = b4
    X = np.random.default_rng(0).standard_normal((7, d))
    logits, loss = O.mlp_forward(p, X, np.array([2] * 7))
    np.testing.assert_allclose(logits, np.tile(p[-4:], (7, 1)))
    z = p[-4:]
    assert loss == pytest.approx(-(z[2] - np.log(np.exp(z).sum())))
    # one hidden unit path: W1[0,0]=1, W2[0,0]=1, W3[0,0]=1, W4[1,0]=3 -> logit1 = 3 relu(x0)
    q = np.zeros(O.mlp_param_count(d))
    q[0] = 1.0
    o2 = 64 * d + 64
    q[o2] = 1.0
    o3 = o2 + 64 * 64 + 64
    q[o3] = 1.0
    o4 = o3 + 64 * 64 + 64
    q[o4 + 64] = 3.0
    X = np.array([[2.0] + [0.0] * (d - 1), [-1.0] + [0.0] * (d - 1)])
    logits, _ = O.mlp_forward(q, X)
    np.testing.assert_allclose(logits[:, 1], [6.0, 0.0])


def test_backward_matches_finite_differences():
    d, B = 10, 9
    rng = np.random.default_rng(1)
    p = rand_params(d, 2)
    X = rng.standard_normal((B, d))
    lab = rng.integers(0, 4, B)
    loss, g = O.mlp_backward(p, X, lab)
    _, loss_f = O.mlp_forward(p, X, lab)
    assert loss == pytest.approx(loss_f, rel=1e-14)
    idx = rng.choice(p.size, 200, replace=False)
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (O.mlp_forward(pp, X, lab)[1] - O.mlp_forward(pm, X, lab)[1]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_features_column_norm_closed_form():
    m, n = 2000, 40
    pr = P.make_problem(m, n, 10.0, 0.0, 3)
    scale = np.exp2(np.arange(n) % 7)
    A = np.asfortranarray(pr.A * scale[None, :])
    f = O.features(A, 5)
    cn = np.log10(np.linalg.norm(A, axis=0))
    assert f[0] == pytest.approx(np.log2(m) / 16) and f[1] == pytest.approx(np.log2(n) / 10)
    assert f[2] == pytest.approx(cn.max() - cn.min(), rel=1e-12)
    assert f[3] == pytest.approx(cn.std(), rel=1e-10)


def test_features_diag_r_against_numpy():
    m, n = 3000, 50
    pr = P.make_problem(m, n, 1e3, 0.0, 4)
    f = O.features(pr.A, 9)
    As, e = O.sketch(pr.A, O.SPARSE_SIGN, 2 * n, 8, 9, O.FP8_E4M3)
    R = np.linalg.qr(As, mode="r") * np.exp2(-e)[None, :]
    ld = np.log10(np.abs(np.diag(R)))
    t = np.arange(n) / n
    assert f[4] == pytest.approx(ld.max() - ld.min(), abs=1e-4)
    assert f[5] == pytest.approx(ld.std(), abs=1e-4)
    assert f[6] == pytest.approx(np.polyfit(t, ld, 1)[0], abs=1e-3)
    q0 = n - (n + 3) // 4
    assert f[7] == pytest.approx(ld[q0:].max() - ld[q0:].min(), abs=1e-4)
    assert f[8] == pytest.approx(np.mean(ld < ld.max() - 2.0))
    assert f[9] == pytest.approx(ld.min() - np.log10(np.linalg.norm(pr.A) / np.sqrt(n)), abs=1e-4)
    # the diag-R spread grows with the conditioning
    f_hi = O.features(P.make_problem(m, n, 1e8, 0.0, 4).A, 9)
    assert f_hi[4] > f[4]
