"""The seeded input generators hold the properties the tests rely on: the
stated singular values and right singular vectors, a least-squares residual
orthogonal to range(A) with the stated relative size, column-major layout."""
import numpy as np
import pytest
import torch

import problems as P


@pytest.mark.parametrize("m,n,kappa,rho", [(1024, 40, 1e4, 1e-3), (4096, 64, 1e8, 0.0), (256, 1, 1.0, 1e-6)])
def test_hadamard_generator(m, n, kappa, rho):
    A, b, x_star, sigma, V = P.make_problem_hadamard_torch(m, n, kappa, rho, 11, device="cpu")
    assert A.shape == (m, n) and A.stride() == (1, m)
    An, s, Vn = A.numpy(), sigma.numpy(), V.numpy()
    sv = np.linalg.svd(An, compute_uv=False)
    # to the rounding of forming A (absolute, ~u ||A||)
    np.testing.assert_allclose(sv, s, rtol=0, atol=1e-13 * s[0])
    assert s[0] == 1.0 and np.isclose(s[0] / s[-1], kappa, rtol=1e-12)
    np.testing.assert_allclose(Vn.T @ Vn, np.eye(n), atol=1e-14)
    np.testing.assert_allclose(An.T @ An, (Vn * s**2) @ Vn.T, atol=1e-14)
    # b - A x_* carries the rounding of A x_* (~u ||A|| ||x_*||)
    r = (b - A @ x_star).numpy()
    nx = np.linalg.norm(x_star.numpy())
    assert abs(np.linalg.norm(r) - rho * s[0] * nx) <= 1e-14 * nx
    assert np.linalg.norm(An.T @ r) <= 1e-14 * nx


def test_hadamard_generator_rejects_bad_shapes():
    with pytest.raises(ValueError):
        P.make_problem_hadamard_torch(1000, 10, 1e2, 0.0, 1, device="cpu")
    with pytest.raises(ValueError):
        P.make_problem_hadamard_torch(64, 64, 1e2, 0.0, 1, device="cpu")


def test_gaussian_generator_matches_its_statement():
    pr = P.make_problem(500, 20, 1e6, 1e-4, 5)
    sv = np.linalg.svd(pr.A, compute_uv=False)
    np.testing.assert_allclose(sv, pr.sigma, rtol=1e-10)
    r = pr.b - pr.A @ pr.x_star
    assert np.linalg.norm(r) == pytest.approx(1e-4 * np.linalg.norm(pr.x_star), rel=1e-10)
    assert np.linalg.norm(pr.A.T @ r) <= 1e-13 * np.linalg.norm(r)
