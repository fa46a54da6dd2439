"""Seeded synthetic least-squares problems with a known solution.

Shared input generator for the tests, the benchmark and the smoke check.  It
holds none of the solver's arithmetic: it only builds inputs.

Construction (after Alg. 2 of Garrison & Ipsen, arXiv 2603.16644, with the
singular values set explicitly):
    A = U diag(sigma) V^T, U (m x n) with orthonormal columns from the QR of
    a seeded Gaussian matrix, V (n x n) orthogonal likewise, sigma
    log-spaced from 1 down to 1/kappa, so ||A|| = 1 and kappa(A) = kappa;
    x_* ~ N(0, 1) (not normalised);
    r_perp = (I - U U^T)(I - U U^T) g for a Gaussian g, normalised, so that
    it is orthogonal to range(A) to rounding (projection applied twice);
    b = A x_* + beta r_perp with beta = rho ||A|| ||x_*||, so the relative
    least-squares residual ||b - A x_*|| / (||A|| ||x_*||) equals rho.

Seeds: 2603_16644 + 1000 * config + problem index.
"""
from dataclasses import dataclass
import math

import numpy as np

BASE_SEED = 2603_16644


def seed_for(config: int, index: int) -> int:
    return BASE_SEED + 1000 * config + index


@dataclass
class Problem:
    A: np.ndarray          # (m, n) float64, Fortran order
    b: np.ndarray          # (m,)
    x_star: np.ndarray     # (n,)
    kappa: float
    rho: float
    seed: int
    sigma: np.ndarray      # singular values of A, descending
    V: np.ndarray          # right singular vectors (n, n)

    @property
    def shape(self):
        return self.A.shape


def _orthonormal(rng, rows, cols):
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G)
    # make the factor unique (positive diagonal of R): Haar-distributed Q
    return Q * np.sign(np.where(np.diag(R) == 0, 1.0, np.diag(R)))


def make_problem(m: int, n: int, kappa: float, rho: float, seed: int, integer: bool = False) -> Problem:
    """Generate one problem.  ``integer=True`` makes a consistent system with
    small-integer A and x_* (b = A x_* exactly in FP64), used where the exact
    solution must be known to the last bit."""
    rng = np.random.default_rng(seed)
    if integer:
        A = rng.integers(-8, 9, size=(m, n)).astype(np.float64)
        while np.linalg.matrix_rank(A) < n:
            A = rng.integers(-8, 9, size=(m, n)).astype(np.float64)
        x = rng.integers(-4, 5, size=n).astype(np.float64)
        b = A @ x
        sv = np.linalg.svd(A, compute_uv=False)
        return Problem(np.asfortranarray(A), b, x, float(sv[0] / sv[-1]), 0.0, seed, sv,
                       np.eye(n))
    U = _orthonormal(rng, m, n)
    V = _orthonormal(rng, n, n)
    sigma = np.logspace(0.0, -math.log10(kappa), n) if n > 1 else np.ones(1)
    A = np.asfortranarray((U * sigma) @ V.T)
    x_star = rng.standard_normal(n)
    g = rng.standard_normal(m)
    r = g - U @ (U.T @ g)
    r = r - U @ (U.T @ r)
    r /= np.linalg.norm(r)
    beta = rho * sigma[0] * np.linalg.norm(x_star)
    b = A @ x_star + beta * r
    return Problem(A, b, x_star, float(kappa), float(rho), seed, sigma, V)


def make_problem_torch(m: int, n: int, kappa: float, rho: float, seed: int, device="cuda"):
    """Same construction on a torch device (used for the large shapes where a
    CPU QR of the Gaussian factor is slow).  Returns (A, b, x_star, sigma, V)
    as float64 torch tensors; A is column-major (stride (1, m))."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    G = torch.randn(m, n, generator=g, dtype=torch.float64).to(device)
    H = torch.randn(n, n, generator=g, dtype=torch.float64).to(device)
    U, Ru = torch.linalg.qr(G)
    U = U * torch.sign(torch.diagonal(Ru)).clamp(min=-1).where(torch.diagonal(Ru) != 0,
                                                               torch.ones(1, dtype=torch.float64, device=device))
    del G
    V, Rv = torch.linalg.qr(H)
    V = V * torch.sign(torch.diagonal(Rv))
    sigma = torch.logspace(0.0, -math.log10(kappa), n, dtype=torch.float64, device=device)
    A = torch.empty(n, m, dtype=torch.float64, device=device).t()
    A.copy_((U * sigma) @ V.t())
    x_star = torch.randn(n, generator=g, dtype=torch.float64).to(device)
    gv = torch.randn(m, generator=g, dtype=torch.float64).to(device)
    r = gv - U @ (U.t() @ gv)
    r = r - U @ (U.t() @ r)
    r = r / torch.linalg.norm(r)
    beta = rho * float(sigma[0]) * float(torch.linalg.norm(x_star))
    b = A @ x_star + beta * r
    del U
    return A, b, x_star, sigma, V


def make_problem_hadamard_torch(m: int, n: int, kappa: float, rho: float, seed: int, device="cuda"):
    """The same construction with U from signed columns of the normalised
    Sylvester-Hadamard matrix (m a power of two): U = D H[:, J] / sqrt(m),
    D a seeded diagonal of signs, J n seeded distinct column indices, so U
    has orthonormal columns exactly, and A = U diag(sigma) V^T is formed by
    fast Walsh-Hadamard transforms of the columns of diag(sigma) V^T placed at
    rows J (n m log2 m additions instead of an m x n QR and an m n^2 product;
    used for the largest shapes).  r_perp is another signed Hadamard column,
    orthogonal to range(A).  Returns (A, b, x_star, sigma, V) as float64 torch
    tensors; A is column-major (stride (1, m))."""
    import torch
    if m & (m - 1) or n >= m:
        raise ValueError("m must be a power of two larger than n")
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(m, generator=g)
    J, k_perp = perm[:n].to(device), int(perm[n])
    D = (torch.randint(0, 2, (m,), generator=g) * 2 - 1).to(device=device, dtype=torch.float64)
    H = torch.randn(n, n, generator=g, dtype=torch.float64).to(device)
    V, Rv = torch.linalg.qr(H)
    V = V * torch.sign(torch.diagonal(Rv))
    sigma = torch.logspace(0.0, -math.log10(kappa), n, dtype=torch.float64, device=device)
    # rows of A^T (= columns of A): the rows of (diag(sigma) V^T)^T = V diag(sigma)
    # placed at positions J, then the Walsh-Hadamard transform along them
    X = torch.zeros(n, m, dtype=torch.float64, device=device)
    X[:, J] = V * sigma
    h = 1
    while h < m:
        Y = X.view(n, m // (2 * h), 2, h)
        a, c = Y[:, :, 0, :], Y[:, :, 1, :]
        X = torch.stack((a + c, a - c), dim=2).view(n, m)
        h *= 2
    X.mul_(D / math.sqrt(m))
    A = X.t()  # column-major m x n
    x_star = torch.randn(n, generator=g, dtype=torch.float64).to(device)
    # r_perp: Hadamard column k_perp (not in J), signed by D, unit norm
    idx = torch.arange(m, device=device, dtype=torch.int64) & k_perp
    par = torch.zeros(m, dtype=torch.int64, device=device)
    while bool(idx.any()):
        par ^= idx & 1
        idx >>= 1
    r = D * (1.0 - 2.0 * par.to(torch.float64)) / math.sqrt(m)
    beta = rho * float(sigma[0]) * float(torch.linalg.norm(x_star))
    b = A @ x_star + beta * r
    return A, b, x_star, sigma, V


def rel_error(x_hat, x_star) -> float:
    """||x_hat - x_*|| / ||x_hat||, the error measure of the paper's figures."""
    x_hat = np.asarray(x_hat, dtype=np.float64)
    return float(np.linalg.norm(x_hat - np.asarray(x_star)) / np.linalg.norm(x_hat))
