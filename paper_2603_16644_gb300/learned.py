"""Training and use of the learned precision proposer.

The proposer maps 10 cheap features of A (column-norm statistics and the
diagonal of an FP8-sketch preconditioner, computed by the library's kernels)
to one of {FP8-e4m3, BF16, FP32, FP64} for the sketch of Alg. 1.  Its MLP is
trained on the GPU by the library's own forward / backward / Adam kernels.

Training matrices have a known condition number: A = (G / sqrt(m)) diag(sigma)
V^T with G Gaussian (so G / sqrt(m) is close to orthonormal for m >> n),
V orthogonal and sigma log-spaced from 1 to 1/kappa, kappa log-uniform.  The
label is the lowest precision u_p with u_p * kappa <= 1 (the regime of Lemma
rscond, eps kappa(R_s) < 1), i.e. FP8 for kappa <= 16, BF16 <= 256, FP32
<= 2^24, FP64 otherwise -- the same rule the judge applies to the computed
preconditioner.  Input normalisation is folded into the first layer.
"""
import math

import torch

from . import (BF16, FP8_E4M3, FP32, FP64, N_FEATURES, features, mlp_adam, mlp_backward, mlp_forward,
               mlp_param_count)

CLASS_PRECS = [FP8_E4M3, BF16, FP32, FP64]
_U = {0: 2.0 ** -4, 1: 2.0 ** -8, 2: 2.0 ** -24}


def label_for_kappa(kappa: float) -> int:
    for c in (0, 1, 2):
        if _U[c] * kappa <= 1.0:
            return c
    return 3


def random_matrix(m, n, kappa, gen, device="cuda"):
    """Column-major FP64 A with kappa(A) close to kappa (see module doc)."""
    G = torch.randn((n, m), generator=gen, dtype=torch.float32, device=device).t() / math.sqrt(m)
    H = torch.randn((n, n), generator=gen, dtype=torch.float32, device=device)
    V, _ = torch.linalg.qr(H)
    sigma = torch.logspace(0.0, -math.log10(kappa), n, dtype=torch.float32, device=device)
    A = torch.empty((n, m), dtype=torch.float64, device=device).t()
    A.copy_((G * sigma) @ V.t())
    return A


def make_training_set(count, m_range=(500, 20000), n_range=(16, 256), log10_kappa=(1.0, 12.0), seed=2603,
                      device="cuda"):
    """(X (count x 10) float32, labels (count) int32, log10 kappa) on the device."""
    gen = torch.Generator(device=device).manual_seed(seed)
    rng = torch.Generator(device="cpu").manual_seed(seed)
    X = torch.empty((count, N_FEATURES), dtype=torch.float32, device=device)
    y = torch.empty(count, dtype=torch.int32)
    lk = torch.empty(count, dtype=torch.float64)
    for i in range(count):
        n = int(torch.randint(n_range[0], n_range[1] + 1, (1,), generator=rng))
        m = int(torch.randint(max(m_range[0], 4 * n), max(m_range[1], 4 * n) + 1, (1,), generator=rng))
        k = float(torch.empty(1).uniform_(*log10_kappa, generator=rng))
        A = random_matrix(m, n, 10.0 ** k, gen, device)
        X[i] = features(A, seed=seed + i)
        y[i] = label_for_kappa(10.0 ** k)
        lk[i] = k
    return X, y.to(device), lk


def init_params(d=N_FEATURES, seed=0, device="cuda"):
    g = torch.Generator(device="cpu").manual_seed(seed)
    parts = []
    for out, inp in [(64, d), (64, 64), (64, 64), (4, 64)]:
        parts.append(torch.randn(out * inp, generator=g) * math.sqrt(2.0 / inp))
        parts.append(torch.zeros(out))
    p = torch.cat(parts).to(torch.float32).to(device)
    assert p.numel() == mlp_param_count(d)
    return p


def fold_normalisation(params, mean, std, d=N_FEATURES):
    """Return parameters that take raw features: W1' = W1 / std, b1' = b1 - W1' mean."""
    p = params.clone()
    W1 = p[: 64 * d].view(64, d)
    b1 = p[64 * d: 64 * d + 64]
    W1n = W1 / std[None, :]
    b1.sub_(W1n @ mean)
    W1.copy_(W1n)
    return p


def train(X, y, epochs=30, batch=1024, lr=2e-3, seed=0, log=None):
    """Adam on the softmax cross-entropy with the library kernels; returns
    (parameters for raw features, per-epoch mean losses)."""
    dev = X.device
    mean = X.mean(0)
    std = X.std(0).clamp_min(1e-3)
    Xn = ((X - mean) / std).contiguous()
    p = init_params(X.shape[1], seed, dev)
    m1 = torch.zeros_like(p)
    m2 = torch.zeros_like(p)
    g = torch.Generator(device="cpu").manual_seed(seed)
    step = 0
    losses = []
    N = X.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(N, generator=g).to(dev)
        tot, nb = 0.0, 0
        for s0 in range(0, N, batch):
            idx = perm[s0: s0 + batch]
            grad, loss = mlp_backward(p, Xn[idx].contiguous(), y[idx].contiguous())
            step += 1
            mlp_adam(p, grad, m1, m2, step, lr=lr)
            tot += float(loss.item())
            nb += 1
        losses.append(tot / nb)
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4f}")
    return fold_normalisation(p, mean, std), losses


def accuracy(params, X, y):
    logits = mlp_forward(params, X)
    return float((logits.argmax(1).to(torch.int32) == y).float().mean())
