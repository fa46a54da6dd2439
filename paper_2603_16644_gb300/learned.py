"""Training and use of the learned precision proposer.

The proposer maps 10 cheap features of A (column-norm statistics and the
diagonal of an FP8-sketch preconditioner, computed by the library's kernels)
to one of {FP8-e4m3, BF16, FP32, FP64} for the sketch of Alg. 1.  Its MLP is
trained on the GPU by the library's own forward / backward / Adam kernels.

Training matrices have a known condition number: A = (G / sqrt(m)) diag(sigma)
V^T with G Gaussian (so G / sqrt(m) is close to orthonormal for m >> n),
V orthogonal (drawn from a small seeded pool per n, so that no QR runs per
sample) and sigma log-spaced from 1 to 1/kappa, kappa log-uniform.  The
label is the lowest precision u_p with u_p * kappa <= 1 (the regime of Lemma
rscond, eps kappa(R_s) < 1), i.e. FP8 for kappa <= 16, BF16 <= 256, FP32
<= 2^24, FP64 otherwise -- the same rule the second-opinion judge applies to
the computed preconditioner.  Input normalisation is folded into the first
layer.  ``train_default`` is the training run of the shipped weights
(``proposer_weights.npy``: 200k matrices with m <= 20000, n <= 256, kappa
log-uniform in [1e1, 1e12]); ``evaluate`` compares the learned solve with the
estimator-only solves on a batch of uneven problems.
"""
import math
import os
import time

import numpy as np
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


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposer_weights.npy")
_V_POOL = {}


def _orthogonal(n, gen, device, pool=8):
    """A pool of `pool` seeded random orthogonal n x n matrices (FP32)."""
    key = (n, str(device))
    if key not in _V_POOL:
        Vs = []
        for _ in range(pool):
            H = torch.randn((n, n), generator=gen, dtype=torch.float32, device=device)
            V, R = torch.linalg.qr(H)
            Vs.append(V * torch.sign(torch.diagonal(R)))
        _V_POOL[key] = Vs
    return _V_POOL[key]


def random_matrix(m, n, kappa, gen, device="cuda", pick=0):
    """Column-major FP64 A with kappa(A) close to kappa (see module doc)."""
    G = torch.randn((n, m), generator=gen, dtype=torch.float32, device=device).t() / math.sqrt(m)
    V = _orthogonal(n, gen, device)[pick % 8]
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
        A = random_matrix(m, n, 10.0 ** k, gen, device, pick=i)
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


def save(params, path=WEIGHTS):
    np.save(path, params.detach().cpu().numpy().astype(np.float32))


def load(path=WEIGHTS, device="cuda"):
    """The shipped weights (raw-feature input), or None if absent."""
    if not os.path.exists(path):
        return None
    return torch.from_numpy(np.load(path)).to(device)


def train_default(count=200000, heldout=20000, seed=2603, epochs=40, log=None):
    """The training run of the shipped weights: `count` generated matrices
    (m <= 20000, n <= 256, kappa log-uniform in [1e1, 1e12]), features and
    training on the GPU by the library's kernels, accuracy on `heldout`
    fresh matrices.  Returns (params, losses, train accuracy, held-out
    accuracy, seconds)."""
    t0 = time.time()
    X, y, _ = make_training_set(count, seed=seed)
    Xh, yh, _ = make_training_set(heldout, seed=seed + 7919)
    params, losses = train(X, y, epochs=epochs, batch=4096, lr=2e-3, seed=seed, log=log)
    return params, losses, accuracy(params, X, y), accuracy(params, Xh, yh), time.time() - t0


def c3_like_problems(count, seed, device="cuda", m_range=(2000, 40000), n_range=(32, 512)):
    """Uneven problems drawn like the batched workload: m, n uniform, kappa
    log-uniform in [1e2, 1e10], relative residual log-uniform in
    [1e-12, 1e-2] (problems.make_problem_torch)."""
    import problems as P

    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        m = int(rng.integers(max(m_range[0], 4 * n), m_range[1] + 1))
        kap = float(10 ** rng.uniform(2, 10))
        rho = float(10 ** rng.uniform(-12, -2))
        A, b, x_star, _, _ = P.make_problem_torch(m, n, kap, rho, seed * 100000 + i, device=device)
        out.append({"A": A, "b": b, "x_star": x_star, "kappa": kap, "rho": rho, "seed": seed * 100000 + i})
    return out


def evaluate(params, problems, sketch_kind=None, log=None):
    """Solve every problem three ways -- the learned proposal judged by the
    estimator on a sketch, the estimator on a sketch alone (AUTO_SKETCH) and
    the paper's estimator on A^T A (AUTO) -- with PNE, a Gaussian sketch of
    s = 2n and one refinement step.  Returns per-arm solves/s (CUDA events
    around the whole batch), errors against x_*, the precisions used and the
    escalation count of the learned arm."""
    from . import AUTO, AUTO_SKETCH, GAUSSIAN, make_opts, pne, pne_learned

    kind = GAUSSIAN if sketch_kind is None else sketch_kind

    def opts(p, prec):
        n = p["A"].shape[1]
        return make_opts(kind=kind, s=2 * n, zeta=min(8, 2 * n), seed=p["seed"], sketch_prec=prec,
                         qr_prec=FP32, refine_steps=1)

    res = {}
    for arm in ("learned", "auto_sketch", "auto"):
        xs, used, esc = [], [], 0
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for p in problems:
            if arm == "learned":
                x, info, u, e = pne_learned(p["A"], p["b"], params, opts(p, FP64))
                used.append(u)
                esc += e
            else:
                x, info = pne(p["A"], p["b"], opts=opts(p, AUTO_SKETCH if arm == "auto_sketch" else AUTO))
            xs.append((x, info))
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1000.0
        errs = [float(torch.linalg.norm(x - p["x_star"]) / torch.linalg.norm(x)) for (x, _), p in zip(xs, problems)]
        infos = [int(i.item()) for _, i in xs]
        res[arm] = {"solves_per_s": len(problems) / sec, "seconds": sec, "errors": errs, "infos": infos,
                    "x": [x.cpu().numpy() for x, _ in xs]}
        if arm == "learned":
            res[arm]["used"] = used
            res[arm]["escalations"] = esc
        if log:
            log(f"{arm}: {len(problems) / sec:.1f} solves/s")
    return res
