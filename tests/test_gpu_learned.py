"""Learned precision proposal on the GPU: MLP forward and gradients against
the FP64 oracle, features against the oracle's, the judge against exact
condition numbers, training that learns, and the learned PNE solve against
the oracle at the precision it ends up using."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import oracle as O
import problems as P
from tests.gpu_util import U_P, assert_solution_parity, dev_colmajor, gpu_realizations, oracle_realizations, to_np

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")


def test_mlp_forward_and_gradient_match_oracle():
    d, B = lsq.N_FEATURES, 333
    rng = np.random.default_rng(0)
    p = rng.standard_normal(O.mlp_param_count(d)) * 0.2
    X = rng.standard_normal((B, d))
    y = rng.integers(0, 4, B).astype(np.int32)
    pt = torch.from_numpy(p).float().cuda()
    Xt = torch.from_numpy(X).float().cuda()
    logits = to_np(lsq.mlp_forward(pt, Xt))
    # oracle on the same FP32-rounded inputs, in FP64
    p32 = p.astype(np.float32).astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    lo, _ = O.mlp_forward(p32, X32)
    assert np.max(np.abs(logits - lo)) <= 1e-5 * max(1.0, np.abs(lo).max())
    g, loss = lsq.mlp_backward(pt, Xt, torch.from_numpy(y).cuda())
    lo_loss, go = O.mlp_backward(p32, X32, y)
    assert abs(float(to_np(loss)[0]) - lo_loss) <= 1e-5 * max(1.0, lo_loss)
    g = to_np(g).astype(np.float64)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)


def test_features_match_oracle():
    for (m, n, kap) in [(3000, 50, 1e3), (2048, 128, 1e8), (700, 20, 10.0)]:
        pr = P.make_problem(m, n, kap, 0.0, 5)
        f = to_np(lsq.features(dev_colmajor(pr.A), seed=9)).astype(np.float64)
        fo = O.features(pr.A, 9)
        np.testing.assert_allclose(f[:4], fo[:4], rtol=1e-5, atol=1e-5)
        # diag R: same bit-exact FP8 sketch, FP32 QR in another order
        np.testing.assert_allclose(f[4:], fo[4:], rtol=2e-2, atol=2e-2)


def test_judge_is_a_lower_bound_and_decides_by_lemma():
    for kap, prec, want in [(1e1, O.FP32, 1), (1e6, O.FP32, 1), (1e8, O.FP32, 0), (1e3, O.BF16, 0), (1.2, O.FP8_E4M3, 1), (5.0, O.FP8_E4M3, 0)]:
        n = 64
        rng = np.random.default_rng(int(np.log10(kap)) + prec)
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        Rn = np.linalg.qr(Q @ np.diag(np.logspace(0, -np.log10(kap), n)) @ Q.T, mode="r")
        R = Rn * np.sign(np.diag(Rn))[:, None]
        acc, k1 = lsq.judge_preconditioner(dev_colmajor(R), prec)
        k1 = float(to_np(k1)[0])
        exact = np.abs(R).sum(0).max() * np.abs(np.linalg.inv(R)).sum(0).max()
        assert k1 <= exact * (1 + 1e-3)
        assert k1 >= exact / 10
        u = {O.FP8_E4M3: 2.0 ** -4, O.BF16: 2.0 ** -8, O.FP32: 2.0 ** -24}[prec]
        assert int(to_np(acc)[0]) == int(u * k1 <= 1.0) == want


def test_training_learns_and_generalises():
    from paper_2603_16644_gb300 import learned

    X, y, lk = learned.make_training_set(800, m_range=(500, 2000), n_range=(16, 48), seed=11)
    params, losses = learned.train(X, y, epochs=40, batch=128, lr=3e-3)
    assert losses[-1] < 0.8 * losses[0]
    # accuracy on fresh matrices, not the training set
    Xh, yh, _ = learned.make_training_set(400, m_range=(500, 2000), n_range=(16, 48), seed=12)
    assert learned.accuracy(params, Xh, yh) > 0.6


def forced(cls):
    """MLP parameters whose proposal is class `cls` (0 FP8, 1 BF16, 2 FP32,
    3 FP64) for every input: zero weights, a large bias on that class."""
    p = torch.zeros(lsq.mlp_param_count(), dtype=torch.float32, device="cuda")
    p[-4 + cls] = 10.0
    return p


@pytest.mark.parametrize("cls,kap,want,esc_min", [(0, 1e5, O.FP32, 1), (3, 1e1, O.FP64, 0), (1, 1e1, O.BF16, 0),
                                                  (0, 1e10, O.FP64, 1)])
def test_estimator_judges_proposals(cls, kap, want, esc_min):
    # a proposal below the estimate's choice is replaced by it (the fallback);
    # an FP64 proposal is taken as it is
    pr = P.make_problem(3000, 40, kap, 1e-6, 77)
    opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=160, zeta=8, seed=5, refine_steps=1)
    x, info, used, esc = lsq.pne_learned(dev_colmajor(pr.A), torch.from_numpy(pr.b).cuda(), forced(cls), opts)
    assert int(to_np(info)[0]) == 0
    assert used == want and esc >= esc_min, (used, esc)
    k0, ch, _, _ = O.condest_sketch(pr.A, 5)
    # never below the estimator's choice, except by the proposal being higher
    assert used >= min(ch, O.FP64)


def test_learned_solve_matches_oracle_and_gains_over_the_estimate_on_AtA():
    from paper_2603_16644_gb300 import learned

    params = learned.load()
    if params is None:
        pytest.skip("no shipped weights")
    probs = learned.c3_like_problems(24, seed=41, m_range=(2000, 8000), n_range=(32, 128))
    res = learned.evaluate(params, probs)
    lower = 0
    for k, p in enumerate(probs):
        used = res["learned"]["used"][k]
        assert res["learned"]["infos"][k] == 0
        A, b, xs_ = p["A"].cpu().numpy(), p["b"].cpu().numpy(), p["x_star"].cpu().numpy()
        kw = dict(kind=O.GAUSSIAN, s=2 * A.shape[1], seed=p["seed"], sketch_prec=used,
                  qr_prec=O.FP64 if used == O.FP64 else O.FP32, refine_steps=1)
        ref = O.solve(A, b, **kw)
        # solution tolerance of the method at the precision the judged proposal used
        pr = SimpleNamespace(A=A, b=b)
        assert_solution_parity(res["learned"]["x"][k], ref["x"], xs_, p["kappa"], p["rho"], f"problem {k}",
                               refined=True, u_p=used, realizations=oracle_realizations(pr, k=8, **kw),
                               gpu_realizations=gpu_realizations(pr, k=8, **kw))
        ch = O.condest(A)[1]
        lower += used < ch
    # the gain: problems the estimate on A^T A sends to a higher precision
    # than the judged proposal needed (the FP32 Cholesky of A^T A breaks down
    # once kappa(A)^2 > 1/u32), at the same accuracy
    assert lower >= 1, lower
    print("learned vs estimate on A^T A (solves/s):", res["learned"]["solves_per_s"], res["auto"]["solves_per_s"],
          "escalations:", res["learned"]["escalations"], "lower precision on", lower, "of", len(probs))
