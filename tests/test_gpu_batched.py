"""Batched solver (many uneven problems in one cached CUDA-graph launch):
every problem's result equals the single-problem call bit for bit (same
kernels, same inputs), replays reuse the graph and see new data, AUTO
precisions are resolved per problem, and the results meet the solution
tolerance against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import problems as P
from tests.gpu_util import assert_solution_parity, dev_colmajor, oracle_realizations, to_np

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")


def make_batch(count, seed, auto=False):
    rng = np.random.default_rng(seed)
    probs, opts = [], []
    for i in range(count):
        n = int(rng.integers(16, 129))
        m = int(rng.integers(max(500, 4 * n), 5001))
        kap = float(10 ** rng.uniform(2, 8 if not auto else 10))
        rho = float(10 ** rng.uniform(-12, -2))
        pr = P.make_problem(m, n, kap, rho, seed * 1000 + i)
        kind = lsq.SPARSE_SIGN if i % 2 == 0 else lsq.GAUSSIAN
        s = (2 if i % 3 else 4) * n
        prec = lsq.AUTO if auto else [lsq.BF16, lsq.FP32, lsq.FP64, lsq.FP16][i % 4]
        opts.append(lsq.make_opts(kind=kind, s=s, zeta=min(8, s), seed=7 + i, sketch_prec=prec,
                                  qr_prec=lsq.FP64 if prec == lsq.FP64 else lsq.FP32, refine_steps=i % 2))
        probs.append(pr)
    return probs, opts


def test_batched_equals_single_calls_bitwise():
    probs, opts = make_batch(12, 1)
    As = [dev_colmajor(p.A) for p in probs]
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    xs = [torch.empty(p.shape[1], dtype=torch.float64, device="cuda") for p in probs]
    infos = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in probs]
    desc = lsq.batch_descriptors(As, bs, xs, infos, opts)
    ws = lsq.batched_workspace(desc)
    lsq.solve_batched(desc, ws)
    xb = [to_np(x).copy() for x in xs]
    for i, p in enumerate(probs):
        assert int(to_np(infos[i])[0]) == 0
        x1, info1 = lsq.pne(As[i], bs[i], opts=opts[i])
        np.testing.assert_array_equal(to_np(x1), xb[i])
    # replay (cached graph) gives the same bits; new data in the same buffers is used
    lsq.solve_batched(desc, ws)
    for i in range(len(probs)):
        np.testing.assert_array_equal(to_np(xs[i]), xb[i])
    bs[0].mul_(2.0)
    lsq.solve_batched(desc, ws)
    np.testing.assert_allclose(to_np(xs[0]), 2 * xb[0], rtol=1e-9)


@pytest.mark.parametrize("hpne", [False, True])
def test_batched_against_oracle(hpne):
    probs, opts = make_batch(6, 2)
    As = [dev_colmajor(p.A) for p in probs]
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    xs = [torch.empty(p.shape[1], dtype=torch.float64, device="cuda") for p in probs]
    infos = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in probs]
    desc = lsq.batch_descriptors(As, bs, xs, infos, opts)
    ws = lsq.batched_workspace(desc, hpne=hpne)
    lsq.solve_batched(desc, ws, hpne=hpne)
    for i, p in enumerate(probs):
        o = opts[i]
        ref = O.solve(p.A, p.b, hpne=hpne, kind=o.kind, s=o.s, zeta=o.zeta, seed=o.seed, sketch_prec=o.sketch_prec,
                      qr_prec=o.qr_prec, refine_steps=o.refine_steps)
        assert int(to_np(infos[i])[0]) == ref["info"] == 0
        more = oracle_realizations(p, hpne=hpne, kind=o.kind, s=o.s, zeta=o.zeta, seed=o.seed,
                                   sketch_prec=o.sketch_prec, qr_prec=o.qr_prec, refine_steps=o.refine_steps)
        assert_solution_parity(to_np(xs[i]), ref["x"], p.x_star, p.kappa, p.rho, f"problem {i}",
                               refined=o.refine_steps > 0, u_p=o.sketch_prec, realizations=more)


def test_batched_auto_precision_per_problem():
    probs, opts = make_batch(8, 3, auto=True)
    As = [dev_colmajor(p.A) for p in probs]
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    xs = [torch.empty(p.shape[1], dtype=torch.float64, device="cuda") for p in probs]
    infos = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in probs]
    desc = lsq.batch_descriptors(As, bs, xs, infos, opts)
    ws = lsq.batched_workspace(desc)
    lsq.solve_batched(desc, ws)
    for i in range(len(probs)):
        x1, _ = lsq.pne(As[i], bs[i], opts=opts[i])
        np.testing.assert_array_equal(to_np(x1), to_np(xs[i]))


def test_batched_bad_input():
    probs, opts = make_batch(2, 4)
    As = [dev_colmajor(p.A) for p in probs]
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    xs = [torch.empty(p.shape[1], dtype=torch.float64, device="cuda") for p in probs]
    infos = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in probs]
    opts[1].s = 1  # s < n
    desc = lsq.batch_descriptors(As, bs, xs, infos, opts)
    with pytest.raises(lsq.LsqError):
        lsq.batched_workspace(desc)
    with pytest.raises(lsq.LsqError):
        lsq.solve_batched(desc, torch.empty(1024, dtype=torch.uint8, device="cuda"))


def test_autotuner_picks_a_candidate(tmp_path):
    from paper_2603_16644_gb300.autotune import CANDIDATES, Autotuner

    tuner = Autotuner(path=str(tmp_path / "tune.json"))
    kind, s = tuner.choose(3000, 100, prec=lsq.FP32)
    assert (kind, s // 100) in CANDIDATES
    again = Autotuner(path=str(tmp_path / "tune.json"))
    assert again.choose(3000, 100, prec=lsq.FP32) == (kind, s)
