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


def test_batched_sketch_and_qr_equal_single_calls():
    # lsq_sketch_batched / lsq_precond_qr_batched: one captured fan-out, the
    # results of separate calls bit for bit
    rng = np.random.default_rng(9)
    As, opts = [], []
    for i in range(10):
        n = int(rng.integers(8, 200))
        m = int(rng.integers(4 * n, 6000))
        A = dev_colmajor(np.asfortranarray(rng.standard_normal((m, n)) * np.exp2(rng.integers(-8, 8, n))[None, :]))
        kind = lsq.SPARSE_SIGN if i % 2 else lsq.GAUSSIAN
        prec = [lsq.FP8_E4M3, lsq.BF16, lsq.FP16, lsq.FP32, lsq.FP64][i % 5]
        As.append(A)
        opts.append(lsq.make_opts(kind=kind, s=(2 + i % 3) * n, zeta=min(8, 2 * n), seed=100 + i, sketch_prec=prec))
    outs = lsq.sketch_batched(As, opts)
    for A, o, (Asb, ceb, infob) in zip(As, opts, outs):
        As1, ce1, info1 = lsq.sketch(A, o)
        assert int(to_np(infob)[0]) == int(to_np(info1)[0]) == 0
        np.testing.assert_array_equal(to_np(Asb), to_np(As1))
        np.testing.assert_array_equal(to_np(ceb), to_np(ce1))
    qr = lsq.precond_qr_batched([(Asb, ceb) for Asb, ceb, _ in outs])
    for (Asb, ceb, _), (Rb, infob), o in zip(outs, qr, opts):
        qp = lsq.FP64 if o.sketch_prec == lsq.FP64 else lsq.FP32
        R1, info1 = lsq.precond_qr(Asb, ceb, qp)
        assert int(to_np(infob)[0]) == int(to_np(info1)[0]) == 0
        np.testing.assert_array_equal(np.triu(to_np(Rb)), np.triu(to_np(R1)))


def test_batched_auto_sketch_per_problem():
    probs, opts = make_batch(8, 5, auto=True)
    for o in opts:
        o.sketch_prec = lsq.AUTO_SKETCH
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


def test_batched_full_size_uneven_batch():
    # the batched workload at full size: 512 problems, m uniform in [2000, 40000],
    # n uniform in [32, 512], kappa log-uniform in [1e2, 1e10], relative
    # residual log-uniform in [1e-12, 1e-2]; sketch kind and s in {2n, 4n} from
    # the autotuner, precision per problem from the estimate on a sketch
    from types import SimpleNamespace

    from paper_2603_16644_gb300.autotune import Autotuner

    rng = np.random.default_rng(2603)
    tuner = Autotuner()
    As, bs, xs, infos, opts, meta = [], [], [], [], [], []
    for i in range(512):
        n = int(rng.integers(32, 513))
        m = int(rng.integers(max(2000, 4 * n), 40001))
        kap = float(10 ** rng.uniform(2, 10))
        rho = float(10 ** rng.uniform(-12, -2))
        seed = P.seed_for(3, i)
        A, b, x_star, _, _ = P.make_problem_torch(m, n, kap, rho, seed)
        kind, s = tuner.choose(m, n, prec=lsq.FP32)
        As.append(A)
        bs.append(b)
        xs.append(torch.empty(n, dtype=torch.float64, device="cuda"))
        infos.append(torch.zeros(1, dtype=torch.int32, device="cuda"))
        opts.append(lsq.make_opts(kind=kind, s=s, zeta=min(8, s), seed=seed, sketch_prec=lsq.AUTO_SKETCH,
                                  qr_prec=lsq.FP32, refine_steps=0))
        meta.append((kap, rho, x_star))
    desc = lsq.batch_descriptors(As, bs, xs, infos, opts)
    ws = lsq.batched_workspace(desc)
    lsq.solve_batched(desc, ws)  # estimate pass, capture, first launch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lsq.solve_batched(desc, ws)  # estimate pass and one cached graph launch
    e1.record()
    torch.cuda.synchronize()
    print(f"512 uneven problems: {512 / (e0.elapsed_time(e1) / 1000):.1f} solves/s")
    assert all(int(to_np(f)[0]) == 0 for f in infos)
    # bit-identical to single calls on a sample
    for i in range(0, 512, 37):
        x1, _ = lsq.pne(As[i], bs[i], opts=opts[i])
        np.testing.assert_array_equal(to_np(x1), to_np(xs[i]))
    # against the oracle on a subset, at the precision the estimate chose
    for i in range(3, 512, 16):
        kap, rho, x_star = meta[i]
        _, ch = lsq.condest_sketch(As[i], seed=opts[i].seed)
        prec = int(to_np(ch)[0])
        A_np, b_np = to_np(As[i]), to_np(bs[i])
        kw = dict(kind=opts[i].kind, s=opts[i].s, zeta=opts[i].zeta, seed=opts[i].seed, sketch_prec=prec,
                  qr_prec=O.FP64 if prec == O.FP64 else O.FP32, refine_steps=0)
        ref = O.solve(A_np, b_np, **kw)
        assert ref["info"] == 0
        more = oracle_realizations(SimpleNamespace(A=A_np, b=b_np), **kw)
        assert_solution_parity(to_np(xs[i]), ref["x"], to_np(x_star), kap, rho, f"problem {i}", refined=False,
                               u_p=prec, realizations=more)
