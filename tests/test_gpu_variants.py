"""The alternative solution methods and the condition estimate on a sketch,
through the C ABI, against the oracle:
  * HPNE through a QR of A_p^T A (lsq_hpne_qr_solve), the seminormal
    equations with R = L^T R_s (lsq_sne_solve), the not-normal equations with
    B = A U_s^{-1} from the LU of the sketch (lsq_nne_solve): solutions under
    the solution tolerance of the method, U_s of the not-normal equations
    against the oracle's, the LU pivots' breakdown index bit-exact;
  * the estimate on the sketch (lsq_condest_sketch): kappa0 close to the
    oracle's, the same precision chosen, and AUTO_SKETCH solves that use it.
"""
import numpy as np
import pytest
import torch

import oracle as O
import problems as P
from tests.gpu_util import assert_solution_parity, dev_colmajor, oracle_realizations, to_np

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")

CASES = [
    # m, n, kappa, rho, kind, s, zeta, prec, refine
    (2048, 128, 1e2, 0.0, O.SPARSE_SIGN, 512, 8, O.BF16, 1),
    (2048, 128, 1e4, 1e-6, O.GAUSSIAN, 256, 0, O.FP32, 0),
    (3000, 200, 1e6, 1e-8, O.SPARSE_SIGN, 600, 8, O.FP32, 1),
    (1037, 113, 1e8, 1e-10, O.GAUSSIAN, 339, 0, O.FP64, 0),
    (4096, 256, 1e3, 1e-3, O.GAUSSIAN, 512, 0, O.FP16, 1),
]


@pytest.mark.parametrize("method", ["hpne_qr", "sne", "nne_lu"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-k{c[2]:.0e}-r{c[3]:.0e}-p{c[7]}-f{c[8]}")
def test_method_matches_oracle(method, case):
    m, n, kap, rho, kind, s, zeta, prec, refine = case
    pr = P.make_problem(m, n, kap, rho, P.seed_for(1, 300 + n + int(np.log10(kap))))
    qr = O.FP64 if prec == O.FP64 else O.FP32
    kw = dict(kind=kind, s=s, zeta=zeta, seed=7, sketch_prec=prec, qr_prec=qr, refine_steps=refine)
    opts = lsq.make_opts(**kw)
    Rs = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
    x, info = lsq.solve(dev_colmajor(pr.A), torch.from_numpy(pr.b).cuda(), method=method, opts=opts, Rs_out=Rs)
    ref = O.solve(pr.A, pr.b, method=method, **kw)
    assert int(to_np(info)[0]) == ref["info"] == 0
    if method == "nne_lu":
        # U_s: both are LU factors of the same sketch (FP32 or FP64 arithmetic,
        # different update order); tall LU is backward stable with growth <= 2^n
        # in theory and small in practice: compare normwise with the oracle's.
        Ug, Uo = np.triu(to_np(Rs)), ref["Rs"]
        u = 2.0 ** -53 if qr == O.FP64 else 2.0 ** -24
        assert np.linalg.norm(Ug - Uo) <= 64 * s * u * np.linalg.norm(Uo) * max(1.0, np.log2(n)), \
            np.linalg.norm(Ug - Uo) / np.linalg.norm(Uo)
    more = oracle_realizations(pr, method=method, **kw)
    assert_solution_parity(to_np(x), ref["x"], pr.x_star, kap, rho, f"{method}", refined=refine > 0, u_p=prec,
                           realizations=more)


def test_sne_shows_kappa_squared_and_corrected_sne_recovers():
    pr = P.make_problem(3000, 80, 1e6, 1e-8, 77)
    A, b = dev_colmajor(pr.A), torch.from_numpy(pr.b).cuda()
    kw = dict(kind=lsq.SPARSE_SIGN, s=320, zeta=8, seed=5, sketch_prec=lsq.FP64, qr_prec=lsq.FP64)
    e = {}
    for meth, ref in (("pne", 0), ("sne", 0), ("sne", 1)):
        x, info = lsq.solve(A, b, method=meth, opts=lsq.make_opts(refine_steps=ref, **kw))
        assert int(to_np(info)[0]) == 0
        e[(meth, ref)] = P.rel_error(to_np(x), pr.x_star)
    assert e[("sne", 0)] >= 100 * e[("pne", 0)], e
    assert e[("sne", 1)] <= 10 * e[("pne", 0)] + 1e-14, e


def test_nne_zero_column_reports_breakdown():
    pr = P.make_problem(500, 20, 1e2, 0.0, 81)
    A = pr.A.copy(order="F")
    A[:, 7] = 0.0
    opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=40, zeta=4, seed=1, sketch_prec=lsq.FP32)
    x, info = lsq.solve(dev_colmajor(A), torch.from_numpy(pr.b).cuda(), method="nne_lu", opts=opts)
    ref = O.solve(A, pr.b, method="nne_lu", kind=O.SPARSE_SIGN, s=40, zeta=4, seed=1, sketch_prec=O.FP32)
    assert int(to_np(info)[0]) == ref["info"] == 8


@pytest.mark.parametrize("m,n", [(4000, 64), (8000, 256), (6000, 1000)])
def test_condest_sketch_matches_oracle(m, n):
    for kap in (1e1, 1e3, 1e5, 1e7, 1e10):
        pr = P.make_problem(m, n, kap, 0.0, 5)
        k0, ch = lsq.condest_sketch(dev_colmajor(pr.A), seed=3)
        k0, ch = float(to_np(k0)[0]), int(to_np(ch)[0])
        ok0, och, ok1, rc = O.condest_sketch(pr.A, 3)
        assert rc == 0
        if np.isinf(ok0):
            assert np.isinf(k0) and ch == och == O.FP64, (kap, k0, ok0)
        else:
            # the same sketch bit for bit; FP32 QR, Gram and Hager in another order
            assert abs(k0 - ok0) <= 0.02, (kap, k0, ok0)
            # next to a threshold of the table the two may round apart
            if min(abs(ok0 - t) for t in (2.0, 3.0, 4.0, 8.0)) > 0.02:
                assert ch == och, (kap, k0, ok0)


@pytest.mark.parametrize("kap,want", [(1e2, O.FP16), (1e4, O.FP32), (1e10, O.FP64)])
def test_auto_sketch_solve(kap, want):
    pr = P.make_problem(4096, 64, kap, 1e-6, 93)
    opts = lsq.make_opts(kind=lsq.GAUSSIAN, s=192, seed=8, sketch_prec=lsq.AUTO_SKETCH, qr_prec=lsq.FP32)
    x, info = lsq.solve(dev_colmajor(pr.A), torch.from_numpy(pr.b).cuda(), opts=opts)
    ref = O.solve(pr.A, pr.b, kind=O.GAUSSIAN, s=192, seed=8, sketch_prec=O.AUTO_SKETCH, qr_prec=O.FP32)
    assert ref["prec"] == want
    assert int(to_np(info)[0]) == 0
    assert_solution_parity(to_np(x), ref["x"], pr.x_star, kap, 1e-6, refined=False, u_p=want)


@pytest.mark.parametrize("hpne", [False, True])
@pytest.mark.parametrize("m,n,kap,rho,prec", [(6000, 200, 1e6, 1e-8, O.FP32), (100000, 400, 1e7, 1e-6, O.FP32),
                                              (3000, 100, 1e2, 0.0, O.FP16), (5000, 150, 1e10, 1e-6, O.FP64)])
def test_srft_solve_matches_oracle(hpne, m, n, kap, rho, prec):
    # the paper's own sketch (Eq. e_sketch) with d = 3n (Sec. 6.2); 100000 x 400
    # at kappa = 1e7, residual 1e-6 is the shape of the paper's GPU timing
    # experiment (Fig. 6) with its smallest n
    pr = P.make_problem(m, n, kap, rho, P.seed_for(5, n + int(np.log10(kap))))
    qr = O.FP64 if prec == O.FP64 else O.FP32
    kw = dict(kind=O.SRFT, s=3 * n, zeta=0, seed=13, sketch_prec=prec, qr_prec=qr, refine_steps=0)
    x, info = lsq.solve(dev_colmajor(pr.A), torch.from_numpy(pr.b).cuda(), hpne=hpne, opts=lsq.make_opts(**kw))
    ref = O.solve(pr.A, pr.b, hpne=hpne, **kw)
    assert int(to_np(info)[0]) == ref["info"] == 0
    more = oracle_realizations(pr, hpne=hpne, **kw)
    assert_solution_parity(to_np(x), ref["x"], pr.x_star, kap, rho, "srft", refined=False, u_p=prec,
                           realizations=more)
