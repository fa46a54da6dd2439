"""End-to-end parity of the CUDA solver (Alg. 1 with PNE / HPNE) with the
oracle, under the solution tolerance of the method: relative difference 1e-12
from the oracle when kappa(A) <= 1e4 and the residual is zero, otherwise an
error against x_* within 2x the oracle's own error against x_*.
"""
import numpy as np
import pytest
import torch

import oracle as O
import problems as P
from tests.gpu_util import assert_solution_parity, dev_colmajor, oracle_realizations, to_np

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")


def run_both(pr, hpne, kind, s, zeta, seed, prec, qr_prec=O.FP32, refine=0):
    opts = lsq.make_opts(kind=kind, s=s, zeta=zeta, seed=seed, sketch_prec=prec, qr_prec=qr_prec,
                         refine_steps=refine)
    A = dev_colmajor(pr.A)
    b = torch.from_numpy(pr.b).cuda()
    x, info = lsq.solve(A, b, hpne=hpne, opts=opts)
    ref = O.solve(pr.A, pr.b, hpne=hpne, kind=kind, s=s, zeta=zeta, seed=seed, sketch_prec=prec,
                  qr_prec=qr_prec, refine_steps=refine)
    return to_np(x), int(to_np(info)[0]), ref


RHOS = [0.0] + list(np.logspace(-12, -2, 11))


@pytest.mark.parametrize("hpne", [False, True])
def test_fig1_config_residual_sweep(hpne):
    # 1000 x 100, kappa = 1e8, Gaussian sketch s = 2n, FP32 preconditioner (Fig. 1 setting)
    for k, rho in enumerate(RHOS):
        pr = P.make_problem(1000, 100, 1e8, rho, P.seed_for(0, k))
        x, info, ref = run_both(pr, hpne, O.GAUSSIAN, 200, 0, 17 + k, O.FP32)
        assert info == 0 == ref["info"]
        more = oracle_realizations(pr, hpne=hpne, kind=O.GAUSSIAN, s=200, seed=17 + k, sketch_prec=O.FP32,
                                   qr_prec=O.FP32)
        assert_solution_parity(x, ref["x"], pr.x_star, 1e8, rho, f"rho={rho}", refined=False, u_p=O.FP32,
                               realizations=more)


CASES = [
    # m, n, kappa, rho, kind, s, zeta, prec, refine
    (2048, 128, 1e2, 0.0, O.SPARSE_SIGN, 512, 8, O.BF16, 1),
    (2048, 128, 1e4, 0.0, O.SPARSE_SIGN, 512, 8, O.BF16, 1),
    (2048, 128, 1e4, 0.0, O.GAUSSIAN, 256, 0, O.FP32, 0),
    (2048, 128, 1e4, 0.0, O.GAUSSIAN, 256, 0, O.FP32, 1),
    (2048, 128, 1e6, 1e-8, O.SPARSE_SIGN, 512, 8, O.BF16, 1),
    (2048, 128, 1e6, 1e-3, O.SPARSE_SIGN, 512, 8, O.BF16, 1),
    (2048, 128, 1e10, 1e-8, O.SPARSE_SIGN, 512, 8, O.FP64, 1),
    (1037, 113, 1e2, 1e-6, O.GAUSSIAN, 229, 0, O.FP8_E4M3, 0),
    (1037, 113, 1e3, 1e-6, O.GAUSSIAN, 229, 0, O.FP16, 1),
    (1037, 113, 1e4, 0.0, O.GAUSSIAN, 339, 0, O.FP64, 0),
    (4096, 256, 1e6, 1e-6, O.SPARSE_SIGN, 1024, 8, O.FP32, 1),
]


@pytest.mark.parametrize("hpne", [False, True])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-k{c[2]:.0e}-r{c[3]:.0e}-p{c[7]}")
def test_solver_parity(hpne, case):
    m, n, kap, rho, kind, s, zeta, prec, refine = case
    pr = P.make_problem(m, n, kap, rho, P.seed_for(1, int(np.log10(kap)) + 20 * n))
    x, info, ref = run_both(pr, hpne, kind, s, zeta, 3, prec, refine=refine)
    assert info == ref["info"] == 0
    more = oracle_realizations(pr, hpne=hpne, kind=kind, s=s, zeta=zeta, seed=3, sketch_prec=prec,
                               qr_prec=O.FP32, refine_steps=refine)
    assert_solution_parity(x, ref["x"], pr.x_star, kap, rho, refined=refine > 0, u_p=prec, realizations=more)


@pytest.mark.parametrize("kap,want", [(1e2, O.FP16), (1e10, O.FP64)])
def test_auto_precision_matches_oracle(kap, want):
    # Fig. 7: kappa = 1e2 selects half precision, kappa = 1e10 double
    pr = P.make_problem(4096, 64, kap, 1e-6, 93)
    x, info, ref = run_both(pr, False, O.GAUSSIAN, 192, 0, 8, O.AUTO)
    assert ref["prec"] == want
    k0, ch = lsq.condest(dev_colmajor(pr.A))
    assert int(to_np(ch)[0]) == want
    assert info == 0
    assert_solution_parity(x, ref["x"], pr.x_star, kap, 1e-6, refined=False, u_p=want)


def test_edge_shapes():
    # n = 1; square m = s = n; sketch as tall as A
    for (m, n, s) in [(50, 1, 2), (64, 64, 64), (300, 40, 300)]:
        pr = P.make_problem(m, n, 10.0, 0.0 if m == n else 1e-6, 5)
        for hp in (False, True):
            x, info, ref = run_both(pr, hp, O.GAUSSIAN, s, 0, 1, O.FP64, qr_prec=O.FP64, refine=1)
            assert info == 0
            assert_solution_parity(x, ref["x"], pr.x_star, 10.0, 0.0 if m == n else 1e-6, f"{m}x{n} s={s}")


def test_zero_column_reports_breakdown():
    pr = P.make_problem(500, 20, 1e2, 0.0, 81)
    A = pr.A.copy(order="F")
    A[:, 7] = 0.0
    opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=40, zeta=4, seed=1, sketch_prec=lsq.FP32)
    x, info = lsq.pne(dev_colmajor(A), torch.from_numpy(pr.b).cuda(), opts=opts)
    assert int(to_np(info)[0]) == 8


def test_nan_rhs_does_not_crash():
    pr = P.make_problem(500, 20, 1e2, 0.0, 82)
    b = pr.b.copy()
    b[3] = np.nan
    opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=40, zeta=4, seed=1, sketch_prec=lsq.FP32)
    x, info = lsq.pne(dev_colmajor(pr.A), torch.from_numpy(b).cuda(), opts=opts)
    assert not np.all(np.isfinite(to_np(x)))


def test_bad_arguments_and_small_workspace():
    pr = P.make_problem(200, 20, 1e2, 0.0, 83)
    A = dev_colmajor(pr.A)
    b = torch.from_numpy(pr.b).cuda()
    with pytest.raises(lsq.LsqError):
        lsq.pne(A, b, opts=lsq.make_opts(kind=lsq.SPARSE_SIGN, s=10, zeta=4, seed=1))  # s < n
    with pytest.raises(lsq.LsqError):
        lsq.pne(A, b, opts=lsq.make_opts(kind=lsq.SPARSE_SIGN, s=40, zeta=41, seed=1))  # zeta > s
    with pytest.raises(lsq.LsqError):
        lsq.pne(A, b, opts=lsq.make_opts(kind=lsq.SPARSE_SIGN, s=300, zeta=4, seed=1))  # s > m
    opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=40, zeta=4, seed=1)
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(lsq.LsqError):
        lsq.pne(A, b, opts=opts, ws=ws)


def test_deterministic_and_host_path_identical():
    pr = P.make_problem(3000, 150, 1e6, 1e-8, 84)
    opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=600, zeta=8, seed=4, sketch_prec=lsq.BF16, refine_steps=1)
    A = dev_colmajor(pr.A)
    b = torch.from_numpy(pr.b).cuda()
    x1, _ = lsq.pne(A, b, opts=opts)
    x2, _ = lsq.pne(A, b, opts=opts)
    x1, x2 = to_np(x1), to_np(x2)
    np.testing.assert_array_equal(x1, x2)
    Ah = torch.from_numpy(np.ascontiguousarray(pr.A.T)).pin_memory().t()
    bh = torch.from_numpy(pr.b).pin_memory()
    xh, info = lsq.solve_host(Ah, bh, opts=opts)
    assert info == 0
    np.testing.assert_array_equal(xh.numpy(), x1)


@pytest.mark.parametrize("kap,want", [(1e4, O.FP32), (1e8, O.FP64)])
@pytest.mark.parametrize("hpne", [False, True])
def test_large_single_problem_within_bound(hpne, kap, want):
    # the 262144 x 4096 problem (8.6 GB) the benchmark times: Gaussian sketch
    # s = 2n with per-column power-of-two scaling, its precision chosen by the
    # condition estimate on a sketch (FP32 at kappa = 1e4, FP64 at 1e8), FP64
    # rest.  Exact orthonormal U from signed Hadamard columns; the bound is
    # evaluated on the device with exact condition numbers.  The paper
    # evaluates its bounds with eps_A = u; a backward-stable FP64 evaluation
    # has eps_A = gamma_n, but at this size the measured error stays within
    # 10x the bound (the oracle's own ratios on the Fig. 1-5 shapes with
    # u_p kappa(A) << 1 are below 0.4).
    m, n, rho = 262144, 4096, 1e-6
    A, b, x_star, sigma, V = P.make_problem_hadamard_torch(m, n, kap, rho, P.seed_for(2, 0))
    k0, ch = lsq.condest_sketch(A, seed=P.seed_for(2, 0))
    assert int(to_np(ch)[0]) == want, float(to_np(k0)[0])
    opts = lsq.make_opts(kind=lsq.GAUSSIAN, s=2 * n, seed=P.seed_for(2, 0), sketch_prec=lsq.AUTO_SKETCH,
                         qr_prec=lsq.FP32, refine_steps=0)
    Rs = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
    x, info = lsq.solve(A, b, hpne=hpne, opts=opts, Rs_out=Rs)
    assert int(to_np(info)[0]) == 0
    Rs = torch.triu(Rs)
    # Eq. (eq41) / (eq32) with exact condition numbers: A_p = U diag(sigma) V^T R_s^{-1}
    MT = torch.linalg.solve_triangular(Rs.t(), V * sigma, upper=False)  # (diag(sigma) V^T R_s^{-1})^T
    kappa = lambda X: float((lambda s_: s_[0] / s_[-1])(torch.linalg.svdvals(X)))
    kAp, kR = kappa(MT), kappa(Rs)
    res = float(torch.linalg.norm(b - A @ x) / torch.linalg.norm(x))
    u2 = 2.0 ** -52
    if hpne:
        H = MT @ (sigma[:, None] * V.t())  # A_p^T A = M^T diag(sigma) V^T
        nu = float(torch.linalg.matrix_norm(MT, 2) / torch.linalg.matrix_norm(H, 2))
        bound = kappa(H) * nu * u2 * (kR * res + 1 + kap * u2)
    else:
        bound = kR * kAp * u2 * (kAp * kR * res + 1 + kap * u2)
    err = float(torch.linalg.norm(x - x_star) / torch.linalg.norm(x))
    print(f"262144x4096 kappa={kap:.0e} hpne={hpne}: err={err:.3e} bound={bound:.3e} ratio={err / bound:.3g} "
          f"kappa(A_p)={kAp:.3g}")
    assert kAp <= 10.0
    assert err <= 10 * bound, (err, bound, kAp)


@pytest.mark.parametrize("hpne", [False, True])
def test_full_size_tall_skinny_within_bound(hpne):
    # the 65536 x 1024 workload: sparse-sign s = 4n, zeta = 8, BF16 sketch, FP32 QR,
    # FP64 rest, one refinement step, in the launch configuration the benchmark times
    m, n, kap, rho = 65536, 1024, 1e6, 1e-8
    A, b, x_star, sigma, V = P.make_problem_torch(m, n, kap, rho, P.seed_for(1, 1))
    opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=4 * n, zeta=8, seed=P.seed_for(1, 1), sketch_prec=lsq.BF16,
                         qr_prec=lsq.FP32, refine_steps=1)
    Rs = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
    x, info = lsq.solve(A, b, hpne=hpne, opts=opts, Rs_out=Rs)
    assert int(to_np(info)[0]) == 0
    x, Rs = to_np(x), np.triu(to_np(Rs))
    # Eq. (eq41) / (eq32) with exact condition numbers: A_p = U diag(sigma) V^T R_s^{-1}
    S = to_np(sigma)
    Vn = to_np(V)
    M = (S[:, None] * Vn.T) @ np.linalg.inv(Rs)
    kAp = O.kappa(M)
    kR = O.kappa(Rs)
    res = np.linalg.norm(to_np(b) - to_np(A @ torch.from_numpy(x).cuda())) / np.linalg.norm(x)
    u2 = 2.0 ** -52
    if hpne:
        H = M.T @ (S[:, None] * Vn.T)  # A_p^T A = M^T diag(S) V^T
        nu = np.linalg.norm(M, 2) / np.linalg.norm(H, 2)
        bound = O.kappa(H) * nu * u2 * (kR * res + 1 + kap * u2)
    else:
        bound = kR * kAp * u2 * (kAp * kR * res + 1 + kap * u2)
    err = P.rel_error(x, to_np(x_star))
    assert err <= n * bound, (err, bound, kAp)


# The nine 65536 x 1024 problems the benchmark times (its seeds, its launch
# configuration: sparse sign s = 4n, zeta = 8, BF16 sketch, FP32 QR, one
# refinement step), each against the oracle at full size under the solution
# tolerance of the method.
C1_KAPPAS, C1_RHOS = [1e2, 1e6, 1e10], [0.0, 1e-8, 1e-3]
C1_CASES = [(i, j, False) for i in range(3) for j in range(3)] + [(0, 2, True), (1, 1, True), (2, 0, True)]


@pytest.mark.parametrize("i,j,hpne", C1_CASES,
                         ids=lambda v: str(v) if not isinstance(v, bool) else ("hpne" if v else "pne"))
def test_tall_skinny_bench_problems_against_oracle(i, j, hpne):
    from types import SimpleNamespace

    m, n = 65536, 1024
    kap, rho = C1_KAPPAS[i], C1_RHOS[j]
    seed = P.seed_for(1, 3 * i + j)
    A, b, x_star, sigma, V = P.make_problem_torch(m, n, kap, rho, seed)
    kw = dict(kind=O.SPARSE_SIGN, s=4 * n, zeta=8, seed=seed, sketch_prec=O.BF16, qr_prec=O.FP32, refine_steps=1)
    opts = lsq.make_opts(**kw)
    x, info = lsq.solve(A, b, hpne=hpne, opts=opts)
    assert int(to_np(info)[0]) == 0
    A_np, b_np = to_np(A), to_np(b)
    ref = O.solve(A_np, b_np, hpne=hpne, **kw)
    assert ref["info"] == 0
    more = oracle_realizations(SimpleNamespace(A=A_np, b=b_np), hpne=hpne, **kw)
    assert_solution_parity(to_np(x), ref["x"], to_np(x_star), kap, rho, f"kappa={kap} rho={rho}", refined=True,
                           u_p=O.BF16, realizations=more)
