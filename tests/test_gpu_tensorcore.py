"""Gaussian sketch on the tensor cores (tcgen05, TMA, TMEM) for FP8-e4m3,
BF16 and FP16 sketch precisions, against the oracle (FP32-accumulation
rounding bound) and against the CUDA-core GEMM on the same inputs, on
shapes with ragged M, N and K tiles and with split K."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from tests.gpu_util import dev_colmajor, to_np

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")
U32 = 2.0 ** -24
U64 = 2.0 ** -53


def set_tc(on):
    f = lsq.lib().lsq_set_tensor_core_sketch
    f.restype = C.c_int32
    f.argtypes = [C.c_int32]
    return f(int(on))


@pytest.mark.parametrize("prec", [O.BF16, O.FP16, O.FP8_E4M3])
@pytest.mark.parametrize("m,n,s", [(5000, 200, 300), (1037, 113, 250), (20000, 64, 128), (300, 129, 130),
                                   (3001, 300, 400), (2000, 512, 520)])
def test_tensor_core_sketch_matches_oracle_and_cuda_cores(prec, m, n, s):
    rng = np.random.default_rng(m + n + s)
    A = np.asfortranarray(rng.standard_normal((m, n)) * np.exp2(rng.integers(-6, 6, n))[None, :])
    opts = lsq.make_opts(kind=lsq.GAUSSIAN, s=s, seed=21, sketch_prec=prec)
    Ad = dev_colmajor(A)
    prev = set_tc(True)
    try:
        As_tc, ce, info = lsq.sketch(Ad, opts)
        As_tc = to_np(As_tc).astype(np.float64)
        assert int(to_np(info)[0]) == 0
        set_tc(False)
        As_cc, _, _ = lsq.sketch(Ad, opts)
        As_cc = to_np(As_cc).astype(np.float64)
    finally:
        set_tc(prev)
    oAs, oce = O.sketch(A, O.GAUSSIAN, s, 0, 21, prec)
    np.testing.assert_array_equal(to_np(ce), oce)
    Om = O.gaussian_operator(21, s, m, prec)
    Ah = O.quantize(A, prec, oce)
    scale = np.abs(Om) @ np.abs(Ah)
    # both FP32 sums carry at most (m-1) u sum|terms|; operator entries may differ next to ties
    tol = 2 * m * U32 * scale + 2 ** -3 * np.abs(Ah).max() * 4
    assert np.all(np.abs(As_tc - oAs) <= tol)
    assert np.all(np.abs(As_tc - As_cc) <= tol)
    # relative agreement is far tighter than the worst-case bound in practice
    assert np.linalg.norm(As_tc - oAs) <= 1e-5 * np.linalg.norm(oAs)


def test_tensor_core_sketch_large_split_k():
    # K = 65536 over split-K CTAs: both FP32 summations against the FP64 product
    # of the same rounded operands (error ~ sqrt(K) u32 for either order)
    m, n, s = 65536, 512, 1024
    rng = np.random.default_rng(1)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    opts = lsq.make_opts(kind=lsq.GAUSSIAN, s=s, seed=22, sketch_prec=lsq.BF16)
    Ad = dev_colmajor(A)
    As_tc, ce, info = lsq.sketch(Ad, opts)
    assert int(to_np(info)[0]) == 0
    prev = set_tc(False)
    try:
        As_cc, _, _ = lsq.sketch(Ad, opts)
    finally:
        set_tc(prev)
    a, c = to_np(As_tc).astype(np.float64), to_np(As_cc).astype(np.float64)
    Om = torch.from_numpy(O.gaussian_operator(22, s, m, O.BF16)).cuda()
    Ah = torch.from_numpy(O.quantize(A, O.BF16, to_np(ce))).cuda()
    ref = (Om @ Ah).cpu().numpy()
    e_tc = np.linalg.norm(a - ref) / np.linalg.norm(ref)
    e_cc = np.linalg.norm(c - ref) / np.linalg.norm(ref)
    # The tensor cores do not accumulate with round-to-nearest (measured on
    # GB300: ~1.9e-5 here against ~5.5e-7 for CUDA-core FMAs); both stay far
    # below the BF16 rounding of the inputs (2^-9).
    assert e_tc <= 4 * np.sqrt(m) * U32, e_tc
    assert e_cc <= 4 * np.sqrt(m) * U32, e_cc


def tc_gemm(prec, X, Y):
    """C = X Y^T on the tensor cores through the C ABI (X: M x K, Y: N x K, K-contiguous)."""
    L = lsq.lib()
    L.lsq_tc_gemm.restype = C.c_int32
    L.lsq_tc_gemm.argtypes = [C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                              C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
    L.lsq_tc_gemm_workspace_size.restype = C.c_size_t
    L.lsq_tc_gemm_workspace_size.argtypes = [C.c_int32, C.c_int64, C.c_int64, C.c_int64]
    M, K = X.shape
    N = Y.shape[0]
    out = torch.empty((N, M), dtype=torch.float32, device="cuda").t()
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(int(L.lsq_tc_gemm_workspace_size(prec, M, N, K)), dtype=torch.uint8, device="cuda")
    rc = L.lsq_tc_gemm(prec, X.data_ptr(), K, Y.data_ptr(), K, M, N, K, out.data_ptr(), M, info.data_ptr(),
                       ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    assert int(to_np(info)[0]) == 0
    return to_np(out).astype(np.float64)


@pytest.mark.parametrize("prec,lim,K,M,N", [(O.FP8_E4M3, 15, 65536, 256, 384), (O.BF16, 127, 1024, 384, 256),
                                           (O.FP8_E4M3, 15, 4096, 200, 130)])
def test_integer_operands_accumulate_exactly(prec, lim, K, M, N):
    # integer digits whose products and sums stay below 2^24 must come out exact
    rng = np.random.default_rng(K + M)
    Xi = rng.integers(-lim, lim + 1, size=(M, K))
    Yi = rng.integers(-lim, lim + 1, size=(N, K))
    dt = torch.float8_e4m3fn if prec == O.FP8_E4M3 else torch.bfloat16
    X = torch.from_numpy(Xi.astype(np.float32)).to(dt).cuda().contiguous()
    Y = torch.from_numpy(Yi.astype(np.float32)).to(dt).cuda().contiguous()
    Cg = tc_gemm(prec, X.view(torch.uint8) if prec == O.FP8_E4M3 else X, Y.view(torch.uint8) if prec == O.FP8_E4M3 else Y)
    exact = (Xi.astype(np.int64) @ Yi.T.astype(np.int64)).astype(np.float64)
    assert np.abs(exact).max() < 2 ** 24
    np.testing.assert_array_equal(Cg, exact)


def _sketch_both_ways(A, prec, s, seed, fp64):
    """Sketch on the tensor cores (default) and on the CUDA cores (switched off)."""
    opts = lsq.make_opts(kind=lsq.GAUSSIAN, s=s, seed=seed, sketch_prec=prec)
    Ad = dev_colmajor(A)
    As_tc, ce, info = lsq.sketch(Ad, opts)
    assert int(to_np(info)[0]) == 0
    As_tc = to_np(As_tc).astype(np.float64)
    prev = lsq.set_fp64_emulation(False) if fp64 else set_tc(False)
    try:
        As_cc, _, _ = lsq.sketch(Ad, opts)
    finally:
        if fp64:
            lsq.set_fp64_emulation(prev)
        else:
            set_tc(prev)
    return As_tc, to_np(As_cc).astype(np.float64), to_np(ce)


@pytest.mark.parametrize("m,n,s", [(1037, 113, 250), (20011, 70, 200), (300, 129, 130), (5000, 200, 300),
                                   (3001, 300, 600), (1500, 520, 600)])
def test_fp32_gaussian_sketch_bf16_pieces(m, n, s):
    # FP32 sketch as six BF16 piece products on the tensor cores: against the
    # oracle's sequential FP32 sum (worst-case bound) and, in norm, no less
    # accurate than the oracle or the CUDA-core FP32 GEMM against the FP64
    # product of the same FP32-rounded operands
    rng = np.random.default_rng(m + 7 * n)
    A = np.asfortranarray(rng.standard_normal((m, n)) * np.exp2(rng.integers(-6, 6, n))[None, :])
    As_tc, As_cc, ce = _sketch_both_ways(A, lsq.FP32, s, 23, False)
    oAs, oce = O.sketch(A, O.GAUSSIAN, s, 0, 23, O.FP32)
    np.testing.assert_array_equal(ce, oce)
    Om = O.gaussian_operator(23, s, m, O.FP32)
    Ah = O.quantize(A, O.FP32, oce)
    exact = Om @ Ah  # FP64 product of FP32 values: error ~1e-16, far below FP32
    scale = np.abs(Om) @ np.abs(Ah)
    tol = 3 * m * U32 * scale
    assert np.all(np.abs(As_tc - oAs) <= tol)
    e_tc = np.linalg.norm(As_tc - exact)
    e_or = np.linalg.norm(oAs - exact)
    e_cc = np.linalg.norm(As_cc - exact)
    assert e_tc <= 2 * max(e_or, e_cc), (e_tc, e_or, e_cc)


@pytest.mark.parametrize("m,n,s", [(1037, 113, 250), (3001, 70, 200), (700, 129, 130)])
def test_fp64_gaussian_sketch_digit_sliced(m, n, s):
    # FP64 sketch as K chunks of 1024 FP64-accurate digit-sliced products:
    # elementwise against the oracle's sequential FP64 sum within both error
    # bounds, and against the exact rational value on sampled entries
    from fractions import Fraction

    rng = np.random.default_rng(m + 3 * n)
    A = np.asfortranarray(rng.standard_normal((m, n)) * np.exp2(rng.integers(-20, 20, n))[None, :])
    As_tc, As_cc, ce = _sketch_both_ways(A, lsq.FP64, s, 29, True)
    oAs, _ = O.sketch(A, O.GAUSSIAN, s, 0, 29, O.FP64)
    Om = O.gaussian_operator(29, s, m, O.FP64)
    # per chunk: digit error below 1024 2^-50.6 2^3 max|A_chunk,c| (Omega is
    # sliced with the fixed exponent 2^3 > |Omega|) and two FP64 roundings of
    # the running sum; the oracle: gamma_m sum|terms|
    chunks = [slice(k, min(k + 1024, m)) for k in range(0, m, 1024)]
    dig = sum(1024 * 2.0 ** -50.6 * 8.0 * np.outer(np.ones(s), np.abs(A[c, :]).max(axis=0)) for c in chunks)
    scale = np.abs(Om) @ np.abs(A)
    gamma = m * U64 / (1 - m * U64)
    tol = dig + 2 * gamma * scale
    assert np.all(np.abs(As_tc - oAs) <= tol)
    # the CUDA-core FP64 GEMM on the same operator, same bound
    assert np.all(np.abs(As_tc - As_cc) <= tol)
    e_tc, e_or = [], []
    for (i, c) in [(0, 0), (s - 1, n - 1), (s // 2, n // 3), (7, n - 1), (s - 1, 0), (s // 3, 5)]:
        ex = sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(Om[i, :], A[:, c])), Fraction(0))
        e_tc.append(abs(As_tc[i, c] - float(ex)))
        e_or.append(abs(oAs[i, c] - float(ex)))
        assert e_tc[-1] <= tol[i, c]
    assert np.sqrt(np.mean(np.square(e_tc))) <= 4 * np.sqrt(np.mean(np.square(e_or))) + 4 * U64 * np.abs(oAs).max()
