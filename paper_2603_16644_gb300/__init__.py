"""Python binding of liblsq: randomized-preconditioned normal equations on
GB300 (Garrison & Ipsen, arXiv 2603.16644, Alg. 1; PNE Eq. e_pne, HPNE
Eq. e_hpne).

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``liblsq.so`` behind the C ABI of ``include/lsq.h``.  PyTorch
supplies device memory and the current stream.  There is no CPU fallback:
importing works without a GPU, but every call needs CUDA tensors and the
built library, and raises otherwise.

Matrices are column-major FP64: an (m, n) tensor with stride (1, lda), lda >= m,
e.g. ``colmajor(A)``.
"""
import ctypes as C
import os

import torch

__all__ = [
    "FP8_E4M3", "BF16", "FP16", "FP32", "FP64", "AUTO", "AUTO_SKETCH", "GAUSSIAN", "SPARSE_SIGN", "SRFT", "METHODS",
    "condest_sketch",
    "Opts", "lib", "colmajor", "workspace", "sketch", "precond_qr", "condest", "trsm_gram",
    "factor_solve", "trsm_tc", "gram_tc", "gemm_tn_tc", "set_fp64_emulation", "pne", "hpne", "solve", "solve_host", "sparse_sign_operator",
    "gaussian_operator", "precision_from_kappa0", "status_string", "LsqError",
]

FP8_E4M3, BF16, FP16, FP32, FP64, AUTO, AUTO_SKETCH = 0, 1, 2, 3, 4, 5, 6
GAUSSIAN, SPARSE_SIGN, SRFT = 0, 1, 2
(OP_SKETCH, OP_PRECOND_QR, OP_CONDEST, OP_PNE, OP_HPNE, OP_TRSM_GRAM, OP_FACTOR_SOLVE, OP_PNE_HOST, OP_HPNE_HOST,
 OP_CONDEST_SKETCH, OP_HPNE_QR, OP_SNE, OP_NNE) = range(13)
# solution methods: entry point and workspace op
METHODS = {"pne": ("lsq_pne_solve", OP_PNE), "hpne": ("lsq_hpne_solve", OP_HPNE),
           "hpne_qr": ("lsq_hpne_qr_solve", OP_HPNE_QR), "sne": ("lsq_sne_solve", OP_SNE),
           "nne_lu": ("lsq_nne_solve", OP_NNE)}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblsq.so")
_lib = None


class LsqError(RuntimeError):
    pass


class Opts(C.Structure):
    _fields_ = [("kind", C.c_int32), ("zeta", C.c_int32), ("s", C.c_int64), ("seed", C.c_uint64),
                ("sketch_prec", C.c_int32), ("qr_prec", C.c_int32), ("refine_steps", C.c_int32),
                ("row_offset", C.c_int32)]


_vp, _i64, _sz = C.c_void_p, C.c_int64, C.c_size_t


def lib():
    """Load liblsq.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LsqError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        sig = {
            "lsq_version": (C.c_int32, []),
            "lsq_status_string": (C.c_char_p, [C.c_int32]),
            "lsq_last_cuda_error": (C.c_char_p, []),
            "lsq_workspace_size": (_sz, [C.c_int32, _i64, _i64, C.POINTER(Opts)]),
            "lsq_precision_from_kappa0": (C.c_int32, [C.c_double]),
            "lsq_sparse_sign_operator": (C.c_int32, [C.c_uint64, _i64, _i64, C.c_int32, _vp, _vp, _vp]),
            "lsq_gaussian_operator": (C.c_int32, [C.c_uint64, _i64, _i64, C.c_int32, _vp, _vp]),
            "lsq_sketch": (C.c_int32, [_vp, _i64, _i64, _i64, C.POINTER(Opts), _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
            "lsq_precond_qr": (C.c_int32, [_vp, _i64, _i64, _i64, C.c_int32, C.c_int32, _vp, _vp, _i64, _vp, _vp,
                                           _sz, _vp]),
            "lsq_condest": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, _vp, _vp, _sz, _vp]),
            "lsq_condest_sketch": (C.c_int32, [_vp, _i64, _i64, _i64, C.c_uint64, _vp, _vp, _vp, _sz, _vp]),
            "lsq_hpne_qr_solve": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, C.POINTER(Opts), _vp, _vp, _vp, _vp, _sz,
                                              _vp]),
            "lsq_sne_solve": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, C.POINTER(Opts), _vp, _vp, _vp, _vp, _sz, _vp]),
            "lsq_nne_solve": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, C.POINTER(Opts), _vp, _vp, _vp, _vp, _sz, _vp]),
            "lsq_trsm_gram": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, _i64, _vp, C.c_int32, _vp, _i64, _vp, _i64,
                                          _vp, _vp, _sz, _vp]),
            "lsq_factor_solve": (C.c_int32, [C.c_int32, _vp, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _sz,
                                             _vp]),
            "lsq_pne_solve": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, C.POINTER(Opts), _vp, _vp, _vp, _vp, _sz, _vp]),
            "lsq_hpne_solve": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, C.POINTER(Opts), _vp, _vp, _vp, _vp, _sz,
                                           _vp]),
            "lsq_pne_solve_host": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, C.POINTER(Opts), _vp, _vp, _vp, _sz,
                                               _vp]),
            "lsq_hpne_solve_host": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, C.POINTER(Opts), _vp, _vp, _vp, _sz,
                                                _vp]),
            "lsq_launch_count": (C.c_int64, []),
            "lsq_profile": (C.c_int32, [C.c_int32]),
            "lsq_profile_collect": (C.c_int32, [C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_int32]),
            "lsq_profile_collect_work": (C.c_int32, [C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                                     C.POINTER(C.c_double), C.c_int32]),
            "lsq_profile_records": (C.c_int32, [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int32]),
            "lsq_trsm_tc_workspace_size": (_sz, [_i64, _i64]),
            "lsq_trsm_tc": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
            "lsq_gram_tc_workspace_size": (_sz, [_i64, _i64]),
            "lsq_gram_tc": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
            "lsq_set_fp64_emulation": (C.c_int32, [C.c_int32]),
            "lsq_test_set_solve_wait_ns": (_i64, [_i64]),
            "lsq_gemm_tn_tc_workspace_size": (_sz, [_i64, _i64]),
            "lsq_gemm_tn_tc": (C.c_int32, [_vp, _i64, _vp, _i64, _i64, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


STAGES = ["condest", "sketch", "qr", "trsm", "gram", "factor", "solve", "refine", "k_ot_update", "k_qr_panel",
          "k_sketch_tc", "k_ot_update3"]


def launch_count() -> int:
    """Kernel launches issued by liblsq since it was loaded."""
    return int(lib().lsq_launch_count())


def profile(enable: bool) -> None:
    """Start (clearing old records) or stop per-stage CUDA-event timing."""
    lib().lsq_profile(int(enable))


def profile_collect(with_work: bool = False) -> dict:
    """{stage: (total ms, records)} since the last collect, or (total ms,
    records, algorithmic flops) with ``with_work``; waits for the events."""
    k = len(STAGES)
    ms = (C.c_double * k)()
    cnt = (C.c_int32 * k)()
    work = (C.c_double * k)()
    _check(lib().lsq_profile_collect_work(ms, cnt, work, k), "lsq_profile_collect_work")
    if with_work:
        return {name: (ms[i], cnt[i], work[i]) for i, name in enumerate(STAGES)}
    return {name: (ms[i], cnt[i]) for i, name in enumerate(STAGES)}


def profile_records(stage: str) -> list:
    """[(ms, work)] of every record of one stage since the last collect."""
    idx = STAGES.index(stage)
    n = int(lib().lsq_profile_records(idx, (C.c_double * 1)(), (C.c_double * 1)(), 0))
    if n < 0:
        raise LsqError(f"lsq_profile_records failed: {status_string(-n)}")
    ms = (C.c_double * max(1, n))()
    work = (C.c_double * max(1, n))()
    lib().lsq_profile_records(idx, ms, work, n)
    return [(ms[i], work[i]) for i in range(n)]


def status_string(rc: int) -> str:
    return lib().lsq_status_string(rc).decode()


def _check(rc, what):
    if rc != 0:
        extra = f" [{lib().lsq_last_cuda_error().decode()}]" if rc == 5 else ""
        raise LsqError(f"{what} failed: {status_string(rc)} ({rc}){extra}")


def _stream(device=None):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise LsqError("liblsq needs CUDA tensors (no CPU fallback)")


def colmajor(A: torch.Tensor, ld: int = None) -> torch.Tensor:
    """Column-major FP64 copy of A (shape (m, n), stride (1, ld))."""
    m, n = A.shape
    ld = m if ld is None else ld
    out = torch.empty((n, ld), dtype=torch.float64, device=A.device).t()[:m]
    out.copy_(A)
    return out


def _ld(A, dtypes=(torch.float64,)):
    m, n = A.shape
    if A.dtype not in dtypes:
        raise LsqError("A must be " + " or ".join(str(d).replace("torch.", "") for d in dtypes))
    if n == 1:
        return m
    if A.stride(0) != 1 or A.stride(1) < m:
        raise LsqError("A must be column-major: stride (1, lda) with lda >= m (see colmajor())")
    return A.stride(1)


def make_opts(*, kind=SPARSE_SIGN, s=None, n=None, zeta=8, seed=0, sketch_prec=FP32, qr_prec=FP32, refine_steps=0,
              row_offset=0):
    if s is None:
        s = 2 * n
    return Opts(kind=kind, zeta=zeta, s=s, seed=seed, sketch_prec=sketch_prec, qr_prec=qr_prec,
                refine_steps=refine_steps, row_offset=row_offset)


# Row-sharded solves: the caller's reduction of partial sums (lsq_set_reduce_hook).
REDUCE_SUM_F32, REDUCE_SUM_F64, REDUCE_MAX_U64 = 0, 1, 2
REDUCE_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p)
_reduce_keep = []


def set_reduce_hook(fn):
    """Register `fn(buf_ptr, count, kind, stream_ptr) -> int` (0 = OK) as the
    reduction of every partial sum over rows, or None to remove it."""
    L = lib()
    L.lsq_set_reduce_hook.restype = C.c_void_p
    L.lsq_set_reduce_hook.argtypes = [REDUCE_FN, C.c_void_p]
    if fn is None:
        L.lsq_set_reduce_hook(REDUCE_FN(), None)
        _reduce_keep.clear()
        return
    cb = REDUCE_FN(lambda buf, count, kind, stream, user: int(fn(buf, count, kind, stream)))
    _reduce_keep[:] = [cb]
    L.lsq_set_reduce_hook(cb, None)


def workspace_size(op, m, n, opts=None) -> int:
    return int(lib().lsq_workspace_size(op, m, n, C.byref(opts) if opts is not None else None))


def workspace(op, m, n, opts=None, device=None) -> torch.Tensor:
    nbytes = workspace_size(op, m, n, opts)
    if nbytes == 0:
        raise LsqError("invalid arguments for the workspace query")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def precision_from_kappa0(k0: float) -> int:
    return int(lib().lsq_precision_from_kappa0(float(k0)))


def sparse_sign_operator(seed, m, s, zeta, device="cuda"):
    idx = torch.empty((m, zeta), dtype=torch.int32, device=device)
    sgn = torch.empty((m, zeta), dtype=torch.int8, device=device)
    _check(lib().lsq_sparse_sign_operator(seed, m, s, zeta, _ptr(idx), _ptr(sgn), _stream()), "lsq_sparse_sign_operator")
    return idx, sgn


def gaussian_operator(seed, s, m, prec=FP64, device="cuda"):
    Om = torch.empty((m, s), dtype=torch.float64, device=device).t()
    _check(lib().lsq_gaussian_operator(seed, s, m, prec, _ptr(Om), _stream()), "lsq_gaussian_operator")
    return Om


def sketch(A, opts: Opts, ws=None):
    """A_s (s x n, float32 unless FP64; column-major), colexp (n int32), info."""
    _need_cuda(A)
    m, n = A.shape
    lda = _ld(A)
    s = opts.s
    dt = torch.float64 if opts.sketch_prec == FP64 else torch.float32
    As = torch.empty((n, s), dtype=dt, device=A.device).t()
    colexp = torch.empty(n, dtype=torch.int32, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    ws = workspace(OP_SKETCH, m, n, opts, A.device) if ws is None else ws
    _check(lib().lsq_sketch(_ptr(A), m, n, lda, C.byref(opts), _ptr(As), s, _ptr(colexp), _ptr(info), _ptr(ws),
                            ws.numel(), _stream()), "lsq_sketch")
    return As, colexp, info


def precond_qr(As, colexp=None, qr_prec=FP32, ws=None):
    """R_s (n x n FP64, upper; strict lower zero), info."""
    _need_cuda(As)
    s, n = As.shape
    as_prec = FP64 if As.dtype == torch.float64 else FP32
    if As.stride(0) != 1:
        raise LsqError("As must be column-major")
    Rs = torch.zeros((n, n), dtype=torch.float64, device=As.device).t()
    info = torch.zeros(1, dtype=torch.int32, device=As.device)
    ws = workspace(OP_PRECOND_QR, s, n, None, As.device) if ws is None else ws
    _check(lib().lsq_precond_qr(_ptr(As), s, n, As.stride(1) if n > 1 else s, as_prec, qr_prec, _ptr(colexp), _ptr(Rs),
                                n, _ptr(info), _ptr(ws), ws.numel(), _stream()), "lsq_precond_qr")
    return Rs, info


def condest(A, ws=None):
    """(kappa0 (1 float64), chosen precision (1 int32)) on the device."""
    _need_cuda(A)
    m, n = A.shape
    lda = _ld(A)
    k0 = torch.empty(1, dtype=torch.float64, device=A.device)
    ch = torch.empty(1, dtype=torch.int32, device=A.device)
    ws = workspace(OP_CONDEST, m, n, None, A.device) if ws is None else ws
    _check(lib().lsq_condest(_ptr(A), m, n, lda, _ptr(k0), _ptr(ch), _ptr(ws), ws.numel(), _stream()), "lsq_condest")
    return k0, ch


def trsm_gram(A, Rs, b, hpne=False, ws=None):
    """A_p = A R_s^{-1}, G = A_p^T A_p (or A_p^T A), c = A_p^T b."""
    _need_cuda(A, Rs, b)
    m, n = A.shape
    lda = _ld(A)
    Ap = torch.empty((n, m), dtype=torch.float64, device=A.device).t()
    G = torch.empty((n, n), dtype=torch.float64, device=A.device).t()
    c = torch.empty(n, dtype=torch.float64, device=A.device)
    ws = workspace(OP_TRSM_GRAM, m, n, None, A.device) if ws is None else ws
    _check(lib().lsq_trsm_gram(_ptr(A), m, n, lda, _ptr(Rs), _ld(Rs), _ptr(b), int(hpne), _ptr(Ap), m, _ptr(G), n,
                               _ptr(c), _ptr(ws), ws.numel(), _stream()), "lsq_trsm_gram")
    return Ap, G, c


def trsm_tc(A, R, out=None):
    """A_p = A R^{-1} in FP64 with tensor-core updates (lsq_trsm_tc); returns (Ap, info).
    ``out`` may be ``A`` itself (in place)."""
    _need_cuda(A, R)
    m, n = A.shape
    Ap = torch.empty((n, m), dtype=torch.float64, device=A.device).t() if out is None else out
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    ws = torch.empty(int(lib().lsq_trsm_tc_workspace_size(m, n)), dtype=torch.uint8, device=A.device)
    _check(lib().lsq_trsm_tc(_ptr(A), m, n, _ld(A), _ptr(R), _ld(R), _ptr(Ap), _ld(Ap), _ptr(info), _ptr(ws),
                             ws.numel(), _stream()), "lsq_trsm_tc")
    return Ap, info


def gram_tc(X):
    """G = X^T X in FP64 on the FP8 tensor cores (lsq_gram_tc); returns (G, info)."""
    _need_cuda(X)
    m, n = X.shape
    G = torch.empty((n, n), dtype=torch.float64, device=X.device).t()
    info = torch.zeros(1, dtype=torch.int32, device=X.device)
    ws = torch.empty(int(lib().lsq_gram_tc_workspace_size(m, n)), dtype=torch.uint8, device=X.device)
    _check(lib().lsq_gram_tc(_ptr(X), m, n, _ld(X), _ptr(G), n, _ptr(info), _ptr(ws), ws.numel(), _stream()),
           "lsq_gram_tc")
    return G, info


def gemm_tn_tc(X, Y):
    """G = X^T Y in FP64 on the FP8 tensor cores (lsq_gemm_tn_tc); returns (G, info)."""
    _need_cuda(X, Y)
    m, n = X.shape
    if Y.shape != (m, n):
        raise LsqError("X and Y must have the same shape")
    G = torch.empty((n, n), dtype=torch.float64, device=X.device).t()
    info = torch.zeros(1, dtype=torch.int32, device=X.device)
    ws = torch.empty(int(lib().lsq_gemm_tn_tc_workspace_size(m, n)), dtype=torch.uint8, device=X.device)
    _check(lib().lsq_gemm_tn_tc(_ptr(X), _ld(X), _ptr(Y), _ld(Y), m, n, _ptr(G), n, _ptr(info), _ptr(ws), ws.numel(),
                                _stream()), "lsq_gemm_tn_tc")
    return G, info


def set_fp64_emulation(enable: bool) -> bool:
    """Route the FP64 Gram (PNE) and A_p = A R^{-1} through the tensor cores
    (True, the default) or the FP64 CUDA cores; returns the previous setting."""
    return bool(lib().lsq_set_fp64_emulation(int(enable)))


def test_set_solve_wait_ns(ns: int) -> int:
    """Test-only: bound (ns) of each wait of the triangular solves for another
    block's solution; a wait that runs out records -2 in info.  Returns the
    previous bound."""
    return int(lib().lsq_test_set_solve_wait_ns(int(ns)))


def factor_solve(G, c, Rs=None, hpne=False):
    """Factor G in place (Cholesky or LU-PP) and solve; returns (x, factors, piv, info)."""
    _need_cuda(G, c, Rs)
    n = G.shape[0]
    F = colmajor(G)
    x = torch.empty(n, dtype=torch.float64, device=G.device)
    piv = torch.zeros(n, dtype=torch.int32, device=G.device)
    info = torch.zeros(1, dtype=torch.int32, device=G.device)
    ws = workspace(OP_FACTOR_SOLVE, 1, n, None, G.device)
    _check(lib().lsq_factor_solve(int(hpne), _ptr(F), n, n, _ptr(c), _ptr(Rs), _ld(Rs) if Rs is not None else n,
                                  _ptr(x), _ptr(piv), _ptr(info), _ptr(ws), ws.numel(), _stream()),
           "lsq_factor_solve")
    return x, F, piv, info


def condest_sketch(A, seed=0, ws=None):
    """Condition estimate on an FP32 sketch (lsq_condest_sketch): (kappa0, chosen) on the device."""
    _need_cuda(A)
    m, n = A.shape
    k0 = torch.empty(1, dtype=torch.float64, device=A.device)
    ch = torch.empty(1, dtype=torch.int32, device=A.device)
    ws = workspace(OP_CONDEST_SKETCH, m, n, None, A.device) if ws is None else ws
    _check(lib().lsq_condest_sketch(_ptr(A), m, n, _ld(A), C.c_uint64(seed), _ptr(k0), _ptr(ch), _ptr(ws),
                                    ws.numel(), _stream()), "lsq_condest_sketch")
    return k0, ch


def solve(A, b, *, hpne=False, method=None, opts: Opts = None, ws=None, Rs_out=None, x=None, info=None, **kw):
    """Alg. 1 end to end.  `method` (pne, hpne, hpne_qr, sne, nne_lu; default
    PNE, or HPNE with hpne=True) picks the entry point.  Returns (x, info)
    device tensors."""
    _need_cuda(A, b)
    m, n = A.shape
    lda = _ld(A)
    opts = opts or make_opts(n=n, **kw)
    name, op = METHODS[method or ("hpne" if hpne else "pne")]
    ws = workspace(op, m, n, opts, A.device) if ws is None else ws
    x = torch.empty(n, dtype=torch.float64, device=A.device) if x is None else x
    info = torch.zeros(1, dtype=torch.int32, device=A.device) if info is None else info
    _check(getattr(lib(), name)(_ptr(A), m, n, lda, _ptr(b), C.byref(opts), _ptr(x), _ptr(Rs_out), _ptr(info),
                                _ptr(ws), ws.numel(), _stream()), name)
    return x, info


def pne(A, b, **kw):
    return solve(A, b, hpne=False, **kw)


def hpne(A, b, **kw):
    return solve(A, b, hpne=True, **kw)


def solve_host(A_host, b_host, *, hpne=False, opts: Opts = None, ws=None, x_host=None, **kw):
    """End to end on HOST tensors (pinned recommended): copies in, solves,
    copies x back; returns (x_host, info)."""
    m, n = A_host.shape
    if A_host.is_cuda or b_host.is_cuda:
        raise LsqError("solve_host takes host tensors")
    lda = _ld(A_host)
    opts = opts or make_opts(n=n, **kw)
    op = OP_HPNE_HOST if hpne else OP_PNE_HOST
    ws = workspace(op, m, n, opts) if ws is None else ws
    x_host = torch.empty(n, dtype=torch.float64, pin_memory=A_host.is_pinned()) if x_host is None else x_host
    info = C.c_int32(0)
    fn = lib().lsq_hpne_solve_host if hpne else lib().lsq_pne_solve_host
    _check(fn(_ptr(A_host), m, n, lda, _ptr(b_host), C.byref(opts), _ptr(x_host), C.cast(C.pointer(info), C.c_void_p),
              _ptr(ws), ws.numel(), _stream()), "lsq_solve_host")
    return x_host, info.value


# ---------------------------------------------------------------------------- batched
class BatchProblem(C.Structure):
    _fields_ = [("A", C.c_void_p), ("m", C.c_int64), ("n", C.c_int64), ("lda", C.c_int64), ("b", C.c_void_p),
                ("x", C.c_void_p), ("info", C.c_void_p), ("reserved0", C.c_int32), ("reserved1", C.c_int32),
                ("opts", Opts)]


def _batch_sigs():
    L = lib()
    L.lsq_batched_workspace_size.restype = C.c_size_t
    L.lsq_batched_workspace_size.argtypes = [C.c_int32, C.c_int32, C.POINTER(BatchProblem)]
    for nm in ("lsq_pne_solve_batched", "lsq_hpne_solve_batched"):
        f = getattr(L, nm)
        f.restype = C.c_int32
        f.argtypes = [C.c_int32, C.POINTER(BatchProblem), C.c_void_p, C.c_size_t, C.c_void_p]
    return L


def batch_descriptors(As, bs, xs, infos, opts_list):
    """ctypes array of lsq_batch_problem for device tensors (A column-major)."""
    arr = (BatchProblem * len(As))()
    for i, (A, b, x, info, o) in enumerate(zip(As, bs, xs, infos, opts_list)):
        _need_cuda(A, b, x, info)
        m, n = A.shape
        arr[i] = BatchProblem(A.data_ptr(), m, n, _ld(A), b.data_ptr(), x.data_ptr(), info.data_ptr(), 0, 0, o)
    return arr


def batched_workspace(desc, hpne=False, device=None):
    L = _batch_sigs()
    nbytes = int(L.lsq_batched_workspace_size(int(hpne), len(desc), desc))
    if nbytes == 0:
        raise LsqError("invalid batch description")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def solve_batched(desc, ws, hpne=False):
    """Alg. 1 on every problem of `desc` (from batch_descriptors): one cached
    CUDA-graph launch of all solves over 16 internal streams."""
    L = _batch_sigs()
    fn = L.lsq_hpne_solve_batched if hpne else L.lsq_pne_solve_batched
    _check(fn(len(desc), desc, _ptr(ws), ws.numel(), _stream()), "lsq_solve_batched")


class SketchProblem(C.Structure):
    _fields_ = [("A", C.c_void_p), ("m", C.c_int64), ("n", C.c_int64), ("lda", C.c_int64), ("As", C.c_void_p),
                ("ldas", C.c_int64), ("colexp", C.c_void_p), ("info", C.c_void_p), ("opts", Opts)]


class QrProblem(C.Structure):
    _fields_ = [("As", C.c_void_p), ("s", C.c_int64), ("n", C.c_int64), ("ldas", C.c_int64),
                ("as_prec", C.c_int32), ("qr_prec", C.c_int32), ("colexp", C.c_void_p), ("Rs", C.c_void_p),
                ("ldr", C.c_int64), ("info", C.c_void_p)]


def _steps_sigs():
    L = lib()
    for nm, T in (("lsq_sketch_batched", SketchProblem), ("lsq_precond_qr_batched", QrProblem)):
        w = getattr(L, nm + "_workspace_size")
        w.restype = C.c_size_t
        w.argtypes = [C.c_int32, C.POINTER(T)]
        f = getattr(L, nm)
        f.restype = C.c_int32
        f.argtypes = [C.c_int32, C.POINTER(T), C.c_void_p, C.c_size_t, C.c_void_p]
    return L


def sketch_batched(As_list, opts_list):
    """lsq_sketch on every (A, opts) in one captured fan-out; returns
    [(A_s, colexp, info)] (A_s float32, or float64 for FP64)."""
    L = _steps_sigs()
    arr = (SketchProblem * len(As_list))()
    outs = []
    for i, (A, o) in enumerate(zip(As_list, opts_list)):
        _need_cuda(A)
        m, n = A.shape
        dt = torch.float64 if o.sketch_prec == FP64 else torch.float32
        As = torch.empty((n, o.s), dtype=dt, device=A.device).t()
        ce = torch.empty(n, dtype=torch.int32, device=A.device)
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
        arr[i] = SketchProblem(A.data_ptr(), m, n, _ld(A), As.data_ptr(), o.s, ce.data_ptr(), info.data_ptr(), o)
        outs.append((As, ce, info))
    nbytes = int(L.lsq_sketch_batched_workspace_size(len(arr), arr))
    if nbytes == 0:
        raise LsqError("invalid batch description")
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _check(L.lsq_sketch_batched(len(arr), arr, _ptr(ws), ws.numel(), _stream()), "lsq_sketch_batched")
    return outs


def precond_qr_batched(items, qr_prec=FP32):
    """lsq_precond_qr on every (A_s, colexp) in one captured fan-out; returns [(R_s, info)]."""
    L = _steps_sigs()
    arr = (QrProblem * len(items))()
    outs = []
    for i, (As, ce) in enumerate(items):
        _need_cuda(As)
        s_, n = As.shape
        ap = FP64 if As.dtype == torch.float64 else FP32
        qp = FP64 if ap == FP64 else qr_prec
        Rs = torch.zeros((n, n), dtype=torch.float64, device=As.device).t()
        info = torch.zeros(1, dtype=torch.int32, device=As.device)
        arr[i] = QrProblem(As.data_ptr(), s_, n, _ld(As, (torch.float64, torch.float32)), ap, qp,
                           ce.data_ptr() if ce is not None else None,
                           Rs.data_ptr(), n, info.data_ptr())
        outs.append((Rs, info))
    nbytes = int(L.lsq_precond_qr_batched_workspace_size(len(arr), arr))
    if nbytes == 0:
        raise LsqError("invalid batch description")
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _check(L.lsq_precond_qr_batched(len(arr), arr, _ptr(ws), ws.numel(), _stream()), "lsq_precond_qr_batched")
    return outs


# ---------------------------------------------------------------------------- learned proposal
N_FEATURES = 10
CLASS_PRECS = [FP8_E4M3, BF16, FP32, FP64]


def _learn_sigs():
    L = lib()
    sigs = {
        "lsq_mlp_param_count": (C.c_int64, [C.c_int32]),
        "lsq_mlp_num_features": (C.c_int32, []),
        "lsq_features_workspace_size": (C.c_size_t, [C.c_int64, C.c_int64]),
        "lsq_features": (C.c_int32, [_vp, _i64, _i64, _i64, C.c_uint64, _vp, _vp, _sz, _vp]),
        "lsq_mlp_forward": (C.c_int32, [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp]),
        "lsq_mlp_backward_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32]),
        "lsq_mlp_backward": (C.c_int32, [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
        "lsq_mlp_adam": (C.c_int32, [_vp, _vp, _vp, _vp, _i64, C.c_float, C.c_float, C.c_float, C.c_float,
                                     C.c_int32, _vp]),
        "lsq_propose_precision": (C.c_int32, [_vp, _i64, _i64, _i64, C.c_uint64, _vp, C.c_int32, _vp, _vp, _vp,
                                              _sz, _vp]),
        "lsq_judge_workspace_size": (C.c_size_t, [C.c_int64]),
        "lsq_judge_preconditioner": (C.c_int32, [_vp, _i64, _i64, C.c_int32, _vp, _vp, _vp, _sz, _vp]),
        "lsq_learned_workspace_size": (C.c_size_t, [_i64, _i64, C.POINTER(Opts)]),
        "lsq_pne_solve_learned": (C.c_int32, [_vp, _i64, _i64, _i64, _vp, C.POINTER(Opts), _vp, C.c_int32, _vp,
                                              _vp, _vp, _vp, _vp, _sz, _vp]),
    }
    for nm, (res, args) in sigs.items():
        f = getattr(L, nm)
        f.restype = res
        f.argtypes = args
    return L


def mlp_param_count(d=N_FEATURES) -> int:
    return int(_learn_sigs().lsq_mlp_param_count(d))


def features(A, seed=0, ws=None):
    """The 10 proposal features of A (float32 device tensor)."""
    L = _learn_sigs()
    _need_cuda(A)
    m, n = A.shape
    f = torch.empty(N_FEATURES, dtype=torch.float32, device=A.device)
    ws = torch.empty(int(L.lsq_features_workspace_size(m, n)), dtype=torch.uint8, device=A.device) if ws is None else ws
    _check(L.lsq_features(_ptr(A), m, n, _ld(A), seed, _ptr(f), _ptr(ws), ws.numel(), _stream()), "lsq_features")
    return f


def mlp_forward(params, X):
    L = _learn_sigs()
    _need_cuda(params, X)
    B, d = X.shape
    logits = torch.empty((B, 4), dtype=torch.float32, device=X.device)
    _check(L.lsq_mlp_forward(_ptr(params), d, B, _ptr(X.contiguous()), _ptr(logits), _stream()), "lsq_mlp_forward")
    return logits


def mlp_backward(params, X, labels, ws=None):
    """(gradient, mean loss) of the softmax cross-entropy."""
    L = _learn_sigs()
    _need_cuda(params, X, labels)
    B, d = X.shape
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    nbytes = int(L.lsq_mlp_backward_workspace_size(d, B))
    ws = torch.empty(nbytes, dtype=torch.uint8, device=X.device) if ws is None or ws.numel() < nbytes else ws
    _check(L.lsq_mlp_backward(_ptr(params), d, B, _ptr(X.contiguous()), _ptr(labels), _ptr(grad), _ptr(loss),
                              _ptr(ws), ws.numel(), _stream()), "lsq_mlp_backward")
    return grad, loss


def mlp_adam(params, grad, m1, m2, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    L = _learn_sigs()
    _check(L.lsq_mlp_adam(_ptr(params), _ptr(grad), _ptr(m1), _ptr(m2), params.numel(), lr, beta1, beta2, eps,
                          step, _stream()), "lsq_mlp_adam")


def propose_precision(A, params, seed=0, ws=None):
    """(proposed precision code, class probabilities) as device tensors."""
    L = _learn_sigs()
    m, n = A.shape
    prec = torch.empty(1, dtype=torch.int32, device=A.device)
    probs = torch.empty(4, dtype=torch.float32, device=A.device)
    ws = torch.empty(int(L.lsq_features_workspace_size(m, n)), dtype=torch.uint8, device=A.device) if ws is None else ws
    _check(L.lsq_propose_precision(_ptr(A), m, n, _ld(A), seed, _ptr(params), N_FEATURES, _ptr(prec), _ptr(probs),
                                   _ptr(ws), ws.numel(), _stream()), "lsq_propose_precision")
    return prec, probs


def judge_preconditioner(Rs, prec):
    """(accept (1 int32), kappa_1 estimate (1 float64)) on the device."""
    L = _learn_sigs()
    n = Rs.shape[0]
    acc = torch.empty(1, dtype=torch.int32, device=Rs.device)
    k1 = torch.empty(1, dtype=torch.float64, device=Rs.device)
    ws = torch.empty(int(L.lsq_judge_workspace_size(n)), dtype=torch.uint8, device=Rs.device)
    _check(L.lsq_judge_preconditioner(_ptr(Rs), n, _ld(Rs), prec, _ptr(acc), _ptr(k1), _ptr(ws), ws.numel(),
                                      _stream()), "lsq_judge_preconditioner")
    return acc, k1


def pne_learned(A, b, params, opts, ws=None, x=None, info=None):
    """PNE with the learned proposal; returns (x, info, used precision, escalations)."""
    L = _learn_sigs()
    _need_cuda(A, b, params)
    m, n = A.shape
    ws = torch.empty(int(L.lsq_learned_workspace_size(m, n, C.byref(opts))), dtype=torch.uint8,
                     device=A.device) if ws is None else ws
    x = torch.empty(n, dtype=torch.float64, device=A.device) if x is None else x
    info = torch.zeros(1, dtype=torch.int32, device=A.device) if info is None else info
    used = C.c_int32(0)
    esc = C.c_int32(0)
    _check(L.lsq_pne_solve_learned(_ptr(A), m, n, _ld(A), _ptr(b), C.byref(opts), _ptr(params), N_FEATURES, _ptr(x),
                                   _ptr(info), C.cast(C.pointer(used), C.c_void_p), C.cast(C.pointer(esc), C.c_void_p),
                                   _ptr(ws), ws.numel(), _stream()), "lsq_pne_solve_learned")
    return x, info, used.value, esc.value
