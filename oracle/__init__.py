"""ctypes wrapper around the plain-C oracle (``oracle/lsq_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously correct CPU
statement of randomized-preconditioned normal equations (Garrison & Ipsen,
arXiv 2603.16644, Alg. 1 and Eqs. e_pne / e_hpne).  Only the tests, the
package smoke check and the benchmark's CPU-baseline leg may import it; the
CUDA library never does, and the two share no code.

All matrices are numpy float64 arrays in Fortran (column-major) order.
"""
import ctypes as C
import math

import numpy as np

from . import build as _build

FP8_E4M3, BF16, FP16, FP32, FP64, AUTO, AUTO_SKETCH = 0, 1, 2, 3, 4, 5, 6
GAUSSIAN, SPARSE_SIGN, SRFT = 0, 1, 2
PREC_NAMES = {FP8_E4M3: "fp8_e4m3", BF16: "bf16", FP16: "fp16", FP32: "fp32", FP64: "fp64", AUTO: "auto",
              AUTO_SKETCH: "auto_sketch"}

_lib = None

_d = C.POINTER(C.c_double)
_i32 = C.POINTER(C.c_int32)
_i8 = C.POINTER(C.c_int8)
_u32 = C.POINTER(C.c_uint32)
_i64 = C.c_int64


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "lsqo_set_threads": (C.c_int, [C.c_int]),
            "lsqo_srft_order": (_i64, [_i64]),
            "lsqo_srft_sign": (C.c_int, [C.c_uint64, _i64]),
            "lsqo_srft_row": (_i64, [C.c_uint64, _i64, _i64]),
            "lsqo_fwht": (None, [_d, _i64]),
            "lsqo_round": (C.c_double, [C.c_double, C.c_int]),
            "lsqo_round_array": (None, [_d, _i64, C.c_int, _d]),
            "lsqo_philox4x32_10": (None, [_u32, _u32, _u32]),
            "lsqo_sparse_sign_column": (C.c_int, [C.c_uint64, _i64, _i64, C.c_int, _i32, _i8]),
            "lsqo_sparse_sign_indices": (C.c_int, [C.c_uint64, _i64, _i64, C.c_int, _i32, _i8]),
            "lsqo_gaussian_entry": (C.c_double, [C.c_uint64, _i64, _i64]),
            "lsqo_zig_tables": (None, [_d, _d]),
            "lsqo_gaussian_operator": (None, [C.c_uint64, _i64, _i64, C.c_int, _d]),
            "lsqo_colexp": (None, [_d, _i64, _i64, _i64, C.c_int, _i32]),
            "lsqo_quantize": (None, [_d, _i64, _i64, _i64, C.c_int, _i32, _d]),
            "lsqo_sketch": (C.c_int, [_d, _i64, _i64, _i64, C.c_int, _i64, C.c_int, C.c_uint64, C.c_int, _d, _i32]),
            "lsqo_qr_r": (C.c_int, [_d, _i64, _i64, _i64, C.c_int, _d]),
            "lsqo_unscale_r": (None, [_d, _i64, _i64, _i32]),
            "lsqo_trsm_right_upper": (C.c_int, [_d, _i64, _i64, _i64, _d, _i64, _d]),
            "lsqo_gram": (None, [_d, _d, _i64, _i64, _i64, _i64, _d, _d, _d]),
            "lsqo_cholesky": (C.c_int, [_d, _i64, _i64]),
            "lsqo_lu": (C.c_int, [_d, _i64, _i64, _i32]),
            "lsqo_solve_lower": (None, [_d, _i64, _i64, C.c_int, _d]),
            "lsqo_solve_lower_t": (None, [_d, _i64, _i64, _d]),
            "lsqo_solve_upper": (None, [_d, _i64, _i64, _d]),
            "lsqo_lu_solve": (None, [_d, _i64, _i64, _i32, _d]),
            "lsqo_lstsq_qr": (C.c_int, [_d, _i64, _i64, _i64, _d, _d]),
            "lsqo_precision_from_kappa0": (C.c_int, [C.c_double]),
            "lsqo_condest": (C.c_int, [_d, _i64, _i64, _i64, _d, _i32, _d, _d]),
            "lsqo_solve": (C.c_int, [_d, _i64, _i64, _i64, _d, C.c_int, C.c_int, _i64, C.c_int, C.c_uint64,
                                     C.c_int, C.c_int, C.c_int, _d, _d, _d, _i32]),
            "lsqo_solve_method": (C.c_int, [_d, _i64, _i64, _i64, _d, C.c_int, C.c_int, _i64, C.c_int, C.c_uint64,
                                            C.c_int, C.c_int, C.c_int, _d, _d, _d, _i32]),
            "lsqo_lu_tall_u": (C.c_int, [_d, _i64, _i64, _i64, C.c_int, _d]),
            "lsqo_condest_sketch": (C.c_int, [_d, _i64, _i64, _i64, C.c_uint64, _d, _i32, _d]),
            "lsqo_kappa1_upper32": (C.c_double, [_d, _i64, _i64]),
            "lsqo_solve_upper_t": (None, [_d, _i64, _i64, _d]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def set_threads(n):
    """Threads of the oracle's parallel loops (n <= 0: unchanged); returns
    the previous count.  Results do not depend on it."""
    return int(lib().lsqo_set_threads(int(n)))


def _p(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


# --- rounding ---------------------------------------------------------------
def round_to(x, prec):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    y = np.empty_like(x)
    lib().lsqo_round_array(_p(x), x.size, prec, _p(y))
    return y


# --- random streams ---------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().lsqo_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def sparse_sign_indices(seed, m, s, zeta):
    """Row indices (m, zeta) int32 and signs (m, zeta) int8 of every column of Omega."""
    idx = np.zeros((m, zeta), dtype=np.int32)
    sgn = np.zeros((m, zeta), dtype=np.int8)
    rc = lib().lsqo_sparse_sign_indices(C.c_uint64(seed), m, s, zeta, _p(idx, C.c_int32), _p(sgn, C.c_int8))
    if rc:
        raise ValueError(f"sparse_sign_indices rc={rc}")
    return idx, sgn


def gaussian_entry(seed, i, j):
    return lib().lsqo_gaussian_entry(C.c_uint64(seed), i, j)


ZIG_N = 256


def zig_tables():
    """The ziggurat's layer bounds x_0..x_256 and f(x_i) = exp(-x_i^2 / 2)
    (f(x_0) stored as 0)."""
    x, f = np.zeros(ZIG_N + 1), np.zeros(ZIG_N + 1)
    lib().lsqo_zig_tables(_p(x), _p(f))
    return x, f


def gaussian_operator(seed, s, m, prec=FP64):
    Om = np.zeros((s, m), dtype=np.float64, order="F")
    lib().lsqo_gaussian_operator(C.c_uint64(seed), s, m, prec, _p(Om))
    return Om


# --- method steps -----------------------------------------------------------
def colexp(A, prec):
    A = _f64(A)
    m, n = A.shape
    e = np.zeros(n, dtype=np.int32)
    lib().lsqo_colexp(_p(A), m, n, m, prec, _p(e, C.c_int32))
    return e


def quantize(A, prec, e):
    A = _f64(A)
    m, n = A.shape
    e = np.ascontiguousarray(e, dtype=np.int32)
    out = np.zeros((m, n), dtype=np.float64, order="F")
    lib().lsqo_quantize(_p(A), m, n, m, prec, _p(e, C.c_int32), _p(out))
    return out


def sketch(A, kind, s, zeta, seed, prec):
    """Returns (A_s (s, n) float64 holding FP32 values unless prec==FP64, colexp)."""
    A = _f64(A)
    m, n = A.shape
    As = np.zeros((s, n), dtype=np.float64, order="F")
    e = np.zeros(n, dtype=np.int32)
    rc = lib().lsqo_sketch(_p(A), m, n, m, kind, s, zeta, C.c_uint64(seed), prec, _p(As), _p(e, C.c_int32))
    if rc:
        raise ValueError(f"sketch rc={rc}")
    return As, e


def qr_r(As, prec):
    As = _f64(As)
    s, n = As.shape
    R = np.zeros((n, n), dtype=np.float64, order="F")
    rc = lib().lsqo_qr_r(_p(As), s, n, s, prec, _p(R))
    if rc:
        raise ValueError(f"qr_r rc={rc}")
    return R


def unscale_r(R, e):
    R = _f64(R).copy(order="F")
    n = R.shape[0]
    e = np.ascontiguousarray(e, dtype=np.int32)
    lib().lsqo_unscale_r(_p(R), n, n, _p(e, C.c_int32))
    return R


def trsm_right_upper(A, R):
    A = _f64(A)
    R = _f64(R)
    m, n = A.shape
    Ap = np.zeros((m, n), dtype=np.float64, order="F")
    lib().lsqo_trsm_right_upper(_p(A), m, n, m, _p(R), n, _p(Ap))
    return Ap


def gram(X, Y, b=None):
    X = _f64(X)
    Y = _f64(Y)
    m, n = X.shape
    G = np.zeros((n, n), dtype=np.float64, order="F")
    c = np.zeros(n, dtype=np.float64)
    bb = _f64(b) if b is not None else None
    lib().lsqo_gram(_p(X), _p(Y), m, n, m, m, _p(bb) if bb is not None else None, _p(G),
                    _p(c) if bb is not None else None)
    return G, (c if bb is not None else None)


def cholesky(G):
    L = _f64(G).copy(order="F")
    n = L.shape[0]
    info = lib().lsqo_cholesky(_p(L), n, n)
    return L, info


def lu(H):
    LU = _f64(H).copy(order="F")
    n = LU.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    info = lib().lsqo_lu(_p(LU), n, n, _p(piv, C.c_int32))
    return LU, piv, info


def solve_lower(L, y, unit=False):
    L = _f64(L)
    y = np.array(y, dtype=np.float64)
    lib().lsqo_solve_lower(_p(L), L.shape[0], L.shape[0], int(unit), _p(y))
    return y


def solve_lower_t(L, y):
    L = _f64(L)
    y = np.array(y, dtype=np.float64)
    lib().lsqo_solve_lower_t(_p(L), L.shape[0], L.shape[0], _p(y))
    return y


def solve_upper(U, y):
    U = _f64(U)
    y = np.array(y, dtype=np.float64)
    lib().lsqo_solve_upper(_p(U), U.shape[0], U.shape[0], _p(y))
    return y


def lu_solve(LU, piv, y):
    LU = _f64(LU)
    y = np.array(y, dtype=np.float64)
    piv = np.ascontiguousarray(piv, dtype=np.int32)
    lib().lsqo_lu_solve(_p(LU), LU.shape[0], LU.shape[0], _p(piv, C.c_int32), _p(y))
    return y


def lstsq_qr(A, b):
    """Reference least-squares solution by FP64 Householder QR (not the method)."""
    A = _f64(A)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n, dtype=np.float64)
    rc = lib().lsqo_lstsq_qr(_p(A), m, n, m, _p(b), _p(x))
    if rc:
        raise ValueError("lstsq_qr: bad shape")
    return x


def precision_from_kappa0(k0):
    return lib().lsqo_precision_from_kappa0(float(k0))


def condest(A):
    """Returns (kappa0, chosen precision, ||G||_1, gamma, cholesky info)."""
    A = _f64(A)
    m, n = A.shape
    k0 = C.c_double()
    ch = C.c_int32()
    nr = C.c_double()
    ga = C.c_double()
    info = lib().lsqo_condest(_p(A), m, n, m, C.byref(k0), C.byref(ch), C.byref(nr), C.byref(ga))
    return k0.value, ch.value, nr.value, ga.value, info


PNE, HPNE, HPNE_QR, SNE, NNE_LU = 0, 1, 2, 3, 4
METHODS = {"pne": PNE, "hpne": HPNE, "hpne_qr": HPNE_QR, "sne": SNE, "nne_lu": NNE_LU}


def solve(A, b, *, hpne=False, method=None, kind=SPARSE_SIGN, s=None, zeta=8, seed=0, sketch_prec=FP32,
          qr_prec=FP32, refine_steps=0):
    """Alg. 1 end to end.  `method` (a code or a name: pne, hpne, hpne_qr,
    sne, nne_lu) overrides `hpne`.  Returns dict(x, Rs, info, kappa0, prec);
    Rs is U_s for the not-normal equations."""
    A = _f64(A)
    m, n = A.shape
    s = 2 * n if s is None else s
    if method is None:
        method = HPNE if hpne else PNE
    method = METHODS.get(method, method)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n, dtype=np.float64)
    Rs = np.zeros((n, n), dtype=np.float64, order="F")
    k0 = C.c_double()
    pr = C.c_int32()
    info = lib().lsqo_solve_method(_p(A), m, n, m, _p(b), int(method), kind, s, zeta, C.c_uint64(seed),
                                   sketch_prec, qr_prec, refine_steps, _p(x), _p(Rs), C.byref(k0), C.byref(pr))
    return {"x": x, "Rs": Rs, "info": info, "kappa0": k0.value, "prec": pr.value}


def condest_sketch(A, seed):
    """Condition estimate on an FP32 sparse-sign sketch: (kappa0, chosen, kappa_1(R_e), rc)."""
    A = _f64(A)
    m, n = A.shape
    k0 = C.c_double()
    ch = C.c_int32()
    k1 = C.c_double()
    rc = lib().lsqo_condest_sketch(_p(A), m, n, m, C.c_uint64(seed), C.byref(k0), C.byref(ch), C.byref(k1))
    return k0.value, ch.value, k1.value, rc


def kappa1_upper32(R):
    """||R||_1 times Hager's FP32 estimate of ||R^{-1}||_1 for upper triangular R."""
    R = _f64(R)
    return float(lib().lsqo_kappa1_upper32(_p(R), R.shape[0], R.shape[0]))


def srft_operator(seed, m, s):
    """(signs (m,), sampled rows (s,), m') of the SRFT sketch S F D."""
    L = lib()
    mp = int(L.lsqo_srft_order(m))
    sg = np.array([L.lsqo_srft_sign(C.c_uint64(seed), j) for j in range(m)], dtype=np.int8)
    rows = np.array([L.lsqo_srft_row(C.c_uint64(seed), t, mp) for t in range(s)], dtype=np.int64)
    return sg, rows, mp


def fwht(x):
    """The oracle's Walsh-Hadamard butterflies (FP64) on a copy of x (length a power of two)."""
    y = np.array(x, dtype=np.float64)
    lib().lsqo_fwht(_p(y), len(y))
    return y


def lu_tall_u(As, prec=FP64):
    """U of the LU with partial pivoting of a tall s x n matrix; returns (U, info)."""
    As = _f64(As)
    s_, n = As.shape
    U = np.zeros((n, n), dtype=np.float64, order="F")
    info = lib().lsqo_lu_tall_u(_p(As), s_, n, s_, prec, _p(U))
    return U, info


def solve_upper_t(U, y):
    U = _f64(U)
    y = np.array(y, dtype=np.float64)
    lib().lsqo_solve_upper_t(_p(U), U.shape[0], U.shape[0], _p(y))
    return y


def kappa(M):
    s = np.linalg.svd(np.asarray(M), compute_uv=False)
    return float(s[0] / s[-1]) if s[-1] > 0 else math.inf


# --- learned precision proposal ----------------------------------------------
N_FEATURES = 10
CLASSES = [FP8_E4M3, BF16, FP32, FP64]


def _mlp_sigs():
    L = lib()
    L.lsqo_mlp_param_count.restype = C.c_int64
    L.lsqo_mlp_param_count.argtypes = [C.c_int]
    L.lsqo_mlp_forward.restype = C.c_double
    L.lsqo_mlp_forward.argtypes = [_d, C.c_int, C.c_int, _d, _i32, _d]
    L.lsqo_mlp_backward.restype = C.c_double
    L.lsqo_mlp_backward.argtypes = [_d, C.c_int, C.c_int, _d, _i32, _d]
    L.lsqo_features.restype = C.c_int
    L.lsqo_features.argtypes = [_d, _i64, _i64, _i64, C.c_uint64, _d]
    return L


def mlp_param_count(d):
    return int(_mlp_sigs().lsqo_mlp_param_count(d))


def mlp_forward(params, X, labels=None):
    """(logits (batch x 4), mean cross-entropy or None)."""
    L = _mlp_sigs()
    X = np.ascontiguousarray(X, dtype=np.float64)
    params = np.ascontiguousarray(params, dtype=np.float64)
    B, d = X.shape
    out = np.zeros((B, 4))
    lab = np.ascontiguousarray(labels, dtype=np.int32) if labels is not None else None
    loss = L.lsqo_mlp_forward(_p(params), d, B, _p(X), _p(lab, C.c_int32) if lab is not None else None, _p(out))
    return out, (loss if lab is not None else None)


def mlp_backward(params, X, labels):
    """(mean cross-entropy, gradient with the packing of params)."""
    L = _mlp_sigs()
    X = np.ascontiguousarray(X, dtype=np.float64)
    params = np.ascontiguousarray(params, dtype=np.float64)
    B, d = X.shape
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    g = np.zeros_like(params)
    loss = L.lsqo_mlp_backward(_p(params), d, B, _p(X), _p(lab, C.c_int32), _p(g))
    return loss, g


def features(A, seed):
    L = _mlp_sigs()
    A = _f64(A)
    m, n = A.shape
    f = np.zeros(N_FEATURES)
    rc = L.lsqo_features(_p(A), m, n, m, C.c_uint64(seed), _p(f))
    if rc:
        raise ValueError(f"features rc={rc}")
    return f
