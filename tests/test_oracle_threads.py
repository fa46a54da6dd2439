"""The oracle spreads loops with independent iterations over host threads
(OpenMP) while every sum keeps its index order, so its results must be
bit-identical for any thread count.  These CPU tests run each oracle step
with one thread and with several and compare the bits."""
import numpy as np
import pytest

import oracle as O
import problems as P


@pytest.fixture
def threads():
    prev = O.set_threads(1)
    yield
    O.set_threads(prev)


def _both(fn):
    O.set_threads(1)
    a = fn()
    O.set_threads(5)
    b = fn()
    O.set_threads(1)
    return a, b


def _same(a, b):
    if isinstance(a, (tuple, list)):
        assert len(a) == len(b)
        for x, y in zip(a, b):
            _same(x, y)
    elif isinstance(a, dict):
        assert a.keys() == b.keys()
        for k in a:
            _same(a[k], b[k])
    elif isinstance(a, np.ndarray):
        assert a.dtype == b.dtype and a.shape == b.shape
        assert a.tobytes() == b.tobytes()
    else:
        assert (a == b) or (a != a and b != b)


@pytest.mark.parametrize("hpne", [False, True])
@pytest.mark.parametrize("kind,prec,refine", [
    (O.SPARSE_SIGN, O.BF16, 1),
    (O.SPARSE_SIGN, O.FP64, 0),
    (O.GAUSSIAN, O.FP32, 1),
    (O.GAUSSIAN, O.FP8_E4M3, 0),
    (O.GAUSSIAN, O.FP64, 1),
    (O.GAUSSIAN, O.AUTO, 0),
])
def test_solve_bits_independent_of_threads(threads, hpne, kind, prec, refine):
    pr = P.make_problem(700, 37, 1e5, 1e-7, 4242)
    s = 111
    kw = dict(hpne=hpne, kind=kind, s=s, zeta=4, seed=9, sketch_prec=prec, qr_prec=O.FP32, refine_steps=refine)
    a, b = _both(lambda: O.solve(pr.A, pr.b, **kw))
    _same(a, b)


def test_steps_bits_independent_of_threads(threads):
    pr = P.make_problem(513, 29, 1e6, 1e-6, 4343)
    for kind in (O.SPARSE_SIGN, O.GAUSSIAN):
        for prec in (O.FP8_E4M3, O.FP16, O.FP32, O.FP64):
            _same(*_both(lambda: O.sketch(pr.A, kind, 64, 3, 5, prec)))
    As, _ = O.sketch(pr.A, O.GAUSSIAN, 64, 0, 5, O.FP64)
    for qp in (O.FP32, O.FP64):
        _same(*_both(lambda: O.qr_r(As, qp)))
    R = O.qr_r(As, O.FP64)
    _same(*_both(lambda: O.trsm_right_upper(pr.A, R)))
    Ap = O.trsm_right_upper(pr.A, R)
    _same(*_both(lambda: O.gram(Ap, pr.A, pr.b)))
    G, _ = O.gram(Ap, Ap, pr.b)
    _same(*_both(lambda: O.cholesky(G)))
    _same(*_both(lambda: O.lu(G)))
    _same(*_both(lambda: O.lstsq_qr(pr.A, pr.b)))
    _same(*_both(lambda: O.condest(pr.A)))
    _same(*_both(lambda: O.sparse_sign_indices(77, 1000, 50, 6)))
    _same(*_both(lambda: O.gaussian_operator(77, 20, 300, O.BF16)))
