"""Row-sharded solves through the reduction hook (lsq_set_reduce_hook): the
library hands every partial sum over rows to the caller's reduction.

  * A hook that multiplies every sum by 4 stands for four identical shards
    (A repeated four times, b likewise): each reduced quantity is then an
    exact power-of-two multiple of the unsharded one, and the solution
    equals the unsharded solve, for every method and both estimates; the
    hook sees exactly the expected sequence of reductions.
  * Two real shards (the rows of A split in two, each with its global row
    offset) solved concurrently from two host threads on two streams, the
    hook summing the two partial results, give the unsharded solution up to
    the order of the sums.
"""
import threading

import numpy as np
import pytest
import torch

import problems as P
from tests.gpu_util import dev_colmajor, to_np

pytestmark = pytest.mark.gpu

lsq = pytest.importorskip("paper_2603_16644_gb300")

TYPESTR = {lsq.REDUCE_SUM_F32: "<f4", lsq.REDUCE_SUM_F64: "<f8", lsq.REDUCE_MAX_U64: "<i8"}


class _Raw:
    """A device buffer the library hands to the hook, seen by torch without a
    copy (CUDA array interface, no stream synchronisation implied)."""

    def __init__(self, ptr, count, kind):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": TYPESTR[kind], "data": (ptr, False),
                                         "version": 3}


def view(buf, count, kind):
    return torch.as_tensor(_Raw(buf, count, kind), device="cuda")


def stream_of(ptr):
    # the library's stream: work queued there runs before its next kernels
    return torch.cuda.ExternalStream(ptr) if ptr else torch.cuda.default_stream()


@pytest.mark.parametrize("method,prec", [("pne", lsq.AUTO_SKETCH), ("hpne", lsq.AUTO), ("sne", lsq.FP64),
                                         ("hpne_qr", lsq.FP32), ("nne_lu", lsq.FP32), ("pne", lsq.FP64),
                                         ("pne", lsq.BF16)])
def test_four_identical_shards_give_the_unsharded_solution(method, prec):
    pr = P.make_problem(3000, 120, 1e5, 1e-7, 91)
    A, b = dev_colmajor(pr.A), torch.from_numpy(pr.b).cuda()
    kind = lsq.SPARSE_SIGN if prec == lsq.BF16 else lsq.GAUSSIAN
    opts = lsq.make_opts(kind=kind, s=360, zeta=8, seed=3, sketch_prec=prec,
                         qr_prec=lsq.FP64 if prec == lsq.FP64 else lsq.FP32, refine_steps=1)
    x0, info0 = lsq.solve(A, b, method=method, opts=opts)
    x0 = to_np(x0)
    calls = []

    def times4(buf, count, kind, stream):
        calls.append((kind, count))
        if kind != lsq.REDUCE_MAX_U64:
            with torch.cuda.stream(stream_of(stream)):
                view(buf, count, kind).mul_(4)
        return 0

    lsq.set_reduce_hook(times4)
    try:
        x1, info1 = lsq.solve(A, b, method=method, opts=opts)
        x1 = to_np(x1)
    finally:
        lsq.set_reduce_hook(None)
    assert int(to_np(info1)[0]) == int(to_np(info0)[0]) == 0
    d = np.linalg.norm(x1 - x0) / np.linalg.norm(x0)
    assert d <= 1e-14, d
    m, n = pr.A.shape
    # column maxima, sketch (the estimate's first, FP32 sparse sign with
    # s = 2n), then A_p^T A_p, A_p^T b and one refinement's A_p^T r
    want = []
    if prec == lsq.AUTO_SKETCH:
        want += [(lsq.REDUCE_MAX_U64, n), (lsq.REDUCE_SUM_F32, 2 * n * n)]
    if prec == lsq.AUTO:
        want += [(lsq.REDUCE_SUM_F32, n * n)]
    # kappa = 1e5: the estimate on a sketch picks FP32, the one on A^T A breaks
    # down and picks FP64
    sk = lsq.REDUCE_SUM_F64 if prec in (lsq.FP64, lsq.AUTO) else lsq.REDUCE_SUM_F32
    want += [(lsq.REDUCE_MAX_U64, n), (sk, 360 * n), (lsq.REDUCE_SUM_F64, n * n), (lsq.REDUCE_SUM_F64, n),
             (lsq.REDUCE_SUM_F64, n)]
    assert calls == want, calls


@pytest.mark.parametrize("kind,prec,kap", [(lsq.SPARSE_SIGN, lsq.BF16, 1e2), (lsq.GAUSSIAN, lsq.FP32, 1e5),
                                           (lsq.GAUSSIAN, lsq.FP64, 1e8), (lsq.SPARSE_SIGN, lsq.AUTO_SKETCH, 1e5)])
def test_two_shards_from_two_threads(kind, prec, kap):
    m, n, m0 = 6000, 150, 2600
    pr = P.make_problem(m, n, kap, 1e-6, 92)
    qr = lsq.FP64 if prec == lsq.FP64 else lsq.FP32
    kw = dict(kind=kind, s=450, zeta=8, seed=11, sketch_prec=prec, qr_prec=qr, refine_steps=1)
    x_full, info = lsq.solve(dev_colmajor(pr.A), torch.from_numpy(pr.b).cuda(), opts=lsq.make_opts(**kw))
    assert int(to_np(info)[0]) == 0
    x_full = to_np(x_full)
    shards = [(0, m0), (m0, m)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    barrier = threading.Barrier(2, timeout=60)
    parts, total, errs = [None, None], [None], []

    def hook(buf, count, kind_, stream):
        try:
            k = 0 if stream == streams[0].cuda_stream else 1
            s = stream_of(stream)
            v = view(buf, count, kind_)
            parts[k] = v
            s.synchronize()  # this shard's partial is in place
            if barrier.wait() == 0:
                # one sum, in one order, for both shards
                with torch.cuda.stream(s):
                    total[0] = torch.maximum(parts[0], parts[1]) if kind_ == lsq.REDUCE_MAX_U64 \
                        else parts[0] + parts[1]
                s.synchronize()
            barrier.wait()  # both partials read
            with torch.cuda.stream(s):
                v.copy_(total[0])
            barrier.wait()  # both copies queued before the total is dropped
            return 0
        except BaseException as e:  # surfaces as the solve's error
            errs.append(e)
            barrier.abort()
            return 1

    xs = [None, None]

    def run(k):
        try:
            r0, r1 = shards[k]
            with torch.cuda.stream(streams[k]):
                A = dev_colmajor(np.asfortranarray(pr.A[r0:r1]))
                b = torch.from_numpy(np.ascontiguousarray(pr.b[r0:r1])).cuda()
                x, inf = lsq.solve(A, b, opts=lsq.make_opts(row_offset=r0, **kw))
                streams[k].synchronize()
                assert int(to_np(inf)[0]) == 0
                xs[k] = to_np(x)
        except BaseException as e:  # reported by the main thread
            errs.append(e)
            barrier.abort()

    lsq.set_reduce_hook(hook)
    try:
        th = [threading.Thread(target=run, args=(k,)) for k in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join(180)
        assert not any(t.is_alive() for t in th)
    finally:
        lsq.set_reduce_hook(None)
    assert not errs, errs
    # both shards end with the same (replicated) solution, the unsharded one
    # up to the order of the sums over rows
    np.testing.assert_array_equal(xs[0], xs[1])
    d = np.linalg.norm(xs[0] - x_full) / np.linalg.norm(x_full)
    assert d <= 1e-8, d
    e_s, e_f = P.rel_error(xs[0], pr.x_star), P.rel_error(x_full, pr.x_star)
    assert e_s <= 4 * e_f + 1e-15, (e_s, e_f)
