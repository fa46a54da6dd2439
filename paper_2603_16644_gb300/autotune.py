"""Autotuner for the batched solver: per shape bucket, the sketch kind and
size s in {2n, 4n} that solve fastest on this device while keeping the
preconditioner effective.

For each bucket (m and n rounded up to powers of two) a seeded synthetic
problem of the bucket's shape is solved with every candidate through the C
ABI; the timing is the median of CUDA-event measurements, and a candidate is
eligible only if its error against the known solution is within 2x of the
best candidate's.  Choices are cached in a JSON file keyed by device name,
bucket and sketch precision ($LSQ_AUTOTUNE_CACHE, default
~/.cache/lsq_autotune.json).
"""
import json
import math
import os

import torch

from . import FP32, FP64, GAUSSIAN, SPARSE_SIGN, OP_PNE, make_opts, solve, workspace_size

CANDIDATES = [(SPARSE_SIGN, 2), (SPARSE_SIGN, 4), (GAUSSIAN, 2), (GAUSSIAN, 4)]


def _cache_path():
    return os.environ.get("LSQ_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "lsq_autotune.json"))


def bucket(m, n):
    return (1 << max(0, math.ceil(math.log2(max(m, 1)))), 1 << max(0, math.ceil(math.log2(max(n, 1)))))


def _tuning_problem(m, n, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    G = torch.randn((n, m), generator=g, dtype=torch.float64, device="cuda").t()
    scale = torch.logspace(0, -6, n, dtype=torch.float64, device="cuda")
    A = torch.empty((n, m), dtype=torch.float64, device="cuda").t()
    A.copy_(G * scale)
    x_star = torch.randn(n, generator=g, dtype=torch.float64, device="cuda")
    b = A @ x_star
    return A, b, x_star


def _time(fn, reps=3):
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


class Autotuner:
    def __init__(self, path=None):
        self.path = path or _cache_path()
        self.table = {}
        try:
            with open(self.path) as f:
                self.table = json.load(f)
        except (OSError, ValueError):
            self.table = {}
        self.dev = torch.cuda.get_device_name()

    def _key(self, bm, bn, prec):
        return f"{self.dev}|{bm}x{bn}|p{prec}"

    def choose(self, m, n, prec=FP32, zeta=8, seed=2603):
        """(kind, s) for an m x n problem sketched in precision `prec`."""
        bm, bn = bucket(m, n)
        key = self._key(bm, bn, prec)
        if key not in self.table:
            self.table[key] = self._tune(min(bm, max(m, 4 * n)), min(bn, n) if bn > n else bn, prec, zeta, seed)
            self.save()
        kind, mult = self.table[key]["kind"], self.table[key]["mult"]
        s = min(mult * n, m)
        return kind, s

    def _tune(self, m, n, prec, zeta, seed):
        m = max(m, 4 * n)
        A, b, x_star = _tuning_problem(m, n, seed)
        results = []
        for kind, mult in CANDIDATES:
            s = min(mult * n, m)
            opts = make_opts(kind=kind, s=s, zeta=min(zeta, s), seed=seed, sketch_prec=prec,
                             qr_prec=FP64 if prec == FP64 else FP32, refine_steps=1)
            ws = torch.empty(workspace_size(OP_PNE, m, n, opts), dtype=torch.uint8, device="cuda")
            x = torch.empty(n, dtype=torch.float64, device="cuda")
            info = torch.zeros(1, dtype=torch.int32, device="cuda")
            solve(A, b, opts=opts, ws=ws, x=x, info=info)
            torch.cuda.synchronize()
            err = float(torch.linalg.vector_norm(x - x_star) / torch.linalg.vector_norm(x))
            ms = _time(lambda: solve(A, b, opts=opts, ws=ws, x=x, info=info))
            ok = int(info.item()) == 0 and math.isfinite(err)
            results.append({"kind": kind, "mult": mult, "ms": ms, "err": err, "ok": ok})
        best_err = min((r["err"] for r in results if r["ok"]), default=math.inf)
        eligible = [r for r in results if r["ok"] and r["err"] <= 2 * best_err + 1e-15] or results
        pick = min(eligible, key=lambda r: r["ms"])
        return {"kind": pick["kind"], "mult": pick["mult"], "candidates": results}

    def save(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            with open(self.path, "w") as f:
                json.dump(self.table, f, indent=1)
        except OSError:
            pass
