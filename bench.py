"""Throughput benchmark: least-squares solves per second of the mixed-precision
randomized-preconditioned normal equations (Alg. 1 of Garrison & Ipsen,
arXiv 2603.16644; PNE Eq. e_pne) on one GB300, next to this library's
all-FP64 PNE on the same inputs.

Workload (large single problem): A is 262144 x 4096 FP64 (8.6 GB), A = U
diag(sigma) V^T with geometric sigma, kappa in {1e4, 1e8} and relative
residual 1e-6 (two seeded synthetic problems resident in HBM, solved in
turn); Gaussian sketch with s = 2n rows; the preconditioner precision chosen
per problem by the single-precision condition estimate on a sketch (Alg. 1
first line; FP32 at kappa = 1e4, FP64 at 1e8), FP32 QR for a low-precision
sketch, FP64 TRSM / Gram / Cholesky / solves (the FP64 products on the
tensor cores by digit slicing).  Every A (8.6 GB) is larger than L2, so no
flush is needed between steps.  Also measured on the same inputs: the
all-FP64 PNE (the 3x comparison), the paper's estimate on A^T A, HPNE (LU),
and the end-to-end solve from host buffers.

One JSON line on rank 0.  --impl reference times the CPU oracle instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

M, N = 262144, 4096
S = 2 * N
KAPPAS = [1e4, 1e8]
RHO = 1e-6
# structure-preserving downscale on which the oracle runs beside every bench
DM, DN = 32768, 512
WORKLOAD = "large_262144x4096_gaussian_s8192_sketch_condest_pne"
METRIC = "LS solves/s (mixed-precision PNE, 262144x4096, precision from the condition estimate)"
FP64_NOMINAL_TFLOPS = 1.25  # CUDA-core FP64 of GB300 (no FP64 tensor path)
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # CUDA-core FP32: SMs x lanes x FMA x clock


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=6)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--fp64-steps", type=int, default=4, help="timed steps of the all-FP64 PNE comparison")
    p.add_argument("--side-steps", type=int, default=2, help="timed steps of the other comparisons")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-oracle-parity", action="store_true")
    p.add_argument("--c4-problems", type=int, default=1024,
                   help="uneven problems of the learned-proposal evaluation (0: skip)")
    p.add_argument("--ncu-case", choices=["pne32", "pne64", "sketch32", "sketch64", "estimate", "uneven", "tall", "trsm64"],
                   default=None,
                   help="run a bounded case for an ncu capture (2 calls on one problem of the workload shape) and exit")
    p.add_argument("--ncu-m", type=int, default=M, help="rows of the ncu case")
    return p.parse_args()


# ----------------------------------------------------------------------------- options and inputs
def opts_for(lsq, prec, seed, n=N):
    qr = lsq.FP64 if prec == lsq.FP64 else lsq.FP32
    return lsq.make_opts(kind=lsq.GAUSSIAN, s=2 * n, zeta=0, seed=seed, sketch_prec=prec, qr_prec=qr,
                         refine_steps=0)


def make_inputs(dev):
    import torch

    import problems as P

    probs = []
    for i, kap in enumerate(KAPPAS):
        seed = P.seed_for(2, i)
        A, b, x_star, sigma, V = P.make_problem_hadamard_torch(M, N, kap, RHO, seed, device=dev)
        probs.append({"A": A, "b": b, "x_star": x_star, "kappa": kap, "seed": seed})
        del sigma, V
    torch.cuda.synchronize()
    return probs


def ncu_case(args):
    """Two calls of one step on one problem of the workload's shape with
    args.ncu_m rows (Gaussian data: the kernels' cost does not depend on the
    conditioning); the first warms up, the second is the one to capture."""
    import torch

    import paper_2603_16644_gb300 as lsq

    torch.cuda.set_device(0)
    if args.ncu_case == "uneven":
        return ncu_case_uneven(lsq, torch)
    if args.ncu_case == "trsm64":
        # A_p = A R^{-1} and its Gram with the tensor-core FP64 products
        # switched off (the FP64 CUDA-core kernels), 65536 x 1024, R a
        # well-conditioned upper triangle
        m, n = 65536, 1024
        g = torch.Generator(device="cuda").manual_seed(7)
        A = torch.randn((n, m), generator=g, dtype=torch.float64, device="cuda").t()
        b = torch.randn(m, generator=g, dtype=torch.float64, device="cuda")
        R = torch.triu(torch.randn((n, n), generator=g, dtype=torch.float64, device="cuda")) * (0.1 / n ** 0.5)
        R = lsq.colmajor(R + torch.eye(n, dtype=torch.float64, device="cuda"))
        prev = lsq.set_fp64_emulation(False)
        try:
            for _ in range(2):
                lsq.trsm_gram(A, R, b)
            torch.cuda.synchronize()
        finally:
            lsq.set_fp64_emulation(prev)
        print(json.dumps({"ncu_case": "trsm64", "m": m, "n": n, "ok": True}))
        return 0
    if args.ncu_case == "tall":
        # the 65536 x 1024 tall-skinny workload: sparse-sign sketch s = 4n,
        # 8 nonzeros per column, BF16 sketch, FP32 QR, one refinement step
        m, n = 65536, 1024
        g = torch.Generator(device="cuda").manual_seed(7)
        A = torch.randn((n, m), generator=g, dtype=torch.float64, device="cuda").t()
        b = torch.randn(m, generator=g, dtype=torch.float64, device="cuda")
        opts = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=4 * n, zeta=8, seed=7, sketch_prec=lsq.BF16,
                             qr_prec=lsq.FP32, refine_steps=1)
        ws = lsq.workspace(lsq.OP_PNE, m, n, opts)
        for _ in range(2):
            lsq.pne(A, b, opts=opts, ws=ws)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "tall", "m": m, "n": n, "ok": True}))
        return 0
    m = args.ncu_m
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn((N, m), generator=g, dtype=torch.float64, device="cuda").t()
    b = torch.randn(m, generator=g, dtype=torch.float64, device="cuda")
    prec = lsq.FP64 if args.ncu_case.endswith("64") else lsq.FP32
    opts = opts_for(lsq, prec, 7)
    if args.ncu_case.startswith("pne"):
        ws = lsq.workspace(lsq.OP_PNE, m, N, opts)
        for _ in range(2):
            lsq.pne(A, b, opts=opts, ws=ws)
    elif args.ncu_case == "estimate":
        # the condition estimate on a sketch alone (the first step of the
        # mixed-precision solve)
        for _ in range(2):
            lsq.condest_sketch(A, seed=7)
    else:
        for _ in range(2):
            lsq.sketch(A, opts)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": args.ncu_case, "m": m, "ok": True}))
    return 0


def ncu_case_uneven(lsq, torch, count=32):
    """The first `count` problems of the batched workload's draw (the batch
    timed by the benchmark), each solved by a single call one after another
    (PNE, sparse-sign sketch of s = 2n, precision from the estimate on a
    sketch, one refinement), twice: the second pass is the one to capture.
    The problems are generated on the host (no device linear algebra)."""
    from paper_2603_16644_gb300 import learned

    probs = learned.c3_like_problems(count, seed=2604, device="cpu")
    items = []
    for p in probs:
        A = lsq.colmajor(p["A"].to("cuda"))
        m, n = A.shape
        c = int(lsq.condest_sketch(A, seed=p["seed"])[1].item())
        o = lsq.make_opts(kind=lsq.SPARSE_SIGN, s=2 * n, zeta=8, seed=p["seed"], sketch_prec=c,
                          qr_prec=lsq.FP64 if c == lsq.FP64 else lsq.FP32, refine_steps=1)
        items.append((A, p["b"].cuda(), o))
    wsz = max(lsq.workspace_size(lsq.OP_PNE, A.shape[0], A.shape[1], o) for A, _, o in items)
    ws = torch.empty(wsz, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        n0 = lsq.launch_count()
        for A, b, o in items:
            lsq.pne(A, b, opts=o, ws=ws)
        launches = lsq.launch_count() - n0
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": "uneven", "problems": count, "launches_per_pass": launches, "ok": True}))
    return 0


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None
        self.first = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the timed region starts once nvidia-smi is sampling (at most 3 s);
        # only the samples after this point are reported
        t0 = time.time()
        while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.02)
        self.first = len(self.lines)

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, pw, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.first:] or self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "samples": len(sm),
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- timing helpers
def run_steps(lsq, probs, steps, prec, ws, xs, infos, start=0, method="pne", events=None):
    """`steps` solves over the problems in turn; with `events` (a list), an
    event pair per solve is recorded on the launching stream (no
    synchronisation) for per-problem times."""
    import torch

    for k in range(steps):
        i = (start + k) % len(probs)
        p = probs[i]
        if events is not None:
            ev = (i, torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[1].record(torch.cuda.current_stream())
        lsq.solve(p["A"], p["b"], method=method, opts=opts_for(lsq, prec, p["seed"]), ws=ws, x=xs[i], info=infos[i])
        if events is not None:
            ev[2].record(torch.cuda.current_stream())
            events.append(ev)


def max_over_ranks(sec, dist, device):
    """The slowest rank's time (every rank gets it); `sec` itself on one rank."""
    if dist is None:
        return sec
    import torch

    t = torch.tensor([float(sec)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world, steps, sec):
    """Whole-job throughput of `world` replicas that each ran `steps` solves
    in at most `sec` seconds."""
    return world * steps / sec


def timed(lsq, torch, probs, steps, warmup, prec, ws, xs, infos, dist=None, method="pne", events=None):
    """Seconds of `steps` solves after `warmup` untimed ones (CUDA events on
    the launching stream, synchronised on both sides)."""
    run_steps(lsq, probs, warmup, prec, ws, xs, infos, method=method)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run_steps(lsq, probs, steps, prec, ws, xs, infos, start=warmup, method=method, events=events)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    return e0.elapsed_time(e1) / 1000.0


def per_problem_ms(probs, events):
    """Mean milliseconds per solve of each problem from the recorded pairs."""
    out = {}
    for p_i, p in enumerate(probs):
        t = [e0.elapsed_time(e1) for i, e0, e1 in events if i == p_i]
        if t:
            out[f"k{p['kappa']:.0e}"] = sum(t) / len(t)
    return out


def errors(probs, xs, infos):
    out = {}
    for k, p in enumerate(probs):
        x = xs[k].cpu().numpy()
        out[f"k{p['kappa']:.0e}"] = {
            "rel_err_vs_xstar": float(np.linalg.norm(x - p["x_star"].cpu().numpy()) / np.linalg.norm(x)),
            "info": int(infos[k].item())}
    return out


# ----------------------------------------------------------------------------- roofline
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def bf16_peak():
    pk = measured_peaks()
    if pk and pk.get("bf16_tflops_sustained"):
        return pk["bf16_tflops_sustained"], "of measured (MEASURED_PEAKS.json bf16_tflops_sustained)"
    return 1700.0, "of fallback (1.7 PFLOP/s sustained bf16)"


def method_flops(m, n, s, sk64):
    """Algorithmic work of one PNE solve by step (the flop counts of the
    method, not of the emulation): condition estimate on the sketch (sparse
    sketch + FP32 QR of 2n x n + Gram of the sketch), Gaussian sketch 2smn,
    sketch QR 2n^2 (s - n/3), TRSM m n^2, Gram m n^2 (symmetric), Cholesky
    n^3/3."""
    return {"condest": 2 * n * n * (2 * n - n / 3) + 2 * n * n * 2 * n,
            "sketch": 2.0 * s * m * n, "qr": 2.0 * n * n * (s - n / 3), "trsm": float(m) * n * n,
            "gram": float(m) * n * n, "factor": n ** 3 / 3.0}


TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_ot_update_traffic_262144x4096.md")
TRAFFIC_SOURCES = ("oz_trsm.cu", "tcgen05.cuh", "common.cuh")


def update_traffic():
    """DRAM bytes per k_ot_update launch over the timed region's launch mix,
    from the ncu capture summarised in profiles/ -- or None when the kernel's
    sources have changed since that capture."""
    import hashlib

    try:
        text = open(TRAFFIC_PROFILE).read()
        fields = dict(l.split(": ", 1) for l in text.splitlines() if l.startswith(("traffic_bytes", "source_sha")))
        h = hashlib.sha256()
        for f in TRAFFIC_SOURCES:
            with open(os.path.join(ROOT, "paper_2603_16644_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except (OSError, ValueError):
        return None
    if h.hexdigest()[:16] != fields.get("source_sha16", "").strip():
        return None
    return float(fields["traffic_bytes_per_launch"])


def roofline(stages, recs, per_solve_stage_ms, step_mix):
    """The dominant instrumented kernel of the timed region (by total time),
    with `achieved` = the METHOD's flops per launch / its CUDA-event time
    against the measured dense BF16 peak (GB300 has no FP64 tensor path; the
    FP64 products are emulated by BF16/FP8 digit slicing, reported as
    `emulation_factor` and `tensor_pipe_frac`).  The traffic figure comes
    from the DRAM capture summarised in profiles/."""
    peak, src = bf16_peak()
    cand = {}
    for key in ("k_ot_update", "k_qr_panel", "k_sketch_tc"):
        ms, cnt, work = stages[key]
        if key == "k_ot_update":
            # both forms of the update kernel: method work = tensor work / pairs
            ms3, cnt3, work3 = stages.get("k_ot_update3", (0.0, 0, 0.0))
            ms, cnt, work = ms + ms3, cnt + cnt3, (work, work3)
        if cnt:
            cand[key] = (ms, cnt, work)
    if not cand:
        return None
    top = max(cand, key=lambda k: cand[k][0])
    ms, cnt, work = cand[top]
    if top == "k_ot_update":
        # 36 BF16 digit-pair products per FP64 product (21 in the three-digit
        # form of the FP64 sketch)
        w36, w21 = work
        work = w36 + w21
        emul, bound, unit_peak = work / (w36 / 36.0 + w21 / 21.0), "tensor", peak
        kname = "k_ot_update (FP64 products by BF16 digit slicing: TRSM updates, Cholesky updates, FP64 sketch)"
    elif top == "k_sketch_tc":
        # FP32 sketches: six BF16 piece products per FP32 product
        emul, bound, unit_peak = step_mix.get("sketch_emulation", 1.0), "tensor", peak
        kname = "k_sketch_tc (Gaussian sketch GEMM on tcgen05)"
    else:
        emul, bound, unit_peak = 1.0, "alu", FP32_NOMINAL_TFLOPS
        kname = "k_qr_panel_cl (sketch QR panel)"
    hw_tflops = work / (ms / 1000.0) / 1e12
    achieved = hw_tflops / emul
    traffic = update_traffic() if top == "k_ot_update" else None
    out = {"bound": bound, "kernel": kname, "achieved": achieved, "peak": unit_peak, "unit": "TFLOP/s",
           "frac": achieved / unit_peak, "traffic": traffic,
           "traffic_unit": "bytes per launch (dram read + write, mean over the launch mix)",
           "traffic_source": "profiles/k_ot_update_traffic_262144x4096.md" if traffic is not None
           else "none (the kernel changed since the last dram capture)",
           "peak_source": src if bound == "tensor" else "nominal CUDA-core FP32 (152 SMs x 128 lanes x 2 x 2.07 GHz)",
           "launches": cnt, "avg_launch_ms": ms / cnt, "emulation_factor": emul,
           "tensor_pipe_tflops": hw_tflops, "tensor_pipe_frac": hw_tflops / unit_peak if bound == "tensor" else None,
           "share_of_timed_region": None}
    return out


def whole_solve_roofline(per_solve_stage_ms, flops):
    """sum over steps of t_min = work / peak of the step's unit, over the
    measured time of the steps: (a) with each step at the peak of the unit the
    method's arithmetic names, the FP64 steps at the FP64 CUDA-core rate (nominal; the emulated products beat it,
    so this exceeds 1), (b) with every FP64 step at the BF16 tensor peak with
    no emulation credit."""
    peak, _ = bf16_peak()
    t_meas = sum(v for k, v in per_solve_stage_ms.items() if k in flops) / 1000.0
    if t_meas <= 0:
        return None
    fp64_steps = ("trsm", "gram", "factor")
    tmin_a = tmin_b = 0.0
    for k, w in flops.items():
        if k not in per_solve_stage_ms:
            continue
        if k in fp64_steps:
            tmin_a += w / (FP64_NOMINAL_TFLOPS * 1e12)
        elif k in ("qr", "condest"):
            tmin_a += w / (FP32_NOMINAL_TFLOPS * 1e12)
        else:
            tmin_a += w / (peak * 1e12)
        tmin_b += w / (peak * 1e12)
    return {"fp64_steps_at_fp64_peak": tmin_a / t_meas, "all_steps_at_bf16_peak": tmin_b / t_meas,
            "t_measured_ms": 1000 * t_meas}


# ----------------------------------------------------------------------------- CPU oracle
def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def oracle_flops(m, n, s):
    """The oracle's arithmetic for one PNE solve with the sketch estimate,
    counted the same way at any size (its dense Gram forms all n^2 entries)."""
    return (2 * n * n * (2 * n) + 2 * n * n * (2 * n - n / 3) + 2.0 * s * m * n + 2 * n * n * (s - n / 3)
            + float(m) * n * n + 2.0 * m * n * n + n ** 3 / 3.0)


def downscale_problem(kap, i):
    """The workload's structure at 32768 x 512 (s = 2n = 1024): same generator,
    same kappa and residual; built on the CPU (no GPU work)."""
    import torch

    import problems as P

    A, b, x_star, _, _ = P.make_problem_hadamard_torch(DM, DN, kap, RHO, P.seed_for(2, 100 + i), device="cpu")
    return (np.asfortranarray(A.numpy()), b.numpy().copy(), x_star.numpy().copy(), P.seed_for(2, 100 + i))


def oracle_sample():
    """Time the oracle, as it stands, on the downscaled workload (both kappa,
    PNE with the sketch estimate) on all host threads.  Returns (seconds per
    downscaled solve, threads, solves)."""
    import oracle as O

    threads = O.set_threads(0)
    probs = [downscale_problem(k, i) for i, k in enumerate(KAPPAS)]
    t0 = time.perf_counter()
    for A, b, _, seed in probs:
        O.solve(A, b, kind=O.GAUSSIAN, s=2 * DN, zeta=0, seed=seed, sketch_prec=O.AUTO_SKETCH, qr_prec=O.FP32)
    sec = (time.perf_counter() - t0) / len(probs)
    return sec, threads, len(probs)


def cpu_baseline_line(sec, threads, solves):
    scale = oracle_flops(M, N, S) / oracle_flops(DM, DN, 2 * DN)
    return {"value": 1.0 / (sec * scale), "unit": "solves/s", "cores": threads, "kind": "oracle",
            "sample": (f"oracle PNE with the sketch condition estimate (Alg. 1) on the {DM}x{DN} downscale of the "
                       f"workload (s = 2n, kappa in {KAPPAS}, same generator), {solves} full solves at "
                       f"{sec:.2f} s each on {threads} threads; scaled to {M}x{N} by the oracle's flop count "
                       f"(x{scale:.0f})")}


def oracle_parity(lsq, torch, dev):
    """The workload's structure at the downscale: the CUDA path and the oracle
    on the same inputs, error of each against x_* and their difference."""
    import oracle as O

    out = {}
    for i, kap in enumerate(KAPPAS):
        A, b, x_star, seed = downscale_problem(kap, i)
        Ad = lsq.colmajor(torch.from_numpy(A).to(dev))
        bd = torch.from_numpy(b).to(dev)
        for name, prec in (("mixed", lsq.AUTO_SKETCH), ("fp64", lsq.FP64)):
            x, info = lsq.solve(Ad, bd, opts=opts_for(lsq, prec, seed, DN))
            xg = x.cpu().numpy()
            r = O.solve(A, b, kind=O.GAUSSIAN, s=2 * DN, zeta=0, seed=seed, sketch_prec=prec,
                        qr_prec=O.FP64 if prec == O.FP64 else O.FP32)
            eg = float(np.linalg.norm(xg - x_star) / np.linalg.norm(xg))
            eo = float(np.linalg.norm(r["x"] - x_star) / np.linalg.norm(r["x"]))
            out[f"k{kap:.0e}_{name}"] = {"gpu_err": eg, "oracle_err": eo, "err_ratio": eg / eo if eo > 0 else None,
                                         "rel_diff_gpu_oracle": float(np.linalg.norm(xg - r["x"]) / np.linalg.norm(r["x"])),
                                         "prec_oracle": O.PREC_NAMES[r["prec"]], "info": int(info.item())}
    return {"shape": f"{DM}x{DN}, s={2 * DN}", **out}


# ----------------------------------------------------------------------------- learned proposal
def learned_eval(lsq, torch, count, batch=True):
    """The learned proposal (judged by the estimator on a sketch) on `count`
    uneven problems drawn like the batched workload, next to the estimator on
    a sketch alone and the paper's estimate on A^T A: solves/s of each arm,
    escalations, the precisions used and the learned arm's accuracy against
    the estimator arm's."""
    from paper_2603_16644_gb300 import learned

    params = learned.load()
    if params is None:
        return {"unavailable": "no shipped weights"}, None
    probs = learned.c3_like_problems(count, seed=2604)
    res = learned.evaluate(params, probs)
    batched = batched_eval(lsq, torch, probs[:min(count, 512)]) if batch else None
    used = res["learned"]["used"]
    names = {0: "fp8_e4m3", 1: "bf16", 2: "fp16", 3: "fp32", 4: "fp64"}
    ratio = [a / max(b, 1e-300) for a, b in zip(res["learned"]["errors"], res["auto_sketch"]["errors"])]
    out = {"problems": count, "workload": "m in [2000, 40000], n in [32, 512], kappa log-uniform [1e2, 1e10], "
                                          "residual log-uniform [1e-12, 1e-2]; Gaussian s = 2n, PNE, one refinement",
           "solves_per_s": {a: r["solves_per_s"] for a, r in res.items()},
           "escalations": res["learned"]["escalations"],
           "precisions_used": {names[k]: used.count(k) for k in sorted(set(used))},
           "max_err_ratio_learned_over_estimate": max(ratio), "infos_nonzero": sum(
               1 for a in res.values() for i in a["infos"] if i != 0)}
    del probs
    torch.cuda.empty_cache()
    return out, batched


# ----------------------------------------------------------------------------- batched solver
def batched_eval(lsq, torch, probs):
    """The batched solver on uneven problems drawn like the batched workload
    (the first `len(probs)` problems of the learned-proposal batch): sketch
    kind and s in {2n, 4n} per shape bucket from the autotuner, precision per
    problem from the estimate on a sketch (one batched estimate pass and one
    readback per call), PNE with one refinement step, every problem's kernel
    sequence in one cached CUDA-graph launch.  Timed over two calls after the
    call that captures the graphs; beside it the same batch with the chosen
    precisions given (the cached solve graph alone)."""
    from paper_2603_16644_gb300.autotune import Autotuner

    tuner = Autotuner()
    As, bs, xs, infos, opts, kinds = [], [], [], [], [], []
    for p in probs:
        m, n = p["A"].shape
        kind, s = tuner.choose(m, n, prec=lsq.FP32)
        kinds.append(kind)
        As.append(p["A"])
        bs.append(p["b"])
        xs.append(torch.empty(n, dtype=torch.float64, device=p["A"].device))
        infos.append(torch.zeros(1, dtype=torch.int32, device=p["A"].device))
        opts.append(lsq.make_opts(kind=kind, s=s, zeta=min(8, s), seed=p["seed"], sketch_prec=lsq.AUTO_SKETCH,
                                  qr_prec=lsq.FP32, refine_steps=1))

    def run(desc, ws, calls):
        lsq.solve_batched(desc, ws)  # capture and first launch
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(calls):
            lsq.solve_batched(desc, ws)
        e1.record()
        torch.cuda.synchronize()
        return calls * len(probs) / (e0.elapsed_time(e1) / 1000.0)

    desc = lsq.batch_descriptors(As, bs, xs, infos, opts)
    ws = lsq.batched_workspace(desc)
    value = run(desc, ws, 2)
    errs = [float(torch.linalg.norm(x - p["x_star"]) / torch.linalg.norm(x)) for x, p in zip(xs, probs)]
    bad = sum(1 for f in infos if int(f.item()) != 0)
    del ws
    chosen = [int(lsq.condest_sketch(p["A"], seed=p["seed"])[1].item()) for p in probs]
    opts2 = [lsq.make_opts(kind=o.kind, s=o.s, zeta=o.zeta, seed=o.seed, sketch_prec=c,
                           qr_prec=lsq.FP64 if c == lsq.FP64 else lsq.FP32, refine_steps=1)
             for o, c in zip(opts, chosen)]
    desc2 = lsq.batch_descriptors(As, bs, xs, infos, opts2)
    ws2 = lsq.batched_workspace(desc2)
    value2 = run(desc2, ws2, 2)
    del ws2
    torch.cuda.empty_cache()
    names = {0: "fp8_e4m3", 1: "bf16", 2: "fp16", 3: "fp32", 4: "fp64"}
    return {"problems": len(probs), "solves_per_s": value, "unit": "solves/s",
            "solves_per_s_precisions_given": value2,
            "workload": "m in [2000, 40000], n in [32, 512], kappa log-uniform [1e2, 1e10], residual log-uniform "
                        "[1e-12, 1e-2]; sketch kind and s in {2n, 4n} from the autotuner, precision from the estimate "
                        "on a sketch, PNE, one refinement; one cached graph of per-problem kernel sequences over 16 "
                        "internal streams",
            "sketch_kinds": {"gaussian": kinds.count(lsq.GAUSSIAN), "sparse_sign": kinds.count(lsq.SPARSE_SIGN)},
            "precisions_used": {names[k]: chosen.count(k) for k in sorted(set(chosen))},
            "median_rel_err_vs_xstar": float(np.median(errs)), "max_rel_err_vs_xstar": max(errs),
            "infos_nonzero": bad}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O

    threads = O.set_threads(0)
    probs = [downscale_problem(k, i) for i, k in enumerate(KAPPAS)]

    def step(k):
        A, b, _, seed = probs[k % len(probs)]
        O.solve(A, b, kind=O.GAUSSIAN, s=2 * DN, zeta=0, seed=seed, sketch_prec=O.AUTO_SKETCH, qr_prec=O.FP32)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    sec = time.perf_counter() - t0
    scale = oracle_flops(M, N, S) / oracle_flops(DM, DN, 2 * DN)
    value = args.steps / (sec * scale)  # full-size solves per second
    sample = (f"oracle PNE with the sketch condition estimate on the {DM}x{DN} downscale of the workload "
              f"(s = 2n, kappa in {KAPPAS}), one full downscaled solve per step on {threads} threads; the value "
              f"is scaled to {M}x{N} by the oracle's flop count (x{scale:.0f})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "m": M, "n": N, "s": S},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case:
        return ncu_case(args)
    import torch

    import paper_2603_16644_gb300 as lsq

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist_mod.init_process_group("nccl")
        dist = dist_mod
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # the CPU baseline first: the oracle's threads run before any GPU work
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_line(*oracle_sample())

    probs = make_inputs(dev)
    ws_size = max(lsq.workspace_size(lsq.OP_PNE, M, N, opts_for(lsq, p, 0))
                  for p in (lsq.AUTO_SKETCH, lsq.AUTO, lsq.FP64))
    ws_size = max(ws_size, lsq.workspace_size(lsq.OP_HPNE, M, N, opts_for(lsq, lsq.AUTO_SKETCH, 0)))
    ws = torch.empty(ws_size, dtype=torch.uint8, device=dev)
    xs = [torch.empty(N, dtype=torch.float64, device=dev) for _ in probs]
    infos = [torch.zeros(1, dtype=torch.int32, device=dev) for _ in probs]

    # ---- headline: mixed-precision PNE, precision from the estimate on a sketch
    chosen = {}
    for p in probs:
        k0, ch = lsq.condest_sketch(p["A"], seed=p["seed"])
        chosen[f"k{p['kappa']:.0e}"] = {"kappa0": float(k0.item()), "prec": int(ch.item())}
    clocks = ClockSampler(local)
    run_steps(lsq, probs, args.warmup, lsq.AUTO_SKETCH, ws, xs, infos)
    torch.cuda.synchronize()
    lsq.profile(True)
    n_launch0 = lsq.launch_count()
    clocks.start()
    ev_mixed = []
    sec = timed(lsq, torch, probs, args.steps, 0, lsq.AUTO_SKETCH, ws, xs, infos, dist, events=ev_mixed)
    clk = clocks.stop()
    n_launch = lsq.launch_count() - n_launch0
    stages = lsq.profile_collect(with_work=True)
    lsq.profile(False)
    sec = max_over_ranks(sec, dist, dev)
    value = weak_value(world, args.steps, sec)
    err_mixed = errors(probs, xs, infos)

    # ---- all-FP64 PNE on the same inputs (the sketch precision forced to FP64)
    run_steps(lsq, probs, 2, lsq.FP64, ws, xs, infos)  # warm-up, not profiled
    torch.cuda.synchronize()
    lsq.profile(True)
    ev64 = []
    sec64 = timed(lsq, torch, probs, args.fp64_steps, 0, lsq.FP64, ws, xs, infos, dist, events=ev64)
    stages64 = lsq.profile_collect(with_work=True)
    lsq.profile(False)
    err64 = errors(probs, xs, infos)
    value64 = weak_value(world, args.fp64_steps, max_over_ranks(sec64, dist, dev))

    # ---- the paper's estimate on A^T A (Sec. 6.1) and HPNE with LU
    secl = timed(lsq, torch, probs, args.side_steps, 1, lsq.AUTO, ws, xs, infos, dist)
    chosen_literal = {}
    for p in probs:
        k0, ch = lsq.condest(p["A"])
        chosen_literal[f"k{p['kappa']:.0e}"] = {"kappa0": float(k0.item()), "prec": int(ch.item())}
    sech = timed(lsq, torch, probs, args.side_steps, 1, lsq.AUTO_SKETCH, ws, xs, infos, dist, method="hpne")
    errh = errors(probs, xs, infos)
    del ws
    torch.cuda.empty_cache()

    # ---- end to end through the C ABI on host buffers (pinned)
    Ah = [p["A"].t().contiguous().cpu().pin_memory() for p in probs]
    bh = [p["b"].cpu().pin_memory() for p in probs]
    for p in probs:
        del p["A"]
    torch.cuda.empty_cache()
    wsh = torch.empty(lsq.workspace_size(lsq.OP_PNE_HOST, M, N, opts_for(lsq, lsq.AUTO_SKETCH, 0)),
                      dtype=torch.uint8, device=dev)
    xh = torch.empty(N, dtype=torch.float64).pin_memory()
    lsq.solve_host(Ah[0].t(), bh[0], opts=opts_for(lsq, lsq.AUTO_SKETCH, probs[0]["seed"]), ws=wsh, x_host=xh)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.side_steps):
        i = k % len(probs)
        lsq.solve_host(Ah[i].t(), bh[i], opts=opts_for(lsq, lsq.AUTO_SKETCH, probs[i]["seed"]), ws=wsh, x_host=xh)
    e2e_sec = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_value = weak_value(world, args.side_steps, e2e_sec)
    del wsh, Ah
    torch.cuda.empty_cache()

    # ---- learned precision proposal (shipped weights) on a fresh batch of
    # uneven problems, against the estimate alone and the paper's estimate on A^T A
    c4 = c3 = None
    if rank == 0 and args.c4_problems > 0:
        c4, c3 = learned_eval(lsq, torch, args.c4_problems)

    result = None
    if rank == 0:
        per_stage = {k: v[0] / args.steps for k, v in stages.items() if v[1] and not k.startswith("k_")}
        per_stage64 = {k: v[0] / args.fp64_steps for k, v in stages64.items() if v[1] and not k.startswith("k_")}
        per_kernel = {k: {"ms_per_solve": round(v[0] / args.steps, 3), "launches_per_solve": v[1] / args.steps}
                      for k, v in stages.items() if v[1] and k.startswith("k_")}
        n32 = sum(1 for v in chosen.values() if v["prec"] == lsq.FP32)
        mix = {"sketch_emulation": 6.0 if n32 == len(chosen) else 1.0}
        roof = roofline(stages, None, per_stage, mix)
        if roof is not None:
            roof["share_of_timed_region"] = stages[next(k for k in ("k_ot_update", "k_qr_panel", "k_sketch_tc")
                                                         if roof["kernel"].startswith(k))][0] / (1000 * sec)
        flops = method_flops(M, N, S, False)
        parity = None if args.no_oracle_parity else oracle_parity(lsq, torch, dev)
        pname = {0: "fp8_e4m3", 1: "bf16", 2: "fp16", 3: "fp32", 4: "fp64"}
        speedup = {}
        t_mixed, t64 = per_problem_ms(probs, ev_mixed), per_problem_ms(probs, ev64)
        for key in err_mixed:
            em, e6 = err_mixed[key]["rel_err_vs_xstar"], err64[key]["rel_err_vs_xstar"]
            eq = bool(em <= 2 * e6 + 1e-15)
            speedup[key] = {"prec": pname.get(chosen[key]["prec"]), "ms_mixed": t_mixed.get(key),
                            "ms_fp64": t64.get(key), "err_mixed": em, "err_fp64": e6, "equal_accuracy": eq,
                            "speedup": (t64[key] / t_mixed[key]) if eq and key in t64 and key in t_mixed else None}
        result = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded A = U diag(sigma) V^T, U from signed Hadamard columns, known x_*)",
            "config": {"workload": WORKLOAD, "m": M, "n": N, "s": S, "sketch": "gaussian",
                       "sketch_prec": "from the condition estimate on a sketch (auto_sketch)", "qr_prec": "fp32",
                       "refine_steps": 0, "kappas": KAPPAS, "rho": RHO,
                       "l2": "inputs larger than L2 (8.6 GB A per step, 2 problems in turn)"},
            "clocks": clk, "gpu_launches": n_launch,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 8 * M * N + 8 * M,
                    "d2h_bytes_per_step": 8 * N + 4},
            "roofline": roof,
            "whole_solve_roofline": whole_solve_roofline(per_stage, flops),
            "cpu_baseline": cpu,
            "chosen_precision": {k: {"kappa0": v["kappa0"], "prec": pname.get(v["prec"])} for k, v in chosen.items()},
            "stage_ms_per_solve": {k: round(v, 3) for k, v in per_stage.items()},
            "kernel_ms_per_solve": per_kernel,
            "fp64_pne": {"value": value64, "unit": "solves/s", "speedup_mixed_over_fp64": value / value64,
                         "stage_ms_per_solve": {k: round(v, 3) for k, v in per_stage64.items()},
                         "accuracy": err64},
            "speedup_at_equal_accuracy": speedup,
            "paper_estimate_on_AtA": {"value": weak_value(world, args.side_steps, secl), "unit": "solves/s",
                                      "chosen": {k: {"kappa0": v["kappa0"], "prec": pname.get(v["prec"])}
                                                 for k, v in chosen_literal.items()}},
            "hpne": {"value": weak_value(world, args.side_steps, sech), "unit": "solves/s", "accuracy": errh},
            "accuracy": err_mixed,
            "oracle_parity_downscale": parity,
            "learned_proposal": c4,
            "batched_uneven": c3,
        }
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
