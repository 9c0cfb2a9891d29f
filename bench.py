#!/usr/bin/env python3
"""Benchmark of the block COCR (bl_cocr_rq, Algorithm 3) solve on one or more GB300s.

One step = one complete solve of the 3D 7-point Helmholtz problem on a 64^3 grid
(n = 262,144, k = 20, quadratic absorbing border, p = 16 plane-wave right-hand sides)
from X0 = 0 to ||xi_m||_F/||B||_F <= 1e-10, FP64 complex arithmetic, through the C ABI
(setup residual + QR, all iterations, final true residual).  Metric: right-hand-side
columns solved per second.  Inputs are resident in HBM; the working set (A 37 MB plus
six 67 MB blocks) exceeds the 129 MB L2, so no flush is needed between steps.

``--impl reference`` times the CPU oracle (oracle/blcoc_oracle.py) on the host cores on a
bounded sample of the same workload (a few iterations per step), extrapolated to the
oracle's own iteration count for this problem.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own copy (independent replicas; no collective in
the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "helmholtz3d_64cube_k20_p16_planewaves"
METRIC = "RHS-columns solved/sec to relres 1e-10"
UNIT = "RHS-columns/s"
TOL = 1e-10
MAXIT = 20000
# FP64 peak of a GB300: 2 DFMA per clock per SM (nominal 1.25 TFLOP/s; a DFMA probe
# on this pool measured 1.20 TFLOP/s at about 2.0 GHz) x 152 SMs x 2070 MHz max clock.
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12
# Iterations the CPU oracle takes on this workload to 1e-10: the full oracle solve stored
# by tests/golden/make_golden.py --full3d (bl_cocr_rq; 598 iterations).
GOLDEN_FULL = os.path.join(ROOT, "tests", "golden", "helmholtz3d_n262144_p16.json")


def oracle_iters_to_tol(method):
    if method != "cocr_rq":
        raise SystemExit("--impl reference: the oracle's iteration count is stored for bl_cocr_rq only")
    with open(GOLDEN_FULL) as f:
        return int(json.load(f)["iters"])


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--method", choices=["cocr_rq", "cocg_rq"], default="cocr_rq")
    ap.add_argument("--cpu-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--ncu-case", type=int, default=0, metavar="ITERS",
                    help="profiler case: one solve of the same workload for exactly ITERS iterations, then exit")
    ap.add_argument("--option", action="append", default=[], metavar="KEY=VALUE",
                    help="solver option for the profiler case (blcoc_set_option), e.g. fp64_tc=1")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time (every rank gets it); `dist` is torch.distributed or None."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, columns_per_rank, ms):
    """RHS-columns per second of the whole job: every rank solves its own replica, all of
    them within the slowest rank's time."""
    return world * columns_per_rank / (ms / 1e3)


def problem(method):
    from paper_1601_05362_gb300 import problems as P
    return P.helmholtz3d_n262144_p16(method, maxit=MAXIT)


def kernel_width(p):
    return next(w for w in (1, 2, 4, 8, 16, 32) if p <= w)


def fp64_ops(pr):
    """Per-iteration FP64 operations of bl_cocr_rq per row-pass kernel, as (FMAs, adds),
    counted from the arithmetic the kernels evaluate.  Kernel widths from 8 up take three
    real products per complex MAC (Gauss) in the p x p applies and in the self-Grams U^T U
    and W^H W, plus one add per row, k and 8-column sweep (re + im of the input) and two per
    output column (the shared term into both parts; the Gram's companion tile likewise);
    the SpMM's gather and its W^T Y Gram take four products.  Narrower kernels take four
    products everywhere."""
    n, p, nnz = pr.n, pr.p, pr.A.nnz
    tri = p * (p + 1) // 2
    sweeps = range(0, p, 8)
    if kernel_width(p) >= 8:
        full = (3 * p * p, len(sweeps) * p + 2 * p)
        tri_apply = (3 * tri, sum(j0 + min(8, p - j0) for j0 in sweeps) + 2 * p)
        self_gram = (3 * tri, 2 * p)
    else:
        full, tri_apply, self_gram = (4 * p * p, 0), (4 * tri, 0), (4 * tri, 0)
    gram4 = (4 * tri, 0)

    def rows(*parts):
        return [n * sum(x[0] for x in parts), n * sum(x[1] for x in parts)]

    ops = {"cocr_passA": rows(full, self_gram), "spmm_gram": rows(tri_apply, gram4),
           "cocr_passC": rows(tri_apply, full, full, full, self_gram)}
    ops["spmm_gram"][0] += 4 * nnz * p
    return {k: tuple(v) for k, v in ops.items()}


def algorithmic(pr):
    """Per-iteration FP64 flops (FMA = 2, add = 1; from fp64_ops) and HBM bytes of
    bl_cocr_rq (A read once, 14 block passes of n*p*16 bytes: pass A reads Q, U and writes
    W; the SpMM reads W and writes V; pass C reads W, S, X, V, U and writes Q, X, S, U)."""
    n, p = pr.n, pr.p
    a_bytes = pr.A.nbytes(16)
    nps = n * p * 16
    bytes_ = {"cocr_passA": 3 * nps, "spmm_gram": a_bytes + 2 * nps, "cocr_passC": 9 * nps}
    flops = {k: 2.0 * f + a for k, (f, a) in fp64_ops(pr).items()}
    return flops, bytes_, a_bytes + 14 * nps, sum(flops.values())


# The sources that define the FP64 row-pass kernels the traffic figures belong to (the
# tensor-core header is compiled into the same unit but not into these kernels).
ROWPASS_SOURCES = ("blcoc_common.cuh", "blcoc_rowpass.cuh", "kset_p16.cu")


def code_of(text):
    """C/C++ source without comments and blank lines (what the compiler sees of the kernels)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1601_05362_gb300", "csrc")
    for fn in ROWPASS_SOURCES:
        with open(os.path.join(csrc, fn), encoding="utf-8") as f:
            h.update(fn.encode())
            h.update(code_of(f.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, only if it was
    taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch")


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
def cpu_sample(method, iters):
    """Time `iters` iterations of the oracle on this workload (runs in a subprocess)."""
    import numpy as np  # noqa: F401
    import oracle.blcoc_oracle as O
    pr = problem(method)
    A = pr.A.to_scipy()
    f = O.bl_cocr_rq if method == "cocr_rq" else O.bl_cocg_rq
    t0 = time.perf_counter()
    f(A, pr.B, tol=0.0, maxit=0)          # setup only
    t1 = time.perf_counter()
    f(A, pr.B, tol=0.0, maxit=iters)
    t2 = time.perf_counter()
    setup = t1 - t0
    per_iter = (t2 - t1 - setup) / iters
    print(json.dumps({"setup_s": setup, "per_iter_s": per_iter, "iters": iters}))


def run_cpu_sample(method, iters):
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(iters), "--method", method],
                         capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    d = json.loads(out.stdout.strip().splitlines()[-1])
    d["cores"] = cores
    return d


# ----------------------------------------------------------------------------- variants
def _timed_solves(h, B, X, method, tol, maxit, reps, stream):
    import torch
    ms, iters, trr = [], [], []
    for _ in range(reps):
        X.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = h.solve(B, X, method=method, tol=tol, maxit=maxit)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        info = h.info(hist_len=1)
        iters.append(info["iters"])
        trr.append(info["relres_true"])
    from paper_1601_05362_gb300 import blcoc
    return {"status": blcoc.status_string(st), "ms_per_solve": statistics.median(ms), "iters": iters[-1],
            "relres_true": trr[-1]}


def run_variants(h, B, X, pr, args, stream):
    """Same-run measurements next to the headline (not part of it), on the headline
    workload: Algorithm 3 with U_{m+1} = A S_{m+1} formed by a second sparse product, the
    p x p block updates on the bf16 tensor cores by exact integer slicing (option fp64_tc),
    and both together; and
    the mixed-precision refinement against plain FP64 on the 27-point random complex
    symmetric family (n = 262,144, p = 16), where complex64 inner solves converge."""
    import torch
    from paper_1601_05362_gb300 import blcoc, problems as P
    out = {}
    for name, opts in (("explicit_U", {"u_explicit": 1}), ("fp64_tc", {"fp64_tc": 1}),
                       ("fp64_tc_explicit_U", {"fp64_tc": 1, "u_explicit": 1})):
        for k, v in opts.items():
            h.set_option(k, v)
        _timed_solves(h, B, X, args.method, TOL, MAXIT, 1, stream)
        r = _timed_solves(h, B, X, args.method, TOL, MAXIT, 2, stream)
        for k in opts:
            h.set_option(k, 0)
        r["value"] = pr.p / (r["ms_per_solve"] / 1e3)
        r["unit"] = UNIT
        r["workload"] = WORKLOAD
        out[args.method + "_" + name] = r
    A2 = P.random_symmetric_27pt(64, 64, 64, seed=2)
    B2 = torch.from_numpy(P.complex_normal(A2.n, 16, 5)).cuda()
    X2 = torch.zeros_like(B2)
    with blcoc.Handle.from_csr(A2) as h2:
        for name, meth in (("fp64_cocr_rq", "cocr_rq"), ("mixed_cocr_rq", "cocr_rq_mixed")):
            _timed_solves(h2, B2, X2, meth, TOL, MAXIT, 1, stream)
            r = _timed_solves(h2, B2, X2, meth, TOL, MAXIT, 3, stream)
            if meth.endswith("mixed"):
                r["outer_iters"] = h2.stat("outer_iters")
            r["value"] = 16 / (r["ms_per_solve"] / 1e3)
            r["unit"] = UNIT
            r["workload"] = "random27pt_64cube_p16 (27-point pattern, 10% pairs dropped, diag 4+0.5i)"
            out[name + "_random27pt"] = r
    out["autograd_random27pt_n1048576_p8"] = run_autograd_variant(stream)
    out["cocr_rq_helmholtz3d_128cube_p32_fixed_iters"] = run_large_variant(args, stream)
    out["batched_helmholtz2d_64_systems"] = run_batched_variant(args)
    return out


def run_batched_variant(args):
    """64 independent 2D Helmholtz systems (grid side 64-512, k 5-30, damping 0.02-0.1,
    p in {1, 2, 4, 8, 16}; 5.87M rows in total), bl_cocr_rq to 1e-10: 64 separate solves,
    the CUDA-graph batch, the same batch with the tensor-core updates and explicit U per
    system, and the persistent kernel.  Host wall time around each call (each blocks
    until its batch is done)."""
    import torch
    from paper_1601_05362_gb300 import blcoc, problems as P
    probs = P.helmholtz2d_batch(64)
    hs = [blcoc.Handle.from_csr(pr.A) for pr in probs]
    Bs = [torch.from_numpy(pr.B).cuda() for pr in probs]
    out = {"systems": len(probs), "rows": int(sum(pr.n for pr in probs))}

    def run(label, fn, tc=0, ue=0):
        for h in hs:
            h.set_option("fp64_tc", tc)
            h.set_option("u_explicit", ue)
        Xs = [torch.zeros_like(B) for B in Bs]
        torch.cuda.synchronize()
        t = time.perf_counter()
        st = fn(Xs)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        info = [h.info(hist_len=1) for h in hs]
        out[label] = {"status": blcoc.status_string(st), "s": dt,
                      "system_iterations": int(sum(i["iters"] for i in info)),
                      "max_relres_true": max(i["relres_true"] for i in info)}

    def separate(Xs):
        return max(h.solve(B, X, method=args.method, tol=TOL, maxit=MAXIT) for h, B, X in zip(hs, Bs, Xs))

    def batched(persistent):
        def f(Xs):
            st, _, _ = blcoc.solve_batched(hs, Bs, Xs, method=args.method, tol=TOL, maxit=MAXIT, autotune=False,
                                           persistent=persistent)
            return st
        return f

    run("separate_fp64", separate)
    run("graph_fp64", batched(False))
    if args.method == "cocr_rq":
        run("graph_fp64_tc_explicit_U", batched(False), tc=1, ue=1)
    run("persistent_fp64", batched(True))
    for h in hs:
        h.close()
    return out


def run_large_variant(args, stream, iters=24, warm=4):
    """The n >= 2M case: 3D Helmholtz 128^3 (n = 2,097,152, k = 40), p = 32, FP64
    bl_cocr_rq.  A full solve takes minutes, so this times a fixed iteration count: the
    per-iteration time is (t(warm + iters) - t(warm)) / iters with CUDA events, against
    the algorithmic FP64 flops and HBM bytes of one iteration."""
    import torch
    from paper_1601_05362_gb300 import blcoc, problems as P
    pr = P.helmholtz3d_n2097152_p32(args.method)
    B = torch.from_numpy(pr.B).cuda()
    X = torch.zeros_like(B)
    ms = {}
    with blcoc.Handle.from_csr(pr.A) as h:
        for m in (warm, warm + iters, warm, warm + iters):
            X.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.solve(B, X, method=args.method, tol=0.0, maxit=m)
            e1.record(stream)
            torch.cuda.synchronize()
            ms[m] = e0.elapsed_time(e1)
        relres = h.info(hist_len=1)["relres"]
    t_iter = (ms[warm + iters] - ms[warm]) / iters / 1e3
    _, _, it_bytes, it_flops = algorithmic(pr)
    del B, X
    torch.cuda.empty_cache()
    return {"n": pr.n, "nnz": pr.A.nnz, "p": pr.p, "iters_timed": iters, "ms_per_iter": t_iter * 1e3,
            "alg_fp64_tflops": it_flops / t_iter / 1e12, "frac_of_fp64_peak": it_flops / t_iter / 1e12 / FP64_PEAK_TFLOPS,
            "alg_bytes_per_iter": it_bytes, "alg_hbm_gbs": it_bytes / t_iter / 1e9,
            "relres_after": relres}


def run_autograd_variant(stream):
    """Differentiable solve on the 27-point random family at n = 1,048,576 (128x128x64),
    p = 8, loss sum |C^T X|^2: forward solve, then forward + backward (adjoint solve +
    sampled outer product), both to 1e-10; CUDA-event times."""
    import torch
    from paper_1601_05362_gb300 import problems as P
    from paper_1601_05362_gb300.autograd import SymmetricCSR, blcoc_solve
    A = P.random_symmetric_27pt(128, 128, 64, seed=2)
    op = SymmetricCSR(A.row_ptr, A.col_idx, A.n, A.vals)
    B = torch.from_numpy(P.complex_normal(A.n, 8, 3)).cuda()
    Cm = torch.from_numpy(P.complex_normal(A.n, 8, 4)).cuda()
    vals0 = torch.from_numpy(A.vals).cuda()

    def once(backward):
        vals = vals0.clone().requires_grad_(backward)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        X = blcoc_solve(vals, B, op, tol=1e-10, maxit=5000)
        L = (Cm.transpose(0, 1) @ X).abs().pow(2).sum()
        if backward:
            L.backward()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), op.handle.info(hist_len=1)["iters"]

    once(True)
    fwd = [once(False) for _ in range(2)]
    both = [once(True) for _ in range(2)]
    op.close()
    return {"n": A.n, "nnz": A.nnz, "p": 8, "forward_ms": min(f[0] for f in fwd),
            "forward_backward_ms": min(b[0] for b in both), "forward_iters": fwd[-1][1],
            "adjoint_iters": both[-1][1]}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pr = problem(args.method)
    iters_to_tol = oracle_iters_to_tol(args.method)
    sample_iters = 4
    samples = []
    for i in range(args.warmup + args.steps):
        d = run_cpu_sample(args.method, sample_iters)
        if i >= args.warmup:
            samples.append(d)
    per_iter = statistics.median(s["per_iter_s"] for s in samples)
    setup = statistics.median(s["setup_s"] for s in samples)
    t_solve = setup + per_iter * iters_to_tol
    value = pr.p / t_solve
    cores = samples[0]["cores"]
    sample = (f"{sample_iters} iterations of the oracle's bl_cocr_rq per step on the same {pr.n}-row problem, "
              f"extrapolated to the oracle's {iters_to_tol} iterations to 1e-10")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": pr.n, "nnz": pr.A.nnz, "p": pr.p, "method": "bl_" + args.method,
                   "tol": TOL, "device": "host CPU"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1601_05362_gb300 import blcoc, build
    build.build()
    pr = problem(args.method)
    h = blcoc.Handle.from_csr(pr.A)
    B = torch.from_numpy(pr.B).cuda()
    X = torch.zeros_like(B)

    def solve_once():
        X.zero_()
        st = h.solve(B, X, method=args.method, tol=TOL, maxit=MAXIT)
        if st != blcoc.BLCOC_OK:
            raise RuntimeError(f"solve failed: {blcoc.status_string(st)} {h.last_error()}")

    for _ in range(args.warmup):
        solve_once()
    h.set_option("timing", 3)        # events around the dominant row pass only (the roofline's kernel)
    solve_once()                     # capture the timed graph once, outside the timed region
    kt = {}
    launches = 0
    iters = []
    stream = torch.cuda.current_stream()
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            solve_once()
            launches += h.stat("launches")
            iters.append(h.info()["iters"])
            for k in ("cocr_passA", "spmm_gram", "cocr_passC", "cocg_pass1", "cocg_pass2", "reduce",
                      "small_alpha", "small_chol", "small_beta"):
                ns, cnt = h.stat("kt_ns." + k), h.stat("kt_n." + k)
                if cnt:
                    a = kt.setdefault(k, [0, 0])
                    a[0] += ns
                    a[1] += cnt
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    info = h.info()
    ms_per_step = ms / args.steps
    value = whole_job_value(world, pr.p * args.steps, ms)

    # end to end through the C ABI with pinned host buffers
    h.set_option("timing", 0)
    Bh = torch.from_numpy(pr.B).pin_memory()
    Xh = torch.zeros_like(Bh).pin_memory()
    e2e_ms = []
    for i in range(3):
        Xh.zero_()
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        st = h.solve(Bh, Xh, method=args.method, tol=TOL, maxit=MAXIT)
        s1.record(stream)
        torch.cuda.synchronize()
        if st != blcoc.BLCOC_OK:
            raise RuntimeError("e2e solve failed")
        if i > 0:
            e2e_ms.append(s0.elapsed_time(s1))
    e2e_step = max_over_ranks(statistics.median(e2e_ms), dist, "cuda")
    nbytes = pr.n * pr.p * 16

    flops, bytes_, it_bytes, it_flops = algorithmic(pr)
    mean_iters = statistics.mean(iters)
    kern = {}
    for k, (ns, cnt) in kt.items():
        avg_s = ns / cnt / 1e9
        kern[k] = {"launches": cnt, "avg_ms": avg_s * 1e3, "share_of_kernel_time": None,
                   "tflops": flops.get(k, 0.0) / avg_s / 1e12 if k in flops else None,
                   "alg_gbs": bytes_.get(k, 0) / avg_s / 1e9 if k in bytes_ else None}
    total_ns = sum(v[0] for v in kt.values()) or 1
    for k, (ns, cnt) in kt.items():
        kern[k]["share_of_kernel_time"] = ns / total_ns
    dom = max(((k, v) for k, v in kt.items() if k in flops), key=lambda kv: kv[1][0])[0] if kt else None
    roof = None
    if dom:
        ach = kern[dom]["tflops"]
        traffic = ncu_traffic(dom)
        slots = sum(fp64_ops(pr)[dom])
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": f"k_{dom}<16>",
                "flops_per_launch": flops[dom], "alg_bytes_per_launch": bytes_[dom],
                "avg_launch_ms": kern[dom]["avg_ms"],
                "fp64_pipe_frac": slots / (kern[dom]["avg_ms"] / 1e3) / (FP64_PEAK_TFLOPS * 1e12 / 2),
                "peak_note": "FP64: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (derived; probe measured 1.20 TFLOP/s); "
                             "flops count an FMA as 2 and an add as 1, fp64_pipe_frac counts both as one "
                             "of the pipe's 2 operations per clock per SM"}
    t_iter = ms_per_step / mean_iters / 1e3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": pr.n, "nnz": pr.A.nnz, "p": pr.p, "method": "bl_" + args.method,
                   "tol": TOL, "iters": iters, "relres_true": info["relres_true"],
                   "l2": "working set 440 MB > 129 MB L2 (no flush)", "parallelism": f"replicas x{world}"},
        "per_iteration": {"ms": t_iter * 1e3, "alg_bytes": it_bytes, "alg_hbm_gbs": it_bytes / t_iter / 1e9,
                          "frac_of_8tbs": it_bytes / t_iter / 8e12, "alg_fp64_tflops": it_flops / t_iter / 1e12,
                          "frac_of_fp64_peak": it_flops / t_iter / 1e12 / FP64_PEAK_TFLOPS},
        "kernels": kern,
        "roofline": roof,
        "e2e": {"value": whole_job_value(world, pr.p, e2e_step), "unit": UNIT, "h2d_bytes_per_step": 2 * nbytes,
                "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_step},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if not args.no_variants:
        line["variants"] = run_variants(h, B, X, pr, args, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            d = run_cpu_sample(args.method, 4)
            t_cpu = d["setup_s"] + d["per_iter_s"] * mean_iters
            line["cpu_baseline"] = {
                "value": pr.p / t_cpu, "unit": UNIT, "cores": d["cores"], "kind": "oracle",
                "sample": (f"4 iterations of the oracle's bl_cocr_rq on the same {pr.n}-row problem "
                           f"({d['per_iter_s']:.3f} s/iteration, setup {d['setup_s']:.3f} s), extrapolated to "
                           f"this run's {mean_iters:.0f} iterations; scipy's sparse product is single-threaded, "
                           f"BLAS uses {d['cores']} threads")}
        except Exception as e:  # the GPU line still prints
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": f"failed: {e}"[:300]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


def run_ncu_case(args):
    """A short, fixed-length solve of the bench workload for ncu captures (no timing)."""
    import torch
    from paper_1601_05362_gb300 import blcoc, build
    build.build()
    pr = problem(args.method)
    h = blcoc.Handle.from_csr(pr.A)
    B = torch.from_numpy(pr.B).cuda()
    X = torch.zeros_like(B)
    for kv in args.option:
        key, val = kv.split("=", 1)
        h.set_option(key, int(val))
    st = h.solve(B, X, method=args.method, tol=0.0, maxit=args.ncu_case)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case_iters": args.ncu_case, "status": blcoc.status_string(st),
                      "launches": h.stat("launches")}))
    h.close()


def main():
    args = parse()
    if args.ncu_case:
        run_ncu_case(args)
        return
    if args.cpu_sample:
        cpu_sample(args.method, args.cpu_sample)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
