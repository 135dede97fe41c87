"""Throughput benchmark of the FFT/tridiagonal Poisson solve (one JSON line on rank 0).

Default workload (N=1): a 1024^3 cell-centred grid, Neumann x / Dirichlet y / Neumann z,
f i.i.d. U[-1,1] (seeded) with the mean removed, FP64 in/out.  One step = one full solve
(x-forward, y-forward, z tridiagonal, y-inverse, x-inverse), timed with CUDA events on the
launching stream; inputs (8 GiB) exceed the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--n 1024] [--impl ours|reference]

--impl reference times the CPU oracle (naive O(N^2) transforms + Thomas, OpenMP on the host
cores) on a bounded slab of the same workload.  Under torchrun (N>1) every rank solves its own
grid (independent replicas, no collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpoints/s per Poisson solve at 1024^3, FP64 vs mixed; % of HBM roofline"
UNIT = "Gpoints/s"
BC = "NNDDNN"
SEED = 2
STAGES = ["x-forward", "y-forward", "z-solve", "y-inverse", "x-inverse"]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def replica_aggregate(ms_local: float, points_local: int, dist=None, device="cpu"):
    """Whole-job figures of independent replicas: the slowest rank's time per step (max over
    ranks) and the total points of all ranks per that time (Gpoints/s).  No data is exchanged,
    only these two scalars."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms_local, points_local / (ms_local * 1e-3) / 1e9
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(points_local)], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    ms = t.item()
    return ms, p.item() / (ms * 1e-3) / 1e9


# device-code sources of the solve pipeline's kernels (host-side plan code, and the refinement and
# face kernels of pp_misc.cu, which the profiled FP64 solve does not launch, are not part of the hash)
KERNEL_SOURCES = ("pp_arith.cuh", "pp_fft.cuh", "pp_internal.h", "pp_lines.cuh", "pp_lines.cu", "pp_lines_df_tiny.cu",
                  "pp_lines_f32_tiny.cu", "pp_lines_df_small.cu",
                  "pp_lines_df_large.cu", "pp_lines_df_any.cu", "pp_lines_df_any57.cu", "pp_lines_f32_small.cu",
                  "pp_lines_f32_large.cu", "pp_lines_f32_any.cu", "pp_lines_f32_any57.cu", "pp_lines_df_ct3a.cu",
                  "pp_lines_df_ct3b.cu", "pp_lines_f32_ct3a.cu", "pp_lines_f32_ct3b.cu", "pp_zsolve.cu", "pp_zpart.cu",
                  "pp_zfft.cu", "pp_range.cuh", "pp_zmul.cuh")


def _code_only(text: str) -> str:
    """C/C++ source without comments and with whitespace runs collapsed (a comment edit leaves
    the kernels, and so the hash, unchanged)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def _source_hash():
    """Hash of the kernel sources' code (the traffic figures in profiles/ are valid only for these)."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1909_05423_gb300", "csrc", name), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def _traffic(stage: str, n: int):
    """DRAM bytes per launch of `stage` from the committed ncu summary, scaled to n^3, or None when
    the summary is missing, for another workload, or for kernels that have changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic_solve_f64.json")) as fh:
            d = json.load(fh)
    except Exception:
        return None
    if d.get("source_hash") != _source_hash() or d.get("bc") != BC:
        return None
    v = d.get("per_launch_bytes_at_1024", {}).get(stage)
    return None if v is None else v * (n / 1024.0) ** 3


# ---------------------------------------------------------------- ALU roofline of the line kernels
# FP32 operations of the algorithm, counted as issued FP32 lane instructions (an FMA is one):
# double-float in the unnormalised forms the line kernels use: add 8 (TwoSum 6, two lo adds),
# multiply 4 (FMUL, 3 FFMA), complex multiply 32 (two fused a*b -+ c*d of 16: two TwoProds 4,
# TwoSum 6, 6 adds and FMAs of the error terms), complex add 16, halving 2; FP32: add 1, multiply 1,
# complex multiply 4, complex add 2.  Peak: 152 SMs x 128 FP32 lanes x 2.07 GHz (maximum SM clock).
FP32_LANES = 152 * 128
SM_MAX_GHZ = 2.07
_OPS = {"df": {"add": 8, "mul": 4, "cmul": 32, "half": 2}, "f32": {"add": 1, "mul": 1, "cmul": 4, "half": 1}}


def fft_ops(M: int, arith: str) -> float:
    """FP32 operations of one complex FFT of power-of-two length M (radix 8, then 4 or 2; the last
    stage has no twiddles)."""
    o = _OPS[arith]
    cadd = 2 * o["add"]
    dft = {2: 2 * cadd, 4: 8 * cadd, 8: 2 * 8 * cadd + 4 * o["add"] + 4 * o["mul"] + 8 * cadd}
    rads, m = [], M
    while m > 1:
        r = 8 if m % 8 == 0 else (4 if m % 4 == 0 else 2)
        rads.append(r)
        m //= r
    ops = 0.0
    for i, r in enumerate(rads):
        last = i == len(rads) - 1
        ops += (M // r) * (dft[r] + (0 if last else (r - 1) * o["cmul"]))
    return ops


def line_ops_per_real(kind: str, N: int, arith: str) -> float:
    """FP32 operations per real point of one real line transform of length N (complex FFT of N/2
    points plus the pre/post-processing of the kind): DCT-II/DST-II (Hermitian-pair split and
    the quarter-wave twiddle), DCT-III/DST-III (the reverse), as implemented."""
    o = _OPS[arith]
    cadd, cmul, ch = 2 * o["add"], o["cmul"], 2 * o["half"]
    per_pair = {"dct2": (cadd + ch) + cadd + ch + cmul + 2 * cadd + 2 * cmul,
                "dct3": 2 * cmul + cadd + (cadd + cmul) + 4 * o["add"]}[kind]
    return fft_ops(N // 2, arith) / N + per_pair / 4.0


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, world


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        # the raw samples; BENCH_CLOCKS_DIR keeps them (default: the system temporary directory)
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir(),
                                 "bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.read().splitlines()
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_sample(n: int, nz_sample: int, seed: int):
    """Time the CPU oracle on an n x n x nz_sample slab of the workload; returns (seconds, points, threads).
    The per-point cost of the oracle's x/y transforms depends only on n, so the slab's rate is the
    rate of the full n^3 workload (the z part is O(nz) per mode in both)."""
    import numpy as np

    import oracle
    oracle.build()
    f = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(nz_sample, n, n))
    t0 = time.perf_counter()
    oracle.solve(f, BC, (1.0 / n, 1.0 / n, 1.0 / n))
    dt = time.perf_counter() - t0
    return dt, f.size, oracle.num_threads()


def run_reference(args):
    rank, world = _dist()
    if rank != 0:
        return 0
    n = args.n
    nzs = args.oracle_planes
    for _ in range(args.warmup):
        _oracle_sample(n, max(1, nzs // 4), SEED)
    times, pts, threads = [], 0, 1
    for _ in range(args.steps):
        dt, pts, threads = _oracle_sample(n, nzs, SEED)
        times.append(dt)
    tot = sum(times)
    value = pts * len(times) / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded U[-1,1])",
        "config": {"workload": "%d^3 FP64 Neumann-x/Dirichlet-y/Neumann-z, U[-1,1] source" % n,
                   "bc": BC, "n": n, "sample": "%dx%dx%d slab per step" % (n, n, nzs)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "oracle solve of a %dx%dx%d slab per step (naive O(N^2) transforms)" % (n, n, nzs)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _events_ms(fn, reps, warmup=2):
    import torch
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _config3(pp, workloads, args):
    """Mixed precision (FP32 transforms, double-float z) with and without one refinement step, and the
    FP64-class path, at 512^3 and 1024^3: all-periodic and all-Neumann manufactured cos/sin products
    (built on the device).  Errors against the exact discrete solution -- each product term is a
    discrete eigenvector, u = u* sum(k^2) / sum(lambda_d), with lambda_d = -4 sin^2(k h / 2) / h^2
    (the cancellation-free form) -- and rates.  The all-periodic case also times periodic z by
    transform (z_method 2) against Sherman-Morrison (z_method 1)."""
    import math

    import torch
    out = {}
    cases = {
        "PPPPPP": [(1.0, ("cos", 2 * math.pi), ("cos", 2 * math.pi), ("cos", 2 * math.pi)),
                   (0.5, ("sin", 4 * math.pi), ("sin", 2 * math.pi), ("cos", 6 * math.pi))],
        "NNNNNN": [(1.0, ("cos", math.pi), ("cos", 3 * math.pi), ("cos", 6 * math.pi)),
                   (0.5, ("cos", 2 * math.pi), ("cos", math.pi), ("cos", 2 * math.pi))],
    }
    tune = {} if args.no_autotune else {"autotune": 1}
    for n in args.n3:
        sp = (1.0 / n,) * 3
        h = 1.0 / n
        lam = lambda k: -4.0 * math.sin(0.5 * k * h) ** 2 / (h * h)
        for bc, terms in cases.items():
            ref = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
            ft = torch.zeros_like(ref)
            for amp, (fx, kx), (fy, ky), (fz, kz) in terms:
                t, ff = workloads.manufactured_device((n, n, n), sp, [(amp, (fx, kx), (fy, ky), (fz, kz))])
                ref += t * (-(kx * kx + ky * ky + kz * kz) / (lam(kx) + lam(ky) + lam(kz)))
                ft += ff
                del t, ff
            ref -= ref.mean()
            nrm = torch.linalg.vector_norm(ref).item()
            rel = lambda x: torch.linalg.vector_norm(x - ref).item() / nrm
            u = torch.empty_like(ft)
            res = {"n": n}
            zm = [1, 2] if bc[4] == "P" else [0]
            for z in zm:
                tag = "" if z != 2 else "_ztransform"
                opts = dict(tune, z_method=z)
                p64 = pp.Plan((n, n, n), bc, sp, "f64", options=opts)
                t64 = _events_ms(lambda: p64.solve(ft, u), args.steps)
                res["f64%s_ms" % tag] = t64
                res["f64%s_gpoints_s" % tag] = n ** 3 / t64 / 1e6
                res["rel_l2_f64%s" % tag] = rel(u)
                p64.close()
                pm = pp.Plan((n, n, n), bc, sp, "mixed_f64io", options=opts)
                tm = _events_ms(lambda: pm.solve(ft, u), args.steps)
                res["mixed%s_ms" % tag] = tm
                res["mixed%s_gpoints_s" % tag] = n ** 3 / tm / 1e6
                res["rel_l2_mixed%s" % tag] = rel(u)
                if z != 2:
                    tr = _events_ms(lambda: pm.solve_refined(ft, u), args.steps)
                    res["refined_ms"] = tr
                    res["refined_gpoints_s"] = n ** 3 / tr / 1e6
                    res["rel_l2_refined"] = rel(u)
                    res["mixed_speedup_vs_f64"] = t64 / tm
                pm.close()
            out["%s_%d" % (bc, n)] = res
            del ft, ref, u
            torch.cuda.empty_cache()
    return out


def _config2_256(pp, args):
    """The headline workload (Neumann-x / Dirichlet-y / Neumann-z, U[-1,1] source, mean removed) at
    256^3: grids of 128 MiB, about the size of L2, so the HBM fraction is not the target there."""
    import torch
    n = 256
    shape = (n, n, n)
    sp = (1.0 / n,) * 3
    g = torch.Generator(device="cuda")
    g.manual_seed(SEED)
    f = torch.empty(shape, dtype=torch.float64, device="cuda").uniform_(-1.0, 1.0, generator=g)
    f -= f.mean()
    u = torch.empty_like(f)
    tune = {} if args.no_autotune else {"autotune": 1}
    out = {"n": n}
    for dtype in ("f64", "mixed_f64io"):
        plan = pp.Plan(shape, BC, sp, dtype, options=tune)
        ms = _events_ms(lambda: plan.solve(f, u), max(args.steps, 20))
        out[dtype] = {"ms": ms, "gpoints_s": n ** 3 / ms / 1e6}
        plan.close()
    return out


def _zsolver_study(pp, args):
    """The paper's tridiagonal-solver comparison (Sec. "Comparison of Tridiagonal Solvers": 64 x 64
    modes, n_z = 255 .. 4095, one GPU): FP64 solves with the z lines solved by the Thomas sweeps and
    by the partitioned solve the autotuner picks (chunk rows 8 / 16 / 32), timed per solve and for
    the z stage alone (in place, on the plan's spectral buffer)."""
    import ctypes
    import torch
    from paper_1909_05423_gb300 import _lib
    lib = _lib.load()
    out = []
    for nz in (255, 511, 1023, 2047, 4095):
        shape = (nz, 64, 64)
        sp = (1.0 / 64, 1.0 / 64, 1.0 / nz)
        g = torch.Generator(device="cuda")
        g.manual_seed(SEED)
        f = torch.empty(shape, dtype=torch.float64, device="cuda").uniform_(-1.0, 1.0, generator=g)
        u = torch.empty_like(f)
        row = {"nz": nz}
        for name, opt in (("thomas", {"z_split": 1}), ("autotuned", {"autotune": 1})):
            plan = pp.Plan(shape, BC, sp, "f64", options=opt)
            ms = _events_ms(lambda: plan.solve(f, u), 20)
            plan.status()
            fp, up = ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr())
            zms = _events_ms(lambda: lib.pp_run_stage(plan._h, 2, fp, up, None), 20)
            try:
                plan.status()  # repeated in-place z solves of one buffer: the values are discarded
            except _lib.PPError:
                pass
            row[name] = {"solve_ms": ms, "z_ms": zms, "z_split": plan.z_split()}
            plan.close()
        row["solve_speedup"] = row["thomas"]["solve_ms"] / row["autotuned"]["solve_ms"]
        out.append(row)
    return out


def _proto_tc_dft32(pp, lines=1 << 22, reps=10):
    """Prototype tensor-core DFT stage (not on the solve path): 32-point complex DFTs of `lines`
    lines by tcgen05 bf16 slice products (pp_proto_dft32_tc), against the double-float line kernel
    on 32-point complex lines (the y-forward of an all-periodic 1024 x 32 x 4096 plan), per complex
    point; plus its accuracy against numpy's FFT on a sample of lines."""
    import ctypes
    import numpy as np
    import torch
    from paper_1909_05423_gb300 import _lib
    lib = _lib.load()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    g = torch.Generator(device="cuda")
    g.manual_seed(SEED)
    re = torch.empty(lines, 32, dtype=torch.float64, device="cuda").uniform_(-1.0, 1.0, generator=g)
    im = torch.empty(lines, 32, dtype=torch.float64, device="cuda").uniform_(-1.0, 1.0, generator=g)
    ore, oim = torch.empty_like(re), torch.empty_like(im)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    run = lambda: _lib.check(lib.pp_proto_dft32_tc(P(re), P(im), P(ore), P(oim), lines, P(err), None))
    tc_ms = _events_ms(run, reps)
    if int(err.item()) != 0:
        raise RuntimeError("tensor-core DFT prototype: MMA wait limit reached")
    k = min(lines, 4096)
    z = re[:k].cpu().numpy() + 1j * im[:k].cpu().numpy()
    y = ore[:k].cpu().numpy() + 1j * oim[:k].cpu().numpy()
    ref = np.fft.fft(z, axis=1)
    rel = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    del re, im, ore, oim
    shape = (1024, 32, 4096)
    plan = pp.Plan(shape, "PPPPPP", (1.0, 1.0, 1.0), "f64", options={"autotune": 1})
    x = torch.empty(shape, dtype=torch.float64, device="cuda").uniform_(-1.0, 1.0, generator=g)
    u = torch.empty_like(x)
    _lib.check(lib.pp_run_stage(plan._h, 0, P(x), P(u), None))
    y_ms = _events_ms(lambda: _lib.check(lib.pp_run_stage(plan._h, 1, P(x), P(u), None)), reps)
    plan.close()
    ylines = (4096 // 2 + 1) * 1024
    tc_ns, df_ns = tc_ms * 1e6 / (lines * 32), y_ms * 1e6 / (ylines * 32)
    return {"lines": lines, "tc_ms": tc_ms, "tc_ns_per_complex_point": tc_ns, "rel_l2_vs_numpy": rel,
            "df_line_kernel_ms": y_ms, "df_lines": ylines, "df_ns_per_complex_point": df_ns,
            "tc_over_df": tc_ns / df_ns, "adopted": False}


def _config4(pp, workloads, args):
    """64 independent grids, sides drawn from {32,...,256} per axis and boundary conditions per axis/face,
    U[-1,1] sources; one graph launch per batch (FP64 and FP32 I/O), with autotuned plans (each plan
    tuned alone at creation, then the batch graph tuned as a whole on its first call) and with the
    default launch shapes."""
    import torch
    grids = workloads.batched_grids(seed=4, count=64)
    pts = sum(s[0] * s[1] * s[2] for s, _ in grids)
    out = {"grids": 64, "points": pts}
    g = torch.Generator(device="cuda")
    g.manual_seed(4)
    for dtype, tdt in (("f64", torch.float64), ("mixed_f32io", torch.float32)):
        fs = [torch.empty(s, dtype=tdt, device="cuda").uniform_(-1.0, 1.0, generator=g) for s, _ in grids]
        us = [torch.empty_like(x) for x in fs]
        res = {}
        for name, tune in (("autotuned", {"autotune": 1}), ("heuristic", {})):
            if args.no_autotune and tune:
                continue
            plans = [pp.Plan(s, bc, (1.0 / s[2], 1.0 / s[1], 1.0 / s[0]), dtype, options=tune) for s, bc in grids]
            ms = _events_ms(lambda: pp.solve_batched(plans, fs, us), args.steps)
            res[name] = {"ms_per_batch": ms, "gpoints_s": pts / ms / 1e6, "graph_launches_per_batch": 1}
            for p in plans:
                p.close()
        best = min(res, key=lambda k: res[k]["ms_per_batch"])
        out[dtype] = dict(res[best], shapes=best, **{k: v for k, v in res.items()})
        del fs, us
        torch.cuda.empty_cache()
    return out


def _config5(pp, workloads, args):
    """256^3 FP64, periodic x/y, Dirichlet z; f = 16 Gaussian blobs; L = 0.5||S f - u_t||^2:
    forward solve + adjoint solve (the gradient dL/df) through the autograd Function."""
    import numpy as np
    import torch
    n = 256
    sp = (1.0 / n,) * 3
    amp, centre, width = workloads.gaussian_blobs((n, n, n), sp, seed=5, count=16)
    f = torch.from_numpy(workloads.blob_field((n, n, n), sp, amp, centre, width)).cuda().requires_grad_(True)
    ut = torch.from_numpy(np.random.default_rng(6).uniform(-1, 1, size=(n, n, n))).cuda()
    plan = pp.Plan((n, n, n), "PPPPDD", sp, "f64")

    def step():
        f.grad = None
        uu = pp.PoissonSolve.apply(f, plan)
        loss = 0.5 * ((uu - ut) ** 2).sum()
        loss.backward()

    ms = _events_ms(step, args.steps)
    plan.close()
    return {"n": n, "ms_forward_plus_adjoint": ms, "gpoints_s_forward_plus_adjoint": n ** 3 / ms / 1e6}


def _copy_gbs(fh, uh, dev):
    """Plain pinned host<->device copy bandwidth of the e2e buffers (one whole-grid copy each way,
    CUDA events on the current stream), GB/s."""
    import torch
    st = torch.cuda.current_stream()
    out = []
    for src, dst in ((fh, dev), (dev, uh)):
        dst.copy_(src, non_blocking=True)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        dst.copy_(src, non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        out.append(src.numel() * src.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return out[0], out[1]


class HostPlacement:
    """The GPU's CPU and NUMA affinity (nvidia-smi topo -m) and where the pinned pages live
    (/proc/self/numa_maps).  bind() restricts this process to the GPU-local CPUs while the pinned
    buffers are allocated and touched; unbind() restores the previous affinity."""

    def __init__(self, index):
        self.index = index
        self.cpus, self.numa, self.saved = None, None, None
        try:
            txt = subprocess.run(["nvidia-smi", "topo", "-m"], capture_output=True, text=True, timeout=20).stdout
            lines = [ln for ln in txt.splitlines() if ln.strip()]
            head = lines[0].split("\t")
            row = next(ln for ln in lines[1:] if ln.split("\t")[0].strip() == "GPU%d" % index).split("\t")
            cols = {h.strip(): i for i, h in enumerate(head)}
            # a header without an empty leading cell (for the row names) is shifted by one
            sh = 0 if head[0].strip() == "" else 1
            cpu_s = row[cols["CPU Affinity"] + sh].strip() if "CPU Affinity" in cols else ""
            self.numa = row[cols["NUMA Affinity"] + sh].strip() if "NUMA Affinity" in cols else None
            cpus = set()
            for part in cpu_s.split(","):
                if "-" in part:
                    lo, hi = part.split("-")
                    cpus.update(range(int(lo), int(hi) + 1))
                elif part.strip().isdigit():
                    cpus.add(int(part))
            self.cpus = sorted(cpus & os.sched_getaffinity(0)) or None
        except Exception:
            pass

    def bind(self):
        try:
            self.saved = os.sched_getaffinity(0)
            if self.cpus:
                os.sched_setaffinity(0, self.cpus)
        except Exception:
            self.saved = None

    def unbind(self):
        if self.saved:
            try:
                os.sched_setaffinity(0, self.saved)
            except Exception:
                pass

    @staticmethod
    def _pages(addr):
        """N<node>=pages of the mapping that holds addr."""
        try:
            best = None
            with open("/proc/self/numa_maps") as fh:
                for ln in fh:
                    start = int(ln.split()[0], 16)
                    if start <= addr and (best is None or start > best[0]):
                        best = (start, ln)
            return {kv.split("=")[0]: int(kv.split("=")[1]) for kv in best[1].split() if kv[:1] == "N" and "=" in kv}
        except Exception:
            return None

    def report(self, *addrs):
        return {"gpu_cpu_affinity": (("%d-%d" % (self.cpus[0], self.cpus[-1])) if self.cpus else None),
                "gpu_numa_affinity": self.numa, "bound_to_gpu_cpus": bool(self.cpus),
                "pinned_pages_per_node": [self._pages(a) for a in addrs]}


def run_ours(args):
    import numpy as np
    import torch

    import paper_1909_05423_gb300 as pp
    from paper_1909_05423_gb300 import _lib, workloads

    rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = args.n
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else (n, n, n)
    nz_, ny_, nx_ = shape
    sp = (1.0 / nx_, 1.0 / ny_, 1.0 / nz_)
    npts = nx_ * ny_ * nz_
    lib = _lib.load()

    # input: seeded U[-1,1], mean removed, generated on the device
    g = torch.Generator(device="cuda")
    g.manual_seed(SEED + rank)
    f = torch.empty(shape, dtype=torch.float64, device="cuda").uniform_(-1.0, 1.0, generator=g)
    f -= f.mean()
    u = torch.empty_like(f)
    stream = torch.cuda.current_stream()
    sh = _lib.ctypes.c_void_p(stream.cuda_stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def nvtx(name=None):
        # an NVTX range around the timed steps lets a profiler capture exactly those launches
        try:
            if name is None:
                torch.cuda.nvtx.range_pop()
            else:
                torch.cuda.nvtx.range_push(name)
        except Exception:
            pass

    def timed(plan, fin, uout, steps, warmup, tag="timed"):
        """Run warmup + steps solves stage by stage with events between stages.
        Returns (ms per step, per-stage mean ms)."""
        h = plan.handle
        fp, up = _lib.ctypes.c_void_p(fin.data_ptr()), _lib.ctypes.c_void_p(uout.data_ptr())
        for _ in range(warmup):
            _lib.check(lib.pp_solve(h, fp, up, sh))
        barrier()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(steps)]
        nvtx(tag)
        for s in range(steps):
            ev[s][0].record(stream)
            for st in range(5):
                _lib.check(lib.pp_run_stage(h, st, fp, up, sh))
                ev[s][st + 1].record(stream)
        nvtx()
        barrier()
        tot = sum(ev[s][0].elapsed_time(ev[s][5]) for s in range(steps))
        per = [sum(ev[s][k].elapsed_time(ev[s][k + 1]) for s in range(steps)) / steps for k in range(5)]
        return tot / steps, per

    # ---------------------------------------------------------------- FP64 path (headline)
    # launch shapes picked by the library's autotuner at plan creation (timed once, cached)
    tune = {} if args.no_autotune else {"autotune": 1}
    plan = pp.Plan(shape, BC, sp, "f64", options=tune)
    clocks = Clocks(local)
    barrier()
    clocks.start()
    ms, per = timed(plan, f, u, args.steps, args.warmup, "timed_f64")
    clk = clocks.stop()
    ms_all, value = replica_aggregate(ms, npts, dist, device="cuda")
    plan.status()
    shapes = {k: {"threads": t, "lines_per_cta": l} for k, (t, l) in plan.launch_shapes().items()}

    # roofline of the dominant kernel: algorithmic bytes = read input once + write output once
    elem = 8  # FP64 I/O and double-float spill: 8 bytes per real
    xs = (nx_ + 2) / nx_ if BC[0] == "P" else 1.0
    alg_bytes = {"x-forward": npts * elem * (1 + xs), "y-forward": 2 * npts * elem * xs,
                 "z-solve": 2 * npts * elem * xs, "y-inverse": 2 * npts * elem * xs,
                 "x-inverse": npts * elem * (1 + xs)}
    dom = max(range(5), key=lambda k: per[k])
    dname = STAGES[dom]
    peak, peak_kind = _peaks()
    achieved = alg_bytes[dname] / (per[dom] * 1e-3) / 1e9
    path_gbs = 32.0 * npts / (ms * 1e-3) / 1e9
    # the line kernels are bound by FP32 instruction issue (double-float arithmetic): ALU roofline
    kinds = {"x-forward": "dct2", "y-forward": "dct2", "y-inverse": "dct3", "x-inverse": "dct3"}  # NN-x, DD-y
    alu_peak = FP32_LANES * SM_MAX_GHZ * 1e9 / 1e12
    per_stage = {}
    for k, name in enumerate(STAGES):
        d = {"ms": per[k], "hbm_gbs": alg_bytes[name] / (per[k] * 1e-3) / 1e9}
        d["hbm_frac"] = d["hbm_gbs"] / peak
        if name in kinds:
            opr = line_ops_per_real(kinds[name], nx_ if name[0] == "x" else ny_, "df")
            d["fp32_ops_per_point"] = opr
            d["alu_tops"] = opr * npts / (per[k] * 1e-3) / 1e12
            d["alu_frac"] = d["alu_tops"] / alu_peak
        per_stage[name] = d
    # the roofline block is the dominant kernel's HBM fraction (algorithmic bytes of that launch over
    # its CUDA-event time, against the measured copy bandwidth); the line kernels are in fact bound by
    # FP32 instruction issue in double-float arithmetic, so that fraction is reported beside it
    roof = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)" % peak_kind,
            "traffic": None if args.shape else _traffic(dname, n), "alg_bytes_per_launch": alg_bytes[dname],
            "alg_bytes_per_point": alg_bytes[dname] / npts}
    if dname in kinds:
        roof["alu"] = {"achieved": per_stage[dname]["alu_tops"], "peak": alu_peak,
                       "unit": "T FP32 lane instructions/s", "frac": per_stage[dname]["alu_frac"],
                       "alg_fp32_instr_per_point": per_stage[dname]["fp32_ops_per_point"],
                       "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz; algorithmic double-float "
                                      "operations counted as the FP32 lane instructions they issue (FMA = 1)"}

    # ---------------------------------------------------------------- mixed precision variants
    variants = {}
    if not args.no_mixed:
        pm = pp.Plan(shape, BC, sp, "mixed_f64io", options=tune)
        um = torch.empty_like(f)
        ms_m, per_m = timed(pm, f, um, args.steps, args.warmup, "timed_mixed")
        torch.cuda.synchronize()
        err_m = (torch.linalg.vector_norm(um - u) / torch.linalg.vector_norm(u)).item()
        variants["mixed_f64io"] = {"value": npts / (ms_m * 1e-3) / 1e9, "ms_per_step": ms_m,
                                   "stage_ms": dict(zip(STAGES, per_m)), "speedup_vs_f64": ms / ms_m,
                                   "rel_l2_vs_f64_path": err_m}
        # mixed solve + one refinement step (exact residual, FP32 correction solve)
        ms_r = _events_ms(lambda: pm.solve_refined(f, um), args.steps, warmup=args.warmup)
        err_r = (torch.linalg.vector_norm(um - u) / torch.linalg.vector_norm(u)).item()
        variants["refined_f64io"] = {"value": npts / (ms_r * 1e-3) / 1e9, "ms_per_step": ms_r,
                                     "speedup_vs_f64": ms / ms_r, "rel_l2_vs_f64_path": err_r}
        pm.close()
        del um

    # ---------------------------------------------------------------- config 3: mixed precision on MMS
    if not args.no_variants:
        del u
        torch.cuda.empty_cache()
        variants["config2_256"] = _config2_256(pp, args)
        variants["config3_mixed_mms"] = _config3(pp, workloads, args)
        variants["config4_batched"] = _config4(pp, workloads, args)
        variants["config5_adjoint"] = _config5(pp, workloads, args)
        variants["zsolver_study_64x64"] = _zsolver_study(pp, args)
        variants["proto_tc_dft32"] = _proto_tc_dft32(pp)
        u = torch.empty_like(f)
        plan.solve(f, u)

    # ---------------------------------------------------------------- end to end through host buffers
    e2e = None
    if not args.no_e2e:
        host = HostPlacement(local)
        host.bind()  # pinned buffers allocated (and first touched) by a thread on the GPU's own NUMA node
        fh = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        uh = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        fh.copy_(f.cpu())
        uh.zero_()
        h2d, d2h = _copy_gbs(fh, uh, f)
        plan.solve_host(fh, uh)
        barrier()
        # each call timed on its own (it synchronises); the median is reported, since the host side
        # of these shared machines is not quiet (one run saw 230 ms where others saw 93-98 ms)
        calls = []
        for _ in range(max(3, min(args.steps, 5))):
            t0 = time.perf_counter()
            plan.solve_host(fh, uh)
            calls.append(time.perf_counter() - t0)
        dt = statistics.median(calls)
        e2e = {"value": npts / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": npts * 8, "d2h_bytes_per_step": npts * 8,
               "ms_per_step": dt * 1e3, "ms_per_call": [round(c * 1e3, 2) for c in calls], "h2d_gbs": h2d, "d2h_gbs": d2h,
               "copy_floor_ms": npts * 8 / (h2d * 1e9) * 1e3 + npts * 8 / (d2h * 1e9) * 1e3,
               "host": host.report(fh.data_ptr(), uh.data_ptr())}
        host.unbind()
        del fh, uh

    cpu = None
    if rank == 0 and not args.no_cpu:
        dt, pts, threads = _oracle_sample(n, args.oracle_planes, SEED)
        cpu = {"value": pts / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "oracle solve of a %dx%dx%d slab of the same workload (naive O(N^2) transforms, "
                         "per-point cost independent of nz)" % (n, n, args.oracle_planes)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 I/O, double-float (2xf32) transforms and z-solve",
            "data": "synthetic (seeded U[-1,1], mean removed; generated on device)",
            "config": {"workload": "%s FP64 Neumann-x/Dirichlet-y/Neumann-z, U[-1,1] source" %
                                   ("%d^3" % n if not args.shape else "%dx%dx%d (nz x ny x nx)" % shape), "bc": BC,
                       "n": n, "shape_zyx": list(shape), "points": npts,
                       "l2": "inputs (%.1f GiB/grid) exceed L2; no flush" % (npts * 8 / 2 ** 30),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "stage_ms": dict(zip(STAGES, per)), "launch_shapes": shapes,
                       "path_hbm_gbs_32B_per_point": path_gbs,
                       "path_hbm_frac_32B_per_point": path_gbs / peak},
            "roofline": roof,
            "kernels": per_stage,
            "variants": variants,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 5 * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--shape", default=None, help="nz,ny,nx of a non-cubic grid (profiling captures; overrides --n)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--oracle-planes", type=int, default=8)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="fixed launch-shape heuristics instead of the autotuner")
    ap.add_argument("--n3", type=int, nargs="+", default=[512, 1024],
                    help="grid sides of the config-3 mixed-precision variant")
    ap.add_argument("--proto-tc", type=int, default=0, metavar="LINES",
                    help="time only the tensor-core DFT prototype on LINES lines (profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.proto_tc:
        import paper_1909_05423_gb300 as pp
        print(json.dumps({"proto_tc_dft32": _proto_tc_dft32(pp, args.proto_tc, max(args.steps, 1))}))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
