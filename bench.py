#!/usr/bin/env python
"""Throughput of the GB300 layered-medium Helmholtz solver: solved unknowns/s.

One step = one hz_solve of the 320 x 320 x 200 workload (h = 1 on every axis, 4
layers of 50 planes, 4 x 4 blocks, 8 Gaussian sources, complex128): steps 1-7 of
the block method of Sec. 2 with the interface correction, every RHS to relative
residual <= 1e-8.  The FP64 path is the headline `value`; the mixed path (FP32
transforms on the tensor cores, FP64 z solves, interface solves and refinement) is
measured on the same workload and reported beside it, and so is the two-block PML
workload (160 x 160 x 128, 4 point sources).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hz|reference]

N > 1 (torchrun): every rank solves its own copy of the workload (replicas,
weak scaling, no collective on the data path); value = all ranks' unknowns /
the slowest rank's time.  `--impl reference` times the CPU FP64 oracle (the
plain block algorithm in numpy/scipy) on a bounded sample of the workload (one
of its 8 right-hand sides per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solved unknowns/s at rel. residual <=1e-8, mixed vs FP64 path on 1 GB300 (FP64 path as value; mixed beside it)"
UNIT = "unknowns/s"
RTOL = 1e-8
FP64_FLOPS_PER_CLK_SM = 4          # 2 DFMA per SM per clock (1.25 TFLOP/s nominal at 2070 MHz)
N_SM = 152
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hz", choices=["hz", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nrhs", type=int, default=0,
                    help="right-hand sides of an extra workload (default: the workload's own count)")
    ap.add_argument("--workload", default="uniform320",
                    choices=["uniform320", "pml160", "adjoint192", "uniform32", "batch48", "scaling", "perturbed160",
                             "uniform320x40", "longz"],
                    help="uniform320 is the benchmark line; the others are extra measurements")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = sorted(float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit())
        mx = max(float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    """HBM GB/s and bf16 TFLOP/s measured on this machine (MEASURED_PEAKS.json), with fallbacks."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6786.2)), "measured"
    except (OSError, ValueError):
        return 6800.0, "fallback"


def tf32_peak():
    """TF32 dense TFLOP/s: the measured bf16 burst figure x the nominal TF32 / bf16 ratio."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16 = float(json.load(fh).get("bf16_tflops", 1900.0))
        src = "measured bf16 burst x 1.1/2.25 (nominal TF32/bf16)"
    except (OSError, ValueError):
        bf16, src = 1900.0, "fallback bf16 x 1.1/2.25 (nominal TF32/bf16)"
    return bf16 * 1.1 / 2.25, src


def max_over_ranks(value: float, dist, device=None) -> float:
    """The slowest rank's time: all-reduce(MAX) of a per-rank scalar (identity without dist)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(unknowns_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job solved unknowns/s: every rank's unknowns over the slowest rank's time."""
    return world * unknowns_per_rank / seconds_max


def block_sizes(n, ifaces):
    edges = [-1] + [int(p) for p in ifaces] + [int(n)]
    return [edges[b + 1] - edges[b] - 1 for b in range(len(edges) - 1)]


def bulk_macs(w, nrhs):
    """Complex multiply-adds of the four bulk transform launches (X1..X4) of one solve."""
    bx = [int(n) for n in block_sizes(w.nx, w.x_iface)]
    by = [int(n) for n in block_sizes(w.ny, w.y_iface)]
    sx, sy = sum(n * n for n in bx), sum(n * n for n in by)
    rows_x = w.ny - len(w.y_iface)        # rows transformed along x (interface rows skipped)
    rows_y = w.nx - len(w.x_iface)
    per = nrhs * w.nz
    return [per * rows_x * sx, per * rows_y * sy, per * rows_y * sy, per * rows_x * sx]


def real_block_flags(h, ifaces):
    """Per block of one axis: True when all its steps are real (a real eigenvector table)."""
    import numpy as np
    edges = [-1] + [int(p) for p in ifaces] + [len(h)]
    return [bool(np.all(np.imag(h[edges[b] + 1:edges[b + 1]]) == 0)) for b in range(len(edges) - 1)]


def tc_mma_flops(w, nrhs, real_tables):
    """Tensor-pipe flops of the four bulk transform launches of one solve (3 TF32 products).

    Interleaved complex GEMM (K = N = 2 n): 8 real flops per complex multiply-add; the
    real-table kernel (real blocks, when enabled): Re and Im parts times the real table, 4.
    """
    rx = real_block_flags(w.hx, w.x_iface) if real_tables else None
    ry = real_block_flags(w.hy, w.y_iface) if real_tables else None
    bx = [int(n) for n in block_sizes(w.nx, w.x_iface)]
    by = [int(n) for n in block_sizes(w.ny, w.y_iface)]
    fx = sum(n * n * (4 if rx and rx[b] else 8) for b, n in enumerate(bx))
    fy = sum(n * n * (4 if ry and ry[b] else 8) for b, n in enumerate(by))
    per = nrhs * w.nz
    rows_x, rows_y = w.ny - len(w.y_iface), w.nx - len(w.x_iface)
    return 3 * per * (2 * rows_x * fx + 2 * rows_y * fy)


def tc_bytes_per_launch(w, nrhs, nref):
    """Algorithmic HBM bytes of a tensor-core transform launch, averaged over a mixed step.

    A step is 1 + nref solves of 4 launches over the block values (interface rows and
    columns excluded): forward x 24 B per value (complex128 in, complex64 out), forward y
    and inverse y 16 B, inverse x 24 B, or 40 B when it accumulates a correction into u.
    """
    values = (w.nx - len(w.x_iface)) * (w.ny - len(w.y_iface)) * w.nz * nrhs
    return values * (80 + 96 * nref) / (4 * (1 + nref))


def kernel_source_hash(fname: str = "hz_xform.cu"):
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_1909_01299_gb300", "csrc", fname), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str, fname: str = "hz_xform.cu"):
    """dram bytes per launch from the committed ncu summary, if it matches this source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            data = json.load(fh)
        ent = data.get(kernel, {})
        if ent.get("source_sha") == kernel_source_hash(fname) and ent.get("workload") == workload:
            return ent.get("bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(budget_s: float = 12.0, max_runs: int = 3, w=None, of: str = "4"):
    """Time the CPU oracle's block solver on 1 RHS of the workload (bounded sample)."""
    import numpy as np
    from oracle import hz_oracle as O
    from paper_1909_01299_gb300 import workloads as W
    if w is None:
        w = W.pml_160x160x128(nrhs=1)
    P = O.Problem.from_workload(w)
    A, _ = O.assemble(P)
    times = []
    t_all = time.perf_counter()
    while len(times) < max_runs and (time.perf_counter() - t_all) < budget_s:
        t0 = time.perf_counter()
        u = O.block_solve(P, w.f, A)
        times.append(time.perf_counter() - t0)
    res = float(np.max(O.residual(P, u, w.f, A)))
    best = min(times)
    return {"value": w.unknowns / best, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 of {of} RHS of {w.name} through the full 7-step block algorithm, "
                      f"{len(times)} run(s), best {best:.2f} s, residual {res:.1e}; BLAS threads = "
                      f"cores, per-mode z solves single-threaded"}, best, w.unknowns


def oracle_single_thread(workload: str, timeout_s: float = 90.0):
    """The same oracle sample with one BLAS thread, in a child process (thread counts are
    fixed when numpy loads); None if it does not finish in time."""
    import subprocess
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, bench\n"
            "from paper_1909_01299_gb300 import workloads as W\n"
            f"w = W.NAMED[{workload!r}]()\n"
            "r = bench.oracle_sample(budget_s=30.0, max_runs=1, w=type(w)(**{**w.__dict__, 'f': w.f[:1]}), "
            "of=str(w.nrhs))[0]\n"
            "r['cores'] = 1\n"
            "print(json.dumps(r))\n")
    try:
        res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=timeout_s)
        return json.loads(res.stdout.strip().splitlines()[-1]) if res.returncode == 0 else None
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        return None


def bench_workload():
    """The benchmark workload: 320 x 320 x 200, h = 1, 4 layers, 4 x 4 blocks, 8 Gaussian sources
    (the largest single-GPU configuration)."""
    from paper_1909_01299_gb300 import workloads as W
    return W.uniform_320x320x200()


def one_rhs(w, r: int = 0):
    """The same workload restricted to its RHS r (the oracle's bounded sample)."""
    import dataclasses
    return dataclasses.replace(w, f=w.f[r:r + 1].copy())


def run_reference(args, wall_limit_s: float = 420.0):
    """The CPU oracle's block solver on 1 of the 8 RHS of the benchmark workload per step.

    Each step is one full 7-step solve of one RHS (about 10 s on 16 Grace cores).  A wall-clock
    guard stops the timed loop early if the machine is much slower than that; the line then
    reports the steps actually timed."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import hz_oracle as O
    w = one_rhs(bench_workload())
    P = O.Problem.from_workload(w)
    A, _ = O.assemble(P)
    t_all = time.perf_counter()
    for _ in range(args.warmup):
        O.block_solve(P, w.f, A)
    done = 0
    t0 = time.perf_counter()
    u = None
    while done < args.steps:
        u = O.block_solve(P, w.f, A)
        done += 1
        if time.perf_counter() - t_all > wall_limit_s:
            break
    dt = (time.perf_counter() - t0) / done
    res = float(np.max(O.residual(P, u, w.f, A)))
    value = w.unknowns / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": done, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)",
            "data": "synthetic",
            "config": {"workload": w.name + " (1 of 8 RHS per step)", "nx": w.nx, "ny": w.ny, "nz": w.nz,
                       "blocks": "4x4", "nrhs": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"RHS 0 of 8 per step through the full 7-step block algorithm, "
                                       f"residual {res:.1e}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if done < args.steps:
        line["steps_note"] = f"wall-clock guard: {done} of {args.steps} steps timed"
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def time_path(torch, hz, plan, f, u, steps, warmup, dist, world, device):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.solve(f, out=u)
    torch.cuda.synchronize()
    plan.set_stage_timing(True)
    l0 = plan.info()["kernel_launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(device) as clk:
        e0.record(stream)
        for _ in range(steps):
            plan.solve(f, out=u)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist, "cuda")
    launches = plan.info()["kernel_launches"] - l0
    stages = plan.stage_times()
    plan.set_stage_timing(False)
    return ms, launches, stages, clk.summary()


def launch_ms(st):
    """Average CUDA-event time of one bulk transform launch (steps 1 and 7) from the stage timers."""
    return (st["fwd"][0] + st["inv"][0]) / max(1, st["fwd"][1] + st["inv"][1])


def real_tables(w):
    """True when every block of both axes has real eigenvectors (all block steps real)."""
    import numpy as np
    return bool(np.all(np.imag(w.hx) == 0) and np.all(np.imag(w.hy) == 0))


def fast_sine_ok(n):
    """A uniform block of width n takes the FFT-based sine transform: n >= 2 and n + 1 <= 128
    with no prime factor above 5."""
    N = n + 1
    if n < 2 or N > 128:
        return False
    for q in (2, 3, 5):
        while N % q == 0:
            N //= q
    return N == 1


def fast_sine_flops(n):
    """Algorithmic flops of the fast sine transform of one row of a block of width n: one
    complex FFT of length N = n + 1 at the standard 5 N log2 N count, the pre step (6 flops per
    value) and the post step (3 per value)."""
    import math
    N = n + 1
    return 5 * N * math.log2(N) + 9 * (N - 1)


def uniform_blocks(h, ifaces):
    """Per block of the axis: True when all its steps are equal, real and positive."""
    import numpy as np
    edges = [-1] + [int(p) for p in ifaces] + [len(h) - 1]
    out = []
    for b in range(len(edges) - 1):
        s, n = edges[b] + 1, edges[b + 1] - edges[b] - 1
        st = np.asarray(h[s:s + n + 1])
        out.append(bool(np.all(st.imag == 0) and st[0].real > 0 and np.all(st == st[0])))
    return out


def fp64_transform_work(w, nrhs):
    """Per bulk launch of the FP64 path (average of the 4 launches of a solve): algorithmic flops
    of the dense products (4 n real flops per complex value for real tables, 8 n for complex
    ones) and of the fast sine transforms, and whether every block is a fast-sine block."""
    import numpy as np
    dense, fast, all_fast = 0.0, 0.0, True
    for h, ifc, other_n, other_ifc in ((w.hx, w.x_iface, w.ny, w.y_iface), (w.hy, w.y_iface, w.nx, w.x_iface)):
        rows = nrhs * w.nz * (other_n - len(other_ifc))
        real = bool(np.all(np.imag(h) == 0))
        for n, uni in zip(block_sizes(len(h) - 1, ifc), uniform_blocks(h, ifc)):
            if uni and fast_sine_ok(n):
                fast += 2 * rows * fast_sine_flops(n)            # forward and inverse launches
            else:
                all_fast = False
                dense += 2 * rows * n * n * (4 if (real or uni) else 8)
    return dense / 4, fast / 4, all_fast


def fp64_roofline(w, R, st, traffic_workload=None):
    """Roofline of the FP64 path's bulk transforms (its dominant kernels), bound by the FP64 pipe.

    Algorithmic flops per launch: for blocks on the fast sine transform the FFT count of
    fast_sine_flops per row; for the others the dense product, 4 n real flops per complex value
    for a real table (2 FMA per multiply-add) and 8 n for a complex one.  Four launches per
    solve; the launch time is the stage timers' average.
    """
    dense, fast, all_fast = fp64_transform_work(w, R)
    flops = dense + fast
    t = launch_ms(st)
    achieved = flops / (t * 1e-3) / 1e12
    peak = N_SM * SM_MAX_MHZ * 1e6 * FP64_FLOPS_PER_CLK_SM / 1e12
    total_ms = sum(v[0] for v in st.values())
    if all_fast:
        kernel, fname = "dst_kernel (FP64 fast sine transforms of the uniform blocks)", "hz_dst.cu"
        count = "fast sine transform: 5 N log2 N + 9 (N - 1) real flops per row of a block of width n, N = n + 1"
    elif fast == 0:
        kernel, fname = "xform_kernel<double> (FP64 bulk x/y transforms)", "hz_xform.cu"
        count = ("dense product: 4 n real flops per complex value for real tables, 8 n for complex ones "
                 "(n = block width)")
    else:
        kernel, fname = "xform_kernel<double> + dst_kernel (FP64 bulk x/y transforms)", "hz_xform.cu"
        count = "dense product for the non-uniform blocks, fast sine transform count for the uniform ones"
    return {"bound": "alu", "kernel": kernel,
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flop_count": count,
            "peak_note": "FP64 pipe: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s); "
                         "probe measured 1.197 TFLOP/s at ~1.97 GHz",
            "flops_per_launch": flops, "launch_ms": t,
            "traffic": profiled_traffic(kernel.split(" ")[0], traffic_workload or w.name, fname),
            "share_of_step": (st["fwd"][0] + st["inv"][0]) / max(total_ms, 1e-9)}


def tc_roofline(w, R, st, refinements, real_tables=False):
    """Roofline of the mixed path's bulk transform kernel (tensor cores, 3xTF32), HBM-bound.

    Algorithmic bytes per transformed value: forward x reads complex128 f and writes complex64
    (24 B), forward y and inverse y complex64 both ways (16 B), inverse x reads complex64 and
    writes complex128 u (24 B), or also reads u when it accumulates a correction (40 B);
    averaged over the 4 (1 + refinements) launches of a step.  The same launches against the
    tensor pipe: the MMA flops of tc_mma_flops (3 TF32 products; the real-table kernel issues
    half the interleaved form's per complex multiply-add).  (The mixed path's FP32 fast sine
    transform of uniform blocks is opt-in and not used here.)
    """
    hbm_peak, hbm_src = measured_peaks()
    t = launch_ms(st)
    b = tc_bytes_per_launch(w, R, refinements)
    nreal = sum(real_block_flags(w.hx, w.x_iface)) + sum(real_block_flags(w.hy, w.y_iface)) if real_tables else 0
    nblk = len(w.x_iface) + len(w.y_iface) + 2
    if nreal == nblk:
        kernel, fname = "xform_tcr_kernel (tcgen05 3xTF32 bulk x/y transforms, real tables)", "hz_xform_tc.cu"
    elif nreal:
        kernel, fname = "xform_tc_kernel + xform_tcr_kernel (tcgen05 3xTF32 bulk x/y transforms)", "hz_xform_tc.cu"
    else:
        kernel, fname = "xform_tc_kernel (tcgen05 3xTF32 bulk x/y transforms)", "hz_xform_tc.cu"
    out = {"bound": "hbm", "kernel": kernel,
           "achieved": b / (t * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
           "frac": b / (t * 1e-3) / 1e9 / hbm_peak, "peak_source": hbm_src,
           "bytes_per_launch": b, "launch_ms": t,
           "traffic": profiled_traffic(kernel.split(" ")[0], w.name, fname)}
    tc_flops = tc_mma_flops(w, R, real_tables) / 4
    tpk, tsrc = tf32_peak()
    out["tensor"] = {"achieved": tc_flops / (t * 1e-3) / 1e12, "peak": tpk, "unit": "TFLOP/s",
                     "frac": tc_flops / (t * 1e-3) / 1e12 / tpk, "peak_source": tsrc,
                     "flops_per_launch": tc_flops}
    return out


def measure_both(torch, hz, w, args, dist, world, device):
    """FP64 and mixed paths on one workload: times, stages, residuals, rooflines."""
    import numpy as np
    R = w.nrhs
    f = torch.from_numpy(w.f).to(device)
    u = torch.empty_like(f)
    plan = hz.Plan.from_workload(w, precision="fp64")
    plan_ms = plan.info()["plan_ms"]
    ms64, l64, st64, clk64 = time_path(torch, hz, plan, f, u, args.steps, args.warmup, dist, world, device)
    res64 = float(np.max(plan.residual(f, u)))
    plan.set_options(precision="mixed", rtol=RTOL, max_refine=10)
    msmx, lmx, stmx, clkmx = time_path(torch, hz, plan, f, u, args.steps, args.warmup, dist, world, device)
    infomx = plan.info()
    resmx = float(np.max(plan.residual(f, u)))
    plan.set_options(precision="fp64")
    unknowns = w.unknowns * R
    out = {
        "fp64": {"value": job_throughput(unknowns, world, ms64 * 1e-3), "ms_per_step": ms64,
                 "rel_residual_max": res64, "gpu_launches": l64, "roofline": fp64_roofline(w, R, st64),
                 "stages_ms_per_step": {k: v[0] / args.steps for k, v in st64.items() if v[1]},
                 "clocks": clk64},
        "mixed": {"value": job_throughput(unknowns, world, msmx * 1e-3), "ms_per_step": msmx,
                  "roofline": tc_roofline(w, R, stmx, int(infomx.get("refinements", 0)),
                                          bool(infomx.get("real_tables", 0))),
                  "speedup_vs_fp64": ms64 / msmx, "refinements": infomx["refinements"],
                  "rel_residual_max": resmx, "gpu_launches": lmx, "dtype": "c64 transforms + f64",
                  "stages_ms_per_step": {k: v[0] / args.steps for k, v in stmx.items() if v[1]},
                  "clocks": clkmx},
        "plan_ms": plan_ms,
    }
    return plan, f, u, out


def run_hz(args):
    import torch
    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    device = torch.cuda.current_device()
    from paper_1909_01299_gb300 import build as B
    B.build()
    from paper_1909_01299_gb300 import hz, workloads as W

    w = bench_workload()
    R = w.nrhs
    plan, f, u, m = measure_both(torch, hz, w, args, dist, world, device)
    del f, u

    # end to end through the host-buffer entry point (H2D of f and D2H of u inside the call)
    fh = torch.from_numpy(w.f).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    for _ in range(2):
        plan.solve_host(fh, out=uh)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(e2e_steps):
        plan.solve_host(fh, out=uh)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, "cuda")
    plan.close()
    del fh, uh

    # the two-block PML workload (160 x 160 x 128, 4 point sources) beside it
    w2 = W.pml_160x160x128()
    p2, f2, u2, m2 = measure_both(torch, hz, w2, args, dist, world, device)
    p2.close()
    del f2, u2

    unknowns = w.unknowns * R
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu, _, _ = oracle_sample(budget_s=8.0, max_runs=2, w=one_rhs(w), of=str(R))
        one = oracle_single_thread("pml160")
        if one:
            cpu["single_thread_pml160"] = {"value": one["value"], "sample": one["sample"]}
    line = {
        "metric": METRIC, "value": m["fp64"]["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["fp64"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nz": w.nz, "blocks": "4x4", "nrhs": R,
                   "grid": "uniform h = 1 on every axis (uniform blocks: sine eigenvectors); 4 layers of "
                           "50 planes; 8 Gaussian sources (sigma 2 nodes)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "working set ~8 GB (f, u, 3 volume buffers, factors) > 129 MB L2; no flush",
                   "rel_residual_max": m["fp64"]["rel_residual_max"], "plan_ms": m["plan_ms"]},
        "gpu_launches": m["fp64"]["gpu_launches"],
        "roofline": m["fp64"]["roofline"],
        "stages_ms_per_step": m["fp64"]["stages_ms_per_step"],
        "mixed": m["mixed"],
        "e2e": {"value": world * unknowns / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(w.f.size * 16),
                "d2h_bytes_per_step": int(w.f.size * 16), "ms_per_step": e2e_s * 1e3,
                "entry_point": "hz_solve_host (pinned host buffers, FP64 path)"},
        "clocks": m["fp64"]["clocks"],
        "pml160": {"workload": w2.name, "fp64": {k: m2["fp64"][k] for k in ("value", "ms_per_step",
                                                                         "rel_residual_max", "roofline")},
                   "mixed": {k: m2["mixed"][k] for k in ("value", "ms_per_step", "rel_residual_max",
                                                         "refinements", "speedup_vs_fp64", "roofline")}},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_extra(args):
    """Single-GPU measurements of the other named workloads (not the benchmark line)."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_1909_01299_gb300 import build as B
    B.build()
    from paper_1909_01299_gb300 import hz, workloads as W
    out = {"workload": args.workload}
    if args.workload == "scaling":
        def survey_split(n):
            """Interfaces of the paper's split of a survey axis (rim | uniform core | rim, Sec. 2 cost
            paragraph): the uniform nodes 17..n-18 of rim_axis(n - 32) carry core blocks of width s
            (s + 1 with no prime factor above 5, s <= 127, so that they take the fast sine
            transform), interface nodes between them, and the rest of the axis goes to the two
            rim blocks."""
            lo, hi = 17, n - 17                          # uniform nodes [lo, hi)
            C = hi - lo
            k = max(1, -(-(C + 1) // 128))
            s = max(m for m in range(2, 128) if fast_sine_ok(m) and k * m + (k - 1) <= C)
            used = k * s + (k - 1)
            start = lo + (C - used) // 2
            ifc = [start - 1]
            for b in range(1, k):
                ifc.append(start + b * (s + 1) - 1)
            ifc.append(start + used)
            return ifc, s, k

        # the two regimes of the cost estimate in Sec. 2, FP64 path: one block per axis (dense
        # N x N transforms, work per unknown ~ N) against the automatic ~sqrt(N) partition
        # (work per unknown ~ sqrt(N)); survey-type axes (uniform core + 16-node rim), nz = 64
        rows = []
        for n in (64, 96, 128, 192, 256, 320, 384):
            hx = W.rim_axis(n - 32, rim_nodes=16, ratio=1.3, pml_nodes=8)
            hzz = W.ramp_z(64)
            rng = np.random.default_rng(n)
            f = torch.from_numpy(rng.standard_normal((2, 64, n, n)) + 1j * rng.standard_normal((2, 64, n, n))).cuda()
            u = torch.empty_like(f)
            row = {"n": n, "unknowns_x_rhs": n * n * 64 * 2}
            ifc, s_core, k_core = survey_split(n)
            for label, nb in (("one_block", 1), ("auto", 0), ("survey_fast", None)):
                if nb is None:       # rim | k uniform core blocks of width s (fast sine transform) | rim
                    plan = hz.Plan(hx, hx, hzz, [0, 32, 64], [0.2 + 0.004j, 0.35 + 0.007j], x_iface=ifc,
                                   y_iface=ifc, precision="fp64")
                else:
                    plan = hz.Plan(hx, hx, hzz, [0, 32, 64], [0.2 + 0.004j, 0.35 + 0.007j], nbx=nb, nby=nb,
                                   precision="fp64")
                ms, launches, st, clk = time_path(torch, hz, plan, f, u, args.steps, args.warmup, None, 1, 0)
                row[label] = {"blocks": plan.info()["nbx"], "ms": ms, "value": n * n * 64 * 2 / (ms * 1e-3),
                              "ns_per_unknown": ms * 1e6 / (n * n * 64 * 2),
                              "fast_sine": plan.info()["fast_sine"],
                              "rel_residual_max": float(np.max(plan.residual(f, u)))}
                if nb is None:
                    row[label]["core_blocks"] = f"{k_core} x {s_core}"
                plan.close()
            rows.append(row)
        out.update({"path": "fp64", "sweep": rows, "unit": UNIT})
        print(json.dumps(out), flush=True)
        return
    if args.workload == "perturbed160":
        # pml-160 with a local inhomogeneity: dk2 on a 64 x 64 x 48 box in the survey core,
        # 0.3 x the mean layer k^2 (the layered solve as the operator of GMRES)
        w = W.pml_160x160x128()
        rng = np.random.default_rng(1909)
        dk2 = np.zeros((w.nz, w.ny, w.nx), np.complex128)
        amp = 0.3 * float(np.mean(np.real(w.k2)))
        dk2[40:88, 48:112, 48:112] = amp * (rng.uniform(0.5, 1.0, (48, 64, 64)) + 0.1j * rng.uniform(0, 1, (48, 64, 64)))
        d = torch.from_numpy(dk2).cuda()
        f = torch.from_numpy(w.f).cuda()
        out["workload"] = "pml-160x160x128-2x2blocks-4rhs + 64x64x48 perturbation box"
        for prec in ("fp64", "mixed"):
            plan = hz.Plan.from_workload(w, precision=prec)
            u, iters, rel = plan.solve_perturbed(d, f, rtol=1e-8, max_iter=300, restart=20)   # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                u, iters, rel = plan.solve_perturbed(d, f, rtol=1e-8, max_iter=300, restart=20)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / args.steps
            out[prec] = {"ms_per_step": dt * 1e3, "iterations": iters, "value": w.unknowns * w.nrhs / dt,
                         "rel_residual_max": float(np.max(rel)), "ms_per_iteration": dt * 1e3 / max(iters, 1)}
            plan.close()
        out["unit"] = UNIT
        print(json.dumps(out), flush=True)
        return
    if args.workload == "batch48":
        items = W.batched_models(48)
        plans, fs, us, nrhs = [], [], [], []
        t0 = time.perf_counter()
        for w, omegas in items:
            f = torch.from_numpy(w.f).cuda()
            for om in omegas:
                p = hz.Plan.from_workload(w, precision="mixed", rtol=RTOL)
                p.set_frequency(float(om))
                plans.append(p)
                fs.append(f)
                us.append(torch.empty_like(f))
                nrhs.append(w.nrhs)
        plan_s = time.perf_counter() - t0
        batch = hz.Batch(plans, nrhs)
        lanes = batch.autotune(fs, us)
        for _ in range(args.warmup):
            batch.solve(fs, us)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rel = None
        for _ in range(args.steps):
            rel = batch.solve(fs, us)
        dt = (time.perf_counter() - t0) / args.steps
        unknowns = sum(p.nx * p.ny * p.nz * r for p, r in zip(plans, nrhs))
        out.update({"items": len(plans), "unknowns_x_rhs": unknowns, "lanes": lanes,
                    "s_per_batch": dt, "value": unknowns / dt, "unit": UNIT,
                    "graph_replay_ms": batch.info()["last_ms"], "launches_per_replay":
                    batch.info()["launches_per_replay"], "rel_residual_max": float(np.max(rel)),
                    "plan_seconds": plan_s})
        if not args.no_cpu_baseline:
            # the oracle on a 4-model subset (first 4 models, omega = 1, 1 RHS each), extrapolated
            # to the batch at the subset's unknowns/s
            from oracle import hz_oracle as O
            done, secs = 0, 0.0
            for w, _ in items[:4]:
                P = O.Problem.from_workload(w)
                A, _ = O.assemble(P)
                t1 = time.perf_counter()
                O.block_solve(P, w.f[:1], A)
                secs += time.perf_counter() - t1
                done += w.unknowns
            out["cpu_baseline"] = {"value": done / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                   "sample": f"4-model subset of the batch ({done} unknowns, 1 RHS each, omega = 1), "
                                             f"{secs:.1f} s; extrapolated to the batch: "
                                             f"{unknowns / (done / secs):.0f} s per batch"}
    else:
        gen = {"uniform320": W.uniform_320x320x200, "adjoint192": W.adjoint_192x192x128,
               "uniform32": W.single_block_32, "pml160": W.pml_160x160x128,
               "uniform320x40": W.uniform_320x320x40, "longz": W.long_z}[args.workload]
        w = gen(args.nrhs) if args.nrhs else gen()
        f = torch.from_numpy(w.f).cuda()
        u = torch.empty_like(f)
        plan = hz.Plan.from_workload(w, precision="fp64")
        for prec in ("fp64", "mixed"):
            plan.set_options(precision=prec, rtol=RTOL)
            ms, launches, st, clk = time_path(torch, hz, plan, f, u, args.steps, args.warmup, None, 1, 0)
            res = float(np.max(plan.residual(f, u)))
            out[prec] = {"value": w.unknowns * w.nrhs / (ms * 1e-3), "ms_per_step": ms,
                         "rel_residual_max": res, "refinements": plan.info()["refinements"],
                         "stages_ms_per_step": {k: v[0] / args.steps for k, v in st.items() if v[1]},
                         "clocks": clk}
        if args.workload == "adjoint192":
            # misfit gradient: forward solves, adjoint solves and the layer reduction
            rec = torch.from_numpy(w.extra["rec_flat"]).cuda()
            def grad_step():
                uu = plan.solve(f)
                flat = uu.reshape(w.nrhs, -1)
                g = torch.zeros_like(flat)
                g[:, rec] = flat[:, rec]
                lam = plan.solve_adjoint(g.reshape(uu.shape))
                return plan.grad_layers(uu, lam)

            for prec in ("fp64", "mixed"):
                plan.set_options(precision=prec, rtol=RTOL)
                grad_step()                                  # warm-up (buffers, allocator)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(args.steps):
                    grad_step()
                e1.record()
                torch.cuda.synchronize()
                out[prec]["gradient_ms"] = e0.elapsed_time(e1) / args.steps
        out["unit"] = UNIT
        if not args.no_cpu_baseline:
            # the oracle on the machine's host cores, one right-hand side of the same workload
            out["cpu_baseline"] = oracle_sample(budget_s=20.0, max_runs=2, w=gen(1), of=str(w.nrhs))[0]
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "uniform320":
        run_extra(args)
    else:
        run_hz(args)


if __name__ == "__main__":
    main()
