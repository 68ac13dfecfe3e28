#!/usr/bin/env python
"""Benchmark: density-matrix amplitude-updates/s, the fused path against the plain FP64 path at stated error.

Headline workload: the superconducting-like 2 x 7 grid (n = 14), the full depth-60 program of 6494 native ops
(Rz.SX.Rz layers, ZX(pi/2) cross-resonance brickwork, static ZZ crosstalk of 50 kHz on idle edges, T1/T2 idle
decay with T1 log-uniform in 50-200 us and T2 = 0.7 T1, a 2 % readout flip; seeded synthetic program from
workloads.config2_sc_grid).  One step = reset to |0><0|, the whole program through the fused path (stages of
operators on shared-memory tiles) with float-float storage and arithmetic (every real and imaginary part a
pair of FP32 numbers, about 48 significant bits: FP64-class accuracy on the FP32 pipes), then the FP64
reductions (14-qubit Z-basis probabilities, trace, purity) read back to the host.

Metric: amplitude-updates/s = sum over the program's native ops of 4^n, divided by the time.  The state
(4.3 GB in float-float) is larger than L2 (129 MB), so no L2 flush is needed between steps.

Beside the headline the JSON line reports, each with its error against the plain FP64 (complex128) run of
the same program (max-abs, Frobenius norm, the trace-distance bound 1/2 2^(n/2) ||rho - sigma||_F and the
super-fidelity): the plain FP64 path, the fused FP64 path, plain float-float, the fused and plain complex64
paths; the 15-qubit ion-trap program through the tensor-core blocks (tcgen05, 3xTF32 and BF16x3, k = 4..6)
and through the CUDA-core fused path; the 16-qubit spin chain (34 GB complex64 density matrix) fused in
complex64 and float-float; the 1024-instance batch with an autotuned fusion width and tile shape; the
trajectory, device-compiler and noise-sweep workloads; the roofline of each path's dominant kernel; the
oracle timed on the host cores (single thread and all cores); and the SM clocks during the timed region.

--impl reference times the FP64 oracle (its C loops, all host cores) on a bounded sample of the same workload.
With --gpus N > 1 every rank runs an independent replica of the workload (the path has no data exchange).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "density-matrix amplitude-updates/s & HBM roofline %, fused vs plain FP64 at stated error"
UNIT = "amp-updates/s"
WORKLOAD = ("superconducting-like 2x7 grid, 14 qubits, full depth-60 program (6494 native ops: Rz/SX layers, "
            "ZX(pi/2) brickwork, ZZ crosstalk 50 kHz, T1/T2 idle decay, readout flip 2e-2)")
PREC_NAMES = {"split": "f32x2", "f64": "f64", "f32": "f32"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vqd", choices=["vqd", "reference"])
    ap.add_argument("--path", default="fused", choices=["plain", "fused"], help="path of the headline")
    ap.add_argument("--prec", default="split", choices=["split", "f64", "f32"], help="precision of the headline")
    ap.add_argument("--no-extra", action="store_true", help="only the headline (profiling runs)")
    ap.add_argument("--fixed-shape", action="store_true",
                    help="headline without the autotuner: the library's default fusion width and tile shape (profiling)")
    ap.add_argument("--general", action="store_true",
                    help="fused paths without VQD_HERMITIAN (every tile of every stage; the state need not be Hermitian)")
    ap.add_argument("--no-large", action="store_true", help="skip the 15- and 16-qubit lines")
    ap.add_argument("--rows", type=int, default=2, help="grid rows (profiling cases only; the benchmark is 2x7)")
    ap.add_argument("--cols", type=int, default=7)
    ap.add_argument("--depth", type=int, default=60)
    ap.add_argument("--batch-count", type=int, default=1024, help="instances of the batched neutral-atom workload")
    ap.add_argument("--fp64-diag", action="store_true",
                    help="time FP64 elementwise passes (real full, dephasing, Rz) on a 14-qubit state and exit")
    ap.add_argument("--precision", default=None, choices=["sc_grid14", "ion15", "spin16"],
                    help="instead of timing: error of the complex64 paths against the FP64 path on one workload")
    ap.add_argument("--prefix", type=int, default=0, help="--precision: only the first N native ops (0 = all)")
    ap.add_argument("--oracle-plan", action="store_true",
                    help="time the oracle on every configuration (single thread and all cores) and exit")
    ap.add_argument("--tc-case", type=int, nargs=2, default=None, metavar=("N", "GATES"),
                    help="profiling case: the ion-trap program on N qubits with GATES gates through the tensor-core "
                         "blocks (k = 4 3xTF32, k = 4 BF16x3, k = 5 3xTF32), block-kernel times, and exit")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}



# ---------------------------------------------------------------- oracle (host) timing
def host_ram_bytes():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError, AttributeError):
        return 0


def oracle_time(prog, n_ops, threads):
    """Seconds the oracle's C loops take for the first n_ops native ops of prog at full size (the state
    allocation and initialisation are not timed)."""
    import numpy as np
    from oracle import cloop, evolve
    from oracle import compile as oc
    cloop.set_threads(threads)
    rho = np.ascontiguousarray(evolve.initial_state(prog), dtype=np.complex128)   # no second copy (68.7 GB at n = 16)
    t = time.perf_counter()
    for o in prog.ops[:n_ops]:
        cloop.apply_steps(rho, oc.compile_op(o.name, o.qubits, o.params))
    dt = time.perf_counter() - t
    del rho
    return dt


def oracle_line(name, prog, n_ops, threads, kind):
    dt = oracle_time(prog, n_ops, threads)
    units = n_ops * 4.0 ** prog.n
    rec = {"config": name, "n": prog.n, "threads": threads, "ops_timed": n_ops, "ops_total": len(prog.ops),
           "seconds": dt, "value": units / dt, "unit": UNIT}
    if n_ops < len(prog.ops):
        rec["extrapolated_full_program_s"] = dt * len(prog.ops) / n_ops
        rec["kind"] = f"{kind}; extrapolated from the first {n_ops} of {len(prog.ops)} ops"
    else:
        rec["kind"] = kind
    return rec


def cpu_baseline_block(quick=True):
    """The FP64 oracle (plain C loops, OpenMP) on the host cores, on bounded samples of the configurations:
    configuration 1 in full (all cores and one thread), the 14-qubit grid on a prefix (all cores and one
    thread), the 15-qubit ion program on a prefix, the 16-qubit spin chain on a prefix when the host has the
    RAM (68.7 GB), and the neutral-atom batch on its first instances, scaled by sum 4^n.  The per-op cost is
    about the same along a program of one op mix, so prefix timings are extrapolated to the full program
    (labelled).  quick = the bench line's bounded samples; otherwise the larger ones of --oracle-plan."""
    from oracle import cloop
    from workloads import (config1_chain6, config2_sc_grid, config3_ion_alltoall, config4_neutral_batch,
                           config5_spin_chain)
    allc = cloop.max_threads()
    out = {"threads_all": allc, "lines": []}
    c1 = config1_chain6()
    out["lines"].append(oracle_line("chain6 (n=6, full)", c1, len(c1.ops), allc, "all cores"))
    out["lines"].append(oracle_line("chain6 (n=6, full)", c1, len(c1.ops), 1, "one thread"))
    c2 = config2_sc_grid()
    out["lines"].append(oracle_line("sc_grid14 (n=14)", c2, 12 if quick else 60, allc, "all cores"))
    out["lines"].append(oracle_line("sc_grid14 (n=14)", c2, 2 if quick else 12, 1, "one thread"))
    c3 = config3_ion_alltoall()
    out["lines"].append(oracle_line("ion15 (n=15)", c3, 3 if quick else 50, allc, "all cores"))
    if host_ram_bytes() > 160e9:
        c5 = config5_spin_chain()
        out["lines"].append(oracle_line("spin16 (n=16)", c5, 1 if quick else 50, allc, "all cores"))
    else:
        out["lines"].append({"config": "spin16 (n=16)", "skipped": "the host has less than 160 GB of RAM for the 68.7 GB FP64 state"})
    progs = config4_neutral_batch(count=1024)
    tu = sum(len(q.ops) * 4.0 ** q.n for q in progs)
    if quick:
        # one instance per qubit count, its first 100 ops: the per-op time of each size, applied to every
        # instance of that size
        t_full = 0.0
        for m in sorted({q.n for q in progs}):
            q = next(x for x in progs if x.n == m)
            k = min(100, len(q.ops))
            per_op = oracle_time(q, k, allc) / k
            t_full += per_op * sum(len(x.ops) for x in progs if x.n == m)
        out["lines"].append({"config": "neutral batch (1024 instances)", "threads": allc, "value": tu / t_full,
                             "unit": UNIT, "scaled_full_batch_s": t_full,
                             "kind": "all cores; per-op time of one instance per qubit count (first 100 ops), "
                                     "scaled to every instance of that size"})
    else:
        sample = progs[:32]
        t = 0.0
        for q in sample:
            t += oracle_time(q, len(q.ops), allc)
        su = sum(len(q.ops) * 4.0 ** q.n for q in sample)
        out["lines"].append({"config": "neutral batch (1024 instances)", "threads": allc, "instances_timed": len(sample),
                             "seconds": t, "value": su / t, "unit": UNIT, "scaled_full_batch_s": t * tu / su,
                             "kind": "all cores; scaled by sum 4^n from the first 32 instances"})
    cloop.set_threads(allc)
    return out


def run_oracle_plan(args):
    print(json.dumps(cpu_baseline_block(quick=False)), flush=True)


def run_reference(args):
    """The oracle arm: its C loops on all host cores, each step the first 4 native ops of the 14-qubit grid
    program at full size (the state is allocated once; the work per op does not depend on its values)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import cloop, evolve
    from oracle import compile as oc
    from workloads import config2_sc_grid
    prog = config2_sc_grid()
    per_step = 4
    threads = cloop.max_threads()
    cloop.set_threads(threads)
    rho = np.array(evolve.initial_state(prog), dtype=np.complex128, order="C")
    steps = [oc.compile_op(o.name, o.qubits, o.params) for o in prog.ops[:per_step]]

    def step():
        for s in steps:
            cloop.apply_steps(rho, s)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = args.steps * per_step * 4.0 ** prog.n / dt
    sample = (f"first {per_step} native ops of the 14-qubit program at full size per step (FP64 oracle, plain C "
              f"loops, {threads} threads)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------- GPU arm helpers
def load_traffic(kernel_class: str):
    """DRAM bytes per launch of a kernel class from a committed ncu summary, if the kernel source still
    matches the hash recorded with the counters; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel_class)
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2306_07342_gb300", "csrc", rec["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return rec["bytes_per_launch"] if h == rec["source_sha256_16"] else None


def state_view(torch, vqd, ctx, prec):
    """Zero-copy complex128-convertible chunks of a context's state: yields complex torch tensors."""
    n = vqd.vqd_num_qubits(ctx, 0)
    N = 4 ** n
    ptr = vqd.vqd_state_ptr(ctx, 0)
    if prec == vqd.VQD_F32_SPLIT:
        v = split_view(torch, ptr, N)
        return lambda a, b: torch.complex(v[a:b, 0].double() + v[a:b, 1].double(), v[a:b, 2].double() + v[a:b, 3].double())
    v = device_view(torch, ptr, N, prec == vqd.VQD_F32)
    return lambda a, b: v[a:b].to(torch.complex128)


def state_error(torch, vqd, ref_ctx, ref_prec, ctx, prec):
    """Error of a state against a reference state on the device: max-abs, Frobenius norm, the trace-distance
    bound 1/2 2^(n/2) ||rho - sigma||_F, and the super-fidelity tr(rho sigma) + sqrt((1 - tr rho^2)(1 - tr sigma^2))
    (an upper bound of the Uhlmann fidelity), with the total-variation distance of the Z-basis probabilities."""
    import numpy as np
    n = vqd.vqd_num_qubits(ctx, 0)
    N = 4 ** n
    a_of, b_of = state_view(torch, vqd, ref_ctx, ref_prec), state_view(torch, vqd, ctx, prec)
    maxabs, fro2, overlap = 0.0, 0.0, 0.0
    chunk = 1 << 25
    for i in range(0, N, chunk):
        a, b = a_of(i, min(N, i + chunk)), b_of(i, min(N, i + chunk))
        d = b - a
        maxabs = max(maxabs, float(d.abs().max()))
        fro2 += float((d.real ** 2 + d.imag ** 2).sum())
        overlap += float((a.conj() * b).real.sum())          # tr(rho sigma) for Hermitian rho, sigma
        del a, b, d
    pr, pa = vqd.vqd_purity(ref_ctx, 0), vqd.vqd_purity(ctx, 0)
    qr, qa = vqd.vqd_prob(ref_ctx, 0, list(range(n))), vqd.vqd_prob(ctx, 0, list(range(n)))
    return {"max_abs": maxabs, "frobenius": fro2 ** 0.5, "trace_distance_bound": 0.5 * 2 ** (n / 2) * fro2 ** 0.5,
            "super_fidelity": overlap + float(np.sqrt(max(0.0, (1 - pr) * (1 - pa)))),
            "prob_tv_distance": 0.5 * float(np.abs(qa - qr).sum()),
            "trace_err": abs(vqd.vqd_trace(ctx, 0).real - vqd.vqd_trace(ref_ctx, 0).real)}


def roofline_hbm(stats, peak, peak_src, steps=1, exclude=("reduce", "init", "tc_compose")):
    """Dominant kernel class (by device time) as an HBM-bound kernel: algorithmic bytes (2 x state bytes per
    full pass, the touched fraction for elementwise passes) per launch over its average launch time."""
    kern = {k: v for k, v in stats.items() if k not in exclude and v["launches"]}
    dom = max(kern, key=lambda k: kern[k]["total_ms"])
    s = kern[dom]
    per_launch = s["alg_bytes"] / s["launches"]
    avg_ms = s["total_ms"] / s["launches"]
    achieved = per_launch / (avg_ms * 1e-3) / 1e9
    total = sum(v["total_ms"] for v in stats.values())
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": load_traffic(dom), "kernel": dom, "peak_source": peak_src,
            "launches": s["launches"] // max(1, steps), "share_of_kernel_time": s["total_ms"] / total if total else None,
            "alg_bytes_per_launch": per_launch, "avg_launch_ms": avg_ms}


DOT2_FP32_OPS = 12  # FP32 operations of one float-float multiply-add in the compensated dot product (dot2_step)


def roofline_alu(stats, prec_name, fp32_fma, fp64_fma, kernel="fused_stage", traffic_key=None):
    """The fused stage as an arithmetic-bound kernel: the real multiply-adds its sweeps perform (the library's
    count: structured for FP64 and float-float, dense complex FMAs for complex64) per second of device time,
    against the measured FMA rate of the pipe that executes them.  A float-float multiply-add (one step of the
    compensated dot product) takes 12 FP32 operations, each one issue slot of the FP32 pipe, so its peak is the
    FP32 FMA rate / 12."""
    s = stats.get(kernel)
    if not s or not s["launches"] or not s.get("alg_fma"):
        return None
    achieved = s["alg_fma"] / (s["total_ms"] * 1e-3)
    peak, unit, src = {"split": (fp32_fma / DOT2_FP32_OPS, "float-float multiply-adds/s",
                                 f"measured FP32 FMA rate / {DOT2_FP32_OPS}"),
                       "f64": (fp64_fma, "FP64 multiply-adds/s", "measured FP64 FMA rate"),
                       "f32": (fp32_fma, "FP32 multiply-adds/s", "measured FP32 FMA rate")}[prec_name]
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "kernel": kernel, "peak_source": src, "launches": s["launches"],
            "avg_launch_ms": s["total_ms"] / s["launches"], "alg_fma_per_launch": s["alg_fma"] / s["launches"],
            "alg_bytes_per_launch": s["alg_bytes"] / s["launches"],
            "traffic": load_traffic(traffic_key) if traffic_key else None}


def fp64_alu_roofline(stats, fma_rate):
    """Plain FP64 passes as FP64-arithmetic-bound kernels: the real multiply-adds their structured arithmetic
    issues (the library's count, from the coefficients' zero/one/real/imaginary structure) per second of
    device time, against the FP64 FMA rate measured on this GPU (vqd_measure_fma_rate)."""
    out = {}
    for k, v in stats.items():
        if k in ("reduce", "init") or not v["launches"] or not v.get("alg_fma"):
            continue
        achieved = v["alg_fma"] / (v["total_ms"] * 1e-3)
        out[k] = {"bound": "alu", "achieved": achieved, "peak": fma_rate, "unit": "FP64 FMA/s",
                  "frac": achieved / fma_rate, "peak_source": "measured (vqd_measure_fma_rate)",
                  "hbm_frac": (v["alg_bytes"] / (v["total_ms"] * 1e-3) / 1e9)}
    return out


def per_class(stats, steps=1):
    return {k: {"launches": v["launches"] // max(1, steps), "avg_ms": v["total_ms"] / v["launches"]}
            for k, v in stats.items() if v["launches"]}


def timed_steps(torch, vqd, stream, ctx, step, steps, warmup, clocks=None, sync=None):
    """Warm-up steps, then `steps` steps between CUDA events on the context's stream (no per-launch accounting
    inside the timed region); returns (ms, clock record)."""
    for _ in range(warmup):
        step()
    vqd.vqd_profile(ctx, 0)
    (sync or torch.cuda.synchronize)()
    if clocks:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop() if clocks else None
    return e0.elapsed_time(e1), ck


def profiled_step(torch, vqd, ctx, step):
    """One step with every launch timed by CUDA events (the library's accounting): per-class device times."""
    vqd.vqd_profile(ctx, 2)
    vqd.vqd_profile_reset(ctx)
    step()
    torch.cuda.synchronize()
    st = vqd.vqd_profile_read(ctx)
    vqd.vqd_profile(ctx, 0)
    return st


def make_step(vqd, ctx, n, native, path, fuse=0, tc=None, flags=0):
    def step():
        vqd.vqd_init_zero(ctx, 0)
        if path == "plain":
            vqd.vqd_apply_native(ctx, 0, native)
        elif path == "fused":
            vqd.vqd_run_program(ctx, 0, native, fuse, flags)
        else:
            vqd.vqd_run_program_tc(ctx, 0, native, tc[0], tc[1])
        vqd.vqd_prob(ctx, 0, list(range(n)))
        vqd.vqd_trace(ctx, 0)
        vqd.vqd_purity(ctx, 0)
    return step


def tensor_roofline(stats, n, k, scheme, bf16_peak_tflops):
    """tcgen05 blocks against the tensor pipe: algorithmic flops of one block application are the real GEMM's
    2 x 4^(n-k) groups x (2 4^k)^2, times the split products (3 for 3xTF32, 6 for BF16x3); the peak is the
    measured dense BF16 rate, halved for TF32 (the nominal ratio of the two, 1.1 vs 2.25 PFLOP/s)."""
    s = stats.get("tc_gemm")
    if not s or not s["launches"]:
        return None
    nprod = 3 if scheme == 0 else 6
    flops = 2.0 * 4 ** (n - k) * (2 * 4 ** k) ** 2 * nprod
    avg_ms = s["total_ms"] / s["launches"]
    peak = bf16_peak_tflops * (0.5 if scheme == 0 else 1.0)
    achieved = flops / (avg_ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "kernel": "tc_gemm (k_tc_block)", "launches": s["launches"], "avg_launch_ms": avg_ms,
            "flops_per_launch": flops, "peak_source": "measured bf16" + (" x 0.5 (TF32)" if scheme == 0 else ""),
            "hbm_GBps_per_launch": s["alg_bytes"] / s["launches"] / (avg_ms * 1e-3) / 1e9}


def measure_trajectories(vqd, torch, prog, native, stream_handle, ntraj=1024):
    """The same program as Monte-Carlo statevector trajectories (one CTA per trajectory, statevector in shared
    memory): <sum_q Z_q> estimated from `ntraj` trajectories against the density-matrix value."""
    import numpy as np
    n = prog.n
    codes = np.zeros((n, n), np.uint8)
    for q in range(n):
        codes[q, q] = 3
    coeffs = np.ones(n)
    t0 = time.perf_counter()
    vals, mean, se = vqd.vqd_traj_expect(n, vqd.VQD_F32, native, ntraj, 2024, codes, coeffs, 0, stream_handle)
    wall = time.perf_counter() - t0
    ctx = vqd.vqd_create(n, vqd.VQD_F32, stream_handle)
    try:
        vqd.vqd_run_program(ctx, 0, native)
        exact = vqd.vqd_expect(ctx, 0, codes, coeffs)
    finally:
        vqd.vqd_destroy(ctx)
    return {"trajectories": ntraj, "seconds": wall, "trajectories_per_s": ntraj / wall,
            "statevector_amp_updates_per_s": ntraj * len(native) * 2.0 ** n / wall,
            "observable": "sum_q Z_q", "mean": mean, "stderr": se, "density_matrix_value": exact,
            "z_score": (mean - exact) / se if se > 0 else None}


def measure_trajectories_spin16(vqd, stream_handle, ntraj=256):
    """Trajectories where the density matrix is 34 GB: the 16-qubit spin chain (4000 native ops) as
    complex64 statevectors of 512 KB, each spread over a cluster of 8 CTAs (distributed shared memory).
    Reported: <sum_q Z_q> with its standard error, and throughput."""
    import numpy as np
    from workloads import config5_spin_chain
    prog = config5_spin_chain()
    n = prog.n
    native = vqd.native_ops(prog.ops)
    codes = np.zeros((n, n), np.uint8)
    for q in range(n):
        codes[q, q] = 3
    coeffs = np.ones(n)
    vqd.vqd_traj_expect(n, vqd.VQD_F32, native[:50], 8, 1, codes, coeffs, 0, stream_handle)   # warm-up
    t0 = time.perf_counter()
    vals, mean, se = vqd.vqd_traj_expect(n, vqd.VQD_F32, native, ntraj, 2025, codes, coeffs, 0, stream_handle)
    wall = time.perf_counter() - t0
    return {"trajectories": ntraj, "seconds": wall, "trajectories_per_s": ntraj / wall,
            "statevector_amp_updates_per_s": ntraj * len(native) * 2.0 ** n / wall,
            "native_ops": len(native), "observable": "sum_q Z_q", "mean": mean, "stderr": se,
            "note": "16-qubit statevectors on 8-CTA clusters; the density matrix (34 GB) is the plain path's"}


def measure_sc_device(vqd, torch, stream_handle, timed, steps, flags=0):
    """A second workload: the superconducting device model of Sec. 8 on a 2x7 transmon grid (App. C
    parameter ranges), a depth-60 hardware-efficient ansatz compiled by vqd_sc_compile (static ZZ on every
    coupling, thermal T1/T2 decay, readout noise), run through the fused path in complex64 from the
    thermal initial state."""
    from workloads.devices import sc_ansatz, sc_grid_device
    dev = sc_grid_device(2, 7)
    logical = sc_ansatz(dev, 60)
    t0 = time.perf_counter()
    native = vqd.vqd_sc_compile(dev, logical, readout=True)
    compile_s = time.perf_counter() - t0
    n = int(dev["n"])
    ctx = vqd.vqd_create(n, vqd.VQD_F32, stream_handle)
    try:
        def step():
            vqd.vqd_init_product_diag(ctx, 0, dev["excited"])
            vqd.vqd_run_program(ctx, 0, native, 0, flags)
            vqd.vqd_prob(ctx, 0, list(range(n)))
            vqd.vqd_trace(ctx, 0)
        ms, st, _ = timed(step, steps, 1, ctx)
        units = len(native) * 4.0 ** n
        return {"value": steps * units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                "logical_gates": len(logical), "native_ops": len(native), "host_compile_s": compile_s,
                "stages_per_step": st.get("fused_stage", {}).get("launches", 0) // steps,
                "hermitian_stages": bool(flags),
                "note": "fused path, default fusion width 6; amp-updates counted over the compiled native ops"}
    finally:
        vqd.vqd_destroy(ctx)


def measure_nv_noise_sweep(vqd, torch, count=256, props=16):
    """A second workload with the shape of the paper's NV-centre study (Sec. 5): a 5-qubit NV centre (App. C
    table) running BCS-shaped propagators of 200 native gates, swept over `count` noise scales (log-uniform
    0.1..10).  Each scale is one instance of one batched run (stage waves replayed as a CUDA graph)."""
    import numpy as np
    from workloads.devices import NV5, nv_bcs_shape, nv_scaled
    scales = np.logspace(-1, 1, count)
    logical = nv_bcs_shape(NV5, props, 200)
    t0 = time.perf_counter()
    arrays = [vqd.vqd_nv_compile(nv_scaled(NV5, float(sc)), logical, readout=True) for sc in scales]
    compile_s = time.perf_counter() - t0
    units = sum(len(a) * 4.0 ** 5 for a in arrays)
    bstream = torch.cuda.Stream()
    ctx = vqd.vqd_create_batch([5] * count, vqd.VQD_F32, bstream.cuda_stream)
    try:
        t0 = time.perf_counter()
        vqd.vqd_run_batch(ctx, arrays)
        bstream.synchronize()
        first = time.perf_counter() - t0
        t0 = time.perf_counter()
        for i in range(count):
            vqd.vqd_init_zero(ctx, i)
        vqd.vqd_run_batch(ctx, arrays)
        probs, trs, purs = vqd.vqd_batch_reduce(ctx, [5] * count)
        wall = time.perf_counter() - t0
        p1 = [float(pr.reshape(-1)[1::2].sum()) for pr in probs]   # electron reads 1
        return {"value": units / wall, "unit": UNIT, "instances": count, "logical_gates": len(logical),
                "native_ops_per_instance": int(np.mean([len(a) for a in arrays])), "host_compile_s": compile_s,
                "first_run_s": first, "wall_s": wall,
                "electron_p1_at_scales": {f"{scales[i]:.3g}": p1[i] for i in (0, count // 2, count - 1)},
                "note": "complex64; value = re-initialise, one graph replay of the batch, batched reductions"}
    finally:
        vqd.vqd_destroy(ctx)



def device_view(torch, ptr: int, count: int, prec_f32: bool):
    """Zero-copy complex torch view of `count` amplitudes at a library device address (measurement only)."""
    class _A:
        pass
    a = _A()
    a.__cuda_array_interface__ = {"shape": (2 * count,), "typestr": "<f4" if prec_f32 else "<f8",
                                  "data": (ptr, False), "version": 3}
    t = torch.as_tensor(a, device="cuda")
    return torch.view_as_complex(t.view(-1, 2))



def split_view(torch, ptr: int, count: int):
    """Zero-copy view of a float-float state as (count, 4) float32 rows: re.hi, re.lo, im.hi, im.lo."""
    class _A:
        pass
    a = _A()
    a.__cuda_array_interface__ = {"shape": (4 * count,), "typestr": "<f4", "data": (ptr, False), "version": 3}
    return torch.as_tensor(a, device="cuda").view(-1, 4)



def run_precision(args):
    """Error of the complex64 and float-float plain and fused paths against the FP64 plain path on one
    workload."""
    import numpy as np
    import torch
    from paper_2306_07342_gb300 import build as _b
    _b.build()
    from paper_2306_07342_gb300 import vqd
    from workloads import config2_sc_grid, config3_ion_alltoall, config5_spin_chain
    prog = {"sc_grid14": config2_sc_grid, "ion15": config3_ion_alltoall, "spin16": config5_spin_chain}[args.precision]()
    ops = prog.ops[: args.prefix] if args.prefix else prog.ops
    native = vqd.native_ops(ops)
    n = prog.n
    N = 4 ** n
    sh = torch.cuda.current_stream().cuda_stream
    out = {"workload": args.precision, "n": n, "native_ops": len(ops)}

    def run(prec, path, fuse=0):
        ctx = vqd.vqd_create(n, prec, sh)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if path == "plain":
            vqd.vqd_apply_native(ctx, 0, native)
        else:
            vqd.vqd_run_program(ctx, 0, native, fuse)
        torch.cuda.synchronize()
        return ctx, time.perf_counter() - t0

    ref, t64 = run(vqd.VQD_F64, "plain")
    r = device_view(torch, vqd.vqd_state_ptr(ref, 0), N, False)
    p_ref = vqd.vqd_prob(ref, 0, list(range(n)))
    pur_ref = vqd.vqd_purity(ref, 0)
    out["f64_plain_s"] = t64
    out["f64_trace"] = vqd.vqd_trace(ref, 0).real
    out["f64_purity"] = pur_ref
    runs = [(vqd.VQD_F32, "plain", 0), (vqd.VQD_F32, "fused", 4), (vqd.VQD_F32, "fused", 5),
            (vqd.VQD_F32, "fused", 6), (vqd.VQD_F32_SPLIT, "plain", 0), (vqd.VQD_F32_SPLIT, "fused", 6)]
    for prec, path, fuse in runs:
        ctx, t = run(prec, path, fuse)
        split = prec == vqd.VQD_F32_SPLIT
        x = (split_view(torch, vqd.vqd_state_ptr(ctx, 0), N) if split
             else device_view(torch, vqd.vqd_state_ptr(ctx, 0), N, True))
        maxabs, fro2, tr_rs = 0.0, 0.0, 0.0
        chunk = 1 << 26
        for i in range(0, N, chunk):
            a = r[i:i + chunk]
            if split:
                w = x[i:i + chunk].to(torch.float64)
                b = torch.complex(w[:, 0] + w[:, 1], w[:, 2] + w[:, 3])
            else:
                b = x[i:i + chunk].to(torch.complex128)
            d = b - a
            maxabs = max(maxabs, float(d.abs().max()))
            fro2 += float((d.real ** 2 + d.imag ** 2).sum())
            tr_rs += float((a.conj() * b).real.sum())      # tr(rho sigma) for Hermitian rho, sigma
        p = vqd.vqd_prob(ctx, 0, list(range(n)))
        pur = vqd.vqd_purity(ctx, 0)
        sup_fid = tr_rs + np.sqrt(max(0.0, (1 - pur_ref) * (1 - pur)))
        key = ("split_" if split else "c64_") + ("plain" if path == "plain" else f"fused_f{fuse}")
        out[key] = {"seconds": t, "max_abs": maxabs, "frobenius": fro2 ** 0.5,
                    "trace_distance_bound": 0.5 * 2 ** (n / 2) * fro2 ** 0.5,
                    "prob_tv_distance": 0.5 * float(np.abs(p - p_ref).sum()),
                    "trace_err": abs(vqd.vqd_trace(ctx, 0).real - out["f64_trace"]),
                    "purity_err": abs(pur - pur_ref), "super_fidelity": sup_fid}
        vqd.vqd_destroy(ctx)
        torch.cuda.empty_cache()
    vqd.vqd_destroy(ref)
    print(json.dumps(out), flush=True)


def measure_ion15(torch, vqd, stream, bf16_peak):
    """The 15-qubit ion-trap program (800 gates: XX on random pairs and R(theta, phi), dephasing after each;
    2000 native ops; complex64 8.6 GB): fused k-qubit blocks on the tensor cores (3xTF32 for k = 4, 5, 6 and
    BF16x3 for k = 4) and the CUDA-core fused path, each with its error against the plain FP64 run."""
    from workloads import config3_ion_alltoall
    prog = config3_ion_alltoall()
    n = prog.n
    native = vqd.native_ops(prog.ops)
    units = len(native) * 4.0 ** n
    sh = stream.cuda_stream
    out = {"workload": "ion-trap all-to-all, 15 qubits, 800 gates (2000 native ops)", "native_ops": len(native)}
    ref = vqd.vqd_create(n, vqd.VQD_F64, sh)
    try:
        ms, _ = timed_steps(torch, vqd, stream, ref, make_step(vqd, ref, n, native, "plain"), 1, 0)
        out["plain_f64"] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms}
        runs = [("tc_3xtf32_k4", "tc", (4, 0)), ("tc_bf16x3_k4", "tc", (4, 1)), ("tc_3xtf32_k5", "tc", (5, 0)),
                ("tc_3xtf32_k6", "tc", (6, 0)), ("fused_c64", "fused", None)]
        for name, path, tc in runs:
            ctx = vqd.vqd_create(n, vqd.VQD_F32, sh)
            try:
                step = make_step(vqd, ctx, n, native, path, tc=tc)
                if path == "fused":
                    step()
                # one step with the library's per-launch CUDA events (a tensor-core block is one long launch,
                # so the events add nothing measurable); its wall time is the step time
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = profiled_step(torch, vqd, ctx, step)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                rec = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                       "error_vs_plain_f64": state_error(torch, vqd, ref, vqd.VQD_F64, ctx, vqd.VQD_F32)}
                rec["per_class"] = per_class(st)
                if tc:
                    rec["blocks"] = vqd.vqd_tc_plan_info(n, native, tc[0])["blocks"]
                    rec["roofline"] = tensor_roofline(st, n, tc[0], tc[1], bf16_peak)
                out[name] = rec
            finally:
                vqd.vqd_destroy(ctx)
                torch.cuda.empty_cache()
    finally:
        vqd.vqd_destroy(ref)
    return out


def measure_spin16(torch, vqd, stream, herm=0):
    """The 16-qubit spin chain (2000 gates, 4000 native ops), the largest single-GPU configuration: the density
    matrix is 34.4 GB in complex64 and 68.7 GB in float-float.  Both through the fused path, once each;
    complex64's error is stated against the float-float run (FP64-class: float-float is within 1e-13 of FP64
    on the 14-qubit program)."""
    from workloads import config5_spin_chain
    prog = config5_spin_chain()
    n = prog.n
    native = vqd.native_ops(prog.ops)
    units = len(native) * 4.0 ** n
    sh = stream.cuda_stream
    out = {"workload": "silicon-spin / NV-like chain, 16 qubits, 2000 gates (4000 native ops)", "native_ops": len(native)}
    ref = vqd.vqd_create(n, vqd.VQD_F32_SPLIT, sh)
    try:
        ms, _ = timed_steps(torch, vqd, stream, ref, make_step(vqd, ref, n, native, "fused", flags=herm), 1, 0)
        out["fused_split"] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                              "state_bytes": vqd.vqd_state_bytes(n, vqd.VQD_F32_SPLIT)}
        ctx = vqd.vqd_create(n, vqd.VQD_F32, sh)
        try:
            step = make_step(vqd, ctx, n, native, "fused")
            ms, _ = timed_steps(torch, vqd, stream, ctx, step, 1, 0)
            out["fused_c64"] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                                "state_bytes": vqd.vqd_state_bytes(n, vqd.VQD_F32),
                                "error_vs_fused_split": state_error(torch, vqd, ref, vqd.VQD_F32_SPLIT, ctx, vqd.VQD_F32)}
        finally:
            vqd.vqd_destroy(ctx)
    finally:
        vqd.vqd_destroy(ref)
        torch.cuda.empty_cache()
    return out


def measure_batch(vqd, torch, count, herm=0):
    """Neutral-atom-like batch: `count` instances with n ~ U{6..12} in one batched run (stage waves of persistent
    kernels replayed as one CUDA graph), with the fusion width and tile shape picked by the batch autotuner
    (candidates timed on the batch itself), against one launch sequence per instance (fused and plain) on every
    16th instance, scaled to the batch."""
    import numpy as np
    from paper_2306_07342_gb300 import autotune
    from workloads import config4_neutral_batch
    progs = config4_neutral_batch(count=count)
    arrays = [vqd.native_ops(p.ops) for p in progs]
    ns = [p.n for p in progs]
    units = sum(len(p.ops) * 4.0 ** p.n for p in progs)
    bstream = torch.cuda.Stream()                          # a capturable stream: the batch becomes a CUDA graph
    choice = autotune.tune_batch(ns, vqd.VQD_F32, arrays, bstream.cuda_stream, flags=herm)
    herm = choice["flags"]
    ctx = vqd.vqd_create_batch(ns, vqd.VQD_F32, bstream.cuda_stream)
    try:
        fuse = autotune.apply(ctx, choice)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vqd.vqd_run_batch(ctx, arrays, fuse, herm)           # first run: compile, plan, capture, launch
        torch.cuda.synchronize()
        first_wall = time.perf_counter() - t0
        vqd.vqd_profile(ctx, 2)
        vqd.vqd_profile_reset(ctx)
        t0 = time.perf_counter()
        for i in range(count):
            vqd.vqd_init_zero(ctx, i)
        vqd.vqd_run_batch(ctx, arrays, fuse, herm)           # same batch again: one graph launch
        bstream.synchronize()
        t1 = time.perf_counter()
        probs, trs, purs = vqd.vqd_batch_reduce(ctx, ns)     # every instance's results, one launch, one read-back
        wall = time.perf_counter() - t0
        reduce_wall = time.perf_counter() - t1
        assert np.abs(trs - 1).max() < 1e-3 and all(abs(p.sum() - 1) < 1e-3 for p in probs)
        st = vqd.vqd_profile_read(ctx)["batch"]
        vqd.vqd_profile(ctx, 0)
        kern_s = st["total_ms"] * 1e-3
        sample = list(range(0, count, 16))
        sunits = sum(len(progs[i].ops) * 4.0 ** progs[i].n for i in sample)
        res = {}
        for path in ("fused", "plain"):
            for i in sample[:2]:
                if path == "fused":
                    vqd.vqd_run_program(ctx, i, arrays[i], fuse, herm)
                else:
                    vqd.vqd_apply_native(ctx, i, arrays[i])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in sample:
                if path == "fused":
                    vqd.vqd_run_program(ctx, i, arrays[i], fuse, herm)
                else:
                    vqd.vqd_apply_native(ctx, i, arrays[i])
            torch.cuda.synchronize()
            w = time.perf_counter() - t0
            res[path] = {"value": sunits / w, "scaled_batch_s": w * units / sunits}
        return {"value": units / wall, "unit": UNIT, "kernel_value": units / kern_s,
                "first_run_value": units / first_wall, "first_run_s": first_wall,
                "instances": count, "native_ops": int(sum(len(a) for a in arrays)), "amp_updates": units,
                "kernel_s": kern_s, "wall_s": wall, "batch_reduce_s": reduce_wall,
                "autotuned": {k: choice[k] for k in ("fuse_qubits", "tile_bits", "passenger_bits", "hermitian")},
                "autotune_trials": choice["trials"],
                "state_bytes": int(sum(vqd.vqd_state_bytes(n, vqd.VQD_F32) for n in ns)),
                "one_launch_sequence_per_instance": {
                    "instances_timed": len(sample), **res,
                    "note": "every 16th instance timed one launch sequence after another; value = their amp-updates "
                            "over their wall clock, scaled_batch_s = that rate applied to the whole batch"},
                "note": "value = wall clock of re-initialising every state, one vqd_run_batch of a batch seen before "
                        "(one CUDA-graph launch of all stage waves) and one vqd_batch_reduce reading every instance's "
                        "probabilities, trace and purity back to the host; first_run_value includes host compile, "
                        "fusion planning and graph capture; kernel_value = CUDA-event time of the waves only"}
    finally:
        vqd.vqd_destroy(ctx)


def run_fp64_diag():
    """FP64 elementwise passes on a 14-qubit complex128 state: a real diagonal superoperator that changes every
    amplitude, a dephasing and an Rz (both leave half of the amplitudes untouched); 20 timed passes each after 3
    warm-up passes, CUDA events through the library's launch accounting."""
    import numpy as np
    import torch
    from paper_2306_07342_gb300 import build as _b
    _b.build()
    from paper_2306_07342_gb300 import vqd
    from workloads.circuits import NativeOp
    n = 14
    ctx = vqd.vqd_create(n, vqd.VQD_F64, torch.cuda.current_stream().cuda_stream)
    real = np.diag([0.9, 0.8, 0.7, 0.6]).astype(complex)
    cases = {"real_full": lambda: vqd.vqd_apply_superop(ctx, 0, [7], real),
             "deph_half": lambda: vqd.vqd_apply_native(ctx, 0, [NativeOp("deph1", (7,), (0.1,))]),
             "rz_complex_half": lambda: vqd.vqd_apply_native(ctx, 0, [NativeOp("rz", (7,), (0.3,))])}
    out = {"fp64_fma_per_s": vqd.vqd_measure_fma_rate(0), "fp32_fma_per_s": vqd.vqd_measure_fma_rate(1)}
    try:
        for name, f in cases.items():
            for _ in range(3):
                f()
            torch.cuda.synchronize()
            vqd.vqd_profile(ctx, 2)
            vqd.vqd_profile_reset(ctx)
            for _ in range(20):
                f()
            torch.cuda.synchronize()
            st = vqd.vqd_profile_read(ctx)["elem"]
            vqd.vqd_profile(ctx, 0)
            ms = st["total_ms"] / st["launches"]
            out[name] = {"avg_ms": ms, "alg_GBps": st["alg_bytes"] / st["launches"] / (ms * 1e-3) / 1e9}
    finally:
        vqd.vqd_destroy(ctx)
    print(json.dumps(out), flush=True)


def run_tc_case(args):
    """The ion-trap program through the tensor-core blocks on a chosen size: per scheme and k, the block
    kernel's average time (the library's CUDA events)."""
    import torch
    from paper_2306_07342_gb300 import build as _b
    _b.build()
    from paper_2306_07342_gb300 import vqd
    from workloads import config3_ion_alltoall
    n, gates = args.tc_case
    prog = config3_ion_alltoall(n=n, n_gates=gates)
    native = vqd.native_ops(prog.ops)
    ctx = vqd.vqd_create(n, vqd.VQD_F32, torch.cuda.current_stream().cuda_stream)
    out = {"n": n, "native_ops": len(native)}
    try:
        for k, sc in ((4, vqd.VQD_TC_3XTF32), (4, vqd.VQD_TC_BF16X3), (5, vqd.VQD_TC_3XTF32)):
            vqd.vqd_run_program_tc(ctx, 0, native[:20], k, sc)
            vqd.vqd_profile(ctx, 2)
            vqd.vqd_profile_reset(ctx)
            vqd.vqd_run_program_tc(ctx, 0, native, k, sc)
            st = vqd.vqd_profile_read(ctx)
            vqd.vqd_profile(ctx, 0)
            g = st["tc_gemm"]
            out[f"k{k}_{'3xtf32' if sc == 0 else 'bf16x3'}"] = {"blocks": g["launches"], "gemm_ms_avg": g["total_ms"] / g["launches"],
                                                            "compose_ms_total": st["tc_compose"]["total_ms"]}
    finally:
        vqd.vqd_destroy(ctx)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.tc_case:
        run_tc_case(args)
        return
    if args.fp64_diag:
        run_fp64_diag()
        return
    if args.precision:
        run_precision(args)
        return
    if args.oracle_plan:
        run_oracle_plan(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2306_07342_gb300 import build as _b
    if rank == 0:
        _b.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2306_07342_gb300 import autotune, replicas, vqd
    from workloads import config2_sc_grid

    prog = config2_sc_grid(rows=args.rows, cols=args.cols, depth=args.depth)
    n = prog.n
    native = vqd.native_ops(prog.ops)
    units_per_step = len(prog.ops) * 4.0 ** n
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    def sync_all():
        torch.cuda.synchronize()
        replicas.barrier()

    prec = {"split": vqd.VQD_F32_SPLIT, "f64": vqd.VQD_F64, "f32": vqd.VQD_F32}[args.prec]
    layer_ops = len(prog.ops) // prog.meta["depth"]
    # every state here is a density matrix: the fused paths use its Hermiticity (VQD_HERMITIAN)
    herm = 0 if args.general else vqd.VQD_HERMITIAN

    # ---- headline: the FP64-class fused path (float-float) on the full program
    ctx = vqd.vqd_create(n, prec, sh)
    fuse = 0
    choice = None
    if args.path == "fused" and not args.fixed_shape:
        choice = autotune.tune(n, prec, native, sh, prefix=3 * layer_ops, flags=herm)   # outside the timed region
        fuse = autotune.apply(ctx, choice)
    run_flags = choice["flags"] if choice else (herm if args.path == "fused" else 0)
    step = make_step(vqd, ctx, n, native, args.path, fuse, flags=run_flags)
    clocks = ClockSampler(local)
    ms, ck = timed_steps(torch, vqd, stream, ctx, step, args.steps, args.warmup, clocks, sync_all)
    ms = replicas.max_over_ranks(ms)
    value = world * args.steps * units_per_step / (ms * 1e-3)
    stats = profiled_step(torch, vqd, ctx, step)                         # per-class times, outside the timed region
    fp64_fma = vqd.vqd_measure_fma_rate(0, sh)
    fp32_fma = vqd.vqd_measure_fma_rate(1, sh)
    roof_hbm = roofline_hbm(stats, hbm_peak, peak_src)
    # DRAM bytes per launch from a committed ncu capture of this kernel (profiles/traffic.json), if current
    tkey = f"fused_stage_{args.prec}" + ("_herm" if run_flags & vqd.VQD_HERMITIAN else "")
    roof_alu = roofline_alu(stats, args.prec, fp32_fma, fp64_fma, traffic_key=tkey) if args.path == "fused" else None
    # the fused stage is bound by its arithmetic, not by HBM: its roofline is the arithmetic one
    roof = roof_alu if roof_alu else roof_hbm
    launches = int(sum(v["launches"] for v in stats.values()))

    # ---- end to end through the C ABI with host buffers (wall clock; results read back every step)
    e2e_steps = min(args.steps, 3)
    sync_all()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step()
    torch.cuda.synchronize()
    e2e_s = replicas.max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * e2e_steps * units_per_step / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(native.nbytes), "d2h_bytes_per_step": int(8 * 2 ** n + 16 + 8), "steps": e2e_steps,
           "note": "wall clock through vqd_init_zero/vqd_run_program/vqd_prob/vqd_trace/vqd_purity; the native op "
                   "list is a host array compiled and marshalled every step; results copied to host every step"}

    extra, error = {}, None
    if not args.no_extra:
        # ---- the plain FP64 path on the full program: the reference state for every error below
        ref = vqd.vqd_create(n, vqd.VQD_F64, sh)
        rstep = make_step(vqd, ref, n, native[:layer_ops], "plain")
        rstep()                                                           # warm-up on the first layer
        rms, _ = timed_steps(torch, vqd, stream, ref, make_step(vqd, ref, n, native, "plain"), 1, 0)
        st64 = profiled_step(torch, vqd, ref, make_step(vqd, ref, n, native[:2 * layer_ops], "plain"))
        vqd.vqd_init_zero(ref, 0)
        vqd.vqd_apply_native(ref, 0, native)
        f64_rate = units_per_step / (rms * 1e-3)
        extra["plain_f64"] = {
            "value": world * f64_rate, "unit": UNIT, "ms_per_step": rms,
            "roofline_hbm": roofline_hbm(st64, hbm_peak, peak_src),
            "roofline_fp64_alu_per_class": fp64_alu_roofline(st64, fp64_fma),
            "per_class_first_two_layers": per_class(st64),
            "fp64_fma_per_s_measured": fp64_fma, "fp32_fma_per_s_measured": fp32_fma,
            "note": "complex128 plain kernels (one pass per native op), the full program; per-class times from a "
                    "profiled pass over the first two layers"}
        error = state_error(torch, vqd, ref, vqd.VQD_F64, ctx, prec)
        error["vs"] = "plain FP64 (complex128) run of the same program on the same GPU"
        # ---- the other paths on the full program, each with its error against the FP64 state
        paths = [("fused_f64", vqd.VQD_F64, "fused", 1, herm), ("plain_split", vqd.VQD_F32_SPLIT, "plain", 1, 0),
                 ("fused_c64", vqd.VQD_F32, "fused", min(args.steps, 5), herm), ("plain_c64", vqd.VQD_F32, "plain", 2, 0)]
        if herm:   # the same fused paths without the Hermitian stages
            paths += [("fused_split_general", vqd.VQD_F32_SPLIT, "fused", 1, 0),
                      ("fused_f64_general", vqd.VQD_F64, "fused", 1, 0),
                      ("fused_c64_general", vqd.VQD_F32, "fused", min(args.steps, 5), 0)]
        for name, pp, path, nsteps, fl in paths:
            if pp == prec and path == args.path and fl == herm:
                continue
            c2 = vqd.vqd_create(n, pp, sh)
            try:
                f2 = 0
                tuned = None
                if path == "fused":
                    tuned = autotune.tune(n, pp, native, sh, prefix=(10 if pp == vqd.VQD_F32 else 3) * layer_ops,
                                          flags=fl)
                    f2 = autotune.apply(c2, tuned)
                    fl = tuned["flags"]
                s2 = make_step(vqd, c2, n, native, path, f2, flags=fl)
                ms2, _ = timed_steps(torch, vqd, stream, c2, s2, nsteps, 1 if nsteps > 1 else 0)
                rec = {"value": world * nsteps * units_per_step / (ms2 * 1e-3), "unit": UNIT, "ms_per_step": ms2 / nsteps,
                       "steps": nsteps, "error_vs_plain_f64": state_error(torch, vqd, ref, vqd.VQD_F64, c2, pp)}
                rec["speedup_vs_plain_f64"] = rec["value"] / (world * f64_rate)
                if tuned:
                    rec["autotuned"] = {k: tuned[k] for k in ("fuse_qubits", "tile_bits", "passenger_bits")}
                if path == "fused":
                    rec["hermitian_stages"] = bool(fl & vqd.VQD_HERMITIAN)
                if path == "fused":  # per-class accounting from one more step, outside the timed region
                    st2 = profiled_step(torch, vqd, c2, s2)
                    rec["roofline"] = roofline_hbm(st2, hbm_peak, peak_src)
                    rec["roofline_alu"] = roofline_alu(st2, {vqd.VQD_F32: "f32", vqd.VQD_F64: "f64",
                                                             vqd.VQD_F32_SPLIT: "split"}[pp], fp32_fma, fp64_fma)
                    rec["stages_per_step"] = st2.get("fused_stage", {}).get("launches", 0)
                extra[name] = rec
            finally:
                vqd.vqd_destroy(c2)
        vqd.vqd_destroy(ref)
        torch.cuda.empty_cache()
    headline_rec = {"speedup_vs_plain_f64": (value / extra["plain_f64"]["value"]) if "plain_f64" in extra else None,
                    "hermitian_stages": bool(run_flags & vqd.VQD_HERMITIAN)}
    if "fused_split_general" in extra and args.prec == "split":
        headline_rec["speedup_vs_fused_general"] = value / extra["fused_split_general"]["value"]
    if choice:
        headline_rec["autotuned"] = {k: choice[k] for k in ("fuse_qubits", "tile_bits", "passenger_bits", "hermitian")}
    vqd.vqd_destroy(ctx)
    torch.cuda.empty_cache()

    if not args.no_extra and not args.no_large:
        extra["ion15_tensor_core"] = measure_ion15(torch, vqd, stream, bf16_peak)
        extra["spin16"] = measure_spin16(torch, vqd, stream, herm)
    if not args.no_extra:
        extra["trajectories_c64"] = measure_trajectories(vqd, torch, prog, native, sh)
        extra["sc_device_compiled_c64"] = measure_sc_device(vqd, torch, sh, timed_legacy(torch, vqd, stream), 3)
        extra["trajectories_spin16_c64"] = measure_trajectories_spin16(vqd, sh)
        extra["nv5_noise_sweep_batch_c64"] = measure_nv_noise_sweep(vqd, torch)
        if args.batch_count > 0:
            extra["batch_c64"] = measure_batch(vqd, torch, args.batch_count, herm)

    cpu = None
    if rank == 0 and not args.no_extra:
        blk = cpu_baseline_block(quick=True)
        grid_all = next(l for l in blk["lines"] if l["config"].startswith("sc_grid14") and l["threads"] > 1)
        cpu = {"value": grid_all["value"], "unit": UNIT, "cores": grid_all["threads"], "kind": "oracle",
               "sample": f"first {grid_all['ops_timed']} native ops of the 14-qubit program at full size, FP64 oracle "
                         f"(plain C loops, {grid_all['threads']} threads), {grid_all['seconds']:.1f} s",
               "lines": blk["lines"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": PREC_NAMES[args.prec], "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_qubits": n, "native_ops": len(prog.ops),
                       "path": f"{args.path} ({'float-float pairs' if args.prec == 'split' else args.prec})",
                       "state_bytes": vqd.vqd_state_bytes(n, prec),
                       "l2": "inputs larger than L2 (state of 2.1-4.3 GB vs 129 MB L2), no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "error": error, "headline": headline_rec,
            "roofline": roof, "roofline_hbm": roof_hbm, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": ck, "paths": extra, "per_class": per_class(stats),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def timed_legacy(torch, vqd, stream):
    """Timer with the per-class accounting of the side workloads: (ms, stats, None)."""
    def timed(step, steps, warmup, ctx):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        vqd.vqd_profile(ctx, 1)
        vqd.vqd_profile_reset(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        st = vqd.vqd_profile_read(ctx)
        vqd.vqd_profile(ctx, 0)
        return e0.elapsed_time(e1), st, None
    return timed


if __name__ == "__main__":
    main()
