#!/usr/bin/env python
"""Benchmark: density-matrix amplitude-updates per second on the 14-qubit superconducting-grid workload.

Workload: a 2 x 7 grid of transmon-like qubits (n = 14, complex64 state of 2.15 GB), depth-60 brickwork of
native ZX(pi/2) cross-resonance gates and Rz.SX.Rz layers, static ZZ crosstalk (50 kHz) on idle grid edges,
T1 log-uniform in 50-200 us with T2 = 0.7 T1 as passive decay after every sublayer, and a 2 % readout flip
(6494 native ops; seeded synthetic program from workloads.config2_sc_grid).  One step = reset to |0><0|,
the whole program through the plain unfused kernels (one pass over the state per native op), then the
FP64 reductions (14-qubit Z-basis probabilities, trace, purity) read back to the host.

Metric: amplitude-updates/s = sum over the program's native ops of 4^n, divided by the time.  The state
(2.15 GB) is larger than L2 (129 MB), so no L2 flush is needed between steps.

The JSON line also reports the fused path (stages of ops on shared-memory tiles) and the plain FP64
(complex128) path on a sample of the same program, the roofline of the dominant kernel, the oracle timed
on the host cores, and the SM clocks sampled during the timed region.

--impl reference times the FP64 numpy oracle on the host cores on a bounded sample of the same workload.
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

METRIC = "density-matrix amplitude-updates/s (sum over native ops of 4^n per second)"
UNIT = "amp-updates/s"
WORKLOAD = ("superconducting-like 2x7 grid, 14 qubits, depth-60 ZX(pi/2)+Rz/SX brickwork, ZZ crosstalk 50 kHz, "
            "T1/T2 idle decay, readout flip 2e-2; complex64 state; plain unfused kernels")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vqd", choices=["vqd", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="skip the fused / FP64 / oracle side measurements")
    ap.add_argument("--error", action="store_true", help="also measure the complex64 error against an FP64 run")
    ap.add_argument("--rows", type=int, default=2, help="grid rows (profiling cases only; the benchmark is 2x7)")
    ap.add_argument("--cols", type=int, default=7)
    ap.add_argument("--depth", type=int, default=60)
    ap.add_argument("--batch-count", type=int, default=1024, help="instances of the batched neutral-atom workload")
    ap.add_argument("--fp64-diag", action="store_true",
                    help="time FP64 elementwise passes (real full, dephasing, Rz) on a 14-qubit state and exit")
    ap.add_argument("--precision", default=None, choices=["sc_grid14", "ion15", "spin16"],
                    help="instead of timing: error of the complex64 paths against the FP64 path on one workload")
    ap.add_argument("--prefix", type=int, default=0, help="--precision: only the first N native ops (0 = all)")
    ap.add_argument("--path", default="plain", choices=["plain", "fused"],
                    help="path of the headline measurement (profiling cases; the benchmark is plain)")
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
def oracle_rate(prog, n_ops: int):
    """Time the FP64 numpy oracle on the first n_ops native ops of prog at full size."""
    from oracle import evolve
    t = time.perf_counter()
    evolve.run_program(prog, max_ops=n_ops)
    dt = time.perf_counter() - t
    return n_ops * 4.0 ** prog.n / dt, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from workloads import config2_sc_grid
    prog = config2_sc_grid()
    per_step = 2
    for _ in range(args.warmup):
        oracle_rate(prog, per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rate(prog, per_step)
    dt = time.perf_counter() - t0
    value = args.steps * per_step * 4.0 ** prog.n / dt
    cores = os.cpu_count()
    sample = f"first {per_step} native ops of the 14-qubit program at full size per step (FP64 numpy oracle)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------- GPU arm
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


def measure_sc_device(vqd, torch, stream_handle, timed, steps):
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
            vqd.vqd_run_program(ctx, 0, native)
            vqd.vqd_prob(ctx, 0, list(range(n)))
            vqd.vqd_trace(ctx, 0)
        ms, st, _ = timed(step, steps, 1, ctx)
        units = len(native) * 4.0 ** n
        return {"value": steps * units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                "logical_gates": len(logical), "native_ops": len(native), "host_compile_s": compile_s,
                "stages_per_step": st.get("fused_stage", {}).get("launches", 0) // steps,
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


def measure_batch(vqd, torch, stream_handle, count):
    """Neutral-atom-like batch: `count` instances with n ~ U{6..12} in one batched run (stage waves of
    persistent kernels), against one launch sequence per instance (fused and plain) on a sample."""
    import numpy as np
    from workloads import config4_neutral_batch
    progs = config4_neutral_batch(count=count)
    arrays = [vqd.native_ops(p.ops) for p in progs]
    ns = [p.n for p in progs]
    units = sum(len(p.ops) * 4.0 ** p.n for p in progs)
    bstream = torch.cuda.Stream()                          # a capturable stream: the batch becomes a CUDA graph
    ctx = vqd.vqd_create_batch(ns, vqd.VQD_F32, bstream.cuda_stream)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vqd.vqd_run_batch(ctx, arrays)                       # first run: compile, plan, capture, launch
        torch.cuda.synchronize()
        first_wall = time.perf_counter() - t0
        vqd.vqd_profile(ctx, 2)
        vqd.vqd_profile_reset(ctx)
        t0 = time.perf_counter()
        for i in range(count):
            vqd.vqd_init_zero(ctx, i)
        vqd.vqd_run_batch(ctx, arrays)                       # same batch again: one graph launch
        bstream.synchronize()
        t1 = time.perf_counter()
        probs, trs, purs = vqd.vqd_batch_reduce(ctx, ns)     # every instance's results, one launch, one read-back
        wall = time.perf_counter() - t0
        reduce_wall = time.perf_counter() - t1
        assert np.abs(trs - 1).max() < 1e-3 and all(abs(p.sum() - 1) < 1e-3 for p in probs)
        st = vqd.vqd_profile_read(ctx)["batch"]
        vqd.vqd_profile(ctx, 0)
        kern_s = st["total_ms"] * 1e-3
        # one launch sequence per instance, on every 16th instance (all sizes represented)
        sample = list(range(0, count, 16))
        sunits = sum(len(progs[i].ops) * 4.0 ** progs[i].n for i in sample)
        res = {}
        for path in ("fused", "plain"):
            for i in sample[:2]:
                (vqd.vqd_run_program if path == "fused" else vqd.vqd_apply_native)(ctx, i, arrays[i])
            torch.cuda.synchronize()
            vqd.vqd_profile(ctx, 2)
            vqd.vqd_profile_reset(ctx)
            t0 = time.perf_counter()
            for i in sample:
                if path == "fused":
                    vqd.vqd_run_program(ctx, i, arrays[i])
                else:
                    vqd.vqd_apply_native(ctx, i, arrays[i])
            torch.cuda.synchronize()
            w = time.perf_counter() - t0
            ps = vqd.vqd_profile_read(ctx)
            vqd.vqd_profile(ctx, 0)
            kms = sum(v["total_ms"] for k, v in ps.items() if k not in ("reduce", "init"))
            res[path] = {"value": sunits / w, "kernel_value": sunits / (kms * 1e-3),
                         "launches": int(sum(v["launches"] for v in ps.values()))}
        return {"value": units / wall, "unit": "amp-updates/s", "kernel_value": units / kern_s,
                "first_run_value": units / first_wall, "first_run_s": first_wall,
                "instances": count, "native_ops": int(sum(len(a) for a in arrays)), "amp_updates": units,
                "kernel_s": kern_s, "wall_s": wall, "host_init_replay_s": wall - reduce_wall - kern_s,
                "batch_reduce_s": reduce_wall,
                "state_bytes": int(sum(vqd.vqd_state_bytes(n, vqd.VQD_F32) for n in ns)),
                "per_instance_sample": {"instances": len(sample), **res},
                "note": "value = wall clock of re-initialising every state, one vqd_run_batch of a batch seen "
                        "before (one CUDA-graph launch of all stage waves) and one vqd_batch_reduce reading every "
                        "instance's probabilities, trace and purity back to the host; first_run_value includes host compile, "
                        "fusion planning and graph capture; kernel_value = CUDA-event time of the waves only"}
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


def fp64_alu_roof(stats, n):
    """FP64 elementwise passes as an ALU-bound kernel: a complex phase multiply is 4 FP64 instructions per
    amplitude it changes (2 DMUL + 2 DFMA; amplitudes with factor 1 are skipped), against 0.625e12 FP64 FMA
    instructions/s (the GPU's nominal 1.25 TFLOP/s FP64; no measured FP64 peak is on file)."""
    s = stats.get("elem")
    if not s or not s.get("launches"):
        return None
    per_launch_s = s["total_ms"] * 1e-3 / s["launches"]
    amps = s["alg_bytes"] / s["launches"] / 32.0        # amplitudes each launch reads and writes (16 B each way)
    achieved = 4.0 * amps / per_launch_s
    peak = 0.625e12
    return {"bound": "alu", "kernel": "elem (k_diag1/k_diag2, complex factors)", "achieved": achieved, "peak": peak,
            "unit": "FP64 instructions/s", "frac": achieved / peak, "peak_source": "nominal 1.25 TFLOP/s FP64",
            "instructions_per_changed_amplitude": 4}


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
    out = {}
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


def main():
    args = parse()
    if args.fp64_diag:
        run_fp64_diag()
        return
    if args.precision:
        run_precision(args)
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
    from paper_2306_07342_gb300 import vqd
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
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    from paper_2306_07342_gb300 import replicas

    def sync_all():
        torch.cuda.synchronize()
        replicas.barrier()

    max_over_ranks = replicas.max_over_ranks

    def make_step(ctx, path, ops=native):
        def step():
            vqd.vqd_init_zero(ctx, 0)
            if path == "plain":
                vqd.vqd_apply_native(ctx, 0, ops)
            else:
                vqd.vqd_run_program(ctx, 0, ops)
            vqd.vqd_prob(ctx, 0, list(range(n)))
            vqd.vqd_trace(ctx, 0)
            vqd.vqd_purity(ctx, 0)
        return step

    def timed(step, steps, warmup, ctx, clocks=None):
        for _ in range(warmup):
            step()
        vqd.vqd_profile(ctx, 0)
        vqd.vqd_profile_reset(ctx)
        vqd.vqd_profile(ctx, 2)
        sync_all()
        if clocks:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ck = clocks.stop() if clocks else None
        ms = max_over_ranks(e0.elapsed_time(e1))
        stats = vqd.vqd_profile_read(ctx)
        vqd.vqd_profile(ctx, 0)
        return ms, stats, ck

    def roofline(stats, steps):
        kern = {k: v for k, v in stats.items() if k not in ("reduce", "init")}
        dom = max(kern, key=lambda k: kern[k]["total_ms"])
        s = kern[dom]
        per_launch_bytes = s["alg_bytes"] / s["launches"]
        avg_ms = s["total_ms"] / s["launches"]
        achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9
        total_ms = sum(v["total_ms"] for v in stats.values())
        return dom, {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": load_traffic(dom), "kernel": dom,
                     "peak_source": peak_src, "launches": s["launches"] // max(1, steps),
                     "share_of_kernel_time": s["total_ms"] / total_ms if total_ms else None,
                     "alg_bytes_per_launch": per_launch_bytes, "avg_launch_ms": avg_ms}

    # ---- headline: plain complex64 kernels
    ctx = vqd.vqd_create(n, vqd.VQD_F32, sh)
    clocks = ClockSampler(local)
    ms, stats, ck = timed(make_step(ctx, args.path), args.steps, args.warmup, ctx, clocks)
    value = world * args.steps * units_per_step / (ms * 1e-3)
    dom, roof = roofline(stats, args.steps)
    launches = int(sum(v["launches"] for v in stats.values()) / args.steps)

    # ---- end to end through the C ABI with host buffers (wall clock; results read back every step)
    step = make_step(ctx, args.path)
    sync_all()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * args.steps * units_per_step / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(native.nbytes), "d2h_bytes_per_step": int(8 * 2 ** n + 16 + 8),
           "note": "wall clock through vqd_init_zero/vqd_apply_native/vqd_prob/vqd_trace/vqd_purity; the native "
                   "op list is a host array marshalled into kernel parameters; results copied to host every step"}

    extra = {}
    if not args.no_extra:
        # ---- fused path, complex64, with the autotuned fusion width and tile shape (tuned on the first
        # 10 layers, outside the timed region)
        from paper_2306_07342_gb300 import autotune
        layer_ops = len(prog.ops) // prog.meta["depth"]
        choice = autotune.tune(n, vqd.VQD_F32, native, sh, prefix=10 * layer_ops)
        fuse = autotune.apply(ctx, choice)

        def fused_step():
            vqd.vqd_init_zero(ctx, 0)
            vqd.vqd_run_program(ctx, 0, native, fuse)
            vqd.vqd_prob(ctx, 0, list(range(n)))
            vqd.vqd_trace(ctx, 0)
            vqd.vqd_purity(ctx, 0)

        fms, fstats, _ = timed(fused_step, args.steps, 1, ctx)
        fdom, froof = roofline(fstats, args.steps)
        extra["fused_c64"] = {"value": world * args.steps * units_per_step / (fms * 1e-3), "unit": UNIT,
                              "ms_per_step": fms / args.steps, "speedup_vs_plain": ms / fms,
                              "stages_per_step": fstats.get("fused_stage", {}).get("launches", 0) // args.steps,
                              "autotuned": {k: choice[k] for k in ("fuse_qubits", "tile_bits", "passenger_bits")},
                              "roofline": froof}
    vqd.vqd_destroy(ctx)
    if not args.no_extra:
        # ---- plain FP64 (complex128) kernels on the first two layers of the program
        layer_ops = len(prog.ops) // prog.meta["depth"]
        sample = native[:2 * layer_ops]
        ctx64 = vqd.vqd_create(n, vqd.VQD_F64, sh)
        dms, dstats, _ = timed(make_step(ctx64, "plain", sample), 1, 1, ctx64)
        ddom, droof = roofline(dstats, 1)
        kern_ms = sum(v["total_ms"] for k, v in dstats.items() if k not in ("reduce", "init"))
        fp64_rate = len(sample) * 4.0 ** n / (kern_ms * 1e-3)
        droof["bound"] = "alu" if ddom in ("sup1", "uni2", "sup2") else "hbm"
        # the same sample through the fused path in FP64
        fms64, fst64, _ = timed(make_step(ctx64, "fused", sample), 1, 1, ctx64)
        fk64 = sum(v["total_ms"] for k, v in fst64.items() if k not in ("reduce", "init"))
        extra["fused_f64_sample"] = {"value": world * len(sample) * 4.0 ** n / (fk64 * 1e-3), "unit": UNIT,
                                     "sample": f"first 2 of 60 layers ({len(sample)} native ops), kernel time only",
                                     "stages": fst64.get("fused_stage", {}).get("launches", 0)}
        extra["plain_f64_sample"] = {"value": world * fp64_rate, "unit": UNIT,
                                     "sample": f"first 2 of 60 layers ({len(sample)} native ops), kernel time only",
                                     "roofline_hbm": droof,
                                     "roofline_fp64_alu": fp64_alu_roof(dstats, n),
                                     "per_class": {k: {"launches": v["launches"], "avg_ms": v["total_ms"] / v["launches"]}
                                                   for k, v in dstats.items()}}
        vqd.vqd_destroy(ctx64)
        # ---- the same sample with float-float storage (FP64-class accuracy on the FP32 pipes)
        ctxs = vqd.vqd_create(n, vqd.VQD_F32_SPLIT, sh)
        for path in ("plain", "fused"):
            tms, tst, _ = timed(make_step(ctxs, path, sample), 1, 1, ctxs)
            kms = sum(v["total_ms"] for k, v in tst.items() if k not in ("reduce", "init"))
            extra[f"{path}_split_sample"] = {
                "value": world * len(sample) * 4.0 ** n / (kms * 1e-3), "unit": UNIT,
                "sample": f"first 2 of 60 layers ({len(sample)} native ops), kernel time only",
                "vs_f64_plain": (len(sample) * 4.0 ** n / (kms * 1e-3)) / fp64_rate}
        vqd.vqd_destroy(ctxs)

    if not args.no_extra:
        extra["trajectories_c64"] = measure_trajectories(vqd, torch, prog, native, sh)
        extra["sc_device_compiled_c64"] = measure_sc_device(vqd, torch, sh, timed, args.steps)
        extra["trajectories_spin16_c64"] = measure_trajectories_spin16(vqd, sh)
        extra["nv5_noise_sweep_batch_c64"] = measure_nv_noise_sweep(vqd, torch)

    if not args.no_extra and args.batch_count > 0:
        extra["batch_c64"] = measure_batch(vqd, torch, sh, args.batch_count)

    cpu = None
    if rank == 0 and not args.no_extra:
        rate, dt = oracle_rate(prog, 2)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"first 2 native ops of the 14-qubit program at full size, FP64 numpy, {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_qubits": n, "native_ops": len(prog.ops), "state_bytes": 8 * 4 ** n,
                       "l2": "inputs larger than L2 (2.15 GB state vs 129 MB L2), no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": ck, "paths": extra,
            "per_class": {k: {"launches": v["launches"] // args.steps, "avg_ms": v["total_ms"] / v["launches"]}
                          for k, v in stats.items()},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
