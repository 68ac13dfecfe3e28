"""Autotuner of the fused and batched paths: fusion width, tile shape and Hermitian stages, picked by timing.

A candidate is (fuse_qubits, tile_bits, passenger_bits, hermitian). The tuner runs a prefix of the program
through ``vqd_run_program`` on a scratch state of the same size, for every candidate. It times the
stage kernels with the library's CUDA-event launch accounting and returns the fastest candidate.
When the caller allows Hermitian stages (flags with VQD_HERMITIAN: the state is a density matrix), both
the Hermitian and the general plans are candidates, because halving a stage's arithmetic pays only where
the arithmetic, not the memory traffic, bounds the stage (FP64 and float-float; rarely complex64).
The choice's "flags" are the vqd_run_program flags to run with.
Results can be cached in a JSON file, keyed by the qubit count, the precision, the flags and the program's
gate structure (op codes and qubits, not angles).
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Iterable, Optional

import numpy as np

from . import vqd

CANDIDATES = {
    vqd.VQD_F32: [(f, tb, p) for f in (4, 5, 6) for (tb, p) in ((13, 3), (13, 2), (12, 2))],
    vqd.VQD_F64: [(f, tb, p) for f in (5, 6) for (tb, p) in ((12, 2), (12, 1), (11, 1))],
    vqd.VQD_F32_SPLIT: [(f, tb, p) for f in (5, 6) for (tb, p) in ((12, 2), (12, 1), (11, 1))],
}
# Hermitian runs (VQD_HERMITIAN): symmetric tiles of an even bit count whose passengers carry their column bits
# too, so fewer passengers keep the same number of stage qubits.
HERM_CANDIDATES = {
    vqd.VQD_F32: [(f, tb, p) for f in (5, 6) for (tb, p) in ((12, 1), (12, 2), (12, 3))],
    vqd.VQD_F64: [(f, tb, p) for f in (5, 6) for (tb, p) in ((12, 1), (12, 0), (12, 2))],
    vqd.VQD_F32_SPLIT: [(f, tb, p) for f in (5, 6) for (tb, p) in ((12, 1), (12, 0), (12, 2))],
}
# The batched path: whole batches are timed, so fewer candidates (fusion width x tile shape).
BATCH_CANDIDATES = {
    vqd.VQD_F32: [(6, 13, 3), (5, 13, 3), (6, 12, 2), (4, 13, 3)],
    vqd.VQD_F64: [(6, 12, 2), (5, 12, 2), (6, 11, 1)],
    vqd.VQD_F32_SPLIT: [(6, 12, 2), (5, 12, 2), (6, 11, 1)],
}
HERM_BATCH_CANDIDATES = {
    vqd.VQD_F32: [(6, 12, 1), (6, 12, 2), (5, 12, 2), (6, 13, 3)],
    vqd.VQD_F64: [(6, 12, 1), (5, 12, 1), (6, 12, 2)],
    vqd.VQD_F32_SPLIT: [(6, 12, 1), (5, 12, 1), (6, 12, 2)],
}


def _candidates(given, herm: bool, herm_default, general_default):
    """(fuse_qubits, tile_bits, passenger_bits, hermitian) tuples: the caller's (3-tuples take `herm`), else the
    defaults, with the Hermitian ones first when Hermitian stages are allowed."""
    if given is not None:
        return [tuple(c) if len(c) == 4 else (*c, herm) for c in given]
    out = [(*c, True) for c in herm_default] if herm else []
    return out + [(*c, False) for c in general_default]


def _run_flags(flags: int, hermitian: bool) -> int:
    return (flags | vqd.VQD_HERMITIAN) if hermitian else (flags & ~vqd.VQD_HERMITIAN)


def structure_key(n: int, prec: int, native: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(native["code"]).tobytes())
    h.update(np.ascontiguousarray(native["q"]).tobytes())
    return f"n{n}-p{prec}-{len(native)}-{h.hexdigest()[:16]}"


def tune(n: int, prec: int, ops, stream: int = 0, prefix: int = 0, candidates: Optional[Iterable] = None,
         cache_path: Optional[str] = None, flags: int = 0) -> dict:
    """Fastest (fuse_qubits, tile_bits, passenger_bits) for this program run with these vqd_run_program flags;
    runs on a scratch state (|0><0|, Hermitian)."""
    native = ops if isinstance(ops, np.ndarray) else vqd.native_ops(ops)
    sample = native[:prefix] if prefix else native
    key = structure_key(n, prec, sample) + f"-f{flags}"
    herm = bool(flags & vqd.VQD_HERMITIAN)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    cands = _candidates(candidates, herm, HERM_CANDIDATES[prec], CANDIDATES[prec])
    ctx = vqd.vqd_create(n, prec, stream)
    trials = []
    try:
        for f, tb, p, h in cands:
            fl = _run_flags(flags, h)
            vqd.vqd_set_tile_shape(ctx, tb, p)
            vqd.vqd_run_program(ctx, 0, sample, f, fl)      # warm-up (and plan)
            vqd.vqd_sync(ctx)
            vqd.vqd_profile(ctx, 2)
            vqd.vqd_profile_reset(ctx)
            vqd.vqd_run_program(ctx, 0, sample, f, fl)
            st = vqd.vqd_profile_read(ctx).get("fused_stage", {"total_ms": 0.0, "launches": 0})
            vqd.vqd_profile(ctx, 0)
            trials.append({"fuse_qubits": f, "tile_bits": tb, "passenger_bits": p, "hermitian": h, "flags": fl,
                           "ms": st["total_ms"], "stages": st["launches"]})
    finally:
        vqd.vqd_destroy(ctx)
    best = min(trials, key=lambda t: t["ms"])
    result = dict(best, trials=trials, sample_ops=int(len(sample)))
    if cache_path:
        cache[key] = result
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return result


def tune_batch(ns, prec: int, arrays, stream: int = 0, candidates: Optional[Iterable] = None,
               flags: int = 0) -> dict:
    """Fastest (fuse_qubits, tile_bits, passenger_bits) for a batch of programs (one per instance, n qubits
    each) run with these vqd_run_batch flags: every candidate runs the whole batch once (planning and graph
    capture) and is then timed on a replay of its CUDA graph with the library's CUDA-event accounting of the
    batch waves."""
    herm = bool(flags & vqd.VQD_HERMITIAN)
    cands = _candidates(candidates, herm, HERM_BATCH_CANDIDATES[prec], BATCH_CANDIDATES[prec])
    ctx = vqd.vqd_create_batch(list(ns), prec, stream)
    trials = []
    try:
        for f, tb, p, h in cands:
            fl = _run_flags(flags, h)
            vqd.vqd_set_tile_shape(ctx, tb, p)
            vqd.vqd_run_batch(ctx, arrays, f, fl)        # plan, capture
            vqd.vqd_sync(ctx)
            vqd.vqd_profile(ctx, 2)
            vqd.vqd_profile_reset(ctx)
            vqd.vqd_run_batch(ctx, arrays, f, fl)        # replay
            st = vqd.vqd_profile_read(ctx).get("batch", {"total_ms": 0.0, "launches": 0})
            vqd.vqd_profile(ctx, 0)
            trials.append({"fuse_qubits": f, "tile_bits": tb, "passenger_bits": p, "hermitian": h, "flags": fl,
                           "ms": st["total_ms"]})
    finally:
        vqd.vqd_destroy(ctx)
    best = min(trials, key=lambda t: t["ms"])
    return dict(best, trials=trials)


def apply(ctx, choice: dict) -> int:
    """Set the tuned tile shape on a context; returns the fuse width to pass to vqd_run_program (with the
    flags in choice["flags"])."""
    vqd.vqd_set_tile_shape(ctx, choice["tile_bits"], choice["passenger_bits"])
    return int(choice["fuse_qubits"])
