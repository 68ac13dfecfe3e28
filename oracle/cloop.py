"""Oracle evolution in plain C loops (test infrastructure only).

``c/kraus_loop.c`` writes the update rho <- sum_j K_j rho K_j^dagger of Sec. 2 as FP64 loops over the
(row, column) blocks of the target qubits; this module compiles it with the host C compiler (gcc, OpenMP)
and applies the oracle's own compiled steps (``compile.compile_op``) with it, in program order, exactly
as ``evolve.run_program`` does.  The result equals ``evolve``'s up to the rounding of the summation order;
``tests/test_oracle_pins.py`` holds the two together on random programs and runs the closed-form pins
through this evaluation as well.  It makes full-size (14- to 16-qubit) oracle runs affordable, and it
is the oracle that ``bench.py`` times single-threaded and on all host cores.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import compile as _compile
from . import evolve

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c", "kraus_loop.c")
LIB = os.path.join(HERE, "c", "_kraus_loop.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2 -fopenmp, no machine-specific flags) if it is missing or stale."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"oracle C build failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(LIB)
        _lib.oracle_apply_kraus.restype = ctypes.c_int
        _lib.oracle_apply_kraus.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_int, ctypes.c_void_p]
        _lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib.oracle_max_threads.restype = ctypes.c_int
    return _lib


def set_threads(threads: int) -> None:
    """Number of OpenMP threads of the following calls (the results do not depend on it)."""
    lib().oracle_set_threads(int(threads))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def apply_kraus(rho: np.ndarray, qubits, kraus) -> np.ndarray:
    """In place: rho <- sum_j K_j rho K_j^dagger (rho C-contiguous complex128, 2^n x 2^n)."""
    assert rho.dtype == np.complex128 and rho.flags["C_CONTIGUOUS"]
    n = int(round(np.log2(rho.shape[0])))
    t = np.ascontiguousarray(np.asarray(qubits, dtype=np.int32))
    K = np.ascontiguousarray(np.stack([np.asarray(k, dtype=np.complex128) for k in kraus]))
    rc = lib().oracle_apply_kraus(rho.ctypes.data, n, len(t), t.ctypes.data, K.shape[0], K.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_apply_kraus: bad arguments")
    return rho


def apply_steps(rho: np.ndarray, steps) -> np.ndarray:
    for kind, qubits, m in steps:
        apply_kraus(rho, qubits, [m] if kind == "U" else m)
    return rho


def run_program(prog, t2_is_total: bool = False, rho0: np.ndarray | None = None, max_ops: int | None = None,
                threads: int | None = None) -> np.ndarray:
    """Compile every native op of ``prog`` and apply the steps in order (optionally only the first
    ``max_ops``), as ``evolve.run_program`` does."""
    if threads is not None:
        set_threads(threads)
    rho = np.array(evolve.initial_state(prog) if rho0 is None else rho0, dtype=np.complex128, order="C", copy=True)
    ops = prog.ops if max_ops is None else prog.ops[:max_ops]
    for o in ops:
        apply_steps(rho, _compile.compile_op(o.name, o.qubits, o.params, t2_is_total))
    return rho
