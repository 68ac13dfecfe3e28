"""Device tables and logical circuits for the device-family compilers (input generators only).

SC6 is the superconducting device of the paper's App. C table: six transmons on a ladder with their
T1, T2, excited populations, frequencies, anharmonicities, couplings, readout fidelities and gate
durations. sc_grid_device is a larger synthetic device of the same shape for benchmark-sized
programs.
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

from .circuits import NativeOp, _rng, grid_edges

SC6 = {  # App. C, table of the virtual superconducting qubits (MHz, us)
    "n": 6,
    "t1": [63.0, 93.0, 109.0, 115.0, 68.0, 125.0],
    "t2": [113.0, 149.0, 185.0, 161.0, 122.0, 200.0],
    "excited": [3.2e-2, 2.1e-2, 0.8e-2, 0.9e-2, 2.5e-2, 0.7e-2],
    "freq": [4.5e3, 4.9e3, 4.7e3, 5.1e3, 4.9e3, 5.3e3],
    "couple": [(0, 1), (0, 2), (1, 3), (2, 3), (2, 4), (3, 5), (4, 5)],
    "coupling": [4.0, 1.5, 1.5, 4.0, 1.5, 1.5, 4.0],
    "anharm": [296.7, 298.6, 297.4, 298.3, 297.2, 299.1],
    "fid_read": [0.9, 0.92, 0.96, 0.97, 0.93, 0.97],
    "dur_meas": 5.0,
    "dur_rxy": 0.05,
    "dur_zx": 0.5,
    "dur_zz": 0.5,
}


def sc_grid_device(rows: int, cols: int, seed: int = 11) -> Dict:
    """Synthetic rows x cols transmon grid with SC6's parameter ranges (qubit = cols * row + col)."""
    r = _rng(seed)
    n = rows * cols
    edges = [e for cls in grid_edges(rows, cols) for e in cls]
    u = lambda lo, hi, k: [float(x) for x in r.uniform(lo, hi, size=k)]
    return {
        "n": n, "t1": u(60, 130, n), "t2": u(110, 200, n), "excited": u(0.005, 0.035, n),
        "freq": u(4.5e3, 5.3e3, n), "anharm": u(296.0, 300.0, n),
        "couple": [tuple(e) for e in edges], "coupling": u(1.5, 4.0, len(edges)),
        "fid_read": u(0.9, 0.97, n), "dur_meas": 5.0, "dur_rxy": 0.05, "dur_zx": 0.5, "dur_zz": 0.5,
    }


def sc_ansatz(dev: Dict, depth: int, seed: int = 3, sizzle_every: int = 3) -> List[NativeOp]:
    """Hardware-efficient ansatz in the superconducting native gates: per layer Ry, Rz on every qubit,
    then ZX(pi/2) on a greedy matching of the couplings (rotating its start), and every
    ``sizzle_every``-th layer ZZ(pi/2) instead of ZX on the matched pairs."""
    r = _rng(seed)
    n = int(dev["n"])
    couple = [tuple(int(q) for q in e) for e in dev["couple"]]
    ops: List[NativeOp] = []
    for layer in range(depth):
        for q in range(n):
            ops.append(NativeOp("ry", (q,), (float(r.uniform(0, 2 * math.pi)),)))
            ops.append(NativeOp("rz", (q,), (float(r.uniform(0, 2 * math.pi)),)))
        used = set()
        k0 = layer % max(1, len(couple))
        for k in range(len(couple)):
            c, t = couple[(k0 + k) % len(couple)]
            if c in used or t in used:
                continue
            used.update((c, t))
            name = "zz" if sizzle_every and layer % sizzle_every == sizzle_every - 1 else "zx"
            ops.append(NativeOp(name, (c, t), (math.pi / 2,)))
    return ops
