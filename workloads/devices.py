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


SI6 = {  # App. C, table of the virtual silicon qubits (MHz, us); ratios depolarising:dephasing 0:1
    "n": 6,
    "t1": [1e4] * 6,
    "t2": [14.0, 21.1, 40.1, 37.2, 44.7, 26.7],
    "freq": [15.62e3, 15.88e3, 16.3e3, 16.1e3, 15.9e3, 15.69e3],
    "rabi": [5.0] * 6,
    "fid_1q": [0.9977, 0.9987, 0.9996, 0.9988, 0.9991, 0.9989],
    "x_1q": 0.0,
    "freq_cz": [12.1, 11.1, 6.6, 9.8, 5.4],
    "fid_cz": [0.937, 0.934, 0.929, 0.997, 0.979],
    "x_cz": 0.0,
    "xtalk_on": [[0, 0.023, 0.018, 0.03, 0.04],
                 [0.05, 0, 0.03, 0.03, 0.04],
                 [0.05, 0.03, 0, 0.07, 0.042],
                 [0.038, 0.03, 0.031, 0, 0.25],
                 [0.033, 0.03, 0.02, 0.03, 0]],
    "xtalk_off": [0.039, 0.015, 0.03, 0.02, 0.028],
}


def si_circuit(dev: Dict, n_gates: int, seed: int = 9) -> List[NativeOp]:
    """Random circuit in the silicon native gates: Rx, Ry (angles up to pi), virtual Rz, and CZ or CPh
    on neighbour pairs, about one two-qubit gate in three."""
    r = _rng(seed)
    n = int(dev["n"])
    ops: List[NativeOp] = []
    for _ in range(n_gates):
        u = r.uniform()
        if u < 1 / 3:
            k = int(r.integers(0, n - 1))
            pair = (k, k + 1) if r.uniform() < 0.5 else (k + 1, k)
            ops.append(NativeOp("cz", pair) if r.uniform() < 0.5
                       else NativeOp("cph", pair, (float(r.uniform(0.1, math.pi)),)))
        else:
            name = ("rx", "ry", "rz")[int(r.integers(0, 3))]
            ops.append(NativeOp(name, (int(r.integers(0, n)),), (float(r.uniform(-math.pi, math.pi)),)))
    return ops


NV5 = {  # App. C, table of the virtual NV centre (seconds, Hz); qubit 0 = electron, 1..4 = 13C nuclear spins
    "n": 5,
    "t1": [3600.0, 60.0, 60.0, 60.0, 60.0],
    "t2": [1.5, 10.0, 10.0, 10.0, 9.0],
    "freq_zz": 3.0,
    "freq_xy": [15000e3, 0.5e3, 0.5e3, 0.5e3, 0.5e3],
    "freq_z": [32e6, 0.4e6, 0.4e6, 0.4e6, 0.4e6],
    "freq_crot": [1.5e3, 2.8e3, 0.8e3, 2e3],
    "fid_crot": [0.98, 0.98, 0.98, 0.98],
    "fid_xy": [0.9995, 0.995, 0.995, 0.99, 0.99],
    "fid_z": [1.0] * 5,
    "x_xy": 0.75,          # depolarising:dephasing 0.75:0.25
    "x_crot": 0.9,         # depolarising:dephasing 0.9:0.1
    "fid_meas": 0.946,
    "dur_meas": 2e-5,
}


def nv_scaled(dev: Dict, scale: float) -> Dict:
    """The device with every error scaled by `scale` (infidelities times scale, T1 and T2 divided by it),
    as in the paper's sweeps over the scale of noise."""
    d = dict(dev)
    for k in ("fid_xy", "fid_z", "fid_crot"):
        d[k] = [1.0 - scale * (1.0 - f) for f in dev[k]]
    d["fid_meas"] = 1.0 - scale * (1.0 - dev["fid_meas"])
    d["t1"] = [t / scale for t in dev["t1"]]
    d["t2"] = [t / scale for t in dev["t2"]]
    d["freq_zz"] = dev["freq_zz"] * scale
    return d


def nv_bcs_shape(dev: Dict, n_props: int = 64, gates_per_prop: int = 200, seed: int = 13) -> List[NativeOp]:
    """Synthetic circuit with the shape of the paper's BCS propagators on the NV star (Sec. 5): n_props
    propagators of `gates_per_prop` native gates; about one gate in three is a conditional rotation
    CRx+- / CRy+- from the electron to a nuclear spin, the rest single rotations on any spin."""
    r = _rng(seed)
    n = int(dev["n"])
    ops: List[NativeOp] = []
    for _ in range(n_props * gates_per_prop):
        th = float(r.uniform(-math.pi, math.pi))
        if r.uniform() < 1 / 3:
            ops.append(NativeOp(("zx", "zy")[int(r.integers(0, 2))], (0, int(r.integers(1, n))), (th,)))
        else:
            ops.append(NativeOp(("rx", "ry", "rz")[int(r.integers(0, 3))], (int(r.integers(0, n)),), (th,)))
    return ops


ION = {  # App. C, table of the virtual trapped ions (us, MHz); every ion identical; ratios depolarising:dephasing
    "n": 8,
    "t1": 3e9,
    "t2s": 10e5,
    "rabi": 10.0,
    "fid_xy": 0.99999,
    "x_xy": 1.0,           # 1:0
    "freq_cz": 0.1,
    "fid_cz": 0.999,
    "x_cz": 0.1,           # 0.1:0.9
    "bf_read": 0.001,
    "dur_read": 50.0,
}


def ion_circuit(dev: Dict, n_gates: int, seed: int = 17) -> List[NativeOp]:
    """Random circuit in the trapped-ion native gates: Rx, Ry (angles up to pi), virtual Rz, and CZ on any
    pair of ions, about one gate in four a CZ."""
    r = _rng(seed)
    n = int(dev["n"])
    ops: List[NativeOp] = []
    for _ in range(n_gates):
        if n > 1 and r.uniform() < 0.25:
            a, b = (int(x) for x in r.choice(n, size=2, replace=False))
            ops.append(NativeOp("cz", (a, b)))
        else:
            name = ("rx", "ry", "rz")[int(r.integers(0, 3))]
            ops.append(NativeOp(name, (int(r.integers(0, n)),), (float(r.uniform(-math.pi, math.pi)),)))
    return ops


NA_CLUSTER12 = {  # App. C, neutral atoms, 1D cluster-state setting (us, MHz, lattice units)
    "n": 12,
    "sites": [(float(i), 0.0) for i in range(12)],
    "blockade": 1.0,
    "t2": 100e6,
    "t_vac": 100e6,
    "rabi": 0.1,
    "p10": 0.001,          # p(1 -> 0); the table repeats the label, read as p(1 -> 0) then p(0 -> 1)
    "p01": 0.03,
    "leak_init": 0.01,
    "leak_cz": (0.02, 0.0001),
    "dur_cz": 0.25,        # not tabulated: a stand-in Rydberg gate time
    "fid_meas": 0.975,
}


def na_cluster_circuit(dev: Dict, seed: int = 19, layers: int = 1) -> List[NativeOp]:
    """Linear cluster state in the neutral-atom natives: a pi/2 Raman rotation about y on every atom (phi = pi/2,
    Delta = 0, Omega t = pi/2), then CZ(pi/2) along the chain (CZ(phi) of Sec. 6 is a CZ up to local phases at
    phi = pi/2), repeated `layers` times with seeded small detunings."""
    r = _rng(seed)
    n = int(dev["n"])
    om = float(dev["rabi"])
    ops: List[NativeOp] = []
    for _ in range(layers):
        for q in range(n):
            de = float(r.uniform(-0.01, 0.01))
            ops.append(NativeOp("u", (q,), (math.pi / 2, om, de, (math.pi / 2) / om)))
        for q in range(0, n - 1, 2):
            ops.append(NativeOp("czphi", (q, q + 1), (math.pi / 2,)))
        for q in range(1, n - 1, 2):
            ops.append(NativeOp("czphi", (q, q + 1), (math.pi / 2,)))
    return ops
