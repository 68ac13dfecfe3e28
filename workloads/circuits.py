"""Deterministic, seeded generators of native-operation programs.

A program is a list of ``NativeOp(name, qubits, params)``.  Names are the
device vocabulary of the paper (native gates of Sec. 4-8 and the noise
processes of Sec. 3); parameters are physical quantities (angles in radians,
durations in microseconds, frequencies in MHz, probabilities).  Nothing here
builds a matrix or evaluates a decay law.

Every generator takes a ``seed`` and uses numpy's PCG64 stream, so the same
seed yields the same program on every machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

# name -> (number of qubits, parameter names).  The order of the table is the
# numeric op code used at the C boundary (the library header repeats it).
OP_NAMES = {
    # native gates (unitaries)
    "rx": (1, ("theta",)),            # Rx(theta) = exp(-i theta X/2)
    "ry": (1, ("theta",)),
    "rz": (1, ("theta",)),
    "sx": (1, ()),                    # sqrt(X) := Rx(pi/2)
    "h": (1, ()),
    "u": (1, ("phi", "omega", "delta", "t")),   # Raman U(phi, Delta, t), Sec. 6 Eq. (u)
    "r": (1, ("theta", "phi")),       # ion R(theta, phi) = U(phi, Delta=0, Omega t = theta)
    "cz": (2, ()),
    "cph": (2, ("phi",)),             # controlled phase diag(1,1,1,e^{i phi})
    "czphi": (2, ("phi",)),           # Rydberg CZ(phi), Sec. 6
    "zx": (2, ("theta",)),            # cross resonance exp(-i theta/2 Z_c X_t), control = first qubit
    "zz": (2, ("theta",)),            # exp(-i theta/2 Z Z)
    "xx": (2, ("theta",)),            # Molmer-Sorensen exp(-i theta/2 X X)
    "zzphase": (2, ("alpha",)),       # ZZ crosstalk exp(-i alpha Z Z), Eq. (weak_dephasing_zz)
    "zz_idle": (2, ("dt", "xi")),     # static ZZ crosstalk of rate xi (MHz) over an idle of dt (us)
    "crz_xtalk": (2, ("alpha",)),     # conditional Rz crosstalk, Eq. (weak_dephasing); control = first
    "exchange": (2, ("theta",)),      # exchange crosstalk, Eq. (exchange_pauli)
    # noise processes (Kraus channels)
    "depol1": (1, ("p",)),
    "depol2": (2, ("p",)),
    "deph1": (1, ("p",)),
    "deph2": (2, ("p",)),
    "amp": (1, ("p",)),
    "bitflip": (1, ("b",)),
    "bitflip2": (2, ("b",)),
    "gamp": (1, ("dt", "t1", "p0")),          # generalised damping towards p0|0><0| + (1-p0)|1><1|
    "idle": (1, ("dt", "t1", "t2")),          # passive T1 damping + T2 dephasing
    "idle_depol": (1, ("dt", "t1", "t2")),    # passive T1 as depolarising + T2 dephasing
    "stderr1": (1, ("fbar", "x")),            # standard error from average gate fidelity
    "stderr2": (2, ("fbar", "x")),
    "ampdeph2": (2, ("dt", "t1", "t2")),      # T1/T2 decay of both qubits of a pair as one 2-qubit channel
    "leak_init": (1, ("gamma",)),             # CPTN init leakage L
    "leak_cz": (2, ("alpha", "beta")),        # CPTN Rydberg decay K
    # device-family crosstalk unitaries
    "offres": (1, ("omega", "delta", "t")),    # off-resonant Rabi drive on a passive qubit, Eq. (off_resonant)
    "zz_static": (2, ("j", "delta", "alpha_t", "alpha_c")),  # SC static ZZ exp(-i beta Z Z), beta from J, Delta, alpha
    "zy": (2, ("theta",)),            # NV conditional CRy+-(theta) = exp(-i theta/2 Z_c Y_t), Eq. (conditional_rots)
    "idle_t2s": (1, ("dt", "t1", "t2s")),   # passive T1 as depolarising + Gaussian T2* dephasing, Eqs. (depolt1),(depht2s)
    "bitflip_asym": (1, ("p10", "p01")),     # asymmetric bit flip: |1> -> |0> with p10, |0> -> |1> with p01 (Sec. 6)
}


@dataclass(frozen=True)
class NativeOp:
    name: str
    qubits: Tuple[int, ...]
    params: Tuple[float, ...] = ()

    def __post_init__(self):
        nq, pn = OP_NAMES[self.name]
        if len(self.qubits) != nq or len(self.params) != len(pn):
            raise ValueError(f"bad native op {self}")


@dataclass
class Program:
    """One device program on ``n`` qubits.

    ``ops`` is the native-op list; ``measure`` is the list of qubits whose
    Z-basis probabilities are reported at the end; ``meta`` records the
    generator, seed and physical constants used.
    """
    n: int
    ops: List[NativeOp]
    measure: Tuple[int, ...] = ()
    meta: dict = field(default_factory=dict)
    init_excited: Tuple[float, ...] = ()   # optional thermal product init, excited population per qubit

    @property
    def n_gates(self) -> int:
        return sum(1 for o in self.ops if o.name in GATE_NAMES)


GATE_NAMES = frozenset(["rx", "ry", "rz", "sx", "h", "u", "r", "cz", "cph", "czphi", "zx", "zz", "xx"])


def program_stats(prog: Program) -> dict:
    """Counts of native ops by name and by arity (no arithmetic of the method)."""
    by_name = {}
    for o in prog.ops:
        by_name[o.name] = by_name.get(o.name, 0) + 1
    return {"n": prog.n, "ops": len(prog.ops), "gates": prog.n_gates, "by_name": by_name}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------------------------
# Config 1: 6-qubit chain, 200 gates, depolarising gate noise, T1/T2 idle per sublayer.
# --------------------------------------------------------------------------------------------
def config1_chain6(seed: int = 1, n: int = 6, n_gates: int = 200, p1: float = 1e-3, p2: float = 1e-2,
                   t1: float = 100.0, t2: float = 50.0, dt1: float = 0.02, dt2: float = 0.2) -> Program:
    """Linear chain: per layer a random-axis rotation on every qubit then CZ on alternating pairs.

    After each 1q gate depol1(p1); after each CZ depol2(p2); after each sublayer an idle of
    dt1 (rotations) or dt2 (CZs) on every qubit.  Stops exactly at ``n_gates`` gates; the
    sublayer in which the last gate falls still receives its idle.
    """
    r = _rng(seed)
    ops: List[NativeOp] = []
    g = 0
    layer = 0
    while g < n_gates:
        for q in range(n):
            if g >= n_gates:
                break
            axis = ("rx", "ry", "rz")[int(r.integers(0, 3))]
            theta = float(r.uniform(0.0, 2.0 * math.pi))
            ops.append(NativeOp(axis, (q,), (theta,)))
            ops.append(NativeOp("depol1", (q,), (p1,)))
            g += 1
        for q in range(n):
            ops.append(NativeOp("idle", (q,), (dt1, t1, t2)))
        if g >= n_gates:
            break
        start = 0 if layer % 2 == 0 else 1
        for a in range(start, n - 1, 2):
            if g >= n_gates:
                break
            ops.append(NativeOp("cz", (a, a + 1)))
            ops.append(NativeOp("depol2", (a, a + 1), (p2,)))
            g += 1
        for q in range(n):
            ops.append(NativeOp("idle", (q,), (dt2, t1, t2)))
        layer += 1
    return Program(n, ops, measure=tuple(range(n)),
                   meta={"config": "chain6", "seed": seed, "p1": p1, "p2": p2, "t1": t1, "t2": t2,
                         "dt1": dt1, "dt2": dt2, "gates": n_gates})


# --------------------------------------------------------------------------------------------
# Config 2: superconducting-like 2 x C grid, brickwork ZX(pi/2) + Rz/SX, ZZ crosstalk, T1/T2, readout flip.
# --------------------------------------------------------------------------------------------
def grid_edges(rows: int, cols: int):
    """Edges of a rows x cols grid (qubit = cols*row + col) split into 4 colour classes."""
    classes = [[], [], [], []]
    for rr in range(rows):
        for c in range(cols - 1):
            classes[c % 2].append((cols * rr + c, cols * rr + c + 1))
    for c in range(cols):
        for rr in range(rows - 1):
            classes[2 + c % 2].append((cols * rr + c, cols * (rr + 1) + c))
    return classes


def config2_sc_grid(seed: int = 2, rows: int = 2, cols: int = 7, depth: int = 60, xi_mhz: float = 0.05,
                    t1_lo: float = 50.0, t1_hi: float = 200.0, t2_over_t1: float = 0.7,
                    readout_flip: float = 2e-2, dur_1q: float = 0.05, dur_zx: float = 0.5) -> Program:
    """Brickwork of native ZX(pi/2) cross-resonance gates and Rz.SX.Rz single-qubit layers.

    Per layer: Rz(a) SX Rz(b) on every qubit (Rz virtual, 0 us; SX lasts ``dur_1q``), then
    ZX(pi/2) on one of four edge colour classes (cycling; control = lower index, ``dur_zx``).
    After each sublayer every grid edge that carries no ZX gets the static ZZ crosstalk
    unitary for the sublayer's duration and every qubit gets T1/T2 idle decay.  T1 is
    log-uniform in [t1_lo, t1_hi] us per qubit and T2 = t2_over_t1 * T1.  The program
    ends with a readout bit flip on every qubit.
    """
    r = _rng(seed)
    n = rows * cols
    t1 = np.exp(r.uniform(math.log(t1_lo), math.log(t1_hi), size=n))
    t2 = t2_over_t1 * t1
    classes = grid_edges(rows, cols)
    all_edges = [e for cl in classes for e in cl]
    ops: List[NativeOp] = []
    for layer in range(depth):
        for q in range(n):
            ops.append(NativeOp("rz", (q,), (float(r.uniform(0, 2 * math.pi)),)))
            ops.append(NativeOp("sx", (q,)))
            ops.append(NativeOp("rz", (q,), (float(r.uniform(0, 2 * math.pi)),)))
        for (a, b) in all_edges:
            ops.append(NativeOp("zz_idle", (a, b), (dur_1q, xi_mhz)))
        for q in range(n):
            ops.append(NativeOp("idle", (q,), (dur_1q, float(t1[q]), float(t2[q]))))
        active = classes[layer % 4]
        for (a, b) in active:
            ops.append(NativeOp("zx", (a, b), (math.pi / 2,)))
        act = set(active)
        for (a, b) in all_edges:
            if (a, b) not in act:
                ops.append(NativeOp("zz_idle", (a, b), (dur_zx, xi_mhz)))
        for q in range(n):
            ops.append(NativeOp("idle", (q,), (dur_zx, float(t1[q]), float(t2[q]))))
    for q in range(n):
        ops.append(NativeOp("bitflip", (q,), (readout_flip,)))
    return Program(n, ops, measure=tuple(range(n)),
                   meta={"config": f"sc_grid{rows}x{cols}", "seed": seed, "depth": depth, "xi_mhz": xi_mhz,
                         "t1": [float(x) for x in t1], "t2": [float(x) for x in t2],
                         "readout_flip": readout_flip, "dur_1q": dur_1q, "dur_zx": dur_zx})


# --------------------------------------------------------------------------------------------
# Config 3: ion-trap-like all-to-all, XX(theta) on random pairs + R(theta, phi), dephasing per gate.
# --------------------------------------------------------------------------------------------
def config3_ion_alltoall(seed: int = 3, n: int = 15, n_gates: int = 800, p_deph: float = 5e-4) -> Program:
    r = _rng(seed)
    ops: List[NativeOp] = []
    for _ in range(n_gates):
        if r.uniform() < 0.5:
            a, b = (int(x) for x in r.choice(n, size=2, replace=False))
            ops.append(NativeOp("xx", (a, b), (float(r.uniform(0, 2 * math.pi)),)))
            ops.append(NativeOp("deph1", (a,), (p_deph,)))
            ops.append(NativeOp("deph1", (b,), (p_deph,)))
        else:
            q = int(r.integers(0, n))
            ops.append(NativeOp("r", (q,), (float(r.uniform(0, 2 * math.pi)), float(r.uniform(0, 2 * math.pi)))))
            ops.append(NativeOp("deph1", (q,), (p_deph,)))
    return Program(n, ops, measure=tuple(range(n)),
                   meta={"config": f"ion_alltoall{n}", "seed": seed, "gates": n_gates, "p_deph": p_deph})


# --------------------------------------------------------------------------------------------
# Config 4: batch of neutral-atom-like instances of uneven size.
# --------------------------------------------------------------------------------------------
def _neutral_instance(r: np.random.Generator, n: int, depth: int, radius: float,
                      dur_rx: float, dur_cz: float) -> Program:
    side = int(math.ceil(math.sqrt(n))) + 1
    sites = r.choice(side * side, size=n, replace=False)
    pos = [(int(s) % side, int(s) // side) for s in sites]
    t1 = float(math.exp(r.uniform(math.log(50.0), math.log(500.0))))
    t2 = float(math.exp(r.uniform(math.log(20.0), math.log(200.0))))
    p1 = float(math.exp(r.uniform(math.log(1e-4), math.log(1e-3))))
    p2 = float(math.exp(r.uniform(math.log(1e-3), math.log(1e-2))))
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)
             if (pos[a][0] - pos[b][0]) ** 2 + (pos[a][1] - pos[b][1]) ** 2 <= radius * radius]
    ops: List[NativeOp] = []
    for layer in range(depth):
        for q in range(n):
            ops.append(NativeOp("rx", (q,), (float(r.uniform(0, 2 * math.pi)),)))
            ops.append(NativeOp("deph1", (q,), (p1,)))
        for q in range(n):
            ops.append(NativeOp("idle_depol", (q,), (dur_rx, t1, t2)))
        # one global Rydberg pulse: a maximal set of disjoint in-radius pairs, random greedy order
        order = r.permutation(len(pairs)) if pairs else []
        used = set()
        for i in order:
            a, b = pairs[int(i)]
            if a in used or b in used:
                continue
            used.add(a)
            used.add(b)
            ops.append(NativeOp("czphi", (a, b), (float(r.uniform(0, 2 * math.pi)),)))
            ops.append(NativeOp("depol2", (a, b), (p2,)))
        for q in range(n):
            ops.append(NativeOp("idle_depol", (q,), (dur_cz, t1, t2)))
    return Program(n, ops, measure=tuple(range(n)),
                   meta={"t1": t1, "t2": t2, "p1": p1, "p2": p2, "positions": pos})


def config4_neutral_batch(seed: int = 4, count: int = 1024, n_lo: int = 6, n_hi: int = 12, depth: int = 20,
                          radius: float = 1.5, dur_rx: float = 0.5, dur_cz: float = 0.25) -> List[Program]:
    """``count`` independent instances with n ~ U{n_lo..n_hi}; per-instance T1, T2 and gate errors
    log-uniform over a decade."""
    r = _rng(seed)
    ns = r.integers(n_lo, n_hi + 1, size=count)
    progs = []
    for i, n in enumerate(ns):
        sub = _rng(seed * 1_000_003 + i)
        p = _neutral_instance(sub, int(n), depth, radius, dur_rx, dur_cz)
        p.meta.update({"config": "neutral_batch", "seed": seed, "instance": i})
        progs.append(p)
    return progs


# --------------------------------------------------------------------------------------------
# Config 5: silicon-spin-like chain: CPh(phi) on neighbours, Rx/Rz, 2-qubit damping+dephasing Kraus.
# --------------------------------------------------------------------------------------------
def config5_spin_chain(seed: int = 5, n: int = 16, n_gates: int = 2000, p1: float = 1e-3, t1: float = 1e4,
                       t2_lo: float = 14.0, t2_hi: float = 45.0, dur_1q: float = 0.1,
                       dur_cph: float = 0.05) -> Program:
    r = _rng(seed)
    t2 = r.uniform(t2_lo, t2_hi, size=n)
    ops: List[NativeOp] = []
    g = 0
    layer = 0
    while g < n_gates:
        if layer % 2 == 0:
            for q in range(n):
                if g >= n_gates:
                    break
                name = "rx" if r.uniform() < 0.5 else "rz"
                ops.append(NativeOp(name, (q,), (float(r.uniform(0, 2 * math.pi)),)))
                ops.append(NativeOp("depol1", (q,), (p1,)))
                g += 1
        else:
            start = 0 if (layer // 2) % 2 == 0 else 1
            for a in range(start, n - 1, 2):
                if g >= n_gates:
                    break
                ops.append(NativeOp("cph", (a, a + 1), (float(r.uniform(0, 2 * math.pi)),)))
                ops.append(NativeOp("ampdeph2", (a, a + 1), (dur_cph, t1, float(0.5 * (t2[a] + t2[a + 1])))))
                g += 1
        layer += 1
    return Program(n, ops, measure=tuple(range(n)),
                   meta={"config": f"spin_chain{n}", "seed": seed, "gates": n_gates, "p1": p1, "t1": t1,
                         "t2": [float(x) for x in t2], "dur_1q": dur_1q, "dur_cph": dur_cph})


def random_program(seed: int, n: int, n_ops: int, names: Sequence[str] | None = None) -> Program:
    """Random mix of every native op kind (test workload covering the whole vocabulary)."""
    r = _rng(seed)
    names = list(names) if names is not None else list(OP_NAMES)
    if n < 2:
        names = [x for x in names if OP_NAMES[x][0] == 1]
    ops: List[NativeOp] = []
    for _ in range(n_ops):
        name = names[int(r.integers(0, len(names)))]
        nq, pn = OP_NAMES[name]
        qs = tuple(int(x) for x in r.choice(n, size=nq, replace=False))
        ops.append(NativeOp(name, qs, _random_params(r, name)))
    return Program(n, ops, measure=tuple(range(n)), meta={"config": "random", "seed": seed})


def _random_params(r: np.random.Generator, name: str) -> Tuple[float, ...]:
    u = lambda lo, hi: float(r.uniform(lo, hi))
    table = {
        "rx": lambda: (u(0, 2 * math.pi),), "ry": lambda: (u(0, 2 * math.pi),), "rz": lambda: (u(0, 2 * math.pi),),
        "sx": lambda: (), "h": lambda: (), "cz": lambda: (),
        "u": lambda: (u(0, 2 * math.pi), u(0.5, 2.0), u(-1.0, 1.0), u(0.0, 3.0)),
        "r": lambda: (u(0, 2 * math.pi), u(0, 2 * math.pi)),
        "cph": lambda: (u(0, 2 * math.pi),), "czphi": lambda: (u(0, 2 * math.pi),),
        "zx": lambda: (u(0, 2 * math.pi),), "zz": lambda: (u(0, 2 * math.pi),), "xx": lambda: (u(0, 2 * math.pi),),
        "zzphase": lambda: (u(-1, 1),), "zz_idle": lambda: (u(0.01, 1.0), u(0.01, 0.2)),
        "crz_xtalk": lambda: (u(-1, 1),), "exchange": lambda: (u(-1, 1),),
        "depol1": lambda: (u(0, 0.75),), "depol2": lambda: (u(0, 15 / 16),), "deph1": lambda: (u(0, 0.5),),
        "deph2": lambda: (u(0, 0.75),), "amp": lambda: (u(0, 1),), "bitflip": lambda: (u(0, 0.5),),
        "bitflip2": lambda: (u(0, 0.75),), "gamp": lambda: (u(0.01, 50), u(5, 100), u(0.5, 1.0)),
        "idle": lambda: (u(0.01, 20), u(20, 200), u(10, 100)),
        "idle_depol": lambda: (u(0.01, 20), u(20, 200), u(10, 100)),
        "stderr1": lambda: (u(0.95, 1.0), u(0, 1)), "stderr2": lambda: (u(0.9, 1.0), u(0, 1)),
        "ampdeph2": lambda: (u(0.01, 20), u(20, 200), u(10, 100)),
        "leak_init": lambda: (u(0, 0.1),), "leak_cz": lambda: (u(0, 0.1), u(0, 0.01)),
        "offres": lambda: (u(0.5, 2.0), u(-8.0, 8.0), u(0.0, 3.0)),
        "zz_static": lambda: (u(0.02, 0.2), u(0.2, 1.0), u(-3.0, -2.0), u(-3.0, -2.0)),
        "zy": lambda: (u(0, 2 * math.pi),),
        "idle_t2s": lambda: (u(0.01, 20), u(20, 200), u(10, 100)),
        "bitflip_asym": lambda: (u(0, 0.2), u(0, 0.2)),
    }
    return table[name]()
