"""Oracle of the superconducting device compiler (test infrastructure: only tests, the smoke check and
the benchmark's CPU baseline use it).

It follows the superconducting error model of Sec. 8 and its App. C parameter table, step by step, in
plain Python:

- Gates are exact and run fully in parallel. A gate starts in the first layer where all its qubits
  are free, and a layer lasts as long as its longest gate. Rz is virtual and takes no time.
- Errors come only from passive noise over each layer of length L:
  - the static ZZ of every capacitively coupled pair, exp(-i beta Z Z) with
    beta = J^2 (1/(Delta_ct - alpha_t) - 1/(Delta_ct + alpha_c)). A pair under a siZZle (ZZ) gate
    is exempt: the gate absorbs its static ZZ.
  - on every qubit not busy for the whole layer, for its idle time dt: generalised amplitude damping
    towards the thermal state (Eq. gdamp, ground population 1 - p_j), then the dephasing of
    Eq. (depht2).
- Readout, when asked for: gamp(t_M) then depol(eps), with eps = 1 - F (the part before the
  measurement in Sec. 8's readout circuit).

Readings, also used by the library:
- Table frequencies are in MHz and times in us. The static ZZ phase is beta computed from the angular
  frequencies 2 pi f, times L.
- The ZZ op is handed the four angles 2 pi L (J, f_c - f_t, alpha_t, alpha_c). beta is homogeneous of
  degree one, so beta of these angles is the accumulated phase.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence

from workloads.circuits import NativeOp

from .compile import stderr_params

DURATION_KEYS = {"rx": "dur_rxy", "ry": "dur_rxy", "zx": "dur_zx", "zz": "dur_zz"}


def gate_duration(dev: Dict, op: NativeOp) -> float:
    """Duration of one superconducting native gate (Sec. 8: Rz virtual; App. C durations)."""
    if op.name == "rz":
        return 0.0
    if op.name not in DURATION_KEYS:
        raise ValueError(f"{op.name} is not a superconducting native gate")
    return float(dev[DURATION_KEYS[op.name]])


def asap_layers(n: int, ops: Sequence[NativeOp]) -> List[List[int]]:
    """Indices of the ops in each parallel layer: every op joins the first layer after the last one that
    used any of its qubits."""
    free_from = [0] * n
    layers: List[List[int]] = []
    for i, op in enumerate(ops):
        layer = max(free_from[q] for q in op.qubits)
        for q in op.qubits:
            free_from[q] = layer + 1
        while len(layers) <= layer:
            layers.append([])
        layers[layer].append(i)
    return layers


def thermal_decay(dev: Dict, j: int, dt: float) -> List[NativeOp]:
    """Free-induction decay of qubit j over dt: gamp towards the thermal state, then deph of Eq. (depht2)."""
    p_excited = float(dev["excited"][j])
    return [NativeOp("gamp", (j,), (dt, float(dev["t1"][j]), 1.0 - p_excited)),
            NativeOp("deph1", (j,), (0.5 * (1.0 - math.exp(-dt / float(dev["t2"][j]))),))]


def sc_compile(dev: Dict, ops: Sequence[NativeOp], readout: bool = False) -> List[NativeOp]:
    """Logical circuit -> native op list of the superconducting device (Sec. 8, App. C)."""
    n = int(dev["n"])
    flags = int(dev.get("flags", 0))
    passive, static_zz = not (flags & 1), not (flags & 2)
    out: List[NativeOp] = []
    for layer in asap_layers(n, ops):
        length = max(gate_duration(dev, ops[i]) for i in layer)
        busy_for = [0.0] * n
        for i in layer:
            out.append(ops[i])
            for q in ops[i].qubits:
                busy_for[q] = gate_duration(dev, ops[i])
        if length <= 0:
            continue
        if static_zz:
            sizzle_pairs = {frozenset(ops[i].qubits) for i in layer if ops[i].name == "zz"}
            for (c, t), J in zip(dev["couple"], dev["coupling"]):
                if J == 0 or frozenset((c, t)) in sizzle_pairs:
                    continue
                angle = 2.0 * math.pi * length
                out.append(NativeOp("zz_static", (int(c), int(t)),
                                    (angle * J, angle * (dev["freq"][c] - dev["freq"][t]),
                                     angle * dev["anharm"][t], angle * dev["anharm"][c])))
        if passive:
            for j in range(n):
                idle = length - busy_for[j]
                if idle > 0:
                    out.extend(thermal_decay(dev, j, idle))
    if readout:
        for j in range(n):
            if passive and dev["dur_meas"] > 0:
                out.append(NativeOp("gamp", (j,), (float(dev["dur_meas"]), float(dev["t1"][j]),
                                                   1.0 - float(dev["excited"][j]))))
            if dev.get("fid_read") is not None:
                out.append(NativeOp("depol1", (j,), (1.0 - float(dev["fid_read"][j]),)))
    return out


def scaled_standard_error(nq: int, qubits, fbar: float, x: float, theta: float) -> List[NativeOp]:
    """Standard error of a parameterised gate (Sec. 3.2, App. B) with App. C's angle rule: every severity is
    scaled by |theta| / pi. deph(p) o depol(q) becomes depol(q s) then deph(p s); zero severities are dropped."""
    p, q = stderr_params(fbar, x, nq)
    s = abs(theta) / math.pi
    out = []
    if q * s > 0:
        out.append(NativeOp("depol1" if nq == 1 else "depol2", tuple(qubits), (q * s,)))
    if p * s > 0:
        out.append(NativeOp("deph1" if nq == 1 else "deph2", tuple(qubits), (p * s,)))
    return out


# ------------------------------------------------------------------ silicon spin qubits (Sec. 7, App. C)
def si_compile(dev: Dict, ops: Sequence[NativeOp]) -> List[NativeOp]:
    """Logical circuit -> native op list of the silicon device (Sec. 7, App. C).

    The gates run one at a time. Readings, also used by the library:
    - An x/y rotation by theta takes t = |theta| / (2 pi f_Rabi). A controlled phase theta takes
      t = |theta| / (2 pi f_CZ), with CZ = CPh(pi).
    - The off-resonant drive of a bystander j (Eq. off_resonant) uses the driven qubit's Rabi
      frequency and the frequency difference |f_j - f_q| as a magnitude, both angular.
    - The off-state crosstalk acts on every neighbour pair that does not contain the driven qubit,
      once per x/y rotation. The on-state one acts on every other pair during a controlled phase:
      controlled-Rz(delta[k][j] theta / pi), with row k the active pair and column j the passive pair.
    - Passive qubits decay over each gate by Eq. (depolt1) then Eq. (depht2) (the idle_depol op).
    - Rz is virtual: it takes no time and carries no noise.
    """
    n = int(dev["n"])
    flags = int(dev.get("flags", 0))
    passive, offres = not (flags & 1), not (flags & 2)
    xon, xoff = dev.get("xtalk_on"), dev.get("xtalk_off")
    out: List[NativeOp] = []

    def bystander_decay(active, t):
        if passive and t > 0:
            for j in range(n):
                if j not in active:
                    out.append(NativeOp("idle_depol", (j,), (t, float(dev["t1"][j]), float(dev["t2"][j]))))

    for op in ops:
        if op.name == "rz":
            out.append(op)
        elif op.name in ("rx", "ry"):
            q = op.qubits[0]
            rabi = float(dev["rabi"][q])
            t = abs(op.params[0]) / (2 * math.pi * rabi)
            out.append(op)
            out += scaled_standard_error(1, (q,), float(dev["fid_1q"][q]), float(dev["x_1q"]), op.params[0])
            if offres and t > 0:
                for j in range(n):
                    if j != q:
                        out.append(NativeOp("offres", (j,), (2 * math.pi * rabi,
                                                             2 * math.pi * abs(dev["freq"][j] - dev["freq"][q]), t)))
            bystander_decay((q,), t)
            if xoff is not None:
                for k in range(n - 1):
                    if q not in (k, k + 1) and xoff[k] != 0:
                        out.append(NativeOp("crz_xtalk", (k, k + 1), (float(xoff[k]),)))
        elif op.name in ("cz", "cph"):
            a, b = op.qubits
            if abs(a - b) != 1:
                raise ValueError("controlled phase on non-neighbours")
            k = min(a, b)
            theta = math.pi if op.name == "cz" else op.params[0]
            t = abs(theta) / (2 * math.pi * float(dev["freq_cz"][k]))
            out.append(op)
            out += scaled_standard_error(2, (a, b), float(dev["fid_cz"][k]), float(dev["x_cz"]), theta)
            if xon is not None:
                for j in range(n - 1):
                    d = float(xon[k][j])
                    if j != k and d != 0:
                        out.append(NativeOp("crz_xtalk", (j, j + 1), (d * theta / math.pi,)))
            bystander_decay((a, b), t)
        else:
            raise ValueError(f"{op.name} is not a silicon native gate")
    return out


# ------------------------------------------------------------------ NV centre (Sec. 5, App. C)
def nv_compile(dev: Dict, ops: Sequence[NativeOp], readout: bool = False) -> List[NativeOp]:
    """Logical circuit -> native op list of the NV-centre device (Sec. 5, App. C).

    Qubit 0 is the electron spin, the others are nuclear spins. The gates run one at a time
    (dynamical decoupling keeps the passive qubits at their T2, and gates are serial). Steps:
    - Rx/Ry: the gate, then the standard error of Sec. 3.2 from the gate's fidelity with the table's
      depolarising:dephasing split.
    - Rz: the gate, then a pure dephasing standard error when its fidelity is below 1.
    - CRx+- / CRy+- (zx / zy, control = electron): the gate, then the two-qubit standard error.
    - During a gate, every other qubit: the weak ZZ of every pair of passive nuclear spins
      (zz_idle), then T1 as depolarising and the T2 dephasing (idle_depol).
    - Readout: the electron's bias, amplitude damping between two X gates (Sec. 5), with p = 1 - F
      read as the net probability that |0> is recorded as 1.

    Readings, also used by the library:
    - A rotation by theta lasts |theta| / (2 pi f), with f the table's frequency for that kind of
      rotation and qubit.
    - The weak ZZ rate is a conditional frequency, as for the superconducting grid (pi f dt / 2).
    """
    n = int(dev["n"])
    passive = not (int(dev.get("flags", 0)) & 1)
    out: List[NativeOp] = []

    def outside(active, t):
        if not passive or t <= 0:
            return
        if dev["freq_zz"] != 0:
            for i in range(1, n):
                for k in range(i + 1, n):
                    if i not in active and k not in active:
                        out.append(NativeOp("zz_idle", (i, k), (t, float(dev["freq_zz"]))))
        for j in range(n):
            if j not in active:
                out.append(NativeOp("idle_depol", (j,), (t, float(dev["t1"][j]), float(dev["t2"][j]))))

    for op in ops:
        if op.name in ("rx", "ry", "rz"):
            q = op.qubits[0]
            f = dev["freq_z"][q] if op.name == "rz" else dev["freq_xy"][q]
            t = abs(op.params[0]) / (2 * math.pi * float(f))
            out.append(op)
            if op.name != "rz":
                out += scaled_standard_error(1, (q,), float(dev["fid_xy"][q]), float(dev["x_xy"]), op.params[0])
            elif dev["fid_z"][q] < 1:
                out += scaled_standard_error(1, (q,), float(dev["fid_z"][q]), 0.0, op.params[0])
            outside((q,), t)
        elif op.name in ("zx", "zy"):
            c, j = op.qubits
            if c != 0:
                raise ValueError("conditional rotations are controlled by the electron spin (qubit 0)")
            t = abs(op.params[0]) / (2 * math.pi * float(dev["freq_crot"][j - 1]))
            out.append(op)
            out += scaled_standard_error(2, (0, j), float(dev["fid_crot"][j - 1]), float(dev["x_crot"]), op.params[0])
            outside((0, j), t)
        else:
            raise ValueError(f"{op.name} is not an NV-centre native gate")
    if readout:
        out += [NativeOp("rx", (0,), (math.pi,)), NativeOp("amp", (0,), (1.0 - float(dev["fid_meas"]),)),
                NativeOp("rx", (0,), (math.pi,))]
        outside((0,), float(dev["dur_meas"]))
    return out


# ------------------------------------------------------------------ trapped ions (Sec. 4, App. C)
def ion_compile(dev: Dict, ops: Sequence[NativeOp], readout: bool = False) -> List[NativeOp]:
    """Logical circuit -> native op list of the trapped-ion device (Sec. 4, App. C), without zones or shuttling.

    Serial gates:
    - Rx/Ry last |theta| / (2 pi f_Rabi) and carry the standard error of their fidelity, scaled by |theta|/pi.
    - Rz is virtual: instantaneous and exact.
    - CZ lasts 1 / (2 f_CZ) (a phase pi at the gate frequency) and carries its standard error.
    - The other ions decay passively over each gate: T1 as depolarising, then Gaussian T2* dephasing.
    - Readout flips each ion's bit with the tabulated probability, one ion at a time; the ions not yet
      read decay during each readout.
    """
    n = int(dev["n"])
    passive = not (int(dev.get("flags", 0)) & 1)
    out: List[NativeOp] = []

    def idle_others(active, t, first=0):
        if passive and t > 0:
            for j in range(first, n):
                if j not in active:
                    out.append(NativeOp("idle_t2s", (j,), (t, float(dev["t1"]), float(dev["t2s"]))))

    for op in ops:
        if op.name == "rz":
            out.append(op)
        elif op.name in ("rx", "ry"):
            out.append(op)
            out += scaled_standard_error(1, op.qubits, float(dev["fid_xy"]), float(dev["x_xy"]), op.params[0])
            idle_others(op.qubits, abs(op.params[0]) / (2 * math.pi * float(dev["rabi"])))
        elif op.name == "cz":
            out.append(op)
            out += scaled_standard_error(2, op.qubits, float(dev["fid_cz"]), float(dev["x_cz"]), math.pi)
            idle_others(op.qubits, 1.0 / (2 * float(dev["freq_cz"])))
        else:
            raise ValueError(f"{op.name} is not a trapped-ion native gate")
    if readout:
        for j in range(n):
            if dev["bf_read"] > 0:
                out.append(NativeOp("bitflip", (j,), (float(dev["bf_read"]),)))
            idle_others((), float(dev["dur_read"]), j + 1)
    return out


# ------------------------------------------------------------------ neutral atoms (Sec. 6, App. C)
def na_compile(dev: Dict, ops: Sequence[NativeOp], init: bool = False, readout: bool = False) -> List[NativeOp]:
    """Logical circuit -> native op list of the neutral-atom device (Sec. 6, App. C): static sites, serial gates.

    - Initialisation (optional): the leakage operator L on every atom (the perfect reset before it acts on
      |0> and changes nothing).
    - Raman rotation U(phi, Omega, Delta, t), lasting its own t: phase-type error deph(1 - e^{-t/(2 T2)}) (the
      printed exponent's sign read as a decay), then the asymmetric bit flip scaled by the rotation angle
      Omega_R t / pi (App. C's angle rule).
    - Rydberg CZ(phi) on two atoms within the blockade radius, lasting dur_cz: the leakage map K of Eq. (czleak).
    - During a gate the other atoms decay: T1 = T_vac / N as depolarising (Eq. depolt1), T2 dephasing.
    - Readout (optional): depolarising noise whose misclassification probability 2p/3 is 1 - F, so p = 3(1 - F)/2.
    """
    n = int(dev["n"])
    passive = not (int(dev.get("flags", 0)) & 1)
    t1 = float(dev["t_vac"]) / n
    out: List[NativeOp] = []

    def idle_others(active, t):
        if passive and t > 0:
            for j in range(n):
                if j not in active:
                    out.append(NativeOp("idle_depol", (j,), (t, t1, float(dev["t2"]))))

    if init:
        out += [NativeOp("leak_init", (j,), (float(dev["leak_init"]),)) for j in range(n)]
    for op in ops:
        if op.name == "u":
            q = op.qubits[0]
            phi, om, de, t = op.params
            t = abs(t)
            s = math.sqrt(om * om + de * de) * t / math.pi
            out.append(op)
            out.append(NativeOp("deph1", (q,), (1 - math.exp(-t / (2 * float(dev["t2"]))),)))
            if (dev["p10"] > 0 or dev["p01"] > 0) and s > 0:
                out.append(NativeOp("bitflip_asym", (q,), (float(dev["p10"]) * s, float(dev["p01"]) * s)))
            idle_others((q,), t)
        elif op.name == "czphi":
            a, b = op.qubits
            (xa, ya), (xb, yb) = dev["sites"][a], dev["sites"][b]
            if math.hypot(xa - xb, ya - yb) > dev["blockade"]:
                raise ValueError("CZ(phi) on atoms farther apart than the blockade radius")
            out.append(op)
            out.append(NativeOp("leak_cz", (a, b), (float(dev["leak_cz"][0]), float(dev["leak_cz"][1]))))
            idle_others((a, b), float(dev["dur_cz"]))
        else:
            raise ValueError(f"{op.name} is not a neutral-atom native gate")
    if readout:
        out += [NativeOp("depol1", (j,), (1.5 * (1 - float(dev["fid_meas"])),)) for j in range(n)]
    return out
