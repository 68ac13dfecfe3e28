"""Oracle device compiler: native operations -> unitaries and Kraus sets, in FP64.

Conventions (the paper is silent on them; the readings are stated once here):
* qubit q is bit q of a basis index (little-endian);
* for an operation on ``qubits = (q0, q1, ...)`` the matrix index is little-endian over
  that tuple: q0 is the least significant bit of the 2^k x 2^k matrix index;
* rotations: R_sigma(theta) = exp(-i theta sigma / 2); SX := Rx(pi/2).

A compiled step is ``("U", qubits, U)`` or ``("K", qubits, [K_0, K_1, ...])``.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = {"I": I2, "X": X, "Y": Y, "Z": Z}


def two(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """4x4 matrix acting as ``lo`` on the first qubit (low bit) and ``hi`` on the second (high bit)."""
    return np.kron(hi, lo)


# ------------------------------------------------------------------ native gates (unitaries)
def rx(t):
    """Rx(theta) = cos(theta/2) I - i sin(theta/2) X (rotation convention above)."""
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -1j * s], [-1j * s, c]])


def ry(t):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=complex)


def rz(t):
    return np.array([[np.exp(-0.5j * t), 0], [0, np.exp(0.5j * t)]])


def sx():
    return rx(math.pi / 2)


def hadamard():
    return np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2)


def raman_u(phi, omega, delta, t):
    """Raman single-qubit unitary U(phi, Delta, t) of Sec. 6, Eq. (u), as printed.

    Omega_tilde = sqrt(Omega^2 + Delta^2); diagonal cos -/+ i Delta/Omega_tilde sin; off-diagonals
    -i Omega/Omega_tilde sin(Omega_tilde t / 2) e^{+i phi} (top right) and e^{-i phi} (bottom left).
    """
    om = math.sqrt(omega * omega + delta * delta)
    c, s = math.cos(om * t / 2), math.sin(om * t / 2)
    return np.array([[c - 1j * delta / om * s, -1j * omega / om * s * np.exp(1j * phi)],
                     [-1j * omega / om * s * np.exp(-1j * phi), c + 1j * delta / om * s]])


def ion_r(theta, phi):
    """Ion single-qubit R(theta, phi): Eq. (u) with Delta = 0 and Omega t = theta."""
    return raman_u(phi, 1.0, 0.0, theta)


def cz():
    return np.diag([1, 1, 1, -1]).astype(complex)


def cph(phi):
    """Controlled phase CPh(phi) = diag(1, 1, 1, e^{i phi}); CZ = CPh(pi) (Sec. 7)."""
    return np.diag([1, 1, 1, np.exp(1j * phi)])


def czphi(phi):
    """Rydberg CZ(phi) of Sec. 6 as printed: diag(1, e^{i phi}, e^{i phi}, e^{i(2 phi - pi)})."""
    return np.diag([1, np.exp(1j * phi), np.exp(1j * phi), np.exp(1j * (2 * phi - math.pi))])


def pauli_rot2(sig_lo: np.ndarray, sig_hi: np.ndarray, angle: float) -> np.ndarray:
    """exp(-i angle P) for the Pauli product P = sig_hi (x) sig_lo; P^2 = I so it is cos - i sin P."""
    return math.cos(angle) * np.eye(4) - 1j * math.sin(angle) * two(sig_lo, sig_hi)


def zx(theta):
    """Cross resonance ZX(theta) = exp(-i theta/2 Z_c X_t), control c = first qubit (Sec. 8; reading:
    the printed exp(-i pi/2 Z X) is taken as ZX(pi/2) = exp(-i pi/4 Z X))."""
    return pauli_rot2(Z, X, theta / 2)


def zy(theta):
    """NV conditional rotation CRy+-(theta) of Sec. 5, Eq. (conditional_rots), as printed:
    |0><0|_c (x) Ry(theta)_t + |1><1|_c (x) Ry(-theta)_t, control c = first qubit."""
    p0 = np.diag([1, 0]).astype(complex)
    p1 = np.diag([0, 1]).astype(complex)
    return two(p0, ry(theta)) + two(p1, ry(-theta))


def zz(theta):
    return pauli_rot2(Z, Z, theta / 2)


def xx(theta):
    """Molmer-Sorensen XX(theta) = exp(-i theta/2 X X) (named, not defined, in Sec. 4)."""
    return pauli_rot2(X, X, theta / 2)


def zzphase(alpha):
    """ZZ crosstalk exp(-i alpha Z_p Z_q), Sec. 3.4 Eq. (weak_dephasing_zz)."""
    return pauli_rot2(Z, Z, alpha)


def zz_idle(dt, xi):
    """Static ZZ crosstalk of rate xi (MHz) over dt (us): exp(-i alpha ZZ) with alpha = pi xi dt / 2.

    Reading: xi is the conditional frequency shift, so the conditional phase 2 pi xi dt equals 4 alpha.
    """
    return zzphase(math.pi * xi * dt / 2)


def off_resonant(omega, delta, t):
    """Off-resonant Rabi drive on a passive qubit, Sec. 3.3 Eq. (off_resonant), as printed.

    With Omega_R = sqrt(Omega^2 + Delta^2) and h = Omega_R t / 2: the top row is
    ((cos h - i Delta/Omega_R sin h) e^{ih}, -i Omega/Omega_R sin h e^{ih}) and the bottom row
    (-i Omega/Omega_R sin h e^{-ih}, (cos h + i Delta/Omega_R sin h) e^{-ih}).  It tends to the identity
    for Delta >> Omega; for Delta < 0 the printed frame phase leaves a Z rotation by Omega_R t.
    Omega_R = 0 is the limit of the formula, the identity.
    """
    om_r = math.sqrt(omega * omega + delta * delta)
    if om_r == 0.0:
        return np.eye(2, dtype=complex)
    h = om_r * t / 2
    c, s = math.cos(h), math.sin(h)
    ph = np.exp(1j * h)
    return np.array([[(c - 1j * delta / om_r * s) * ph, -1j * omega / om_r * s * ph],
                     [-1j * omega / om_r * s / ph, (c + 1j * delta / om_r * s) / ph]])


def static_zz_beta(j, delta_ct, alpha_t, alpha_c):
    """Static ZZ strength of two capacitively coupled transmons, Sec. 8:
    beta = J^2 (1/(Delta_ct - alpha_t) - 1/(Delta_ct + alpha_c))."""
    d1, d2 = delta_ct - alpha_t, delta_ct + alpha_c
    if d1 == 0.0 or d2 == 0.0:
        raise ValueError("zz_static: Delta_ct - alpha_t or Delta_ct + alpha_c is zero")
    return j * j * (1.0 / d1 - 1.0 / d2)


def zz_static(j, delta_ct, alpha_t, alpha_c):
    """Static ZZ crosstalk exp(-i beta Z_c Z_t) of Sec. 8 with beta from static_zz_beta.

    Reading: the four parameters are the frequencies times the idle duration (J dt, Delta dt,
    alpha dt), so beta, homogeneous of degree one in them, is the accumulated phase beta dt.
    """
    return zzphase(static_zz_beta(j, delta_ct, alpha_t, alpha_c))


def crz_xtalk(alpha):
    """Conditional-Rz crosstalk |0><0|_p (x) I_q + |1><1|_p (x) Rz(alpha)_q, Eq. (weak_dephasing); p = first."""
    p0 = np.diag([1, 0]).astype(complex)
    p1 = np.diag([0, 1]).astype(complex)
    return two(p0, I2) + two(p1, rz(alpha))


def exchange(theta):
    """Exchange crosstalk exp(-i (XX + YY + ZZ) theta / 4), Eq. (exchange_pauli).

    XX, YY and ZZ commute, so the exponential factorises into three Pauli rotations.
    """
    return pauli_rot2(X, X, theta / 4) @ pauli_rot2(Y, Y, theta / 4) @ pauli_rot2(Z, Z, theta / 4)


# ------------------------------------------------------------------ noise channels (Kraus sets)
def pauli_channel_1(probs):
    """Kraus set of sum_s w_s sigma_s rho sigma_s for weights (w_I, w_X, w_Y, w_Z)."""
    return [math.sqrt(w) * P for w, P in zip(probs, (I2, X, Y, Z)) if w > 0] or [0 * I2]


def depol1(p):
    """One-qubit depolarising, Eq. (depol1): (1-p) rho + p/3 sum_sigma sigma rho sigma."""
    return pauli_channel_1((1 - p, p / 3, p / 3, p / 3))


def depol2(p):
    """Two-qubit depolarising, Eq. (depol2).  Reading: all 15 non-identity Pauli pairs, weight p/15 each."""
    ks = []
    for a, A in enumerate((I2, X, Y, Z)):
        for b, B in enumerate((I2, X, Y, Z)):
            w = (1 - p) if (a == 0 and b == 0) else p / 15
            if w > 0:
                ks.append(math.sqrt(w) * two(A, B))
    return ks


def deph1(p):
    """One-qubit dephasing, Eq. (deph1): (1-p) rho + p Z rho Z."""
    return pauli_channel_1((1 - p, 0, 0, p))


def deph2(p):
    """Two-qubit dephasing, Eq. (deph2): (1-p) rho + p/3 (Z_i rho Z_i + Z_j rho Z_j + Z_i Z_j rho Z_i Z_j)."""
    ks = [math.sqrt(1 - p) * np.eye(4, dtype=complex)]
    if p > 0:
        for A, B in ((Z, I2), (I2, Z), (Z, Z)):
            ks.append(math.sqrt(p / 3) * two(A, B))
    return ks


def amp(p):
    """Amplitude damping, Eq. (damp): {[[1,0],[0,sqrt(1-p)]], [[0,sqrt(p)],[0,0]]}."""
    return [np.array([[1, 0], [0, math.sqrt(1 - p)]], dtype=complex),
            np.array([[0, math.sqrt(p)], [0, 0]], dtype=complex)]


def bitflip(b):
    """Bit flip, Eq. (bf): (1-b) rho + b X rho X."""
    return pauli_channel_1((1 - b, b, 0, 0))


def bitflip2(b):
    """Two-qubit bit flip, Eq. (bf2): (1-b) rho + b/3 (X_i rho X_i + X_j rho X_j + X_i X_j rho X_i X_j)."""
    ks = [math.sqrt(1 - b) * np.eye(4, dtype=complex)]
    if b > 0:
        for A, B in ((X, I2), (I2, X), (X, X)):
            ks.append(math.sqrt(b / 3) * two(A, B))
    return ks


def gamp(dt, t1, p0):
    """Generalised amplitude damping, Eq. (gdamp), gamma = 1 - exp(-dt/T1), p0 = ground population."""
    g = 1 - math.exp(-dt / t1)
    a, b = math.sqrt(p0), math.sqrt(1 - p0)
    return [a * np.array([[1, 0], [0, math.sqrt(1 - g)]], dtype=complex),
            a * np.array([[0, math.sqrt(g)], [0, 0]], dtype=complex),
            b * np.array([[math.sqrt(1 - g), 0], [0, 1]], dtype=complex),
            b * np.array([[0, 0], [math.sqrt(g), 0]], dtype=complex)]


def t1_damping_param(dt, t1):
    """Eq. (ampt1): amp(1 - exp(-dt/T1))."""
    return 1 - math.exp(-dt / t1)


def t1_depol_param(dt, t1):
    """Eq. (depolt1): depol(3/4 (1 - exp(-dt/T1)))."""
    return 0.75 * (1 - math.exp(-dt / t1))


def t2_deph_param(dt, t2):
    """Eq. (depht2): deph(1/2 (1 - exp(-dt/T2)))."""
    return 0.5 * (1 - math.exp(-dt / t2))


def bitflip_asym(p10, p01):
    """Asymmetric bit flip of Sec. 6: |1> decays to |0> with probability p10, |0> is excited to |1> with
    probability p01; Kraus operators diag(sqrt(1-p01), sqrt(1-p10)), sqrt(p10)|0><1|, sqrt(p01)|1><0|."""
    return [np.array([[math.sqrt(1 - p01), 0], [0, math.sqrt(1 - p10)]], dtype=complex),
            np.array([[0, math.sqrt(p10)], [0, 0]], dtype=complex),
            np.array([[0, 0], [math.sqrt(p01), 0]], dtype=complex)]


def t2s_deph_param(dt, t2s):
    """Eq. (depht2s): deph(1/2 (1 - exp(-(dt/T2*)^2))), the Gaussian free-induction decay."""
    return 0.5 * (1 - math.exp(-((dt / t2s) ** 2)))


def pure_dephasing_time(t1, t2):
    """T_phi with 1/T2 = 1/(2 T1) + 1/T_phi (used when T2 is read as the total coherence time)."""
    return 1.0 / (1.0 / t2 - 1.0 / (2.0 * t1))


def leak_init(gamma):
    """CPTN initialisation leakage L = diag(sqrt(1-gamma), 1) (Sec. 6)."""
    return [np.diag([math.sqrt(1 - gamma), 1.0]).astype(complex)]


def leak_cz(alpha, beta):
    """CPTN Rydberg-decay operator K = diag(1, sqrt(1-a), sqrt(1-a), sqrt(1-b)), Eq. (czleak)."""
    return [np.diag([1.0, math.sqrt(1 - alpha), math.sqrt(1 - alpha), math.sqrt(1 - beta)]).astype(complex)]


def compose_kraus(first: Sequence[np.ndarray], second: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Kraus set of (second o first): {B A}."""
    return [B @ A for A in first for B in second]


def tensor_kraus(lo: Sequence[np.ndarray], hi: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Kraus set of the product channel lo (first qubit) (x) hi (second qubit)."""
    return [two(A, B) for A in lo for B in hi]


# ------------------------------------------------------------------ App. B: fidelity -> error parameters
def entanglement_fidelity_from_average(fbar: float, d: int) -> float:
    """Invert Eq. (fidelities_relation): Fbar = (d F_e + 1)/(d + 1)  =>  F_e = ((d + 1) Fbar - 1)/d."""
    return ((d + 1) * fbar - 1) / d


def stderr_params(fbar: float, x: float, nq: int) -> Tuple[float, float]:
    """Standard-error severities from an average gate fidelity (App. B).

    Reading of the printed equation: one unknown eps with dephasing p = (1 - x) eps and
    depolarising q = x eps, so that F_e = 1 - p - q + c p q with c = 4/3 (one qubit, Eq. fe1)
    or 16/15 (two qubits).  This gives c x (1 - x) eps^2 - eps + (1 - F_e) = 0; the smallest
    non-negative root is taken.  Returns (p_deph, q_depol).
    """
    d = 2 ** nq
    c = 4.0 / 3.0 if nq == 1 else 16.0 / 15.0
    fe = entanglement_fidelity_from_average(fbar, d)
    a = c * x * (1 - x)
    if a == 0.0:
        eps = 1 - fe
    else:
        eps = (1 - math.sqrt(1 - 4 * a * (1 - fe))) / (2 * a)
    return (1 - x) * eps, x * eps


# ------------------------------------------------------------------ the compiler
def compile_op(name: str, qubits: Sequence[int], params: Sequence[float], t2_is_total: bool = False):
    """One native operation -> list of steps ("U", qubits, U) / ("K", qubits, [K...]), applied in order."""
    q = tuple(qubits)
    P = tuple(params)
    unitary = {
        "rx": lambda: rx(*P), "ry": lambda: ry(*P), "rz": lambda: rz(*P), "sx": sx, "h": hadamard,
        "u": lambda: raman_u(*P), "r": lambda: ion_r(*P), "cz": cz, "cph": lambda: cph(*P),
        "czphi": lambda: czphi(*P), "zx": lambda: zx(*P), "zz": lambda: zz(*P), "xx": lambda: xx(*P),
        "zzphase": lambda: zzphase(*P), "zz_idle": lambda: zz_idle(*P), "crz_xtalk": lambda: crz_xtalk(*P),
        "exchange": lambda: exchange(*P), "offres": lambda: off_resonant(*P), "zz_static": lambda: zz_static(*P),
        "zy": lambda: zy(*P),
    }
    if name in unitary:
        return [("U", q, unitary[name]())]
    simple = {"depol1": depol1, "depol2": depol2, "deph1": deph1, "deph2": deph2, "amp": amp,
              "bitflip": bitflip, "bitflip2": bitflip2, "leak_init": leak_init, "leak_cz": leak_cz,
              "bitflip_asym": bitflip_asym}
    if name in simple:
        return [("K", q, simple[name](*P))]
    if name == "gamp":
        return [("K", q, gamp(*P))]
    if name in ("idle", "idle_depol", "ampdeph2"):
        dt, t1, t2 = P
        tphi = pure_dephasing_time(t1, t2) if t2_is_total else t2
        dephk = deph1(t2_deph_param(dt, tphi))
        if name == "idle":          # Eq. (ampt1) then Eq. (depht2) on one qubit
            return [("K", q, amp(t1_damping_param(dt, t1))), ("K", q, dephk)]
        if name == "idle_depol":    # Eq. (depolt1) then Eq. (depht2)
            return [("K", q, depol1(t1_depol_param(dt, t1))), ("K", q, dephk)]
        one = compose_kraus(amp(t1_damping_param(dt, t1)), dephk)   # deph o amp on one qubit
        return [("K", q, tensor_kraus(one, one))]
    if name == "idle_t2s":          # Eq. (depolt1) then Eq. (depht2s)
        dt, t1, t2s = P
        return [("K", q, depol1(t1_depol_param(dt, t1))), ("K", q, deph1(t2s_deph_param(dt, t2s)))]
    if name in ("stderr1", "stderr2"):
        nq = 1 if name == "stderr1" else 2
        p, qd = stderr_params(P[0], P[1], nq)
        dep = depol1(qd) if nq == 1 else depol2(qd)
        dph = deph1(p) if nq == 1 else deph2(p)
        return [("K", q, dep), ("K", q, dph)]   # Eq. (stderr): deph(p) o depol(q)
    raise ValueError(f"unknown native op {name}")


def compile_program(ops, t2_is_total: bool = False):
    steps = []
    for o in ops:
        steps.extend(compile_op(o.name, o.qubits, o.params, t2_is_total))
    return steps
