"""Pins of the oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper (section / equation) or the mathematical fact it
relies on.  None of these tests needs a GPU.
"""
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import brute, evolve, measure
from oracle import compile as oc
from workloads.circuits import OP_NAMES, random_program

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
I2, X, Y, Z = oc.I2, oc.X, oc.Y, oc.Z


def rand_state(n, rng, rank=None):
    d = 2 ** n
    rank = rank or d
    A = rng.normal(size=(d, rank)) + 1j * rng.normal(size=(d, rank))
    rho = A @ A.conj().T
    return rho / np.trace(rho)


def rand_unitary(d, rng):
    q, r = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def rand_kraus(d, nk, rng):
    """Random CPTP Kraus set from a random isometry (Stinespring): stacked K's have orthonormal columns."""
    V = rand_unitary(d * nk, rng)[:, :d]
    return [V[i * d:(i + 1) * d, :] for i in range(nk)]


def same_up_to_phase(A, B, tol=1e-12):
    i = np.unravel_index(np.argmax(np.abs(B)), B.shape)
    ph = A[i] / B[i]
    return abs(abs(ph) - 1) < tol and np.allclose(A, ph * B, atol=tol, rtol=0)


# ---------------------------------------------------------------- gate definitions
@pytest.mark.parametrize("theta", [0.0, 0.3, 1.7, math.pi, 5.9])
def test_rotations_match_matrix_exponentials(theta):
    # R_sigma(theta) = exp(-i theta sigma / 2), checked with scipy's matrix exponential
    assert np.allclose(oc.rx(theta), expm(-0.5j * theta * X), atol=1e-14)
    assert np.allclose(oc.ry(theta), expm(-0.5j * theta * Y), atol=1e-14)
    assert np.allclose(oc.rz(theta), expm(-0.5j * theta * Z), atol=1e-14)


@pytest.mark.parametrize("theta", [0.4, math.pi / 2, 2.9])
def test_two_qubit_rotations_match_exponentials(theta):
    # first qubit = low bit of the matrix index, so Z_c X_t with c first is kron(X, Z)
    assert np.allclose(oc.zx(theta), expm(-0.5j * theta * np.kron(X, Z)), atol=1e-14)
    assert np.allclose(oc.zz(theta), expm(-0.5j * theta * np.kron(Z, Z)), atol=1e-14)
    assert np.allclose(oc.xx(theta), expm(-0.5j * theta * np.kron(X, X)), atol=1e-14)
    assert np.allclose(oc.zzphase(theta), expm(-1j * theta * np.kron(Z, Z)), atol=1e-14)
    H = np.kron(X, X) + np.kron(Y, Y) + np.kron(Z, Z)
    assert np.allclose(oc.exchange(theta), expm(-0.25j * theta * H), atol=1e-14)       # Eq. (exchange_pauli)
    # controlled Rz on the second qubit, control first: exp(-i theta/2 |1><1|_c Z_t)
    proj1 = np.diag([0, 1]).astype(complex)
    assert np.allclose(oc.crz_xtalk(theta), expm(-0.5j * theta * np.kron(Z, proj1)), atol=1e-14)


def test_named_gate_identities():
    assert same_up_to_phase(oc.sx() @ oc.sx(), X)
    assert np.allclose(oc.cph(math.pi), oc.cz())                 # CZ = CPh(pi), Sec. 7
    assert same_up_to_phase(oc.czphi(0.0), oc.cz())               # Rydberg CZ(phi=0) is a CZ
    assert same_up_to_phase(oc.hadamard() @ Z @ oc.hadamard(), X)
    # ZX(pi/2) is maximally entangling: it maps |+>|0> ... to a Bell-type state with zero purity of the reduced state
    psi = oc.zx(math.pi / 2) @ np.kron([1, 0], [1, 1]).astype(complex) / math.sqrt(2)
    red = np.einsum("ab,cb->ac", psi.reshape(2, 2), psi.reshape(2, 2).conj())
    assert abs(np.trace(red @ red).real - 0.5) < 1e-14


def test_raman_u_worked_examples_golden():
    """Sec. 6 after Eq. (u): H = U(0, Delta=Omega, pi/Omega_tilde) and Rx(theta) = U(0, 0, theta/Omega)."""
    with open(os.path.join(GOLDEN, "raman_u_examples.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for name, phi, om, de, t, gate in rows:
        U = oc.raman_u(float(phi), float(om), float(de), float(t))
        want = oc.hadamard() if gate == "H" else oc.rx(float(gate[2:]))
        assert same_up_to_phase(U, want), name


def test_ion_r_and_zz_idle_readings():
    assert np.allclose(oc.ion_r(1.1, 0.0), oc.rx(1.1))
    # R(theta, phi) = exp(-i theta/2 (cos(phi) X - sin(phi) Y)) as printed (e^{+i phi} top right)
    th, ph = 0.8, 0.6
    gen = math.cos(ph) * X - math.sin(ph) * Y
    assert np.allclose(oc.ion_r(th, ph), expm(-0.5j * th * gen), atol=1e-14)
    # ZZ crosstalk: conditional phase phi11 - phi10 - phi01 + phi00 equals -2 pi xi dt
    dt, xi = 0.5, 0.05
    d = np.angle(np.diag(oc.zz_idle(dt, xi)))
    cond = d[3] - d[1] - d[2] + d[0]
    assert abs(np.angle(np.exp(1j * (cond + 2 * math.pi * xi * dt)))) < 1e-13


# ---------------------------------------------------------------- embedding and Kraus evolution
@pytest.mark.parametrize("n,targets", [(3, (0,)), (3, (2,)), (4, (1, 3)), (4, (3, 1)), (5, (4, 0)), (5, (2, 3))])
def test_unitary_embedding_matches_kronecker_chain(n, targets):
    rng = np.random.default_rng(10 + n)
    U = rand_unitary(2 ** len(targets), rng)
    rho = rand_state(n, rng)
    full = brute.full_operator(U, targets, n)
    want = full @ rho @ full.conj().T
    for method in ("tensor", "dense"):
        got = evolve.apply_unitary(rho, targets, U, method)
        assert np.abs(got - want).max() < 1e-13, method


@pytest.mark.parametrize("n,targets,nk", [(2, (1,), 3), (3, (0, 2), 4), (4, (3, 0), 5), (4, (2,), 2)])
def test_kraus_matches_brute_superoperator(n, targets, nk):
    """vec(K rho K^dagger) = (conj(K) (x) K) vec(rho): the 4^n x 4^n superoperator, applied to vec(rho)."""
    rng = np.random.default_rng(100 + n + nk)
    ks = rand_kraus(2 ** len(targets), nk, rng)
    rho = rand_state(n, rng)
    S = brute.superop([brute.full_operator(K, targets, n) for K in ks])
    want = brute.unvec(S @ brute.vec(rho))
    got = evolve.apply_kraus(rho, targets, ks)
    assert np.abs(got - want).max() < 1e-13
    # the same superoperator written in the device layout index r + c 2^n
    assert np.allclose(evolve.to_device_layout(got), S @ evolve.to_device_layout(rho), atol=1e-13)


def test_superop_application_matches_kraus_form():
    """A superoperator built as sum conj(K) (x) K (index r | c << k) acts like the Kraus map itself."""
    rng = np.random.default_rng(17)
    for n, qs in [(3, (1,)), (4, (3, 0)), (4, (1, 2))]:
        ks = rand_kraus(2 ** len(qs), 3, rng)
        S = sum(np.kron(K.conj(), K) for K in ks)
        rho = rand_state(n, rng)
        assert np.abs(evolve.apply_superop(rho, qs, S) - evolve.apply_kraus(rho, qs, ks)).max() < 1e-14


def test_tensor_and_dense_methods_agree_on_random_program():
    prog = random_program(7, 5, 120)
    a = evolve.run_program(prog, "tensor")
    b = evolve.run_program(prog, "dense")
    assert np.abs(a - b).max() < 1e-13


def test_device_layout_roundtrip():
    rng = np.random.default_rng(3)
    rho = rand_state(3, rng)
    v = evolve.to_device_layout(rho)
    r, c = 5, 2
    assert v[r + c * 8] == rho[r, c]
    assert np.array_equal(evolve.from_device_layout(v), rho)


# ---------------------------------------------------------------- channel closed forms (Sec. 3.1)
def _golden_ranges():
    with open(os.path.join(GOLDEN, "channel_ranges.txt")) as f:
        return {ln.split()[0]: float(ln.split()[1]) for ln in f if ln.strip() and not ln.startswith("#")}


def _bit(x, q):
    return (x >> q) & 1


def test_extreme_channels_closed_forms():
    g = _golden_ranges()
    rng = np.random.default_rng(5)
    n = 3
    rho = rand_state(n, rng)
    d = 2 ** n
    R, C = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    # depol1(3/4) on qubit 1: tr_1(rho) (x) I/2
    q = 1
    out = evolve.apply_kraus(rho, (q,), oc.depol1(g["depol1"]))
    want = np.zeros_like(rho)
    for r in range(d):
        for c in range(d):
            if _bit(r, q) == _bit(c, q):
                r0, c0 = r & ~(1 << q), c & ~(1 << q)
                want[r, c] = 0.5 * (rho[r0, c0] + rho[r0 | 1 << q, c0 | 1 << q])
    assert np.abs(out - want).max() < 1e-14
    # depol2(15/16) on qubits (0, 2): tr_{02}(rho) (x) I/4
    out = evolve.apply_kraus(rho, (0, 2), oc.depol2(g["depol2"]))
    want = np.zeros_like(rho)
    m = (1 << 0) | (1 << 2)
    for r in range(d):
        for c in range(d):
            if (r & m) == (c & m):
                want[r, c] = 0.25 * sum(rho[(r & ~m) | v, (c & ~m) | v] for v in (0, 1, 4, 5))
    assert np.abs(out - want).max() < 1e-14
    # deph1(1/2) on qubit 2: coherences in qubit 2 vanish, the rest unchanged
    out = evolve.apply_kraus(rho, (2,), oc.deph1(g["deph1"]))
    want = np.where(_bit(R, 2) == _bit(C, 2), rho, 0)
    assert np.abs(out - want).max() < 1e-15
    # deph2(3/4) on (0, 1): coherences in either qubit vanish
    out = evolve.apply_kraus(rho, (0, 1), oc.deph2(g["deph2"]))
    want = np.where((_bit(R, 0) == _bit(C, 0)) & (_bit(R, 1) == _bit(C, 1)), rho, 0)
    assert np.abs(out - want).max() < 1e-15
    # amp(1) resets the qubit: tr_q(rho) (x) |0><0|
    q = 0
    out = evolve.apply_kraus(rho, (q,), oc.amp(g["amp"]))
    want = np.zeros_like(rho)
    for r in range(d):
        for c in range(d):
            if _bit(r, q) == 0 and _bit(c, q) == 0:
                want[r, c] = rho[r, c] + rho[r | 1, c | 1]
    assert np.abs(out - want).max() < 1e-15
    # bitflip(1/2): the result is invariant under X on the qubit
    out = evolve.apply_kraus(rho, (1,), oc.bitflip(g["bitflip"]))
    assert np.abs(out - evolve.apply_unitary(out, (1,), X)).max() < 1e-15


def test_amp_p1_gives_ground_state():
    rho = rand_state(1, np.random.default_rng(9))
    out = evolve.apply_kraus(rho, (0,), oc.amp(1.0))
    assert np.allclose(out, np.diag([1, 0]), atol=1e-15)


# ---------------------------------------------------------------- passive decay (Sec. 3.5)
@pytest.mark.parametrize("t2_is_total", [False, True])
def test_idle_t1_t2_closed_forms(t2_is_total):
    rho = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, 0.7]])
    dt, t1, t2 = 3.0, 40.0, 25.0
    steps = oc.compile_op("idle", (0,), (dt, t1, t2), t2_is_total)
    out = evolve.apply_steps(rho.astype(complex), steps)
    assert abs(out[1, 1] - 0.7 * math.exp(-dt / t1)) < 1e-15            # Eq. (ampt1): rho11 e^{-t/T1}
    coh = math.exp(-dt / t2) if t2_is_total else math.exp(-dt / (2 * t1)) * math.exp(-dt / t2)
    assert abs(out[0, 1] - rho[0, 1] * coh) < 1e-15                     # Eq. (depht2) with amp's sqrt(1-g)
    assert abs(np.trace(out) - 1) < 1e-15


def test_idle_is_a_semigroup():
    rng = np.random.default_rng(11)
    rho = rand_state(2, rng)
    for name in ("idle", "idle_depol"):
        a = evolve.apply_steps(rho, oc.compile_op(name, (1,), (1.5, 30.0, 20.0)))
        a = evolve.apply_steps(a, oc.compile_op(name, (1,), (2.5, 30.0, 20.0)))
        b = evolve.apply_steps(rho, oc.compile_op(name, (1,), (4.0, 30.0, 20.0)))
        assert np.abs(a - b).max() < 1e-14, name


def test_idle_depol_bloch_contraction():
    rho = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, 0.7]])
    dt, t1, t2 = 2.0, 10.0, 30.0
    out = evolve.apply_steps(rho, oc.compile_op("idle_depol", (0,), (dt, t1, t2)))
    lam = math.exp(-dt / t1)                          # Eq. (depolt1): depol(3/4 (1 - e^{-t/T1}))
    assert abs((out[1, 1] - 0.5) - (0.7 - 0.5) * lam) < 1e-15
    assert abs(out[0, 1] - rho[0, 1] * lam * math.exp(-dt / t2)) < 1e-15


def test_gamp_limits():
    """Eq. (gdamp): for dt -> infinity the qubit ends in p|0><0| + (1-p)|1><1|; that state is a fixed point."""
    rho = rand_state(1, np.random.default_rng(12))
    out = evolve.apply_kraus(rho, (0,), oc.gamp(1e6, 1.0, 0.9))
    assert np.allclose(out, np.diag([0.9, 0.1]), atol=1e-14)
    fix = np.diag([0.9, 0.1]).astype(complex)
    assert np.allclose(evolve.apply_kraus(fix, (0,), oc.gamp(0.3, 1.0, 0.9)), fix, atol=1e-15)


# ---------------------------------------------------------------- Bell-state depolarisation
def bell():
    psi = np.zeros(4, dtype=complex)
    psi[0] = psi[3] = 1 / math.sqrt(2)
    return psi


@pytest.mark.parametrize("p", [0.0, 0.05, 0.3, 0.7])
def test_bell_state_fidelities(p):
    psi = bell()
    rho = np.outer(psi, psi.conj())
    f = lambda r: measure.fidelity_pure(r, psi)
    assert abs(f(evolve.apply_kraus(rho, (0, 1), oc.depol2(p))) - (1 - 4 * p / 5)) < 1e-14
    assert abs(f(evolve.apply_kraus(rho, (0,), oc.depol1(p))) - (1 - p)) < 1e-14
    both = evolve.apply_kraus(evolve.apply_kraus(rho, (0,), oc.depol1(p)), (1,), oc.depol1(p))
    assert abs(f(both) - ((1 - p) ** 2 + p * p / 3)) < 1e-14
    if p <= 0.75:
        assert abs(f(evolve.apply_kraus(rho, (0, 1), oc.deph2(p))) - (1 - 2 * p / 3)) < 1e-14


# ---------------------------------------------------------------- App. B
def _golden_fe():
    with open(os.path.join(GOLDEN, "app_b_entanglement_fidelity.txt")) as f:
        return [tuple(float(x) for x in ln.split()) for ln in f if ln.strip() and not ln.startswith("#")]


def _entanglement_fidelity(nq, steps):
    """F_e = <Phi|(E (x) I)(|Phi><Phi|)|Phi> with E on the first nq qubits of 2 nq (Eq. def_entanglement_fidelity)."""
    if nq == 1:
        psi = bell()                               # qubits (0, 1)
        qs = (0,)
    else:
        psi = np.zeros(16, dtype=complex)          # |Phi+>_{0,2} |Phi+>_{1,3}
        for a in (0, 1):
            for b in (0, 1):
                psi[a | (b << 1) | (a << 2) | (b << 3)] = 0.5
        qs = (0, 1)
    rho = np.outer(psi, psi.conj())
    for kind, _, m in steps:
        rho = evolve.apply_kraus(rho, qs, [m] if kind == "U" else m)
    return measure.fidelity_pure(rho, psi)


def test_app_b_entanglement_fidelity_golden():
    for nq, p, q, fe in _golden_fe():
        nq = int(nq)
        dep = oc.depol1(q) if nq == 1 else oc.depol2(q)
        dph = oc.deph1(p) if nq == 1 else oc.deph2(p)
        got = _entanglement_fidelity(nq, [("K", None, dep), ("K", None, dph)])
        assert abs(got - fe) < 1e-14, (nq, p, q)


@pytest.mark.parametrize("nq", [1, 2])
@pytest.mark.parametrize("fbar,x", [(0.999, 0.0), (0.995, 1.0), (0.98, 0.3), (0.9, 0.8)])
def test_stderr_inversion_round_trip(nq, fbar, x):
    """Compiling stderr(Fbar, x) and measuring F_e on |Phi+> gives back Fbar via Eq. (fidelities_relation)."""
    name = "stderr1" if nq == 1 else "stderr2"
    qubits = (0,) if nq == 1 else (0, 1)
    steps = oc.compile_op(name, qubits, (fbar, x))
    fe = _entanglement_fidelity(nq, steps)
    d = 2 ** nq
    assert abs((d * fe + 1) / (d + 1) - fbar) < 1e-13
    p, q = oc.stderr_params(fbar, x, nq)
    assert p >= 0 and q >= 0
    if x == 0.0:
        assert q == 0.0
    if x == 1.0:
        assert p == 0.0


# ---------------------------------------------------------------- device-family crosstalk (Secs. 3.3, 8)
@pytest.mark.parametrize("omega,delta,t", [(1.0, 0.0, 0.7), (0.8, 1.3, 2.1), (2.0, -3.0, 1.1), (0.0, 0.9, 1.7),
                                           (1.5, 40.0, 0.3), (0.0, -0.9, 1.7), (1.2, -25.0, 2.2)])
def test_off_resonant_is_frame_phase_times_detuned_rotation(omega, delta, t):
    """Eq. (off_resonant) as printed is exp(+i Omega_R t Z/2) exp(-i t (Omega X + Delta Z)/2): a detuned Rabi
    rotation seen from a frame turning at Omega_R.  Both factors from the matrix exponential of their generators."""
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)
    om_r = math.hypot(omega, delta)
    want = expm(0.5j * om_r * t * Z) @ expm(-0.5j * t * (omega * X + delta * Z))
    U = oc.off_resonant(omega, delta, t)
    assert np.abs(U - want).max() < 1e-14
    assert np.abs(U.conj().T @ U - np.eye(2)).max() < 1e-14


@pytest.mark.parametrize("delta", [1e2, 1e3, 1e4])
def test_off_resonant_tends_to_identity_for_large_detuning(delta):
    """Sec. 3.3: the passive qubit is left alone when Delta >> Omega; |U - I| <= Omega / Delta.  (As printed the
    frame phase turns with +Omega_R, so the limit is the identity for a positive frequency difference.)"""
    for omega, t in [(1.0, 0.9), (2.5, 3.0)]:
        U = oc.off_resonant(omega, delta, t)
        assert np.abs(U - np.eye(2)).max() <= omega / abs(delta) * 1.0001


def test_off_resonant_special_cases():
    """Omega = Delta = 0: identity (limit of the formula).  Omega = 0: no population transfer.
    Resonance (Delta = 0): Rz(-Omega t) Rx(Omega t) with the textbook rotations."""
    assert np.abs(oc.off_resonant(0.0, 0.0, 5.0) - np.eye(2)).max() == 0.0
    U = oc.off_resonant(0.0, 1.7, 0.6)
    assert abs(U[0, 1]) == 0.0 and abs(U[1, 0]) == 0.0
    w = 1.3 * 0.8
    rz = np.diag([np.exp(-0.5j * -w), np.exp(0.5j * -w)])
    rx = np.array([[math.cos(w / 2), -1j * math.sin(w / 2)], [-1j * math.sin(w / 2), math.cos(w / 2)]])
    assert np.abs(oc.off_resonant(1.3, 0.0, 0.8) - rz @ rx).max() < 1e-15


def test_static_zz_beta_worked_value_and_matrix():
    """J = 0.1, Delta = 0.5, alpha_t = -2.5, alpha_c = -2.0: beta = 0.01 (1/3 + 2/3) = 0.01 (Sec. 8 formula,
    by hand); the op is the matrix exponential of -i beta Z Z."""
    beta = oc.static_zz_beta(0.1, 0.5, -2.5, -2.0)
    assert abs(beta - 0.01) < 1e-17
    Z = np.diag([1.0, -1.0])
    assert np.abs(oc.zz_static(0.1, 0.5, -2.5, -2.0) - expm(-1j * 0.01 * np.kron(Z, Z))).max() < 1e-15


def test_static_zz_invariants():
    """beta is symmetric in the two transmons (swap alpha_c, alpha_t and flip Delta_ct), homogeneous of degree
    one in the frequencies, and zero when the anharmonicities cancel (alpha_c + alpha_t = 0)."""
    r = np.random.default_rng(5)
    for _ in range(20):
        j, d = r.uniform(0.01, 0.3), r.uniform(0.1, 1.5)
        at, ac = r.uniform(-3.5, -1.8), r.uniform(-3.5, -1.8)
        b = oc.static_zz_beta(j, d, at, ac)
        assert abs(oc.static_zz_beta(j, -d, ac, at) - b) < 1e-15
        s = r.uniform(0.1, 10.0)
        assert abs(oc.static_zz_beta(s * j, s * d, s * at, s * ac) - s * b) < 1e-14 * max(1.0, abs(s * b))
        assert abs(oc.static_zz_beta(j, d, at, -at)) < 1e-16
    with pytest.raises(ValueError):
        oc.static_zz_beta(0.1, -2.5, -2.5, -2.0)


def test_nv_conditional_rotations_are_zx_and_zy():
    """Sec. 5, Eq. (conditional_rots): |0><0|_c (x) R(theta)_t + |1><1|_c (x) R(-theta)_t is exp(-i theta/2 Z_c S_t)
    for S = X (CRx+-, the zx op) and S = Y (CRy+-, the zy op); control = first (low) qubit."""
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Y = np.array([[0, -1j], [1j, 0]])
    Z = np.diag([1.0, -1.0]).astype(complex)
    p0, p1 = np.diag([1.0, 0.0]), np.diag([0.0, 1.0])
    for theta in (0.3, 1.9, -2.4):
        crx = np.kron(oc.rx(theta), p0) + np.kron(oc.rx(-theta), p1)
        assert np.abs(oc.zx(theta) - crx).max() < 1e-15
        assert np.abs(oc.zy(theta) - expm(-0.5j * theta * np.kron(Y, Z))).max() < 1e-14
        assert np.abs(oc.zx(theta) - expm(-0.5j * theta * np.kron(X, Z))).max() < 1e-14


@pytest.mark.parametrize("dt,t1,t2s", [(3.0, 50.0, 10.0), (0.5, 1e9, 1.0), (20.0, 40.0, 1e6)])
def test_idle_t2s_closed_forms(dt, t1, t2s):
    """Eqs. (depolt1), (depht2s): after an idle of dt from |+>, <X> = e^{-dt/T1} e^{-(dt/T2*)^2} (depolarising
    shrinks the Bloch vector by 1 - 4p/3 = e^{-dt/T1}, Gaussian dephasing by 1 - 2p = e^{-(dt/T2*)^2}); from |1>,
    the population relaxes towards 1/2 as P(1) = 1/2 + e^{-dt/T1}/2."""
    from workloads.circuits import NativeOp, Program
    rho = evolve.run_program(Program(1, [NativeOp("h", (0,)), NativeOp("idle_t2s", (0,), (dt, t1, t2s))]))
    want = math.exp(-dt / t1) * math.exp(-((dt / t2s) ** 2))
    assert abs(measure.expect(rho, [[1]], [1.0]) - want) < 1e-14
    rho = evolve.run_program(Program(1, [NativeOp("rx", (0,), (math.pi,)), NativeOp("idle_t2s", (0,), (dt, t1, t2s))]))
    assert abs(measure.probs(rho, [0])[1] - (0.5 + 0.5 * math.exp(-dt / t1))) < 1e-14


@pytest.mark.parametrize("p10,p01", [(0.1, 0.0001), (0.001, 0.03), (0.0, 0.0), (1.0, 0.25)])
def test_bitflip_asym_closed_forms(p10, p01):
    """Sec. 6's asymmetric bit flip: from |1>, P(0) = p10; from |0>, P(1) = p01; the coherence of |+> is scaled by
    sqrt((1 - p01)(1 - p10)) (only the no-flip operator keeps it); the map preserves the trace."""
    from workloads.circuits import NativeOp, Program
    rho = evolve.run_program(Program(1, [NativeOp("rx", (0,), (math.pi,)), NativeOp("bitflip_asym", (0,), (p10, p01))]))
    assert abs(measure.probs(rho, [0])[0] - p10) < 1e-14
    rho = evolve.run_program(Program(1, [NativeOp("bitflip_asym", (0,), (p10, p01))]))
    assert abs(measure.probs(rho, [0])[1] - p01) < 1e-14
    rho = evolve.run_program(Program(1, [NativeOp("h", (0,)), NativeOp("bitflip_asym", (0,), (p10, p01))]))
    assert abs(2 * rho[0, 1].real - math.sqrt((1 - p01) * (1 - p10))) < 1e-14
    assert abs(measure.trace(rho) - 1) < 1e-14


def test_parity_measurement_closed_forms():
    """Sec. 7: the Bell state (|00> + |11>)/sqrt 2 has even parity with certainty and the projection leaves it as it is;
    (|01> + |10>)/sqrt 2 is odd with certainty, and the decay map K leaves the pure |10> (the deterministic
    initialisation the section describes); |++> is odd or even with probability 1/2 each."""
    bell = np.zeros(8, dtype=complex)
    bell[0] = bell[0b101] = 1 / math.sqrt(2)                # |q0 q2> in {00, 11}, q1 = 0
    bell_rho = np.outer(bell, bell.conj())
    m, pm, out = measure.parity_collapse(bell_rho, 0, 2, u=0.3, decay=False)
    assert m == 1 and abs(pm - 1) < 1e-14 and np.abs(out - bell_rho).max() < 1e-14
    # K as printed lists |00><00| and |11><11| as separate operators, so it also dephases |00> against |11>
    m, pm, out = measure.parity_collapse(bell_rho, 0, 2, u=0.3)
    assert np.abs(out - np.diag(np.diag(bell_rho))).max() < 1e-14
    psi = np.zeros(8, dtype=complex)
    psi[0b100] = psi[0b001] = 1 / math.sqrt(2)              # (|01> + |10>)/sqrt 2 on (q0, q2)
    m, pm, out = measure.parity_collapse(np.outer(psi, psi.conj()), 0, 2, u=0.99)
    want = np.zeros((8, 8))
    want[0b001, 0b001] = 1.0                                 # q0 = 1, q2 = 0: |10>
    assert m == 0 and abs(pm - 1) < 1e-14 and np.abs(out - want).max() < 1e-14
    plus = np.full(4, 0.5, dtype=complex)
    for u, m_want in ((0.2, 0), (0.7, 1)):
        m, pm, out = measure.parity_collapse(np.outer(plus, plus.conj()), 0, 1, u=u, decay=False)
        assert m == m_want and abs(pm - 0.5) < 1e-14 and abs(np.trace(out).real - 1) < 1e-14


@pytest.mark.parametrize("seed", range(4))
def test_qnd_initialisation_is_deterministic(seed):
    """Sec. 7 (Eq. initqdots): parity readouts of (Q1, Q2) with the decay map, X on Q1 after an even outcome,
    CROT from Q3 to Q2 and X on Q3 after reading it 1, repeated once, leave |Q1 Q2 Q3> = |100> from any state."""
    from ._lib import rand_state
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    CX = np.eye(4, dtype=complex)[[0, 3, 2, 1]]
    rng = np.random.default_rng(700 + seed)
    rho = rand_state(3, rng)
    u = iter(rng.uniform(size=6))
    for _ in range(2):
        p1, _, rho = measure.parity_collapse(rho, 0, 1, next(u))
        if p1 == 1:
            rho = evolve.apply_unitary(rho, (0,), X)
        _, _, rho = measure.parity_collapse(rho, 0, 1, next(u))
        rho = evolve.apply_unitary(rho, (2, 1), CX)
        p3, _, rho = measure.parity_collapse(rho, 0, 1, next(u))
        if p3 == 1:
            rho = evolve.apply_unitary(rho, (2,), X)
    want = np.zeros((8, 8))
    want[0b001, 0b001] = 1.0
    assert np.abs(rho - want).max() < 1e-13


# ---------------------------------------------------------------- unitary circuits, graph states
def test_unitary_circuit_matches_statevector():
    n = 4
    prog = random_program(21, n, 60, names=["rx", "ry", "rz", "sx", "h", "u", "r", "cz", "cph", "czphi",
                                            "zx", "zz", "xx", "zzphase", "zz_idle", "crz_xtalk", "exchange",
                                            "offres", "zz_static", "zy"])
    psi = np.zeros(2 ** n, dtype=complex)
    psi[0] = 1
    for o in prog.ops:
        ((_, qs, U),) = oc.compile_op(o.name, o.qubits, o.params)
        psi = brute.full_operator(U, qs, n) @ psi
    rho = evolve.run_program(prog)
    assert np.abs(rho - np.outer(psi, psi.conj())).max() < 1e-13
    assert abs(measure.purity(rho) - 1) < 1e-13


def test_cluster_state_stabilisers():
    """1D cluster state (H on all, CZ on neighbours): <X_j Z_{j-1} Z_{j+1}> = 1 for every j (Sec. 6, Eq. stab)."""
    n = 5
    from workloads.circuits import NativeOp, Program
    ops = [NativeOp("h", (q,)) for q in range(n)] + [NativeOp("cz", (q, q + 1)) for q in range(n - 1)]
    rho = evolve.run_program(Program(n, ops))
    for j in range(n):
        code = [0] * n
        code[j] = 1
        if j > 0:
            code[j - 1] = 3
        if j < n - 1:
            code[j + 1] = 3
        assert abs(measure.expect(rho, [code], [1.0]) - 1) < 1e-13
        assert abs(measure.expect(rho, [code], [1.0], dense=True) - 1) < 1e-13


# ---------------------------------------------------------------- invariants and reductions
def test_cptp_invariants_on_random_programs():
    cptp = [k for k in OP_NAMES if k not in ("leak_init", "leak_cz")]
    for seed in range(3):
        rho = evolve.run_program(random_program(30 + seed, 4, 150, names=cptp))
        assert abs(measure.trace(rho) - 1) < 1e-13
        assert np.abs(rho - rho.conj().T).max() < 1e-14
        assert np.linalg.eigvalsh(rho).min() > -1e-12


def test_cptn_leakage_decreases_trace():
    rho = evolve.zero_state(1)
    out = evolve.apply_kraus(rho, (0,), oc.leak_init(0.03))
    assert abs(measure.trace(out) - 0.97) < 1e-15                   # L|0> = sqrt(1-gamma)|0>
    rho = evolve.run_program(random_program(41, 3, 80))
    assert measure.trace(rho).real <= 1 + 1e-13


def test_reductions():
    n = 3
    mixed = np.eye(2 ** n, dtype=complex) / 2 ** n
    assert abs(measure.purity(mixed) - 2.0 ** -n) < 1e-16
    rho = rand_state(n, np.random.default_rng(13))
    for q in range(n):
        p = measure.probs(rho, [q])
        code = [0] * n
        code[q] = 3
        assert abs(measure.expect(rho, [code], [1.0]) - (p[0] - p[1])) < 1e-14
    assert abs(measure.probs(rho, range(n)).sum() - measure.trace(rho).real) < 1e-15
    assert np.allclose(measure.probs(rho, [2, 0]), [
        sum(rho[r, r].real for r in range(8) if ((r >> 2) & 1) == a and (r & 1) == b)
        for b in (0, 1) for a in (0, 1)])
    # Pauli expectations by basis action agree with tr(P rho) on dense matrices, all 4^n strings
    import itertools
    for code in itertools.product(range(4), repeat=n):
        a = measure.pauli_expect_term(rho, code)
        b = np.trace(measure.pauli_matrix(code) @ rho)
        assert abs(a - b) < 1e-14
    # <Y> = 1 on (|0> + i|1>)/sqrt(2)
    psi = np.array([1, 1j]) / math.sqrt(2)
    assert abs(measure.expect(np.outer(psi, psi.conj()), [[2]], [1.0]) - 1) < 1e-15


def test_trace_distance_and_fidelity_helpers():
    a = np.diag([1.0, 0.0]).astype(complex)
    b = np.diag([0.0, 1.0]).astype(complex)
    assert abs(measure.trace_distance(a, b) - 1) < 1e-15
    assert abs(measure.uhlmann_fidelity(a, a) - 1) < 1e-12
    psi = bell()
    rho = evolve.apply_kraus(np.outer(psi, psi.conj()), (0, 1), oc.depol2(0.2))
    # square roots of near-zero eigenvalues of a rank-deficient state limit this helper to ~1e-8
    assert abs(measure.uhlmann_fidelity(rho, np.outer(psi, psi.conj())) - (1 - 0.8 * 0.2)) < 1e-7


def test_measure_collapse_bell_and_product_states():
    """Measuring one qubit of |Phi+> gives each outcome with probability 1/2 and leaves |mm><mm|; on a
    product state the other qubit's reduced state is untouched."""
    psi = bell()
    rho = np.outer(psi, psi.conj())
    for u, m_want in ((0.2, 0), (0.7, 1)):
        m, pm, out = measure.measure_collapse(rho, 0, u)
        assert m == m_want and abs(pm - 0.5) < 1e-15
        want = np.zeros((4, 4))
        want[3 * m, 3 * m] = 1.0
        assert np.abs(out - want).max() < 1e-15
    a = np.array([[0.7, 0.2 + 0.1j], [0.2 - 0.1j, 0.3]])
    b = np.array([[0.4, -0.3j], [0.3j, 0.6]])
    rho = np.kron(b, a)                               # qubit 0 in a, qubit 1 in b
    m, pm, out = measure.measure_collapse(rho, 1, force=1)
    assert abs(pm - 0.6) < 1e-15
    assert np.abs(out - np.kron(np.diag([0, 1]), a)).max() < 1e-15


# ---------------------------------------------------------------- the C-loop evaluation of the same update
@pytest.mark.parametrize("n,targets,nk", [(2, (1,), 3), (3, (0, 2), 4), (4, (3, 0), 5), (4, (2,), 2), (4, (3, 0, 1), 3),
                                          (5, (1, 4, 2, 0), 2)])
def test_c_loop_matches_brute_superoperator(n, targets, nk):
    """The loop form (oracle/c/kraus_loop.c) of sum_j K_j rho K_j^dagger against the 4^n x 4^n Kronecker
    superoperator, for one to four target qubits in any order."""
    from oracle import cloop
    rng = np.random.default_rng(300 + n + nk)
    ks = rand_kraus(2 ** len(targets), nk, rng)
    rho = rand_state(n, rng)
    S = brute.superop([brute.full_operator(K, targets, n) for K in ks])
    want = brute.unvec(S @ brute.vec(rho))
    got = cloop.apply_kraus(np.ascontiguousarray(rho), targets, ks)
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("seed,n", [(51, 3), (52, 5), (53, 7)])
def test_c_loop_and_tensor_oracle_agree_on_random_programs(seed, n):
    """Every native op kind, evaluated by the C loops and by the tensor contractions: the same result up to
    the rounding of the summation order, whatever the thread count."""
    from oracle import cloop
    prog = random_program(seed, n, 150)
    want = evolve.run_program(prog)
    for threads in (1, 3):
        got = cloop.run_program(prog, threads=threads)
        assert np.abs(got - want).max() < 1e-13
    cloop.set_threads(cloop.max_threads())


@pytest.mark.parametrize("p", [0.05, 0.7])
def test_c_loop_bell_state_fidelities(p):
    """The depolarised Bell-state fidelities (closed forms from Eqs. depol1/depol2) through the C loops."""
    from oracle import cloop
    psi = bell()
    f = lambda r: measure.fidelity_pure(r, psi)
    rho = np.ascontiguousarray(np.outer(psi, psi.conj()))
    assert abs(f(cloop.apply_kraus(rho.copy(), (0, 1), oc.depol2(p))) - (1 - 4 * p / 5)) < 1e-14
    both = cloop.apply_kraus(cloop.apply_kraus(rho.copy(), (0,), oc.depol1(p)), (1,), oc.depol1(p))
    assert abs(f(both) - ((1 - p) ** 2 + p * p / 3)) < 1e-14
