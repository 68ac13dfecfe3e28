"""Oracle reductions: Z-basis probabilities, Pauli expectation values, trace, purity (FP64).

Sums use numpy's pairwise summation.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from .compile import PAULI

PAULI_CODE = "IXYZ"   # 0 = I, 1 = X, 2 = Y, 3 = Z


def probs(rho: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    """Marginal Z-basis probabilities of ``qubits``: out[m] = sum of Re rho[r, r] over basis states r whose
    bits on ``qubits`` spell m (qubits[0] is the least significant bit of m)."""
    diag = np.real(np.diag(rho))
    idx = np.arange(diag.size)
    m = np.zeros(diag.size, dtype=np.int64)
    for j, q in enumerate(qubits):
        m |= ((idx >> q) & 1) << j
    out = np.zeros(2 ** len(qubits))
    for v in range(out.size):
        out[v] = np.sum(diag[m == v])
    return out


def pauli_matrix(code: Sequence[int]) -> np.ndarray:
    """Full Pauli string P = (x)_q sigma_{code[q]}, qubit n-1 leftmost in the Kronecker product."""
    P = np.ones((1, 1), dtype=complex)
    for q in range(len(code)):
        P = np.kron(PAULI[PAULI_CODE[code[q]]], P)
    return P


def pauli_expect_term(rho: np.ndarray, code: Sequence[int]) -> complex:
    """tr(P rho) for one Pauli string, from the action of P on basis states:
    P|c> = ph(c)|c xor x>, so tr(P rho) = sum_c ph(c) rho[c, c xor x]."""
    n = len(code)
    dim = 2 ** n
    c = np.arange(dim)
    xmask = 0
    ph = np.ones(dim, dtype=complex)
    for q, s in enumerate(code):
        b = (c >> q) & 1
        if s == 1:      # X|b> = |1-b>
            xmask |= 1 << q
        elif s == 2:    # Y|0> = i|1>, Y|1> = -i|0>
            xmask |= 1 << q
            ph *= np.where(b == 0, 1j, -1j)
        elif s == 3:    # Z|b> = (-1)^b |b>
            ph *= np.where(b == 0, 1.0, -1.0)
    return complex(np.sum(ph * rho[c, c ^ xmask]))


def expect(rho: np.ndarray, codes: Sequence[Sequence[int]], coeffs: Sequence[float], dense: bool = False) -> float:
    """Re sum_k c_k tr(P_k rho)."""
    total = 0.0
    for code, ck in zip(codes, coeffs):
        v = np.trace(pauli_matrix(code) @ rho) if dense else pauli_expect_term(rho, code)
        total += ck * float(np.real(v))
    return total


def trace(rho: np.ndarray) -> complex:
    return complex(np.sum(np.diag(rho)))


def purity(rho: np.ndarray) -> float:
    """tr(rho^dagger rho) = sum_ij |rho_ij|^2; equals tr(rho^2) for Hermitian rho."""
    return float(np.sum(np.abs(rho) ** 2))


def fidelity_pure(rho: np.ndarray, psi: np.ndarray) -> float:
    """<psi| rho |psi>."""
    return float(np.real(np.vdot(psi, rho @ psi)))


def trace_distance(a: np.ndarray, b: np.ndarray) -> float:
    """T = 1/2 ||a - b||_1 from the eigenvalues of the Hermitian difference."""
    d = a - b
    d = 0.5 * (d + d.conj().T)
    return 0.5 * float(np.sum(np.abs(np.linalg.eigvalsh(d))))


def uhlmann_fidelity(a: np.ndarray, b: np.ndarray) -> float:
    """F = (tr sqrt(sqrt(a) b sqrt(a)))^2 via Hermitian eigendecompositions."""
    w, v = np.linalg.eigh(0.5 * (a + a.conj().T))
    sa = (v * np.sqrt(np.clip(w, 0, None))) @ v.conj().T
    m = sa @ b @ sa
    ev = np.linalg.eigvalsh(0.5 * (m + m.conj().T))
    return float(np.sum(np.sqrt(np.clip(ev, 0, None))) ** 2)


def measure_collapse(rho: np.ndarray, q: int, u: float = 0.0, force: int = -1):
    """Projective Z measurement of qubit q (selective): outcome m with probability tr(P_m rho)/tr(rho),
    drawn as m = 0 when u tr(rho) < tr(P_0 rho) (or forced), and the collapsed state
    P_m rho P_m / tr(P_m rho).  Returns (m, probability, new rho)."""
    n = int(round(np.log2(rho.shape[0])))
    p = probs(rho, [q])
    tot = p[0] + p[1]
    m = force if force >= 0 else (0 if u * tot < p[0] else 1)
    proj = np.zeros((2, 2), dtype=complex)
    proj[m, m] = 1.0
    from .evolve import apply_kraus
    out = apply_kraus(rho, (q,), [proj]) / p[m]
    return m, p[m] / tot, out


def parity_collapse(rho: np.ndarray, qa: int, qb: int, u: float = 0.0, force: int = -1, decay: bool = True):
    """Silicon parity measurement of Sec. 7 (Eq. m) on qubits (qa, qb): outcome 0 is the odd subspace
    span{|01>, |10>}, outcome 1 the even subspace span{|00>, |11>} (|ab>: qa = a, qb = b).  Drawn as 0 when
    u tr(rho) < tr(P_0 rho) (or forced); the state becomes P_m rho P_m / tr(P_m rho), then, with decay, the
    Kraus map {|00><00|, |11><11|, |10><10|, |10><01|} of Sec. 7.  Returns (m, probability, new rho)."""
    from .evolve import apply_kraus
    p = probs(rho, [qa, qb])                       # index a | b << 1
    p_odd, p_even = p[1] + p[2], p[0] + p[3]
    tot = p_odd + p_even
    m = force if force >= 0 else (0 if u * tot < p_odd else 1)
    keep = (1, 2) if m == 0 else (0, 3)
    proj = np.zeros((4, 4), dtype=complex)
    for r in keep:
        proj[r, r] = 1.0
    pm = p_odd if m == 0 else p_even
    out = apply_kraus(rho, (qa, qb), [proj]) / pm
    if decay:
        ket = lambda a, b: a | (b << 1)
        ks = []
        for (ra, rb), (ca, cb) in [((0, 0), (0, 0)), ((1, 1), (1, 1)), ((1, 0), (1, 0)), ((1, 0), (0, 1))]:
            k = np.zeros((4, 4), dtype=complex)
            k[ket(ra, rb), ket(ca, cb)] = 1.0
            ks.append(k)
        out = apply_kraus(out, (qa, qb), ks)
    return m, pm / tot, out
