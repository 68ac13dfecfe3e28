"""Oracle of the Monte-Carlo trajectory path (Sec. 2: statevector unravelling of the noisy circuit).

Each trajectory starts in |0...0>.  A unitary acts on the statevector; a channel {K_k} is replaced by one
operator: with u the trajectory's uniform draw for this native op, operator k is taken when
sum_{j<k} p_j <= u < sum_{j<=k} p_j, where p_j = ||K_j psi||^2, and psi <- K_k psi / sqrt(p_k).  If u lies
above sum_j p_j (a trace-decreasing channel), the trajectory is lost and contributes 0.  The estimate of
Re tr(H rho) is the mean over trajectories of <psi|H|psi>.

Draws come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011), written here from the paper's round
definition: counter (op index, trajectory, 0, 0), key (seed low, seed high); u takes 53 bits of the first
two output words.  The Kraus operators of a native op are listed in a fixed order: a composite process
(first step A, then B) has operators B_j A_i with i outer, as ``compile.compose_kraus`` builds them.
"""
from __future__ import annotations

import numpy as np

from . import compile as oc
from . import evolve, measure

M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on Python integers: one 4-word block."""
    x0, x1, x2, x3 = ctr
    k0, k1 = key
    for _ in range(10):
        p0 = M0 * x0
        p1 = M1 * x2
        x0, x1, x2, x3 = ((p1 >> 32) ^ x1 ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ x3 ^ k1) & MASK, p0 & MASK
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return x0, x1, x2, x3


def uniform(seed: int, op: int, traj: int) -> float:
    w = philox4x32_10((op & MASK, traj & MASK, 0, 0), (seed & MASK, (seed >> 32) & MASK))
    return ((w[0] >> 5) * 67108864.0 + (w[1] >> 6)) / 9007199254740992.0


def kraus_list(o, t2_is_total: bool = False):
    """("U", qubits, U) or ("K", qubits, [K...]) for one native op, composite processes as one Kraus set."""
    steps = oc.compile_op(o.name, o.qubits, o.params, t2_is_total)
    if len(steps) == 1:
        return steps[0]
    ks = steps[0][2]
    for _, _, nxt in steps[1:]:
        ks = oc.compose_kraus(ks, nxt)
    return ("K", steps[0][1], ks)


def _apply_vec(psi: np.ndarray, n: int, qubits, M: np.ndarray) -> np.ndarray:
    """M acting on ``qubits`` of a statevector (qubit q = bit q; M's index little-endian over qubits)."""
    t = psi.reshape((2,) * n)
    return evolve._apply_on_axes(t, [n - 1 - q for q in qubits], M).reshape(-1)


def trajectory_values(prog, ntraj: int, seed: int, codes, coeffs, t2_is_total: bool = False) -> np.ndarray:
    """Per-trajectory w <psi|H|psi> (w = 0 for lost trajectories)."""
    n = prog.n
    forms = [kraus_list(o, t2_is_total) for o in prog.ops]
    vals = np.zeros(ntraj)
    for t in range(ntraj):
        psi = np.zeros(2 ** n, dtype=complex)
        psi[0] = 1.0
        alive = True
        for oi, (kind, qs, m) in enumerate(forms):
            if kind == "U":
                psi = _apply_vec(psi, n, qs, m)
                continue
            outs = [_apply_vec(psi, n, qs, K) for K in m]
            probs = [float(np.vdot(v, v).real) for v in outs]
            u = uniform(seed, oi, t)
            cum, choice = 0.0, -1
            for j, pj in enumerate(probs):
                cum += pj
                if u < cum:
                    choice = j
                    break
            if choice < 0:
                alive = False
                break
            psi = outs[choice] / np.sqrt(probs[choice])
        if alive:
            rho = np.outer(psi, psi.conj())
            vals[t] = measure.expect(rho, codes, coeffs)
    return vals
