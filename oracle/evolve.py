"""Oracle state evolution: rho <- U rho U^dagger and rho <- sum_k K_k rho K_k^dagger, literally.

rho is an ordinary (2^n x 2^n) complex128 numpy matrix, rho[r, c] with row r and column c.
Qubit q is bit q of r (and of c).  Two equivalent evaluations of the same definition:

* ``method="tensor"`` (default, any n): rho viewed as a tensor with one axis per row bit and
  one per column bit; the local matrix is contracted with the target row axes (K rho) and
  its conjugate with the target column axes (rho K^dagger);
* ``method="dense"`` (n <= 10): the local matrix is embedded in the full 2^n x 2^n space
  by index arithmetic and the matrix products are formed directly.

No blocking, fusion or reordering of operations is done: the compiled steps are applied one
after another in program order (Sec. 2: the noisy circuit is a sequence of unitary and
decohering operators applied to the density matrix).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import compile as _compile


# ------------------------------------------------------------------ initial states
def zero_state(n: int) -> np.ndarray:
    """|0...0><0...0|."""
    rho = np.zeros((2 ** n, 2 ** n), dtype=complex)
    rho[0, 0] = 1.0
    return rho


def classical_state(n: int, basis: int) -> np.ndarray:
    rho = np.zeros((2 ** n, 2 ** n), dtype=complex)
    rho[basis, basis] = 1.0
    return rho


def product_diag_state(n: int, excited: Sequence[float]) -> np.ndarray:
    """Thermal product state of Eq. (thermalstate): (x)_j ((1 - e_j)|0><0| + e_j |1><1|), e_j excited."""
    diag = np.ones(1)
    for q in range(n):          # qubit q is bit q: build from qubit 0 (least significant) upward
        diag = np.kron(np.array([1 - excited[q], excited[q]]), diag)
    return np.diag(diag).astype(complex)


# ------------------------------------------------------------------ tensor evaluation
def _apply_on_axes(t: np.ndarray, axes: Sequence[int], M: np.ndarray) -> np.ndarray:
    """Contract the input index of M (little-endian over ``axes``) with tensor axes ``axes``
    and put M's output index back on the same axes."""
    k = len(axes)
    Mt = M.reshape((2,) * (2 * k))          # axes 0..k-1: output bits k-1..0; k..2k-1: input bits k-1..0
    in_axes = [2 * k - 1 - j for j in range(k)]   # input bit j of M
    out = np.tensordot(Mt, t, axes=(in_axes, list(axes)))
    out_axes = [k - 1 - j for j in range(k)]      # output bit j of M, now at the front
    return np.moveaxis(out, out_axes, list(axes))


def _row_axes(n, qubits):
    return [n - 1 - q for q in qubits]


def _col_axes(n, qubits):
    return [2 * n - 1 - q for q in qubits]


def apply_kraus(rho: np.ndarray, qubits: Sequence[int], kraus: Sequence[np.ndarray],
                method: str = "tensor") -> np.ndarray:
    """sum_k K_k rho K_k^dagger with each K_k acting on ``qubits`` (Sec. 2, general Kraus maps)."""
    n = int(round(np.log2(rho.shape[0])))
    if method == "dense":
        out = np.zeros_like(rho)
        for K in kraus:
            Kf = embed(K, qubits, n)
            out += Kf @ rho @ Kf.conj().T
        return out
    t = rho.reshape((2,) * (2 * n))
    acc = None
    for K in kraus:
        left = _apply_on_axes(t, _row_axes(n, qubits), K)                  # K rho
        both = _apply_on_axes(left, _col_axes(n, qubits), K.conj())        # (K rho) K^dagger
        acc = both.copy() if acc is None else acc + both
    return np.ascontiguousarray(acc).reshape(rho.shape)


def apply_unitary(rho: np.ndarray, qubits: Sequence[int], U: np.ndarray, method: str = "tensor") -> np.ndarray:
    """U rho U^dagger."""
    return apply_kraus(rho, qubits, [U], method)


def apply_superop(rho: np.ndarray, qubits: Sequence[int], S: np.ndarray) -> np.ndarray:
    """Apply a k-qubit superoperator S (4^k x 4^k, index s = r | c << k over the target bits) by its
    definition: for every assignment of the other row and column bits, the 4^k amplitudes
    rho[r, c] spanned by the target bits are replaced by S times them."""
    n = int(round(np.log2(rho.shape[0])))
    k = len(qubits)
    dim = 2 ** n
    mask = sum(1 << q for q in qubits)
    out = np.empty_like(rho)
    offs = [sum(((s >> j) & 1) << q for j, q in enumerate(qubits)) for s in range(2 ** k)]
    rbase = [r for r in range(dim) if not (r & mask)]
    rr = np.array([[rb | o for o in offs] for rb in rbase])          # (groups, 2^k) row indices
    for cb in rbase:
        cc = [cb | o for o in offs]
        # group vector g[s] with s = r | c << k
        g = np.stack([rho[rr[:, r], cc[c]] for c in range(2 ** k) for r in range(2 ** k)], axis=1)
        h = g @ S.T
        for c in range(2 ** k):
            for r in range(2 ** k):
                out[rr[:, r], cc[c]] = h[:, r | (c << k)]
    return out


def embed(M: np.ndarray, qubits: Sequence[int], n: int) -> np.ndarray:
    """Full 2^n x 2^n operator acting as M on ``qubits`` and as identity elsewhere.

    Entry [r', r] is M[sub(r'), sub(r)] if r' and r agree on every non-target bit, else 0,
    where sub() collects the target bits little-endian.
    """
    dim = 2 ** n
    idx = np.arange(dim)
    sub = np.zeros(dim, dtype=np.int64)
    mask = 0
    for j, q in enumerate(qubits):
        sub |= ((idx >> q) & 1) << j
        mask |= 1 << q
    rest = idx & ~mask
    same = rest[:, None] == rest[None, :]
    return np.where(same, M[sub[:, None], sub[None, :]], 0).astype(complex)


# ------------------------------------------------------------------ programs
def apply_steps(rho: np.ndarray, steps, method: str = "tensor") -> np.ndarray:
    for kind, qubits, m in steps:
        if kind == "U":
            rho = apply_unitary(rho, qubits, m, method)
        else:
            rho = apply_kraus(rho, qubits, m, method)
    return rho


def initial_state(prog) -> np.ndarray:
    if getattr(prog, "init_excited", ()):
        return product_diag_state(prog.n, prog.init_excited)
    return zero_state(prog.n)


def run_program(prog, method: str = "tensor", t2_is_total: bool = False, rho0: np.ndarray | None = None,
                max_ops: int | None = None) -> np.ndarray:
    """Compile every native op of ``prog`` and apply the steps in order (optionally only the first
    ``max_ops`` native ops)."""
    rho = initial_state(prog) if rho0 is None else rho0
    ops = prog.ops if max_ops is None else prog.ops[:max_ops]
    for o in ops:
        rho = apply_steps(rho, _compile.compile_op(o.name, o.qubits, o.params, t2_is_total), method)
    return rho


def to_device_layout(rho: np.ndarray) -> np.ndarray:
    """Flat vector v with v[r + c 2^n] = rho[r, c] (column-major vectorisation)."""
    return np.ascontiguousarray(rho.T).reshape(-1)


def from_device_layout(v: np.ndarray) -> np.ndarray:
    dim = int(round(np.sqrt(v.size)))
    return np.ascontiguousarray(v.reshape(dim, dim).T)
