"""Independent full-space constructions used only to pin the oracle.

* ``kron_chain``: a full operator from single-qubit factors by numpy Kronecker products
  (qubit n-1 leftmost), without any index arithmetic.
* ``full_operator``: a k-qubit operator embedded by expanding it in the Pauli basis
  (M = sum_P tr(P M)/2^k P) and writing each Pauli product as a Kronecker chain.
* ``superop``: the 4^n x 4^n matrix S = sum_k conj(K_k) (x) K_k acting on the column-major
  vectorisation, from the textbook identity vec(A X B) = (B^T (x) A) vec(X).
"""
from __future__ import annotations

import itertools
from typing import Sequence

import numpy as np

from .compile import I2, X, Y, Z

_P = (I2, X, Y, Z)


def kron_chain(factors_by_qubit: Sequence[np.ndarray]) -> np.ndarray:
    out = np.ones((1, 1), dtype=complex)
    for f in factors_by_qubit:      # qubit 0 first, each next factor goes to the left (more significant)
        out = np.kron(f, out)
    return out


def full_operator(M: np.ndarray, qubits: Sequence[int], n: int) -> np.ndarray:
    k = len(qubits)
    out = np.zeros((2 ** n, 2 ** n), dtype=complex)
    for labels in itertools.product(range(4), repeat=k):
        # local Pauli product with labels[j] on local bit j (local bit j = qubits[j])
        local = np.ones((1, 1), dtype=complex)
        for j in range(k):
            local = np.kron(_P[labels[j]], local)
        coef = np.trace(local.conj().T @ M) / 2 ** k
        if abs(coef) == 0:
            continue
        factors = [I2] * n
        for j, q in enumerate(qubits):
            factors[q] = _P[labels[j]]
        out += coef * kron_chain(factors)
    return out


def superop(kraus_full: Sequence[np.ndarray]) -> np.ndarray:
    return sum(np.kron(K.conj(), K) for K in kraus_full)


def vec(rho: np.ndarray) -> np.ndarray:
    return rho.reshape(-1, order="F")


def unvec(v: np.ndarray) -> np.ndarray:
    d = int(round(np.sqrt(v.size)))
    return v.reshape((d, d), order="F")
