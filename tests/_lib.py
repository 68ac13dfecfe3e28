"""Shared test helpers: build/load libvqd, oracle comparisons, tolerances."""
import math

import numpy as np

# FP64 parity bar: max-abs difference to the FP64 oracle.
TOL_F64 = 1e-12


def tol_f32(n_ops: int) -> float:
    """FP32 max-abs tolerance after n_ops compiled operators.

    One pass rounds each amplitude (a sum of at most 16 products, |rho_ij| <= 1) with a random error
    of about sqrt(16) * 2^-24 = 2.4e-7; over m passes these add like a random walk.  The bound is
    4x that estimate: 1e-6 * sqrt(m), and never below 1e-6.
    """
    return 1e-6 * math.sqrt(max(1, n_ops))


def tol_split(n_ops: int) -> float:
    """Float-float (VQD_F32_SPLIT) max-abs tolerance after n_ops compiled operators.

    Float-float numbers round at about u^2 = 2^-48 = 3.6e-15 (u = 2^-24), and each operation of the
    double-word sum and product adds a few u^2 of relative error.  One pass forms each amplitude from at
    most 16 products, a random error of about sqrt(16) * 3 u^2 = 4e-14; over m passes these add like a
    random walk.  The bound is 5x that estimate: 2e-13 * sqrt(m), and never below 2e-13.
    """
    return 2e-13 * math.sqrt(max(1, n_ops))


def get_lib():
    from paper_2306_07342_gb300 import build as _b
    _b.build()
    from paper_2306_07342_gb300 import vqd
    vqd.lib()
    return vqd


def rand_state(n, rng):
    d = 2 ** n
    A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    rho = A @ A.conj().T
    return rho / np.trace(rho)


def rand_unitary(d, rng):
    q, r = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def rand_kraus(d, nk, rng):
    V = rand_unitary(d * nk, rng)[:, :d]
    return [V[i * d:(i + 1) * d, :] for i in range(nk)]
