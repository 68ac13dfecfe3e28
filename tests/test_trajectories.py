"""Monte-Carlo trajectories (Sec. 2): oracle pins on CPU, GPU parity (one by one and in the mean)."""
import math
import os

import numpy as np
import pytest

from oracle import evolve, measure
from oracle import compile as oc
from oracle import trajectories as otj
from workloads import config1_chain6
from workloads.circuits import OP_NAMES, NativeOp, Program, random_program

from ._lib import get_lib

UNITARIES = ["rx", "ry", "rz", "sx", "h", "u", "r", "cz", "cph", "czphi", "zx", "zz", "xx", "zzphase", "zz_idle",
             "crz_xtalk", "exchange", "offres", "zz_static", "zy"]


def hamiltonian(n, rng, nterms=6):
    codes = rng.integers(0, 4, size=(nterms, n)).astype(np.uint8)
    codes[0] = 0
    codes[0][0] = 3                       # always include Z_0
    return codes, rng.normal(size=nterms)


# ---------------------------------------------------------------- CPU pins of the oracle
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_philox_known_answer_vectors():
    """The oracle's Philox4x32-10 reproduces the generator's published known-answer vectors: a swapped
    multiplier, key schedule constant or output word changes every one of them."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if ln.strip() and ln[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        assert otj.philox4x32_10(tuple(w[0:4]), tuple(w[4:6])) == tuple(w[6:10])


def test_philox_uniform_draws_are_uniform_and_distinct():
    u = np.array([otj.uniform(12345, op, t) for op in range(40) for t in range(250)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert len(np.unique(u)) == u.size
    hist, _ = np.histogram(u, bins=20, range=(0, 1))
    chi2 = float(((hist - u.size / 20) ** 2 / (u.size / 20)).sum())
    assert chi2 < 50.0                    # 19 degrees of freedom: p ~ 1e-4
    assert abs(u.mean() - 0.5) < 0.01
    assert otj.uniform(1, 2, 3) != otj.uniform(1, 3, 2) and otj.uniform(1, 2, 3) != otj.uniform(2, 2, 3)


def test_oracle_trajectory_mean_converges_to_density_matrix():
    """The unravelling's mean estimates Re tr(H rho) (Sec. 2), including a trace-decreasing channel."""
    rng = np.random.default_rng(5)
    prog = random_program(17, 3, 30)
    prog.ops.append(NativeOp("leak_init", (1,), (0.2,)))
    codes, coeffs = hamiltonian(3, rng)
    exact = measure.expect(evolve.run_program(prog), codes, coeffs)
    vals = otj.trajectory_values(prog, 3000, 99, codes, coeffs)
    se = vals.std(ddof=1) / math.sqrt(vals.size)
    assert abs(vals.mean() - exact) < 5 * se + 1e-12


def test_oracle_unitary_trajectories_are_exact():
    rng = np.random.default_rng(6)
    prog = random_program(18, 4, 40, names=UNITARIES)
    codes, coeffs = hamiltonian(4, rng)
    exact = measure.expect(evolve.run_program(prog), codes, coeffs)
    vals = otj.trajectory_values(prog, 3, 1, codes, coeffs)
    assert np.abs(vals - exact).max() < 1e-13


# ---------------------------------------------------------------- GPU parity
@pytest.fixture(scope="module")
def vqd():
    return get_lib()


@pytest.mark.gpu
@pytest.mark.parametrize("p,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_traj_unitary_program_is_exact_every_trajectory(vqd, p, tol):
    rng = np.random.default_rng(7)
    prog = random_program(19, 6, 80, names=UNITARIES)
    codes, coeffs = hamiltonian(6, rng)
    exact = measure.expect(evolve.run_program(prog), codes, coeffs)
    vals, mean, se = vqd.vqd_traj_expect(6, vqd.VQD_F64 if p == "f64" else vqd.VQD_F32, prog.ops, 8, 3, codes, coeffs)
    assert np.abs(vals - exact).max() < tol
    assert se < tol
    assert abs(mean - vals.mean()) < 1e-15 and abs(se - vals.std(ddof=1) / math.sqrt(vals.size)) < 1e-15


@pytest.mark.gpu
def test_traj_match_oracle_one_by_one_fp64(vqd):
    """Same draws on both sides: every FP64 trajectory equals the oracle's (every native op kind, incl. leakage)."""
    rng = np.random.default_rng(8)
    prog = random_program(21, 4, 60)
    codes, coeffs = hamiltonian(4, rng)
    want = otj.trajectory_values(prog, 48, 2024, codes, coeffs)
    got, mean, se = vqd.vqd_traj_expect(4, vqd.VQD_F64, prog.ops, 48, 2024, codes, coeffs)
    assert np.abs(got - want).max() < 1e-10
    assert abs(mean - want.mean()) < 1e-10


@pytest.mark.gpu
@pytest.mark.parametrize("p", ["f64", "f32"])
def test_traj_mean_converges_to_density_matrix(vqd, p):
    """The six-qubit chain (682 native ops): 4096 trajectories against the density-matrix oracle."""
    rng = np.random.default_rng(9)
    prog = config1_chain6()
    codes, coeffs = hamiltonian(6, rng, nterms=8)
    exact = measure.expect(evolve.run_program(prog), codes, coeffs)
    vals, mean, se = vqd.vqd_traj_expect(6, vqd.VQD_F64 if p == "f64" else vqd.VQD_F32, prog.ops, 4096, 77,
                                         codes, coeffs)
    assert se > 0
    assert abs(mean - exact) < 5 * se + 1e-6


@pytest.mark.gpu
def test_traj_largest_statevector_and_errors(vqd):
    n = 14
    prog = Program(n, [NativeOp("h", (q,)) for q in range(n)] + [NativeOp("depol1", (q,), (0.1,)) for q in range(n)])
    codes = np.zeros((1, n), np.uint8)
    codes[0, 3] = 1                                     # <X_3> = 1 - 4p/3 after H and depol1(p)
    vals, mean, se = vqd.vqd_traj_expect(n, vqd.VQD_F32, prog.ops, 2048, 5, codes, [1.0])
    assert abs(mean - (1 - 4 * 0.1 / 3)) < 5 * se + 1e-6
    for p in (vqd.VQD_F32, vqd.VQD_F64):
        with pytest.raises(vqd.VQDError) as e:
            vqd.vqd_traj_expect(17, p, [], 4, 1, np.zeros((1, 17), np.uint8), [1.0])
        assert e.value.code == vqd.VQD_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("n,p,ntraj", [(14, "f64", 6), (15, "f64", 4), (16, "f64", 2), (15, "f32", 4)])
def test_traj_cluster_statevector_one_by_one(vqd, n, p, ntraj):
    """Statevectors beyond one CTA's shared memory live on a cluster of CTAs (distributed shared memory):
    every trajectory equals the oracle's on the same draws (every op kind, operators on the cluster-rank
    qubits included)."""
    rng = np.random.default_rng(30 + n)
    prog = random_program(40 + n, n, 36)
    hi = [NativeOp("h", (n - 1,)), NativeOp("cz", (n - 1, 0)), NativeOp("depol2", (n - 2, n - 1), (0.2,)),
          NativeOp("amp", (n - 1,), (0.3,)), NativeOp("rx", (n - 3,), (0.7,))]
    prog = Program(n, hi + list(prog.ops))
    codes, coeffs = hamiltonian(n, rng)
    codes[1, n - 1] = 1                                    # a term that flips a cluster-rank bit
    want = otj.trajectory_values(prog, ntraj, 99, codes, coeffs)
    got, mean, se = vqd.vqd_traj_expect(n, vqd.VQD_F64 if p == "f64" else vqd.VQD_F32, prog.ops, ntraj, 99,
                                        codes, coeffs)
    assert np.abs(got - want).max() < (1e-10 if p == "f64" else 5e-5)


@pytest.mark.gpu
def test_traj_cluster_16_qubit_unitary_exact(vqd):
    """n = 16 in complex64 (eight CTAs of 64 KB): a unitary program gives the exact expectation in every
    trajectory."""
    n = 16
    rng = np.random.default_rng(44)
    prog = random_program(45, n, 50, names=UNITARIES)
    codes, coeffs = hamiltonian(n, rng)
    psi = np.zeros(2 ** n, dtype=complex)
    psi[0] = 1
    for o in prog.ops:
        ((_, qs, U),) = oc.compile_op(o.name, o.qubits, o.params)
        psi = otj._apply_vec(psi, n, qs, U)
    exact = 0.0
    for c, row in zip(coeffs, codes):
        v = psi.copy()
        for q, code in enumerate(row):
            if code:
                v = otj._apply_vec(v, n, (q,), [None, np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]),
                                                np.diag([1.0, -1.0])][code])
        exact += c * np.vdot(psi, v).real
    vals, mean, se = vqd.vqd_traj_expect(n, vqd.VQD_F32, prog.ops, 6, 1, codes, coeffs)
    assert np.abs(vals - exact).max() < 5e-5
