"""Tensor-core form of the fused path (vqd_run_program_tc): k-qubit blocks as split-precision GEMMs.

Parity against the FP64 oracle on ion-trap-shaped all-to-all programs (the 15-qubit precision workload's gates
and noise on 7 to 10 qubits), for k = 4, 5, 6 and both limb schemes.  Tolerance: each block replaces an
amplitude by a sum of up to 2 * 4^k products; the split products drop terms of relative size about 2^-22
(3xTF32: lo * lo; BF16x3: the products of order 5 and 6) and the FP32 accumulation rounds at 2^-24, so an
amplitude (|rho_ij| <= 1) moves by a few 1e-7 per block, adding like a random walk over m blocks:
tol_tc(m) = 4e-6 sqrt(m), four times the FP32 bound of tests/_lib.py per pass, since a block pass sums
far more terms than a one- or two-qubit pass.
"""
import math

import numpy as np
import pytest

from oracle import cloop, evolve
from workloads import config3_ion_alltoall
from workloads.circuits import random_program

from ._lib import get_lib

pytestmark = pytest.mark.gpu


def tol_tc(blocks: int) -> float:
    return 4e-6 * math.sqrt(max(1, blocks))


@pytest.fixture(scope="module")
def vqd():
    return get_lib()


def run_tc(vqd, prog, k, scheme):
    ctx = vqd.vqd_create(prog.n, vqd.VQD_F32)
    try:
        vqd.vqd_run_program_tc(ctx, 0, prog.ops, k, scheme)
        return vqd.rho_from_flat(vqd.vqd_get_state(ctx, 0)), vqd.vqd_trace(ctx, 0)
    finally:
        vqd.vqd_destroy(ctx)


@pytest.fixture(scope="module")
def ion_programs():
    progs = {n: config3_ion_alltoall(seed=40 + n, n=n, n_gates=120) for n in (7, 8, 10)}
    return {n: (p, cloop.run_program(p)) for n, p in progs.items()}


@pytest.mark.parametrize("scheme", ["3xtf32", "bf16x3"])
@pytest.mark.parametrize("n,k", [(7, 4), (8, 4), (8, 5), (8, 6), (10, 4), (10, 5)])
def test_tc_blocks_match_oracle(vqd, ion_programs, n, k, scheme):
    prog, want = ion_programs[n]
    sc = vqd.VQD_TC_3XTF32 if scheme == "3xtf32" else vqd.VQD_TC_BF16X3
    got, tr = run_tc(vqd, prog, k, sc)
    blocks = vqd.vqd_tc_plan_info(prog.n, prog.ops, k)["blocks"]
    err = float(np.abs(got - want).max())
    assert err < tol_tc(blocks), (n, k, scheme, err, blocks)
    assert abs(tr - np.trace(want)) < tol_tc(blocks)


def test_tc_every_op_kind_and_matches_fused_path(vqd):
    """Every native op kind (channels, leakage, crosstalk) through the tensor-core blocks, against the oracle
    and against the CUDA-core fused path on the same state."""
    prog = random_program(91, 8, 150)
    want = evolve.run_program(prog)
    got, _ = run_tc(vqd, prog, 4, vqd.VQD_TC_3XTF32)
    blocks = vqd.vqd_tc_plan_info(prog.n, prog.ops, 4)["blocks"]
    assert np.abs(got - want).max() < tol_tc(blocks)
    ctx = vqd.vqd_create(prog.n, vqd.VQD_F32)
    try:
        vqd.vqd_run_program(ctx, 0, prog.ops)
        fused = vqd.rho_from_flat(vqd.vqd_get_state(ctx, 0))
    finally:
        vqd.vqd_destroy(ctx)
    assert np.abs(got - fused).max() < tol_tc(blocks) + 1e-5


def test_tc_repeated_calls_and_odd_block_counts_keep_the_state_in_place(vqd):
    """Two calls in a row on one context (the second starts from the first's output), with programs whose
    block counts are odd and even: the state stays at vqd_state_ptr."""
    p1 = config3_ion_alltoall(seed=5, n=8, n_gates=30)
    p2 = config3_ion_alltoall(seed=6, n=8, n_gates=47)
    want = cloop.run_program(p2, rho0=cloop.run_program(p1))
    ctx = vqd.vqd_create(8, vqd.VQD_F32)
    try:
        ptr = vqd.vqd_state_ptr(ctx, 0)
        vqd.vqd_run_program_tc(ctx, 0, p1.ops, 4)
        vqd.vqd_run_program_tc(ctx, 0, p2.ops, 4)
        assert vqd.vqd_state_ptr(ctx, 0) == ptr
        got = vqd.rho_from_flat(vqd.vqd_get_state(ctx, 0))
    finally:
        vqd.vqd_destroy(ctx)
    blocks = vqd.vqd_tc_plan_info(8, p1.ops, 4)["blocks"] + vqd.vqd_tc_plan_info(8, p2.ops, 4)["blocks"]
    assert np.abs(got - want).max() < tol_tc(blocks)


def test_tc_argument_checks(vqd):
    prog = config3_ion_alltoall(seed=7, n=6, n_gates=10)
    ctx = vqd.vqd_create(6, vqd.VQD_F64)
    try:
        with pytest.raises(vqd.VQDError) as e:
            vqd.vqd_run_program_tc(ctx, 0, prog.ops, 4)
        assert e.value.code == vqd.VQD_ENOTSUP
    finally:
        vqd.vqd_destroy(ctx)
    ctx = vqd.vqd_create(5, vqd.VQD_F32)
    try:
        for k, sc in ((3, 0), (6, 0), (4, 2)):
            with pytest.raises(vqd.VQDError) as e:
                vqd.vqd_run_program_tc(ctx, 0, config3_ion_alltoall(seed=8, n=5, n_gates=5).ops, k, sc)
            assert e.value.code == vqd.VQD_EINVAL
    finally:
        vqd.vqd_destroy(ctx)
