"""Hermitian stages of the fused and batched paths (VQD_HERMITIAN): rho = rho^dagger (Sec. 2, every density
matrix), so a stage updates only the tiles on or above the diagonal of its tile grid and writes each one's
conjugate transpose into the mirror tile.

Parity against the FP64 oracle with the tolerances of tests/_lib.py, in every precision, over tile shapes,
qubit counts whose plans have one to many tile rows, the batched path, and a 14-qubit full-size layer; the
stored state must be exactly Hermitian (lower triangle the bitwise conjugate of the upper one, real diagonal).
"""
import numpy as np
import pytest

from oracle import cloop, evolve, measure
from workloads import config2_sc_grid
from workloads.circuits import Program, random_program

from ._lib import TOL_F64, get_lib, tol_f32, tol_split

pytestmark = pytest.mark.gpu

PRECS = ["f64", "f32", "split"]


@pytest.fixture(scope="module")
def vqd():
    return get_lib()


def prec_code(vqd, p):
    return {"f64": vqd.VQD_F64, "f32": vqd.VQD_F32, "split": vqd.VQD_F32_SPLIT}[p]


def tol(p, nops):
    return {"f64": TOL_F64, "f32": tol_f32(nops), "split": tol_split(nops)}[p]


def run_fused(vqd, prog, p, flags, fuse=0, shape=None):
    ctx = vqd.vqd_create(prog.n, prec_code(vqd, p))
    try:
        if prog.init_excited:
            vqd.vqd_init_product_diag(ctx, 0, prog.init_excited)
        if shape is not None:
            vqd.vqd_set_tile_shape(ctx, *shape)
        vqd.vqd_run_program(ctx, 0, prog.ops, fuse, flags)
        return vqd.rho_from_flat(vqd.vqd_get_state(ctx, 0))
    finally:
        vqd.vqd_destroy(ctx)


def assert_exactly_hermitian(rho):
    assert np.array_equal(rho, rho.conj().T)
    assert not np.any(np.diag(rho).imag)


@pytest.fixture(scope="module")
def programs():
    """Every native op kind at n = 7 (one row of 2 x 2 tiles) to n = 10 (tile grids of 16 x 16 and more)."""
    progs = {n: random_program(500 + n, n, 150) for n in (7, 8, 9, 10)}
    return {n: (q, cloop.run_program(q)) for n, q in progs.items()}


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("n", [7, 8, 9, 10])
def test_hermitian_stages_match_oracle(vqd, programs, p, n):
    prog, want = programs[n]
    got = run_fused(vqd, prog, p, vqd.VQD_HERMITIAN)
    assert np.abs(got - want).max() < tol(p, len(prog.ops)), (p, n)
    assert_exactly_hermitian(got)


@pytest.mark.parametrize("p", PRECS)
def test_hermitian_tile_shapes_and_fusion_widths(vqd, programs, p):
    """Passengers 0..3, odd tile sizes (rounded down to even), fusion widths 2..6."""
    prog, want = programs[9]
    shapes = [(12, 1), (12, 2), (11, 1), (10, 0), (10, 3), (8, 0), (8, 2)]
    if p == "f32":
        shapes += [(13, 2), (13, 3)]
    for shape in shapes:
        for fuse in (2, 4, 6):
            got = run_fused(vqd, prog, p, vqd.VQD_HERMITIAN, fuse, shape)
            assert np.abs(got - want).max() < tol(p, len(prog.ops)), (shape, fuse)
            assert_exactly_hermitian(got)


@pytest.mark.parametrize("p", PRECS)
def test_hermitian_thermal_start_and_general_path_agree(vqd, p):
    """A thermal product start (init_product_diag), then the same program with and without the flag."""
    prog = config2_sc_grid(seed=21, rows=2, cols=4, depth=6)
    prog.init_excited = tuple(0.01 + 0.004 * q for q in range(prog.n))
    want = evolve.run_program(prog)
    herm = run_fused(vqd, prog, p, vqd.VQD_HERMITIAN)
    full = run_fused(vqd, prog, p, 0)
    t = tol(p, len(prog.ops))
    assert np.abs(herm - want).max() < t and np.abs(full - want).max() < t
    assert np.abs(herm - full).max() < 2 * t
    assert_exactly_hermitian(herm)


@pytest.mark.parametrize("p", PRECS)
def test_hermitian_batch_matches_oracle(vqd, p):
    """Uneven batch (single-tile instances and multi-stage ones) through the batched waves with the flag."""
    progs = [random_program(700 + i, n, 60) for i, n in enumerate((3, 5, 6, 7, 8, 9, 10, 8))]
    wants = [cloop.run_program(q) for q in progs]
    ctx = vqd.vqd_create_batch([q.n for q in progs], prec_code(vqd, p))
    try:
        vqd.vqd_run_batch(ctx, [q.ops for q in progs], 0, vqd.VQD_HERMITIAN)
        for i, prog in enumerate(progs):
            got = vqd.rho_from_flat(vqd.vqd_get_state(ctx, i))
            assert np.abs(got - wants[i]).max() < tol(p, len(prog.ops)), i
            if prog.n > 6:
                assert_exactly_hermitian(got)
    finally:
        vqd.vqd_destroy(ctx)


def test_hermitian_stage_accounting_reads_about_half(vqd):
    """Launch accounting of a Hermitian run: each stage reads (K + 1) / 2K of the state (K tile rows) and
    writes all of it, so its counted bytes lie between 1.5 and 2 state sizes."""
    prog = random_program(808, 10, 80)
    ctx = vqd.vqd_create(prog.n, vqd.VQD_F64)
    try:
        vqd.vqd_profile(ctx, 2)
        vqd.vqd_profile_reset(ctx)
        vqd.vqd_run_program(ctx, 0, prog.ops, 0, vqd.VQD_HERMITIAN)
        st = vqd.vqd_profile_read(ctx)["fused_stage"]
        vqd.vqd_profile(ctx, 0)
    finally:
        vqd.vqd_destroy(ctx)
    per_launch = st["alg_bytes"] / st["launches"] / vqd.vqd_state_bytes(prog.n, vqd.VQD_F64)
    assert 1.5 <= per_launch <= 1.75, per_launch


@pytest.fixture(scope="module")
def grid14_first_layer():
    prog = config2_sc_grid()
    first = Program(prog.n, list(prog.ops[:len(prog.ops) // prog.meta["depth"]]))
    return first, cloop.run_program(first)


@pytest.mark.parametrize("p", PRECS)
def test_hermitian_grid14_first_layer_full_size(vqd, grid14_first_layer, p):
    """The first full layer of the 14-qubit grid program (108 native ops) against the oracle at full size."""
    first, want = grid14_first_layer
    ctx = vqd.vqd_create(first.n, prec_code(vqd, p))
    try:
        vqd.vqd_run_program(ctx, 0, first.ops, 0, vqd.VQD_HERMITIAN)
        flat = vqd.vqd_get_state(ctx, 0)
        tr = vqd.vqd_trace(ctx, 0)
    finally:
        vqd.vqd_destroy(ctx)
    dim = 2 ** first.n
    got = flat.reshape(dim, dim).T
    t = tol(p, len(first.ops))
    err = 0.0
    for r0 in range(0, dim, 1024):
        blk = got[r0:r0 + 1024]
        err = max(err, float(np.abs(blk - want[r0:r0 + 1024]).max()))
        # exact Hermiticity on this row block: rho[r][c] = conj(rho[c][r])
        assert np.array_equal(blk, got[:, r0:r0 + 1024].T.conj())
    assert err < t, (p, err)
    assert abs(tr - measure.trace(want)) < t


def test_autotuner_weighs_hermitian_and_general_plans(vqd, programs):
    """With Hermitian stages allowed, the tuner times the Hermitian and the general plans and returns the run
    flags of the fastest; running with its choice matches the oracle."""
    from paper_2306_07342_gb300 import autotune
    prog, want = programs[9]
    choice = autotune.tune(prog.n, vqd.VQD_F64, prog.ops, flags=vqd.VQD_HERMITIAN)
    trials = choice["trials"]
    assert len(trials) == len(autotune.HERM_CANDIDATES[vqd.VQD_F64]) + len(autotune.CANDIDATES[vqd.VQD_F64])
    assert {t["hermitian"] for t in trials} == {True, False}
    assert all(bool(t["flags"] & vqd.VQD_HERMITIAN) == t["hermitian"] for t in trials)
    ctx = vqd.vqd_create(prog.n, vqd.VQD_F64)
    try:
        f = autotune.apply(ctx, choice)
        vqd.vqd_run_program(ctx, 0, prog.ops, f, choice["flags"])
        got = vqd.rho_from_flat(vqd.vqd_get_state(ctx, 0))
    finally:
        vqd.vqd_destroy(ctx)
    assert np.abs(got - want).max() < TOL_F64
