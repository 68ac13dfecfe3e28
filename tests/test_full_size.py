"""GPU parity at the benchmark's full size, and the exact error of the reduced precisions.

* The first full layer of the 14-qubit superconducting-grid program (108 native ops: Rz, SX, ZX(pi/2), the ZZ
  crosstalk idles and the T1/T2 idles), in every precision and through the plain and the fused path, element
  by element against the oracle (its C-loop evaluation, pinned against the tensor one in
  tests/test_oracle_pins.py).  FP64 must agree within 1e-12.
* The complex64 and float-float states of the six-qubit chain and of a 10-qubit reduced grid against the
  oracle by the exact trace distance T = 1/2 ||rho - sigma||_1 and the Uhlmann fidelity
  F = (tr sqrt(sqrt(rho) sigma sqrt(rho)))^2 (both from Hermitian eigensolvers, affordable at n <= 12).
  Bounds: complex64 T <= 1e-5 and 1 - F <= 1e-5 (the reduced-precision error target), float-float
  T <= 1e-10 and |1 - F| <= 1e-10, FP64 T <= 1e-11.
"""
import numpy as np
import pytest

from oracle import cloop, measure
from workloads import config1_chain6, config2_sc_grid
from workloads.circuits import Program

from ._lib import TOL_F64, get_lib, tol_f32, tol_split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vqd():
    return get_lib()


def prec_code(vqd, p):
    return {"f64": vqd.VQD_F64, "f32": vqd.VQD_F32, "split": vqd.VQD_F32_SPLIT}[p]


def run_gpu_flat(vqd, prog, p, path):
    ctx = vqd.vqd_create(prog.n, prec_code(vqd, p))
    try:
        if path == "plain":
            vqd.vqd_apply_native(ctx, 0, prog.ops)
        else:
            vqd.vqd_run_program(ctx, 0, prog.ops)
        red = (vqd.vqd_trace(ctx, 0), vqd.vqd_purity(ctx, 0))
        return vqd.vqd_get_state(ctx, 0), red
    finally:
        vqd.vqd_destroy(ctx)


@pytest.fixture(scope="module")
def grid14_first_layer():
    prog = config2_sc_grid()
    layer = len(prog.ops) // prog.meta["depth"]
    first = Program(prog.n, list(prog.ops[:layer]))
    assert len(first.ops) == 108 and {o.name for o in first.ops} == {"rz", "sx", "zx", "zz_idle", "idle"}
    return first, cloop.run_program(first)


@pytest.mark.parametrize("p", ["f64", "f32", "split"])
@pytest.mark.parametrize("path", ["plain", "fused"])
def test_grid14_first_layer_full_size_vs_oracle(vqd, grid14_first_layer, p, path):
    prog, want = grid14_first_layer
    flat, (tr, pur) = run_gpu_flat(vqd, prog, p, path)
    dim = 2 ** prog.n
    got = flat.reshape(dim, dim).T                     # device layout r + c 2^n -> got[r, c] (a view)
    tol = {"f64": TOL_F64, "f32": tol_f32(len(prog.ops)), "split": tol_split(len(prog.ops))}[p]
    err = 0.0
    for r0 in range(0, dim, 1024):                     # row blocks keep the temporaries small
        err = max(err, float(np.abs(got[r0:r0 + 1024] - want[r0:r0 + 1024]).max()))
    assert err < tol, (p, path, err)
    assert abs(tr - np.trace(want)) < tol
    # purity sums 2^28 squared moduli: complex64 rounding (relative 2^-24 per amplitude) moves it by ~1e-7
    assert abs(pur - float(np.sum(np.abs(want) ** 2))) < (1e-5 if p == "f32" else 1e-11)


@pytest.fixture(scope="module")
def small_programs():
    progs = {"chain6": config1_chain6(), "grid10": config2_sc_grid(seed=11, rows=2, cols=5, depth=20)}
    return {k: (q, cloop.run_program(q)) for k, q in progs.items()}


@pytest.mark.parametrize("name", ["chain6", "grid10"])
@pytest.mark.parametrize("p", ["f64", "f32", "split"])
@pytest.mark.parametrize("path", ["plain", "fused"])
def test_exact_trace_distance_and_fidelity(vqd, small_programs, name, p, path):
    prog, want = small_programs[name]
    flat, _ = run_gpu_flat(vqd, prog, p, path)
    dim = 2 ** prog.n
    got = np.ascontiguousarray(flat.reshape(dim, dim).T)
    T = measure.trace_distance(want, got)
    F = measure.uhlmann_fidelity(want, got)
    print(f"{name} n={prog.n} ops={len(prog.ops)} {p} {path}: T={T:.3e} 1-F={1 - F:.3e}")
    if p == "f32":
        assert T <= 1e-5 and 1 - F <= 1e-5
    elif p == "split":
        assert T <= 1e-10 and abs(1 - F) <= 1e-10
    else:
        assert T <= 1e-11 and abs(1 - F) <= 1e-11
