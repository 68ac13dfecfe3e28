"""Superconducting device compiler (Sec. 8, App. C): library against the oracle, a worked example by hand,
closed forms of the noise it inserts, and GPU parity of a compiled program."""
import math

import numpy as np
import pytest

from oracle import evolve, measure
from oracle.devices import sc_compile
from workloads.circuits import NativeOp, Program
from workloads.devices import SC6, sc_ansatz, sc_grid_device

from ._lib import TOL_F64, get_lib


@pytest.fixture(scope="module")
def vqd():
    return get_lib()


def as_ops(vqd, arr):
    """Native-op array -> NativeOp list (names, qubits, parameters of the op's arity)."""
    from workloads.circuits import OP_NAMES
    out = []
    for r in arr:
        name = vqd.OP_CODES[int(r["code"])]
        nq, pn = OP_NAMES[name]
        out.append(NativeOp(name, tuple(int(q) for q in r["q"][:nq]), tuple(float(x) for x in r["par"][:len(pn)])))
    return out


def same_ops(a, b, tol=0.0):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.name == y.name and tuple(x.qubits) == tuple(y.qubits), (x, y)
        assert len(x.params) == len(y.params) and all(abs(p - q) <= tol for p, q in zip(x.params, y.params)), (x, y)


def small_device(**kw):
    dev = {"n": 3, "t1": [50.0, 60.0, 70.0], "t2": [30.0, 40.0, 50.0], "excited": [0.01, 0.02, 0.03],
           "freq": [4500.0, 4900.0, 4700.0], "anharm": [300.0, 250.0, 280.0], "couple": [(0, 1), (1, 2)],
           "coupling": [2.0, 3.0], "fid_read": [0.9, 0.95, 0.99], "dur_rxy": 0.05, "dur_zx": 0.5, "dur_zz": 0.4,
           "dur_meas": 2.0}
    dev.update(kw)
    return dev


def test_worked_example_by_hand(vqd):
    """rx(q0) and zx(q1,q2) share layer 0 (0.5 us long); rz(q0) is layer 1 (no time, no noise).  Layer 0
    emits its two gates, the static ZZ of both couplings (ZX is not a siZZle gate), then q0's decay over
    0.45 us; q1, q2 are busy the whole layer."""
    dev = small_device()
    ops = [NativeOp("rx", (0,), (0.3,)), NativeOp("zx", (1, 2), (math.pi / 2,)), NativeOp("rz", (0,), (0.7,))]
    w = 2 * math.pi * 0.5
    want = [ops[0], ops[1],
            NativeOp("zz_static", (0, 1), (w * 2.0, w * (4500.0 - 4900.0), w * 250.0, w * 300.0)),
            NativeOp("zz_static", (1, 2), (w * 3.0, w * (4900.0 - 4700.0), w * 280.0, w * 250.0)),
            NativeOp("gamp", (0,), (0.45, 50.0, 0.99)),
            NativeOp("deph1", (0,), (0.5 * (1 - math.exp(-0.45 / 30.0)),)),
            ops[2]]
    same_ops(sc_compile(dev, ops), want, 1e-15)
    same_ops(as_ops(vqd, vqd.vqd_sc_compile(dev, ops)), want, 1e-12)
    # readout: gamp(t_M) then depol(1 - F) on every qubit, after the last layer
    tail = as_ops(vqd, vqd.vqd_sc_compile(dev, ops, readout=True))[len(want):]
    same_ops(tail, [x for j in range(3) for x in (NativeOp("gamp", (j,), (2.0, dev["t1"][j], 1 - dev["excited"][j])),
                                                   NativeOp("depol1", (j,), (1 - dev["fid_read"][j],)))], 1e-15)


def test_sizzle_gate_absorbs_static_zz(vqd):
    dev = small_device()
    ops = [NativeOp("zz", (1, 0), (math.pi / 2,))]   # siZZle on the coupled pair (0, 1), either order
    out = as_ops(vqd, vqd.vqd_sc_compile(dev, ops))
    zz = [o for o in out if o.name == "zz_static"]
    assert [o.qubits for o in zz] == [(1, 2)]
    same_ops(out, sc_compile(dev, ops), 0.0)


def test_flags_off_give_the_logical_circuit(vqd):
    """Without noise the output is the logical circuit in layer order: the same ops, and on every qubit
    the same sequence (so the same channel)."""
    dev = small_device(flags=vqd.VQD_SC_NO_PASSIVE | vqd.VQD_SC_NO_STATIC_ZZ)
    ops = sc_ansatz(dev, 5, seed=4)
    out = as_ops(vqd, vqd.vqd_sc_compile(dev, ops))
    same_ops(out, sc_compile(dev, ops), 0.0)
    assert sorted(map(repr, out)) == sorted(map(repr, ops))
    for q in range(dev["n"]):
        same_ops([o for o in out if q in o.qubits], [o for o in ops if q in o.qubits], 0.0)


@pytest.mark.parametrize("seed", range(4))
def test_library_matches_oracle(vqd, seed):
    for dev, readout in [(SC6, True), (sc_grid_device(2, 3, seed=seed), bool(seed % 2)),
                         (dict(sc_grid_device(3, 3, seed=seed), fid_read=None, flags=seed % 4), True)]:
        ops = sc_ansatz(dev, 6, seed=seed)
        same_ops(as_ops(vqd, vqd.vqd_sc_compile(dev, ops, readout)), sc_compile(dev, ops, readout), 1e-12)


def test_rejects_bad_input(vqd):
    with pytest.raises(vqd.VQDError):
        vqd.vqd_sc_compile(small_device(), [NativeOp("h", (0,))])           # not a native SC gate
    with pytest.raises(vqd.VQDError):
        vqd.vqd_sc_compile(small_device(t1=[50.0, -1.0, 70.0]), [NativeOp("rx", (0,), (0.1,))])
    with pytest.raises(vqd.VQDError):
        vqd.vqd_sc_compile(small_device(couple=[(0, 3), (1, 2)]), [NativeOp("rx", (0,), (0.1,))])


def idle_program(dev, m, first):
    """`first` ops in layer 0, then m - 1 more exact rx(0) layers on qubit 0 (m layers of 0.05 us)."""
    return first + [NativeOp("rx", (0,), (0.0,)) for _ in range(m - 1)]


def test_thermal_relaxation_closed_form():
    """Qubit 1 idles all m layers, T = m * 0.05 us, from |0>: its excited population is p_1 (1 - e^{-T/T1})
    (Eq. gdamp).  Prepared in |+> by a gate of layer 0, it idles T = (m-1) * 0.05 us and its coherence <X>
    decays as e^{-T/(2 T1)} e^{-T/T2} (gamp, then Eq. depht2)."""
    dev = small_device(n=2, t1=[40.0, 20.0], t2=[30.0, 15.0], excited=[0.0, 0.1], couple=[], coupling=[],
                       freq=[4500.0, 4900.0], anharm=[300.0, 250.0], fid_read=None)
    m = 81
    T = m * 0.05
    prog = Program(2, sc_compile(dev, idle_program(dev, m, [NativeOp("rx", (0,), (0.0,))])))
    rho = evolve.run_program(prog)
    p1 = measure.probs(rho, [1])[1]
    assert abs(p1 - 0.1 * (1 - math.exp(-T / 20.0))) < 1e-13
    T = (m - 1) * 0.05
    prog = Program(2, sc_compile(dev, idle_program(dev, m, [NativeOp("rx", (0,), (0.0,)),
                                                            NativeOp("ry", (1,), (math.pi / 2,))])))
    x1 = measure.expect(evolve.run_program(prog), [[0, 1]], [1.0])
    assert abs(x1 - math.exp(-T / 40.0) * math.exp(-T / 15.0)) < 1e-13


def test_static_zz_phase_closed_form():
    """Coupled pair (J = 2, Delta = 500, alpha_t = 300, alpha_c = 250 MHz): beta = 4 (1/200 - 1/750) = 11/750 MHz.
    Both in |+>, 20 layers of 0.05 us: <X_0> = cos(2 * 2 pi beta * 1 us)."""
    first = [NativeOp("ry", (1,), (math.pi / 2,)), NativeOp("ry", (2,), (math.pi / 2,))]
    # the pair is (c, t) = (1, 2); qubit 0 clocks 20 layers with exact rx(0) gates
    dev = small_device(n=3, freq=[4700.0, 5000.0, 4500.0], anharm=[280.0, 250.0, 300.0], couple=[(1, 2)],
                       coupling=[2.0], flags=1, fid_read=None)
    ops = first + [NativeOp("rx", (0,), (0.0,)) for _ in range(20)]
    rho = evolve.run_program(Program(3, sc_compile(dev, ops)))
    phi = 2 * math.pi * (11 / 750) * 1.0
    assert abs(measure.expect(rho, [[0, 1, 0]], [1.0]) - math.cos(2 * phi)) < 1e-13


@pytest.mark.gpu
@pytest.mark.parametrize("dev_name", ["sc6", "grid2x4"])
def test_compiled_program_gpu_parity(vqd, dev_name):
    """A compiled ansatz from the thermal initial state, FP64, plain and fused, against the oracle's compile
    and evolution."""
    dev = SC6 if dev_name == "sc6" else sc_grid_device(2, 4, seed=5)
    ops = sc_ansatz(dev, 8, seed=6)
    lib_ops = vqd.vqd_sc_compile(dev, ops, readout=True)
    prog = Program(int(dev["n"]), sc_compile(dev, ops, readout=True), init_excited=tuple(dev["excited"]))
    want = evolve.run_program(prog)
    for runner in ("plain", "fused"):
        ctx = vqd.vqd_create(prog.n, vqd.VQD_F64)
        try:
            vqd.vqd_init_product_diag(ctx, 0, dev["excited"])
            if runner == "plain":
                vqd.vqd_apply_native(ctx, 0, lib_ops)
            else:
                vqd.vqd_run_program(ctx, 0, lib_ops)
            got = vqd.rho_from_flat(vqd.vqd_get_state(ctx, 0))
            assert np.abs(got - want).max() < TOL_F64, runner
        finally:
            vqd.vqd_destroy(ctx)
