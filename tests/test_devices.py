"""Superconducting device compiler (Sec. 8, App. C): library against the oracle, a worked example by hand,
closed forms of the noise it inserts, and GPU parity of a compiled program."""
import math

import numpy as np
import pytest

from oracle import evolve, measure
from oracle.compile import stderr_params as oc_stderr
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


# ---------------------------------------------------------------- silicon spin qubits (Sec. 7, App. C)
from oracle.devices import si_compile  # noqa: E402
from workloads.devices import SI6, si_circuit  # noqa: E402


def small_si(**kw):
    dev = {"n": 3, "t1": [1e4, 2e4, 3e4], "t2": [20.0, 30.0, 40.0], "freq": [15600.0, 15900.0, 16300.0],
           "rabi": [5.0, 4.0, 6.0], "fid_1q": [0.998, 0.997, 0.999], "x_1q": 0.25, "freq_cz": [12.0, 8.0],
           "fid_cz": [0.95, 0.97], "x_cz": 0.5, "xtalk_on": [[0.0, 0.02], [0.04, 0.0]], "xtalk_off": [0.03, 0.01]}
    dev.update(kw)
    return dev


def test_si_worked_example_by_hand(vqd):
    """Rx(pi/2) on q1 (Rabi 4 MHz: t = 1/16 us); CZ on (0,1) (12 MHz: t = 1/24 us); virtual Rz on q2.  The
    standard errors follow App. C's angle rule: severities times |theta| / pi."""
    dev = small_si()
    ops = [NativeOp("rx", (1,), (math.pi / 2,)), NativeOp("cz", (0, 1)), NativeOp("rz", (2,), (0.4,))]
    t1, t2 = 1 / 16, 1 / 24
    w = 2 * math.pi
    p1, q1 = oc_stderr(0.997, 0.25, 1)                   # App. B inversion (pinned in the oracle tests)
    p2, q2 = oc_stderr(0.95, 0.5, 2)
    want = [ops[0], NativeOp("depol1", (1,), (q1 / 2,)), NativeOp("deph1", (1,), (p1 / 2,)),   # |theta|/pi = 1/2
            NativeOp("offres", (0,), (w * 4.0, w * 300.0, t1)), NativeOp("offres", (2,), (w * 4.0, w * 400.0, t1)),
            NativeOp("idle_depol", (0,), (t1, 1e4, 20.0)), NativeOp("idle_depol", (2,), (t1, 3e4, 40.0)),
            ops[1], NativeOp("depol2", (0, 1), (q2,)), NativeOp("deph2", (0, 1), (p2,)),             # CZ: theta = pi
            NativeOp("crz_xtalk", (1, 2), (0.02,)),
            NativeOp("idle_depol", (2,), (t2, 3e4, 40.0)), ops[2]]
    same_ops(si_compile(dev, ops), want, 1e-13)
    same_ops(as_ops(vqd, vqd.vqd_si_compile(dev, ops)), want, 1e-12)
    # off-state crosstalk: a rotation on q0 leaves the pair (1, 2) passive
    out = si_compile(dev, [NativeOp("ry", (0,), (1.0,))])
    assert [o for o in out if o.name == "crz_xtalk"] == [NativeOp("crz_xtalk", (1, 2), (0.01,))]


@pytest.mark.parametrize("seed", range(3))
def test_si_library_matches_oracle(vqd, seed):
    for dev in (SI6, dict(SI6, flags=seed, xtalk_on=None if seed == 1 else SI6["xtalk_on"]), small_si(flags=3 - seed)):
        ops = si_circuit(dev, 50, seed=seed)
        same_ops(as_ops(vqd, vqd.vqd_si_compile(dev, ops)), si_compile(dev, ops), 1e-12)


def test_si_off_resonant_rabi_population():
    """A bystander in |0> under the off-resonant drive of an Rx(theta) on its neighbour ends with the detuned
    Rabi population (Omega/Omega_R)^2 sin^2(Omega_R t/2), Omega = 2 pi f_Rabi, Omega_R^2 = Omega^2 + Delta^2,
    t = theta/Omega; at zero detuning it follows the driven qubit: sin^2(theta/2)."""
    for df, theta in [(12.0, 2.5), (3.0, 1.1), (0.0, 0.8)]:
        dev = small_si(n=2, freq=[15600.0, 15600.0 + df], rabi=[5.0, 5.0], fid_1q=[1.0, 1.0], freq_cz=[10.0],
                       fid_cz=[1.0], xtalk_on=None, xtalk_off=None, flags=1)
        rho = evolve.run_program(Program(2, si_compile(dev, [NativeOp("rx", (0,), (theta,))])))
        om, de = 2 * math.pi * 5.0, 2 * math.pi * df
        om_r = math.hypot(om, de)
        want = (om / om_r) ** 2 * math.sin(om_r * (theta / om) / 2) ** 2
        assert abs(measure.probs(rho, [1])[1] - want) < 1e-13
        assert abs(measure.probs(rho, [0])[1] - math.sin(theta / 2) ** 2) < 1e-13


def test_si_single_qubit_error_is_dephasing_of_the_tabulated_fidelity():
    """With the table's 0:1 split (pure dephasing) the severity is p = 1 - F_e, F_e = (3F - 1)/2 (App. B), scaled by
    |theta|/pi (App. C): Ry(pi/2) dephases with p/2, so <X> = 1 - p = F_e; Rx(0) adds no error."""
    F = 0.9977
    dev = small_si(n=2, fid_1q=[F, 1.0], x_1q=0.0, freq_cz=[10.0], fid_cz=[1.0], xtalk_on=None, xtalk_off=None,
                   flags=3)
    rho = evolve.run_program(Program(2, si_compile(dev, [NativeOp("ry", (0,), (math.pi / 2,)),
                                                         NativeOp("rx", (0,), (0.0,))])))
    assert abs(measure.expect(rho, [[1, 0]], [1.0]) - (3 * F - 1) / 2) < 1e-13


def test_si_rejects_bad_input(vqd):
    with pytest.raises(vqd.VQDError):
        vqd.vqd_si_compile(small_si(), [NativeOp("cz", (0, 2))])      # not neighbours
    with pytest.raises(vqd.VQDError):
        vqd.vqd_si_compile(small_si(), [NativeOp("h", (0,))])
    with pytest.raises(vqd.VQDError):
        vqd.vqd_si_compile(small_si(rabi=[5.0, 0.0, 6.0]), [NativeOp("rx", (0,), (0.1,))])


@pytest.mark.gpu
def test_si_compiled_program_gpu_parity(vqd):
    ops = si_circuit(SI6, 60, seed=12)
    lib_ops = vqd.vqd_si_compile(SI6, ops)
    want = evolve.run_program(Program(6, si_compile(SI6, ops)))
    for runner in ("plain", "fused"):
        ctx = vqd.vqd_create(6, vqd.VQD_F64)
        try:
            (vqd.vqd_apply_native if runner == "plain" else vqd.vqd_run_program)(ctx, 0, lib_ops)
            got = vqd.rho_from_flat(vqd.vqd_get_state(ctx, 0))
            assert np.abs(got - want).max() < TOL_F64, runner
        finally:
            vqd.vqd_destroy(ctx)


# ---------------------------------------------------------------- NV centre (Sec. 5, App. C)
from oracle.devices import nv_compile  # noqa: E402
from workloads.devices import NV5, nv_bcs_shape, nv_scaled  # noqa: E402


def small_nv(**kw):
    dev = {"n": 3, "t1": [100.0, 50.0, 40.0], "t2": [2.0, 8.0, 6.0], "freq_xy": [1e4, 500.0, 250.0],
           "freq_z": [1e7, 4e5, 2e5], "fid_xy": [0.999, 0.995, 0.99], "fid_z": [1.0, 1.0, 0.999], "x_xy": 0.75,
           "freq_crot": [1000.0, 2000.0], "fid_crot": [0.98, 0.97], "x_crot": 0.9, "freq_zz": 3.0,
           "fid_meas": 0.95, "dur_meas": 2e-5}
    dev.update(kw)
    return dev


def test_nv_worked_example_by_hand(vqd):
    """Rx(pi/2) on nuclear spin 1 (500 Hz: t = 1/2000 s); CRy+-(1.2) from the electron to spin 2 (2000 Hz:
    t = 1.2/(4000 pi) s); Rz(0.4) on the electron (1e7 Hz), during which the passive nuclear pair (1, 2)
    feels the weak ZZ; Rz(0.3) on spin 2 (fidelity 0.999: a dephasing standard error)."""
    dev = small_nv()
    ops = [NativeOp("rx", (1,), (math.pi / 2,)), NativeOp("zy", (0, 2), (1.2,)), NativeOp("rz", (0,), (0.4,)),
           NativeOp("rz", (2,), (0.3,))]
    t1, t2, t3, t4 = 1 / 2000, 1.2 / (4000 * math.pi), 0.4 / (2e7 * math.pi), 0.3 / (4e5 * math.pi)
    pa, qa = oc_stderr(0.995, 0.75, 1)
    pb, qb = oc_stderr(0.97, 0.9, 2)
    pz, _ = oc_stderr(0.999, 0.0, 1)
    sb, sz = 1.2 / math.pi, 0.3 / math.pi                 # App. C: severities times |theta| / pi
    want = [ops[0], NativeOp("depol1", (1,), (qa / 2,)), NativeOp("deph1", (1,), (pa / 2,)),
            NativeOp("idle_depol", (0,), (t1, 100.0, 2.0)), NativeOp("idle_depol", (2,), (t1, 40.0, 6.0)),
            ops[1], NativeOp("depol2", (0, 2), (qb * sb,)), NativeOp("deph2", (0, 2), (pb * sb,)),
            NativeOp("idle_depol", (1,), (t2, 50.0, 8.0)),
            ops[2], NativeOp("zz_idle", (1, 2), (t3, 3.0)),
            NativeOp("idle_depol", (1,), (t3, 50.0, 8.0)), NativeOp("idle_depol", (2,), (t3, 40.0, 6.0)),
            ops[3], NativeOp("deph1", (2,), (pz * sz,)),
            NativeOp("idle_depol", (0,), (t4, 100.0, 2.0)), NativeOp("idle_depol", (1,), (t4, 50.0, 8.0))]
    same_ops(nv_compile(dev, ops), want, 1e-15)
    same_ops(as_ops(vqd, vqd.vqd_nv_compile(dev, ops)), want, 1e-12)
    tail = as_ops(vqd, vqd.vqd_nv_compile(dev, ops, readout=True))[len(want):]
    same_ops(tail[:3], [NativeOp("rx", (0,), (math.pi,)), NativeOp("amp", (0,), (0.05,)),
                        NativeOp("rx", (0,), (math.pi,))], 1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_nv_library_matches_oracle(vqd, seed):
    for dev in (NV5, nv_scaled(NV5, 10.0 ** (seed - 1)), dict(NV5, flags=1), small_nv(freq_zz=0.0)):
        ops = nv_bcs_shape(dev, 2, 60, seed=seed)
        for readout in (False, True):
            same_ops(as_ops(vqd, vqd.vqd_nv_compile(dev, ops, readout)), nv_compile(dev, ops, readout), 1e-12)


def test_nv_readout_bias_closed_form():
    """Sec. 5: the electron readout damps towards |1> between two X gates, so |0> reads 1 with probability
    p = 1 - F and |1> always reads 1."""
    dev = small_nv(fid_xy=[1.0, 1.0, 1.0], flags=1)
    rho = evolve.run_program(Program(3, nv_compile(dev, [], readout=True)))
    assert abs(measure.probs(rho, [0])[1] - 0.05) < 1e-14
    rho = evolve.run_program(Program(3, nv_compile(dev, [NativeOp("rx", (0,), (math.pi,))], readout=True)))
    assert abs(measure.probs(rho, [0])[1] - 1.0) < 1e-14


def test_nv_weak_zz_phase_closed_form():
    """Nuclear spins 1, 2 in |+>, then 50 electron rotations Rx(2 pi) of 1/f = 1 ms each: the passive pair
    accumulates the weak ZZ phase, <X_1> = cos(pi f_zz T) with T = 0.05 s (conditional-frequency reading);
    T1, T2 are made long enough not to matter."""
    dev = small_nv(t1=[1e30] * 3, t2=[1e30] * 3, freq_xy=[1e3, 500.0, 500.0], fid_xy=[1.0] * 3)
    ops = [NativeOp("ry", (1,), (math.pi / 2,)), NativeOp("ry", (2,), (math.pi / 2,))]
    ops += [NativeOp("rx", (0,), (2 * math.pi,)) for _ in range(50)]
    rho = evolve.run_program(Program(3, nv_compile(dev, ops)))
    assert abs(measure.expect(rho, [[0, 1, 0]], [1.0]) - math.cos(math.pi * 3.0 * 0.05)) < 1e-12


def test_nv_rejects_bad_input(vqd):
    with pytest.raises(vqd.VQDError):
        vqd.vqd_nv_compile(small_nv(), [NativeOp("zx", (1, 2), (0.3,))])    # not controlled by the electron
    with pytest.raises(vqd.VQDError):
        vqd.vqd_nv_compile(small_nv(), [NativeOp("cz", (0, 1))])
    with pytest.raises(vqd.VQDError):
        vqd.vqd_nv_compile(small_nv(freq_crot=[1000.0, 0.0]), [NativeOp("rx", (0,), (0.1,))])


@pytest.mark.gpu
@pytest.mark.parametrize("p", ["f64", "split"])
def test_nv_compiled_program_gpu_parity(vqd, p):
    """Four BCS-shaped propagators (800 native gates) on the App. C NV centre, compiled by the library, plain
    and fused, against the oracle's compile and evolution."""
    from ._lib import tol_split
    ops = nv_bcs_shape(NV5, 4, 200, seed=21)
    lib_ops = vqd.vqd_nv_compile(NV5, ops, readout=True)
    want = evolve.run_program(Program(5, nv_compile(NV5, ops, readout=True)))
    t = TOL_F64 if p == "f64" else tol_split(len(lib_ops))
    for runner in ("plain", "fused"):
        ctx = vqd.vqd_create(5, vqd.VQD_F64 if p == "f64" else vqd.VQD_F32_SPLIT)
        try:
            (vqd.vqd_apply_native if runner == "plain" else vqd.vqd_run_program)(ctx, 0, lib_ops)
            got = vqd.rho_from_flat(vqd.vqd_get_state(ctx, 0))
            assert np.abs(got - want).max() < t, runner
        finally:
            vqd.vqd_destroy(ctx)


# ---------------------------------------------------------------- trapped ions (Sec. 4, App. C)
from oracle.devices import ion_compile  # noqa: E402
from workloads.devices import ION, ion_circuit  # noqa: E402


def small_ion(**kw):
    dev = {"n": 3, "t1": 1000.0, "t2s": 20.0, "rabi": 0.25, "fid_xy": 0.999, "x_xy": 1.0, "freq_cz": 0.05,
           "fid_cz": 0.99, "x_cz": 0.1, "bf_read": 0.01, "dur_read": 5.0}
    dev.update(kw)
    return dev


def test_ion_worked_example_by_hand(vqd):
    """Ry(pi/2) on ion 1 (0.25 MHz: t = 1 us), virtual Rz on ion 0, CZ on (2, 0) (0.05 MHz: t = 10 us); readout
    one ion at a time (5 us each)."""
    dev = small_ion()
    ops = [NativeOp("ry", (1,), (math.pi / 2,)), NativeOp("rz", (0,), (0.4,)), NativeOp("cz", (2, 0))]
    p1, q1 = oc_stderr(0.999, 1.0, 1)                     # pure depolarising: p1 = 0
    p2, q2 = oc_stderr(0.99, 0.1, 2)
    idle = lambda j, t: NativeOp("idle_t2s", (j,), (t, 1000.0, 20.0))
    want = [ops[0], NativeOp("depol1", (1,), (q1 / 2,)), idle(0, 1.0), idle(2, 1.0),
            ops[1],
            ops[2], NativeOp("depol2", (2, 0), (q2,)), NativeOp("deph2", (2, 0), (p2,)), idle(1, 10.0),
            NativeOp("bitflip", (0,), (0.01,)), idle(1, 5.0), idle(2, 5.0),
            NativeOp("bitflip", (1,), (0.01,)), idle(2, 5.0),
            NativeOp("bitflip", (2,), (0.01,))]
    assert p1 == 0.0
    same_ops(ion_compile(dev, ops, readout=True), want, 1e-15)
    same_ops(as_ops(vqd, vqd.vqd_ion_compile(dev, ops, readout=True)), want, 1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_ion_library_matches_oracle(vqd, seed):
    for dev in (ION, dict(ION, flags=1), small_ion(bf_read=0.0)):
        ops = ion_circuit(dev, 80, seed=seed)
        for readout in (False, True):
            same_ops(as_ops(vqd, vqd.vqd_ion_compile(dev, ops, readout)), ion_compile(dev, ops, readout), 1e-12)


def test_ion_gaussian_t2s_accumulates_per_gate():
    """Ion 1 in |+> idles through m Rx(pi) gates on ion 0 (t = 2 us each, exact gates): every gate is its own
    Gaussian free-induction interval (Eq. depht2s), so <X_1> = exp(-m t/T1 - m (t/T2*)^2)."""
    dev = small_ion(n=2, fid_xy=1.0)
    m, t = 12, 2.0
    ops = [NativeOp("ry", (1,), (math.pi / 2,))] + [NativeOp("rx", (0,), (math.pi,)) for _ in range(m)]
    rho = evolve.run_program(Program(2, ion_compile(dev, ops)))
    # the Ry(pi/2) itself (1 us) only idles ion 0
    assert abs(measure.expect(rho, [[0, 1]], [1.0]) - math.exp(-m * t / 1000.0 - m * (t / 20.0) ** 2)) < 1e-13


def test_ion_readout_flip_closed_form():
    """Readout flips each ion's outcome with probability b (symmetric bit flip, Eq. bf).  Ion 2 is flipped by an
    Rx(pi) whose standard error is pure depolarising with q = 3(1 - F)/2 (App. B, x = 1), so its population
    error is 2q/3 = 1 - F and it reads 1 with probability F(1 - b) + (1 - F) b; ion 0 reads 1 with probability b."""
    F, b = 0.999, 0.03
    dev = small_ion(flags=1, bf_read=b, fid_xy=F)
    rho = evolve.run_program(Program(3, ion_compile(dev, [NativeOp("rx", (2,), (math.pi,))], readout=True)))
    assert abs(measure.probs(rho, [0])[1] - b) < 1e-14
    assert abs(measure.probs(rho, [2])[1] - (F * (1 - b) + (1 - F) * b)) < 1e-13


def test_ion_rejects_bad_input(vqd):
    with pytest.raises(vqd.VQDError):
        vqd.vqd_ion_compile(small_ion(), [NativeOp("cph", (0, 1), (0.3,))])
    with pytest.raises(vqd.VQDError):
        vqd.vqd_ion_compile(small_ion(freq_cz=0.0), [NativeOp("rx", (0,), (0.1,))])


@pytest.mark.gpu
def test_ion_compiled_program_gpu_parity(vqd):
    ops = ion_circuit(ION, 120, seed=23)
    lib_ops = vqd.vqd_ion_compile(ION, ops, readout=True)
    want = evolve.run_program(Program(8, ion_compile(ION, ops, readout=True)))
    for runner in ("plain", "fused"):
        ctx = vqd.vqd_create(8, vqd.VQD_F64)
        try:
            (vqd.vqd_apply_native if runner == "plain" else vqd.vqd_run_program)(ctx, 0, lib_ops)
            assert np.abs(vqd.rho_from_flat(vqd.vqd_get_state(ctx, 0)) - want).max() < TOL_F64, runner
        finally:
            vqd.vqd_destroy(ctx)


# ---------------------------------------------------------------- neutral atoms (Sec. 6, App. C)
from oracle.devices import na_compile  # noqa: E402
from workloads.devices import NA_CLUSTER12, na_cluster_circuit  # noqa: E402


def small_na(**kw):
    dev = {"n": 3, "sites": [(0.0, 0.0), (1.0, 0.0), (5.0, 0.0)], "blockade": 1.0, "t2": 40.0, "t_vac": 300.0, "rabi": 0.1,
           "p10": 0.01, "p01": 0.02, "leak_init": 0.05, "leak_cz": (0.1, 0.01), "dur_cz": 0.5, "fid_meas": 0.97}
    dev.update(kw)
    return dev


def test_na_worked_example_by_hand(vqd):
    """U(pi/2, 0.1, 0, 5) on atom 2 (a pi/2 rotation lasting 5 us), then CZ(phi) on the neighbours (0, 1); T1 = 300/3
    = 100 us; initialisation leakage first, readout depolarising p = 3(1 - 0.97)/2 last."""
    dev = small_na()
    ops = [NativeOp("u", (2,), (math.pi / 2, 0.1, 0.0, 5.0)), NativeOp("czphi", (0, 1), (0.7,))]
    s = 0.1 * 5.0 / math.pi
    want = [NativeOp("leak_init", (j,), (0.05,)) for j in range(3)]
    want += [ops[0], NativeOp("deph1", (2,), (1 - math.exp(-5.0 / 80.0),)),
             NativeOp("bitflip_asym", (2,), (0.01 * s, 0.02 * s)),
             NativeOp("idle_depol", (0,), (5.0, 100.0, 40.0)), NativeOp("idle_depol", (1,), (5.0, 100.0, 40.0)),
             ops[1], NativeOp("leak_cz", (0, 1), (0.1, 0.01)), NativeOp("idle_depol", (2,), (0.5, 100.0, 40.0))]
    want += [NativeOp("depol1", (j,), (1.5 * 0.03,)) for j in range(3)]
    same_ops(na_compile(dev, ops, init=True, readout=True), want, 1e-15)
    same_ops(as_ops(vqd, vqd.vqd_na_compile(dev, ops, init=True, readout=True)), want, 1e-12)


def test_na_library_matches_oracle(vqd):
    for dev in (NA_CLUSTER12, dict(NA_CLUSTER12, flags=1), small_na(sites=[(0.0, 0.0), (1.0, 0.0), (0.5, 0.5)])):
        ops = na_cluster_circuit(dev, layers=2)
        for init, readout in ((False, False), (True, True)):
            same_ops(as_ops(vqd, vqd.vqd_na_compile(dev, ops, init, readout)), na_compile(dev, ops, init, readout), 1e-12)


def test_na_leakage_and_readout_closed_forms():
    """Sec. 6: initialisation leakage leaves tr = (1 - gamma)^n; readout depolarising reads |0> as 1 with
    probability 1 - F; CZ(phi) on |11> keeps 1 - beta of the trace (Eq. czleak)."""
    dev = small_na(flags=1, p10=0.0, p01=0.0)
    rho = evolve.run_program(Program(3, na_compile(dev, [], init=True)))
    assert abs(measure.trace(rho).real - 0.95 ** 3) < 1e-14
    rho = evolve.run_program(Program(3, na_compile(dev, [], readout=True)))
    assert abs(measure.probs(rho, [1])[1] - 0.03) < 1e-14
    flip = [NativeOp("u", (q,), (0.0, 0.1, 0.0, math.pi / 0.1)) for q in (0, 1)]    # Omega t = pi: |0> -> |1>
    rho = evolve.run_program(Program(3, na_compile(dev, flip + [NativeOp("czphi", (0, 1), (0.3,))])))
    assert abs(measure.trace(rho).real - (1 - 0.01)) < 1e-13


def test_na_blockade_and_bad_input(vqd):
    with pytest.raises(vqd.VQDError):
        vqd.vqd_na_compile(small_na(), [NativeOp("czphi", (0, 2), (0.3,))])   # 5 lattice units apart
    with pytest.raises(vqd.VQDError):
        vqd.vqd_na_compile(small_na(), [NativeOp("cz", (0, 1))])
    with pytest.raises(ValueError):
        na_compile(small_na(), [NativeOp("czphi", (0, 2), (0.3,))])


@pytest.mark.gpu
def test_na_compiled_program_gpu_parity(vqd):
    """The cluster circuit on the first 8 sites of the App. C chain (the FP64 oracle stays quick), with
    initialisation leakage and readout, plain and fused, against the oracle."""
    dev = dict(NA_CLUSTER12, n=8, sites=NA_CLUSTER12["sites"][:8])
    ops = na_cluster_circuit(dev, layers=2)
    lib_ops = vqd.vqd_na_compile(dev, ops, init=True, readout=True)
    want = evolve.run_program(Program(8, na_compile(dev, ops, init=True, readout=True)))
    for runner in ("plain", "fused"):
        ctx = vqd.vqd_create(8, vqd.VQD_F64)
        try:
            (vqd.vqd_apply_native if runner == "plain" else vqd.vqd_run_program)(ctx, 0, lib_ops)
            assert np.abs(vqd.rho_from_flat(vqd.vqd_get_state(ctx, 0)) - want).max() < TOL_F64, runner
        finally:
            vqd.vqd_destroy(ctx)


# ---------------------------------------------------------------- host contract shared by the compilers
def test_compilers_refuse_null_device_and_short_buffers(vqd):
    """Every compiler refuses a NULL device with VQD_EINVAL.  The compilers share one output sink, so the
    capacity check is exercised through one of them: a buffer one op shorter than the compiled program is refused,
    and the exact size is accepted and filled with the same ops as the counting run."""
    import ctypes
    a = vqd.native_ops(si_circuit(SI6, 20))
    cnt = ctypes.c_int()
    lib = vqd.lib()
    calls = {"sc": lambda: lib.vqd_sc_compile(None, len(a), vqd._ptr(a), 0, 0, None, ctypes.byref(cnt)),
             "si": lambda: lib.vqd_si_compile(None, len(a), vqd._ptr(a), 0, None, ctypes.byref(cnt)),
             "nv": lambda: lib.vqd_nv_compile(None, len(a), vqd._ptr(a), 0, 0, None, ctypes.byref(cnt)),
             "ion": lambda: lib.vqd_ion_compile(None, len(a), vqd._ptr(a), 0, 0, None, ctypes.byref(cnt)),
             "na": lambda: lib.vqd_na_compile(None, len(a), vqd._ptr(a), 0, 0, 0, None, ctypes.byref(cnt))}
    for name, call in calls.items():
        assert call() == vqd.VQD_EINVAL, name
    keep = {k: np.ascontiguousarray(np.asarray(SI6[k], np.float64).reshape(-1))
            for k in ("t1", "t2", "freq", "rabi", "fid_1q", "freq_cz", "fid_cz", "xtalk_on", "xtalk_off")}
    d = vqd.si_device(6, vqd._ptr(keep["t1"]), vqd._ptr(keep["t2"]), vqd._ptr(keep["freq"]), vqd._ptr(keep["rabi"]),
                      vqd._ptr(keep["fid_1q"]), float(SI6["x_1q"]), vqd._ptr(keep["freq_cz"]), vqd._ptr(keep["fid_cz"]),
                      float(SI6["x_cz"]), vqd._ptr(keep["xtalk_on"]), vqd._ptr(keep["xtalk_off"]), 0)
    assert lib.vqd_si_compile(ctypes.byref(d), len(a), vqd._ptr(a), 0, None, ctypes.byref(cnt)) == vqd.VQD_OK
    need = cnt.value
    out = np.zeros(need, dtype=vqd.NATIVE_OP_DTYPE)
    assert lib.vqd_si_compile(ctypes.byref(d), len(a), vqd._ptr(a), need - 1, vqd._ptr(out), ctypes.byref(cnt)) \
        == vqd.VQD_EINVAL
    assert lib.vqd_si_compile(ctypes.byref(d), len(a), vqd._ptr(a), need, vqd._ptr(out), ctypes.byref(cnt)) == vqd.VQD_OK
    assert cnt.value == need
    same_ops(as_ops(vqd, out), as_ops(vqd, vqd.vqd_si_compile(SI6, si_circuit(SI6, 20))), 0.0)
