"""GPU parity: libvqd (through its C ABI) against the FP64 oracle on the same seeded inputs.

FP64 states must match within 1e-12 max-abs; FP32 states within tol_f32(#ops) (see tests/_lib.py).
"""
import math

import numpy as np
import pytest

from oracle import cloop, evolve, measure
from oracle import compile as oc
from workloads import config1_chain6, config2_sc_grid, config3_ion_alltoall, config5_spin_chain
from workloads.circuits import NativeOp, OP_NAMES, Program, random_program

from ._lib import TOL_F64, get_lib, rand_kraus, rand_state, rand_unitary, tol_f32, tol_split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vqd():
    return get_lib()


PRECS = ["f64", "f32", "split"]


def prec_code(vqd, p):
    return {"f64": vqd.VQD_F64, "f32": vqd.VQD_F32, "split": vqd.VQD_F32_SPLIT}[p]


def tol(p, nops):
    return {"f64": TOL_F64, "f32": tol_f32(nops), "split": tol_split(nops)}[p]


def gpu_state(vqd, ctx, inst=0):
    return vqd.rho_from_flat(vqd.vqd_get_state(ctx, inst))


def make_ctx(vqd, n, p, rho=None):
    ctx = vqd.vqd_create(n, prec_code(vqd, p))
    if rho is not None:
        vqd.vqd_set_state(ctx, 0, evolve.to_device_layout(rho))
    return ctx


# ---------------------------------------------------------------- single operators, every kernel class
@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("n", [1, 3, 7])
def test_one_qubit_operators(vqd, p, n):
    rng = np.random.default_rng(100 + n)
    rho = rand_state(n, rng)
    ctx = make_ctx(vqd, n, p, rho)
    try:
        for q in range(n):
            U = rand_unitary(2, rng)
            vqd.vqd_apply_unitary(ctx, 0, [q], U)
            rho = evolve.apply_unitary(rho, (q,), U)
            ks = rand_kraus(2, 3, rng)
            vqd.vqd_apply_kraus(ctx, 0, [q], ks)
            rho = evolve.apply_kraus(rho, (q,), ks)
            D = np.diag(np.exp(1j * rng.uniform(0, 6, 2)))      # diagonal -> elementwise kernel
            vqd.vqd_apply_unitary(ctx, 0, [q], D)
            rho = evolve.apply_unitary(rho, (q,), D)
            ks = oc.amp(0.3)                                       # real sparse superoperator
            vqd.vqd_apply_kraus(ctx, 0, [q], ks)
            rho = evolve.apply_kraus(rho, (q,), ks)
        got = gpu_state(vqd, ctx)
        assert np.abs(got - rho).max() < tol(p, 4 * n)
    finally:
        vqd.vqd_destroy(ctx)


@pytest.mark.parametrize("name", list(OP_NAMES))
def test_every_native_op_alone(vqd, name):
    """Each native op of the device vocabulary, compiled by the library and applied by vqd_apply_native to a
    random 5-qubit state in FP64, against the oracle's compiler and evolution (both qubit orders for pairs)."""
    from workloads.circuits import _random_params, _rng
    n = 5
    r = _rng(4000 + list(OP_NAMES).index(name))
    rho = rand_state(n, np.random.default_rng(4100 + list(OP_NAMES).index(name)))
    nq = OP_NAMES[name][0]
    ops = [NativeOp(name, (3,) if nq == 1 else (3, 1), _random_params(r, name)),
           NativeOp(name, (0,) if nq == 1 else (0, 4), _random_params(r, name))]
    ctx = make_ctx(vqd, n, "f64", rho)
    try:
        vqd.vqd_apply_native(ctx, 0, ops)
        want = evolve.run_program(Program(n, ops), rho0=rho)
        assert np.abs(gpu_state(vqd, ctx) - want).max() < TOL_F64
    finally:
        vqd.vqd_destroy(ctx)


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("n,targets", [(2, (0, 1)), (2, (1, 0)), (5, (4, 1)), (7, (2, 6)), (7, (6, 5))])
def test_two_qubit_operators(vqd, p, n, targets):
    rng = np.random.default_rng(200 + n + targets[0])
    rho = rand_state(n, rng)
    ctx = make_ctx(vqd, n, p, rho)
    try:
        U = rand_unitary(4, rng)
        vqd.vqd_apply_unitary(ctx, 0, targets, U)
        rho = evolve.apply_unitary(rho, targets, U)
        ks = rand_kraus(4, 3, rng)
        vqd.vqd_apply_kraus(ctx, 0, targets, ks)
        rho = evolve.apply_kraus(rho, targets, ks)
        D = np.diag(np.exp(1j * rng.uniform(0, 6, 4)))
        vqd.vqd_apply_unitary(ctx, 0, targets, D)
        rho = evolve.apply_unitary(rho, targets, D)
        ks = oc.deph2(0.2)                                         # diagonal superoperator
        vqd.vqd_apply_kraus(ctx, 0, targets, ks)
        rho = evolve.apply_kraus(rho, targets, ks)
        S = sum(np.kron(K.conj(), K) for K in rand_kraus(4, 2, rng))
        vqd.vqd_apply_superop(ctx, 0, targets, S)
        want = evolve.apply_superop(rho, targets, S)
        got = gpu_state(vqd, ctx)
        assert np.abs(got - want).max() < tol(p, 5)
    finally:
        vqd.vqd_destroy(ctx)


# ---------------------------------------------------------------- native programs, plain and fused
def run_gpu(vqd, prog, p, path, fuse=0, max_ops=None):
    ops = prog.ops if max_ops is None else prog.ops[:max_ops]
    ctx = vqd.vqd_create(prog.n, prec_code(vqd, p))
    try:
        if prog.init_excited:
            vqd.vqd_init_product_diag(ctx, 0, prog.init_excited)
        if path == "plain":
            vqd.vqd_apply_native(ctx, 0, ops)
        else:
            vqd.vqd_run_program(ctx, 0, ops, fuse)
        rho = gpu_state(vqd, ctx)
        red = {"probs": vqd.vqd_prob(ctx, 0, list(range(prog.n))), "trace": vqd.vqd_trace(ctx, 0),
               "purity": vqd.vqd_purity(ctx, 0)}
        return rho, red
    finally:
        vqd.vqd_destroy(ctx)


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("path", ["plain", "fused"])
def test_config1_chain6_full(vqd, p, path):
    """Six-qubit chain, 200 gates (~680 native ops), complex128 and complex64."""
    prog = config1_chain6()
    want = evolve.run_program(prog)
    got, red = run_gpu(vqd, prog, p, path)
    t = tol(p, len(prog.ops))
    assert np.abs(got - want).max() < t
    assert np.abs(red["probs"] - measure.probs(want, range(6))).max() < t
    assert abs(red["trace"] - measure.trace(want)) < t
    assert abs(red["purity"] - measure.purity(want)) < t


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("path,fuse", [("plain", 0), ("fused", 2), ("fused", 4), ("fused", 5), ("fused", 6)])
def test_random_programs_every_op_kind(vqd, p, path, fuse):
    """Every native op kind on n = 8 (16 index bits: the fused path needs several stages and tiles)."""
    prog = random_program(77 + fuse, 8, 160)
    want = evolve.run_program(prog)
    got, _ = run_gpu(vqd, prog, p, path, fuse)
    assert np.abs(got - want).max() < tol(p, len(prog.ops))


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("path", ["plain", "fused"])
def test_config2_grid_reduced(vqd, p, path):
    """The superconducting-grid workload on a 2 x 4 grid (n = 8), depth 12."""
    prog = config2_sc_grid(seed=9, rows=2, cols=4, depth=12)
    want = evolve.run_program(prog)
    got, red = run_gpu(vqd, prog, p, path)
    t = tol(p, len(prog.ops))
    assert np.abs(got - want).max() < t
    assert np.abs(red["probs"] - measure.probs(want, range(8))).max() < t


@pytest.mark.parametrize("p", PRECS)
def test_config3_and_5_shapes_reduced(vqd, p):
    for prog in (config3_ion_alltoall(seed=4, n=7, n_gates=60), config5_spin_chain(seed=6, n=7, n_gates=80)):
        want = evolve.run_program(prog)
        for path in ("plain", "fused"):
            got, _ = run_gpu(vqd, prog, p, path)
            assert np.abs(got - want).max() < tol(p, len(prog.ops)), (prog.meta["config"], path)


@pytest.mark.parametrize("p", PRECS)
def test_thermal_init_and_t2_flag(vqd, p):
    prog = random_program(5, 4, 40)
    prog.init_excited = (0.032, 0.021, 0.008, 0.009)
    want = evolve.run_program(prog)
    got, _ = run_gpu(vqd, prog, p, "plain")
    assert np.abs(got - want).max() < tol(p, 40)
    # VQD_T2_IS_TOTAL reads T2 as the total coherence time
    prog = Program(2, [NativeOp("h", (0,)), NativeOp("idle", (0,), (3.0, 40.0, 25.0))])
    ctx = vqd.vqd_create(2, prec_code(vqd, p))
    try:
        vqd.vqd_apply_native(ctx, 0, prog.ops, vqd.VQD_T2_IS_TOTAL)
        got = gpu_state(vqd, ctx)
    finally:
        vqd.vqd_destroy(ctx)
    want = evolve.run_program(prog, t2_is_total=True)
    assert np.abs(got - want).max() < tol(p, 2)
    assert abs(got[0, 1] - 0.5 * math.exp(-3.0 / 25.0)) < tol(p, 2)


def test_split_precision_is_fp64_class(vqd):
    """Float-float storage on the 6-qubit chain (682 native ops): the plain and fused paths stay within
    the float-float bound of the FP64 oracle, at least 10^4 times closer than complex64."""
    prog = config1_chain6()
    want = evolve.run_program(prog)
    err = {}
    for p in ("f32", "split"):
        for path in ("plain", "fused"):
            ctx = vqd.vqd_create(prog.n, prec_code(vqd, p))
            try:
                (vqd.vqd_apply_native if path == "plain" else vqd.vqd_run_program)(ctx, 0, prog.ops)
                err[p, path] = np.abs(gpu_state(vqd, ctx) - want).max()
            finally:
                vqd.vqd_destroy(ctx)
    for path in ("plain", "fused"):
        assert err["split", path] < tol_split(len(prog.ops)), err
        assert err["split", path] < 1e-4 * err["f32", path], err


@pytest.mark.parametrize("p", ["f32", "f64"])
def test_diagonal_passes_touch_only_changed_amplitudes(vqd, p):
    """A phase (Rz, ZZ crosstalk) or a dephasing leaves half of the amplitudes unchanged (factor exactly 1);
    the elementwise pass skips them, so its accounted bytes are half of a full pass, and results match."""
    n = 6
    rng = np.random.default_rng(77)
    rho = rand_state(n, rng)
    ops = [NativeOp("rz", (3,), (0.9,)), NativeOp("zz_idle", (1, 4), (0.3, 0.2)), NativeOp("deph1", (5,), (0.2,)),
           NativeOp("sx", (2,))]
    ctx = make_ctx(vqd, n, p, rho)
    try:
        vqd.vqd_profile(ctx, 2)
        vqd.vqd_profile_reset(ctx)
        vqd.vqd_apply_native(ctx, 0, ops)
        st = vqd.vqd_profile_read(ctx)
        vqd.vqd_profile(ctx, 0)
        full = 2 * vqd.vqd_state_bytes(n, prec_code(vqd, p))
        assert st["elem"]["launches"] == 3 and abs(st["elem"]["alg_bytes"] - 3 * full / 2) < 1
        assert st["sup1"]["launches"] == 1 and abs(st["sup1"]["alg_bytes"] - full) < 1
        want = evolve.run_program(Program(n, ops), rho0=rho)
        assert np.abs(gpu_state(vqd, ctx) - want).max() < tol(p, len(ops))
    finally:
        vqd.vqd_destroy(ctx)


@pytest.mark.parametrize("p", PRECS)
def test_parity_measurement_matches_oracle(vqd, p):
    """Sec. 7 parity readout on a random 5-qubit state: drawn and forced outcomes, with and without the decay map,
    against the oracle (outcome, probability, collapsed state)."""
    rng = np.random.default_rng(91)
    rho = rand_state(5, rng)
    for qa, qb, u, force, decay in ((1, 3, 0.37, -1, True), (4, 0, 0.81, -1, False), (2, 1, 0.0, 0, True),
                                    (2, 1, 0.0, 1, True)):
        mw, pw, want = measure.parity_collapse(rho, qa, qb, u, force, decay)
        ctx = make_ctx(vqd, 5, p, rho)
        try:
            m, pm = vqd.vqd_measure_parity(ctx, 0, qa, qb, u, force, decay)
            assert m == mw and abs(pm - pw) < (1e-13 if p != "f32" else 1e-6)
            assert np.abs(gpu_state(vqd, ctx) - want).max() < (1e-12 if p != "f32" else 1e-5)
        finally:
            vqd.vqd_destroy(ctx)


def qnd_initialise(meas, x_gate, crot, draws):
    """Sec. 7's QND initialisation of Q1, Q2, Q3 (Eq. initqdots) with classical feedback, driven through callbacks:
    meas(u) is the parity readout of (Q1, Q2) with decay, returning the outcome ("0" odd, "1" even); x_gate(q)
    flips qubit q; crot() is the controlled-X from Q3 to Q2.  Two rounds: readout, X on Q1 if even, readout
    (now |10> on Q1 Q2), CROT, readout (= Q3), X on Q3 if it read 1; the second round re-prepares Q1 Q2."""
    outcomes = []
    for _ in range(2):
        p1 = meas(next(draws))
        if p1 == 1:
            x_gate(0)
        meas(next(draws))
        crot()
        p3 = meas(next(draws))
        outcomes.append((p1, p3))
        if p3 == 1:
            x_gate(2)
    return outcomes


def test_qnd_initialisation_with_feedback(vqd):
    """From a random 3-qubit state, the feedback protocol leaves |Q1 Q2 Q3> = |100> whatever the draws, on the GPU
    and in the oracle, with the same outcomes."""
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    CX = np.eye(4, dtype=complex)[[0, 3, 2, 1]]          # control = first target (low bit), target = second
    for seed in range(3):
        rng = np.random.default_rng(500 + seed)
        rho0 = rand_state(3, rng)
        u = list(rng.uniform(size=6))
        ctx = make_ctx(vqd, 3, "f64", rho0)
        try:
            got = qnd_initialise(lambda x: vqd.vqd_measure_parity(ctx, 0, 0, 1, x, -1, True)[0],
                                 lambda q: vqd.vqd_apply_unitary(ctx, 0, [q], X),
                                 lambda: vqd.vqd_apply_unitary(ctx, 0, [2, 1], CX), iter(u))
            state = {"rho": rho0}

            def o_meas(x):
                m, _, state["rho"] = measure.parity_collapse(state["rho"], 0, 1, x, -1, True)
                return m

            def o_x(q):
                state["rho"] = evolve.apply_unitary(state["rho"], (q,), X)

            def o_crot():
                state["rho"] = evolve.apply_unitary(state["rho"], (2, 1), CX)

            want = qnd_initialise(o_meas, o_x, o_crot, iter(u))
            assert got == want
            final = np.zeros((8, 8))
            final[0b001, 0b001] = 1.0                        # Q1 = q0 = 1, Q2 = Q3 = 0
            assert np.abs(state["rho"] - final).max() < 1e-12
            assert np.abs(gpu_state(vqd, ctx) - final).max() < 1e-12
        finally:
            vqd.vqd_destroy(ctx)


# ---------------------------------------------------------------- reductions
@pytest.mark.parametrize("p", PRECS)
def test_reductions(vqd, p):
    rng = np.random.default_rng(31)
    n = 6
    rho = rand_state(n, rng)
    ctx = make_ctx(vqd, n, p, rho)
    try:
        rho_dev = gpu_state(vqd, ctx)           # the stored state (rounded to FP32 in f32 mode)
        t = 1e-13 if p == "f64" else 1e-12
        for qs in ([0], [5, 2], [1, 3, 4], list(range(n)), [4, 0, 5, 1, 2, 3]):
            assert np.abs(vqd.vqd_prob(ctx, 0, qs) - measure.probs(rho_dev, qs)).max() < t
        codes = rng.integers(0, 4, size=(70, n)).astype(np.uint8)   # > 64 terms: two launches
        coeffs = rng.normal(size=70)
        assert abs(vqd.vqd_expect(ctx, 0, codes, coeffs) - measure.expect(rho_dev, codes, coeffs)) < 1e-12
        assert abs(vqd.vqd_trace(ctx, 0) - measure.trace(rho_dev)) < t
        assert abs(vqd.vqd_purity(ctx, 0) - measure.purity(rho_dev)) < t
    finally:
        vqd.vqd_destroy(ctx)


# ---------------------------------------------------------------- batched persistent path
@pytest.fixture(scope="module")
def batch_programs():
    """Uneven instances of the neutral-atom batch workload and their oracle states (computed once): single-tile
    instances (n = 3..8), multi-stage ones (n = 9, 10) and the largest sizes of the batch configuration (n = 11,
    12; one layer each, the oracle's cost growing as 4^n per op)."""
    from workloads import config4_neutral_batch
    progs = config4_neutral_batch(seed=8, count=10, n_lo=3, n_hi=8, depth=3)
    progs += config4_neutral_batch(seed=9, count=2, n_lo=9, n_hi=10, depth=2)
    progs += [config4_neutral_batch(seed=10 + m, count=1, n_lo=m, n_hi=m, depth=1)[0] for m in (11, 12)]
    assert [q.n for q in progs[-2:]] == [11, 12]
    return progs, [cloop.run_program(q) for q in progs]


@pytest.mark.parametrize("p,fuse", [("f64", 0), ("f32", 0), ("f32", 3), ("split", 0)])
def test_batch_matches_per_instance_oracle(vqd, p, fuse, batch_programs):
    """Uneven instances in one batched run, up to the batch configuration's largest size (n = 12), whose
    stages span several waves and tile chunks, each against the oracle."""
    progs, wants = batch_programs
    ctx = vqd.vqd_create_batch([q.n for q in progs], prec_code(vqd, p))
    try:
        vqd.vqd_run_batch(ctx, [q.ops for q in progs], fuse)
        probs, trs, purs = vqd.vqd_batch_reduce(ctx, [q.n for q in progs])
        for i, prog in enumerate(progs):
            want = wants[i]
            got = gpu_state(vqd, ctx, i)
            t = tol(p, len(prog.ops))
            assert np.abs(got - want).max() < t, i
            assert abs(vqd.vqd_trace(ctx, i) - 1) < t
            assert np.abs(probs[i] - measure.probs(want, range(prog.n))).max() < t
            assert abs(trs[i] - measure.trace(want).real) < t and abs(purs[i] - measure.purity(want)) < t
    finally:
        vqd.vqd_destroy(ctx)


# ---------------------------------------------------------------- argument checks and error codes
def test_error_codes(vqd):
    ctx = vqd.vqd_create(3, vqd.VQD_F64)
    try:
        with pytest.raises(vqd.VQDError) as e:
            vqd.vqd_apply_unitary(ctx, 0, [3], np.eye(2))           # target out of range
        assert e.value.code == vqd.VQD_EINVAL
        with pytest.raises(vqd.VQDError) as e:
            vqd.vqd_apply_unitary(ctx, 0, [1, 1], np.eye(4))        # repeated target
        assert e.value.code == vqd.VQD_EINVAL
        with pytest.raises(vqd.VQDError) as e:
            vqd.vqd_apply_unitary(ctx, 0, [0], np.array([[1, 1], [0, 1]]))
        assert e.value.code == vqd.VQD_ENOTCP
        with pytest.raises(vqd.VQDError) as e:
            vqd.vqd_apply_kraus(ctx, 0, [0], [np.eye(2), 0.5 * np.eye(2)])   # sum K^dag K = 1.25 I
        assert e.value.code == vqd.VQD_ENOTCP
        vqd.vqd_apply_kraus(ctx, 0, [0], oc.leak_init(0.1))          # CPTN is accepted
        assert abs(vqd.vqd_trace(ctx, 0) - 0.9) < 1e-15
        with pytest.raises(vqd.VQDError) as e:
            vqd.vqd_prob(ctx, 0, [0, 0])
        assert e.value.code == vqd.VQD_EINVAL
        with pytest.raises(vqd.VQDError) as e:
            vqd.vqd_run_program(ctx, 0, [NativeOp("rx", (0,), (0.1,))], 9)
        assert e.value.code == vqd.VQD_EINVAL
    finally:
        vqd.vqd_destroy(ctx)
    with pytest.raises(vqd.VQDError):
        vqd.vqd_create(17, vqd.VQD_F32)


def test_create_on_caller_memory(vqd):
    torch = pytest.importorskip("torch")
    n = 5
    buf = torch.zeros(2 * 4 ** n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ctx = vqd.vqd_create_on(n, vqd.VQD_F32, buf.data_ptr(), buf.numel() * 4, stream)
    try:
        vqd.vqd_init_zero(ctx, 0)
        vqd.vqd_apply_native(ctx, 0, [NativeOp("h", (q,)) for q in range(n)])
        torch.cuda.synchronize()
        v = buf.view(-1, 2).cpu().numpy()
        assert np.allclose(v[:, 0], 1.0 / 2 ** n, atol=1e-7) and np.allclose(v[:, 1], 0, atol=1e-7)
    finally:
        vqd.vqd_destroy(ctx)


# ---------------------------------------------------------------- full-size workload (14 qubits)
@pytest.fixture(scope="module")
def config2_full_sample():
    """A full-size (14-qubit) sample of the benchmark program: its first three ops plus the first
    op of every other kind it uses (ZZ crosstalk, T1/T2 idle, ZX, readout flip), run by the oracle."""
    prog = config2_sc_grid()
    picked = list(prog.ops[:3])
    for name in ("zz_idle", "idle", "zx", "bitflip"):
        picked.append(next(o for o in prog.ops if o.name == name))
    sample = Program(prog.n, picked)
    return sample, evolve.run_program(sample)


@pytest.mark.parametrize("path", ["plain", "fused"])
def test_config2_full_size_sample_and_invariants(vqd, path, config2_full_sample):
    """At the full 14-qubit size: a sample program element by element against the oracle, and the whole
    program (complex64, the benchmark configuration) against properties that hold at any size."""
    sample, want = config2_full_sample
    got, _ = run_gpu(vqd, sample, "f32", path)
    assert np.abs(got - want).max() < tol_f32(len(sample.ops))
    del got
    prog = config2_sc_grid()
    ctx = vqd.vqd_create(prog.n, vqd.VQD_F32)
    try:
        if path == "plain":
            vqd.vqd_apply_native(ctx, 0, prog.ops)
        else:
            vqd.vqd_run_program(ctx, 0, prog.ops)
        tr = vqd.vqd_trace(ctx, 0)
        assert abs(tr - 1) < 1e-4                              # CPTP program: trace 1
        pr = vqd.vqd_prob(ctx, 0, list(range(14)))
        assert pr.min() > -1e-6 and abs(pr.sum() - tr.real) < 1e-9
        pur = vqd.vqd_purity(ctx, 0)
        assert 2.0 ** -14 - 1e-9 <= pur <= 1.0 + 1e-6
        # Hermiticity on sampled entries: rho[r][c] = conj(rho[c][r])
        flat = vqd.vqd_get_state(ctx, 0)
        rng = np.random.default_rng(3)
        r, c = rng.integers(0, 2 ** 14, 4096), rng.integers(0, 2 ** 14, 4096)
        assert np.abs(flat[r + (c << 14)] - np.conj(flat[c + (r << 14)])).max() < 1e-6
    finally:
        vqd.vqd_destroy(ctx)


# ---------------------------------------------------------------- the largest workloads (15 and 16 qubits)
def test_ion15_full_size_sample_vs_oracle(vqd):
    """15 qubits (complex64 8.6 GB, complex128 17.2 GB): the first gates of the ion-trap program, both precisions,
    element by element against the oracle (compared in the library's flat layout)."""
    prog = config3_ion_alltoall()
    ops = list(prog.ops[:3])
    want = evolve.to_device_layout(evolve.run_program(Program(prog.n, ops)))
    for p in PRECS:
        for path in ("plain", "fused"):
            ctx = vqd.vqd_create(prog.n, prec_code(vqd, p))
            try:
                if path == "plain":
                    vqd.vqd_apply_native(ctx, 0, ops)
                else:
                    vqd.vqd_run_program(ctx, 0, ops)
                got = vqd.vqd_get_state(ctx, 0)
                assert np.abs(got - want).max() < tol(p, 3), (p, path)
                assert abs(vqd.vqd_trace(ctx, 0) - 1) < tol(p, 3)
                del got
            finally:
                vqd.vqd_destroy(ctx)


def test_spin16_max_size_invariants_and_paths_agree(vqd):
    """16 qubits, the largest supported size (complex64 34.4 GB): the first 240 native ops of the spin-chain program
    through the plain path, the fused path and the fused path with Hermitian stages (which must leave an exactly
    Hermitian state); CPTP invariants and agreement of the paths on sampled amplitudes."""
    prog = config5_spin_chain()
    ops = prog.ops[:240]
    n = prog.n
    rng = np.random.default_rng(16)
    r, c = rng.integers(0, 2 ** n, 8192), rng.integers(0, 2 ** n, 8192)
    idx = r + (c << n)
    samples, reds = {}, {}
    for path in ("plain", "fused", "fused_herm"):
        ctx = vqd.vqd_create(n, vqd.VQD_F32)
        try:
            if path == "plain":
                vqd.vqd_apply_native(ctx, 0, ops)
            else:
                vqd.vqd_run_program(ctx, 0, ops, 0, vqd.VQD_HERMITIAN if path == "fused_herm" else 0)
            reds[path] = (vqd.vqd_trace(ctx, 0), vqd.vqd_purity(ctx, 0), vqd.vqd_prob(ctx, 0, [0, 7, 15]))
            flat = vqd.vqd_get_state(ctx, 0)
            samples[path] = flat[idx]
            herm = np.abs(flat[idx] - np.conj(flat[c + (r << n)])).max()
            del flat
        finally:
            vqd.vqd_destroy(ctx)
        tr, pur, pr = reds[path]
        assert abs(tr - 1) < 1e-4 and pur <= 1 + 1e-5 and herm < 1e-6
        assert abs(pr.sum() - tr.real) < 1e-9 and pr.min() > -1e-7
        if path == "fused_herm":
            assert herm == 0.0
    for path in ("fused", "fused_herm"):
        assert np.abs(samples["plain"] - samples[path]).max() < tol_f32(len(ops))
        assert abs(reds["plain"][1] - reds[path][1]) < 1e-5


# ---------------------------------------------------------------- tile shapes and the autotuner
@pytest.mark.parametrize("p", PRECS)
def test_tile_shapes_give_the_same_result(vqd, p):
    prog = random_program(303, 8, 120)
    want = evolve.run_program(prog)
    shapes = [(13, 3), (13, 2), (12, 2), (11, 1), (8, 0)] if p == "f32" else [(12, 2), (11, 1), (8, 0)]
    for tb, L in shapes:
        ctx = vqd.vqd_create(prog.n, prec_code(vqd, p))
        try:
            vqd.vqd_set_tile_shape(ctx, tb, L)
            vqd.vqd_run_program(ctx, 0, prog.ops, 4)
            got = gpu_state(vqd, ctx)
        finally:
            vqd.vqd_destroy(ctx)
        assert np.abs(got - want).max() < tol(p, len(prog.ops)), (tb, L)
    ctx = vqd.vqd_create(4, prec_code(vqd, p))
    try:
        with pytest.raises(vqd.VQDError):
            vqd.vqd_set_tile_shape(ctx, 14, 3)                # above the 64 KB tile
        with pytest.raises(vqd.VQDError):
            vqd.vqd_set_tile_shape(ctx, 5, 2)                 # a 2-qubit operator needs 4 bits + passengers
    finally:
        vqd.vqd_destroy(ctx)


def test_autotuner_picks_a_candidate_and_keeps_results(vqd, tmp_path):
    from paper_2306_07342_gb300 import autotune
    prog = config2_sc_grid(seed=11, rows=2, cols=5, depth=6)
    cache = str(tmp_path / "tune.json")
    choice = autotune.tune(prog.n, vqd.VQD_F32, prog.ops, cache_path=cache)
    assert (choice["fuse_qubits"], choice["tile_bits"], choice["passenger_bits"]) in autotune.CANDIDATES[vqd.VQD_F32]
    assert len(choice["trials"]) == len(autotune.CANDIDATES[vqd.VQD_F32])
    assert autotune.tune(prog.n, vqd.VQD_F32, prog.ops, cache_path=cache) == choice    # cached
    want = evolve.run_program(prog)
    ctx = vqd.vqd_create(prog.n, vqd.VQD_F32)
    try:
        f = autotune.apply(ctx, choice)
        vqd.vqd_run_program(ctx, 0, prog.ops, f)
        got = gpu_state(vqd, ctx)
    finally:
        vqd.vqd_destroy(ctx)
    assert np.abs(got - want).max() < tol_f32(len(prog.ops))


def test_batch_graph_capture_and_replay(vqd):
    """On a non-default stream the batch is captured into a CUDA graph; running the same batch again replays
    it (after re-initialising the states) and a different batch rebuilds it.  Results match the oracle each time."""
    torch = pytest.importorskip("torch")
    from workloads import config4_neutral_batch
    progs = config4_neutral_batch(seed=12, count=6, n_lo=3, n_hi=9, depth=2)
    stream = torch.cuda.Stream()
    ctx = vqd.vqd_create_batch([q.n for q in progs], vqd.VQD_F32, stream.cuda_stream)
    try:
        for round_ in range(3):
            if round_ == 2:     # a different batch: new angles for every instance
                progs = config4_neutral_batch(seed=13, count=6, n_lo=3, n_hi=9, depth=2)
                ctx2 = vqd.vqd_create_batch([q.n for q in progs], vqd.VQD_F32, stream.cuda_stream)
                vqd.vqd_destroy(ctx)
                ctx = ctx2
            for i in range(len(progs)):
                vqd.vqd_init_zero(ctx, i)
            vqd.vqd_profile(ctx, 1)
            vqd.vqd_profile_reset(ctx)
            vqd.vqd_run_batch(ctx, [q.ops for q in progs])
            launches = vqd.vqd_profile_read(ctx)["batch"]["launches"]
            assert launches == 1                          # one graph launch
            vqd.vqd_sync(ctx)
            for i, prog in enumerate(progs):
                want = evolve.run_program(prog)
                assert np.abs(gpu_state(vqd, ctx, i) - want).max() < tol_f32(len(prog.ops)), (round_, i)
    finally:
        vqd.vqd_destroy(ctx)


@pytest.mark.parametrize("p", PRECS)
def test_measure_collapse_matches_oracle(vqd, p):
    from oracle.measure import measure_collapse
    rng = np.random.default_rng(41)
    n = 5
    rho = rand_state(n, rng)
    ctx = make_ctx(vqd, n, p, rho)
    try:
        rho = gpu_state(vqd, ctx)                    # the stored state (FP32-rounded in f32)
        for q, u, force in ((2, 0.31, -1), (0, 0.93, -1), (4, 0.0, 1), (1, 0.5, 0)):
            m, pm = vqd.vqd_measure(ctx, 0, q, u, force)
            mw, pw, rho = measure_collapse(rho, q, u, force)
            assert m == mw and abs(pm - pw) < (1e-13 if p == "f64" else 1e-6)
            assert np.abs(gpu_state(vqd, ctx) - rho).max() < (1e-12 if p == "f64" else 1e-5)
            assert abs(vqd.vqd_trace(ctx, 0) - 1) < (1e-13 if p == "f64" else 1e-5)
        with pytest.raises(vqd.VQDError):
            vqd.vqd_measure(ctx, 0, 4, 0.0, 0)       # qubit 4 was post-selected to 1: outcome 0 is impossible
    finally:
        vqd.vqd_destroy(ctx)
