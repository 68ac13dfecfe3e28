"""CPU-only checks of the C ABI: the library loads, exports every declared symbol, and its device
compiler (host code) agrees with the oracle's compiler.  No GPU call is made here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import compile as oc
from workloads.circuits import OP_NAMES, NativeOp, random_program, _random_params, _rng

from ._lib import get_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vqd.h")


@pytest.fixture(scope="module")
def vqd():
    return get_lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vqd_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function(vqd):
    names = declared_functions()
    assert len(names) >= 30
    L = ctypes.CDLL(vqd.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_op_code_tables_agree():
    """The header enum, the binding's code list and the workload vocabulary name the same ops in one order."""
    from paper_2306_07342_gb300 import vqd as b
    src = open(HEADER).read()
    enum = re.findall(r"VQD_OP_([A-Z0-9_]+)\s*=\s*(\d+)", src)
    enum = [(name.lower(), int(v)) for name, v in enum if name != "COUNT"]
    assert [v for _, v in enum] == list(range(len(enum)))
    assert [name for name, _ in enum] == b.OP_CODES == list(OP_NAMES)


def oracle_superop(steps):
    """Compose the oracle's compiled steps (applied in order) into one superoperator, index r | c << k."""
    k = len(steps[0][1])
    d = 2 ** k
    S = np.eye(d * d, dtype=complex)
    for kind, _, m in steps:
        ks = [m] if kind == "U" else m
        Sk = np.zeros((d * d, d * d), dtype=complex)
        for K in ks:
            Sk += np.kron(K.conj(), K)      # vec(K X K^dag) = (conj(K) (x) K) vec(X), column-major vec
        S = Sk @ S
    return S


@pytest.mark.parametrize("name", list(OP_NAMES))
def test_device_compiler_matches_oracle(vqd, name):
    r = _rng(1234 + list(OP_NAMES).index(name))
    nq = OP_NAMES[name][0]
    for trial in range(4):
        params = _random_params(r, name)
        qs = (0,) if nq == 1 else (1, 0)
        op = NativeOp(name, qs, params)
        for flags in (0, vqd.VQD_T2_IS_TOTAL):
            if flags and name not in ("idle", "idle_depol", "ampdeph2"):
                continue
            if flags and params[2] > 2 * params[1]:
                continue
            kind, t, M = vqd.vqd_compile_op(op, flags)
            steps = oc.compile_op(name, qs, params, bool(flags))
            assert t == qs
            if kind == "U":
                assert len(steps) == 1 and steps[0][0] == "U"
                assert np.abs(M - steps[0][2]).max() < 1e-13, name
            else:
                assert np.abs(M - oracle_superop(steps)).max() < 1e-13, name


@pytest.mark.parametrize("nq", [1, 2])
def test_stderr_params_match_oracle(vqd, nq):
    for fbar, x in [(0.999, 0.3), (0.99, 0.0), (0.95, 1.0), (0.97, 0.75)]:
        got = vqd.vqd_stderr_params(nq, fbar, x)
        want = oc.stderr_params(fbar, x, nq)
        assert abs(got[0] - want[0]) < 1e-15 and abs(got[1] - want[1]) < 1e-15


def test_compile_rejects_bad_ops(vqd):
    with pytest.raises(vqd.VQDError) as e:
        vqd.vqd_compile_op(NativeOp("depol1", (0,), (0.9,)))          # p > 3/4
    assert e.value.code == vqd.VQD_EINVAL
    with pytest.raises(vqd.VQDError) as e:                            # Delta_ct - alpha_t = 0: no finite beta
        vqd.vqd_compile_op(NativeOp("zz_static", (0, 1), (0.1, -2.5, -2.5, -2.0)))
    assert e.value.code == vqd.VQD_EINVAL
    a = vqd.native_ops([NativeOp("rx", (0,), (0.1,))])
    a[0]["code"] = 99
    isu, k = ctypes.c_int(), ctypes.c_int()
    t = np.zeros(2, np.int32)
    m = np.zeros(256, np.complex128)
    rc = vqd.lib().vqd_compile_op(a.ctypes.data_as(ctypes.c_void_p), 0, ctypes.byref(isu), ctypes.byref(k),
                                  t.ctypes.data_as(ctypes.c_void_p), m.ctypes.data_as(ctypes.c_void_p))
    assert rc == vqd.VQD_EINVAL


def test_state_bytes(vqd):
    assert vqd.vqd_state_bytes(14, vqd.VQD_F32) == 8 * 4 ** 14
    assert vqd.vqd_state_bytes(16, vqd.VQD_F64) == 16 * 4 ** 16
    assert vqd.vqd_state_bytes(17, vqd.VQD_F64) == 0
    assert vqd.vqd_state_bytes(14, vqd.VQD_F32_SPLIT) == 16 * 4 ** 14     # float-float pairs, like complex128


def test_precision_enum_matches_header(vqd):
    src = open(HEADER).read()
    assert "VQD_F64 = 0, VQD_F32 = 1, VQD_F32_SPLIT = 2" in src
    assert (vqd.VQD_F64, vqd.VQD_F32, vqd.VQD_F32_SPLIT) == (0, 1, 2)


def test_trajectories_refuse_split_precision(vqd):
    """Checked on the host before any device work: trajectories run in complex64 or complex128 only."""
    with pytest.raises(vqd.VQDError) as e:
        vqd.vqd_traj_expect(3, vqd.VQD_F32_SPLIT, [NativeOp("h", (0,))], 4, 1, np.ones((1, 3), np.uint8), [1.0])
    assert e.value.code == vqd.VQD_EINVAL


def test_schedule_worked_example_and_oracle(vqd):
    """Two layers by hand: rx(q0) 0.1 us and cz(q1,q2) 0.3 us run together (q0 waits 0.2, q3 idles 0.3);
    then cz(q0,q1) 0.3 us (q2, q3 idle 0.3).  Gate noise stays right after its gate."""
    from oracle.schedule import schedule
    t1, t2 = [50.0, 60.0, 70.0, 80.0], [30.0, 40.0, 50.0, 60.0]
    ops = [NativeOp("rx", (0,), (0.5,)), NativeOp("depol1", (0,), (1e-3,)),
           NativeOp("cz", (1, 2)), NativeOp("depol2", (1, 2), (1e-2,)),
           NativeOp("cz", (0, 1))]
    dur = [0.1, -1, 0.3, -1, 0.3]
    want = [("rx", (0,)), ("depol1", (0,)), ("cz", (1, 2)), ("depol2", (1, 2)),
            ("idle", (0,), 0.2), ("idle", (3,), 0.3),
            ("cz", (0, 1)), ("idle", (2,), 0.3), ("idle", (3,), 0.3)]
    orc = schedule(4, ops, dur, t1, t2)
    got = vqd.vqd_schedule(4, ops, dur, t1, t2)
    assert len(orc) == len(want) == len(got)
    for w, o, g in zip(want, orc, got):
        assert o.name == w[0] and o.qubits == w[1]
        assert vqd.OP_CODES[g["code"]] == w[0] and tuple(g["q"][: g["nq"]]) == w[1]
        if len(w) == 3:
            assert abs(o.params[0] - w[2]) < 1e-15 and abs(g["par"][0] - w[2]) < 1e-15
            assert g["par"][1] == t1[w[1][0]] and g["par"][2] == t2[w[1][0]]


@pytest.mark.parametrize("idle", ["idle_depol", "idle_t2s"])
def test_schedule_random_programs_match_oracle(vqd, idle):
    from oracle.schedule import schedule
    r = _rng(77)
    n = 5
    prog = random_program(78, n, 60, names=["rx", "ry", "cz", "zx", "xx", "depol1", "depol2", "amp"])
    dur = [(-1.0 if o.name in ("depol1", "depol2", "amp") else float(r.uniform(0.05, 0.5))) for o in prog.ops]
    # a noise op must follow a gate on the same qubits: make every noise op act on its gate's qubits
    ops, d2 = [], []
    for o, d in zip(prog.ops, dur):
        if d < 0:
            if not ops or d2[-1] < 0:
                continue
            g = ops[-1]
            name = "depol1" if len(g.qubits) == 1 else "depol2"
            o = NativeOp(name, g.qubits, (1e-3,))
        ops.append(o)
        d2.append(d)
    t1, t2 = list(r.uniform(20, 100, n)), list(r.uniform(10, 50, n))
    orc = schedule(n, ops, d2, t1, t2, idle=idle)
    got = vqd.vqd_schedule(n, ops, d2, t1, t2, idle=idle)
    assert len(orc) == len(got)
    for o, g in zip(orc, got):
        assert vqd.OP_CODES[g["code"]] == o.name and tuple(g["q"][: g["nq"]]) == o.qubits
        assert np.allclose(g["par"][: len(o.params)], o.params, rtol=0, atol=1e-15)


def test_fused_plan_splits_tensor_product_channels(vqd):
    """The fused planner applies a two-qubit channel that is a tensor product of one-qubit channels (T1/T2
    decay of both qubits of a pair) as two one-qubit sweeps, and keeps a correlated one (depol2) dense."""
    prod = [NativeOp("ampdeph2", (0, 2), (0.3, 40.0, 30.0))]
    info = vqd.vqd_plan_info(4, vqd.VQD_F32, prod, fuse_qubits=4)
    assert info["sup2"] == 0 and info["sup1"] == 2
    corr = [NativeOp("depol2", (0, 2), (0.1,))]
    info = vqd.vqd_plan_info(4, vqd.VQD_F32, corr, fuse_qubits=4)
    assert info["sup2"] == 1 and info["sup1"] == 0



def test_fused_plan_keeps_slightly_correlated_channels_dense(vqd):
    """A two-qubit channel that is a product only up to 5e-14 (depol2 with p = 2e-13) stays one channel: the
    planner's product test accepts only a few FP64 roundings of an exact product, so no channel is replaced
    by an approximation above FP64 rounding."""
    info = vqd.vqd_plan_info(4, vqd.VQD_F64, [NativeOp("depol2", (0, 2), (2e-13,))], fuse_qubits=4)
    assert info["sup2"] == 1 and info["sup1"] == 0


@pytest.mark.parametrize("prec_name,state_addr,out_addr", [("f64", 0x10008, 0x20000), ("split", 0x10004, 0x20000),
                                                           ("f32", 0x10004, 0x20000), ("f32", 0x10008, 0x20004)])
def test_prob_static_refuses_misaligned_addresses(vqd, prec_name, state_addr, out_addr):
    """Misaligned device addresses are refused with VQD_EINVAL before any CUDA call (these fake addresses
    never reach a GPU), instead of faulting in the kernel."""
    prec = {"f64": vqd.VQD_F64, "f32": vqd.VQD_F32, "split": vqd.VQD_F32_SPLIT}[prec_name]
    with pytest.raises(vqd.VQDError) as e:
        vqd.vqd_prob_static(state_addr, 4, prec, [0, 1], out_addr)
    assert e.value.code == vqd.VQD_EINVAL and "aligned" in str(e.value)



def test_tc_plan_blocks_keep_per_qubit_order_and_cover_every_op(vqd):
    """The tensor-core planner's blocks hold at most k qubits and, for ion-trap all-to-all programs, absorb
    several native ops each; every op lands in exactly one block (host-only planning call)."""
    from workloads import config3_ion_alltoall
    prog = config3_ion_alltoall(seed=3, n=15, n_gates=800)
    prev = None
    for k in (4, 5, 6):
        info = vqd.vqd_tc_plan_info(15, prog.ops, k)
        assert info["native_ops"] == len(prog.ops) and info["max_block_ops"] >= 1
        assert info["blocks"] * k >= 2 * 1 and info["blocks"] < len(prog.ops) / 4
        if prev is not None:
            assert info["blocks"] <= prev                 # wider blocks never need more passes here
        prev = info["blocks"]
    with pytest.raises(vqd.VQDError):
        vqd.vqd_tc_plan_info(15, prog.ops, 7)


def test_hermitian_plan_symmetric_tiles(vqd):
    """VQD_HERMITIAN plans (host only): symmetric tiles have an even bit count within the tile budget, the
    stage count stays close to the general plan's (the passengers' column bits take the place of one
    passenger row bit), and a shape without room for a two-qubit operator beside the passengers' row and
    column bits is refused."""
    from workloads import config2_sc_grid
    prog = config2_sc_grid()
    for prec in (vqd.VQD_F64, vqd.VQD_F32_SPLIT, vqd.VQD_F32):
        gen = vqd.vqd_plan_info(14, prec, prog.ops)
        herm = vqd.vqd_plan_info(14, prec, prog.ops, flags=vqd.VQD_HERMITIAN)
        assert herm["max_tile_bits"] % 2 == 0 and herm["max_tile_bits"] <= 12
        assert herm["native_ops"] == gen["native_ops"]
        assert 0.8 * gen["stages"] <= herm["stages"] <= 1.35 * gen["stages"], (prec, gen, herm)
    small = random_program(12, 8, 40).ops
    assert vqd.vqd_plan_info(8, vqd.VQD_F64, small, tile_bits=6, passenger_bits=2)["stages"] > 0
    with pytest.raises(vqd.VQDError) as e:
        vqd.vqd_plan_info(8, vqd.VQD_F64, small, flags=vqd.VQD_HERMITIAN, tile_bits=6, passenger_bits=2)
    assert e.value.code == vqd.VQD_EINVAL


def test_plans_of_long_programs_respect_the_stage_budgets(vqd):
    """Long random programs of every op kind plan without tripping the stage budgets' internal checks: at most
    kCoefCap coefficients, kOpCap operators and 64 blocks (shared-memory sweeps) per stage, the planner splitting
    larger stages; in every precision, general and Hermitian, over fusion widths."""
    prog = random_program(4242, 8, 2000)
    for prec in (vqd.VQD_F64, vqd.VQD_F32_SPLIT, vqd.VQD_F32):
        for flags in (0, vqd.VQD_HERMITIAN):
            for fuse in (2, 4, 6):
                info = vqd.vqd_plan_info(8, prec, prog.ops, fuse_qubits=fuse, flags=flags)
                assert info["native_ops"] == 2000 and 0 < info["stages"] <= 2000
                assert info["blocks"] >= info["stages"]


def test_autotuner_candidates_and_run_flags(vqd):
    """Host logic of the autotuner (no GPU): with Hermitian stages allowed, the Hermitian shapes come first and the
    general shapes follow; without, only the general ones; explicit 3-tuples take the caller's flag and 4-tuples keep
    their own; the run flags set or clear VQD_HERMITIAN and keep every other bit."""
    from paper_2306_07342_gb300 import autotune
    for prec in (vqd.VQD_F64, vqd.VQD_F32, vqd.VQD_F32_SPLIT):
        both = autotune._candidates(None, True, autotune.HERM_CANDIDATES[prec], autotune.CANDIDATES[prec])
        assert both == [(*c, True) for c in autotune.HERM_CANDIDATES[prec]] + [(*c, False) for c in autotune.CANDIDATES[prec]]
        gen = autotune._candidates(None, False, autotune.HERM_CANDIDATES[prec], autotune.CANDIDATES[prec])
        assert gen == [(*c, False) for c in autotune.CANDIDATES[prec]]
        for f, tb, p, h in both:
            assert tb <= (13 if prec == vqd.VQD_F32 else 12) and 4 + p <= tb
            if h:
                assert 2 * (p + 2) <= (tb & ~1)        # a Hermitian tile has room for a two-qubit operator
    assert autotune._candidates([(6, 12, 1)], True, [], []) == [(6, 12, 1, True)]
    assert autotune._candidates([(6, 12, 1, False)], True, [], []) == [(6, 12, 1, False)]
    extra = vqd.VQD_T2_IS_TOTAL
    assert autotune._run_flags(extra, True) == extra | vqd.VQD_HERMITIAN
    assert autotune._run_flags(extra | vqd.VQD_HERMITIAN, False) == extra


def test_single_tile_states_plan_the_same_with_or_without_hermitian_stages(vqd):
    """A state whose whole index fits one tile (2n <= 12 bits: n <= 6) is planned on whole-state tiles (split only
    by the per-stage coefficient and block budgets), in every precision; VQD_HERMITIAN changes nothing there (a
    single tile is its own mirror)."""
    for n in (1, 3, 6):
        prog = random_program(600 + n, n, 80)
        for prec in (vqd.VQD_F64, vqd.VQD_F32_SPLIT, vqd.VQD_F32):
            gen = vqd.vqd_plan_info(n, prec, prog.ops)
            herm = vqd.vqd_plan_info(n, prec, prog.ops, flags=vqd.VQD_HERMITIAN)
            assert gen["max_tile_bits"] == 2 * n and gen == herm, (n, prec, gen, herm)
