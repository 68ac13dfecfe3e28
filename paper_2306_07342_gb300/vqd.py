"""Thin ctypes binding of libvqd (include/vqd.h): the same entry points, arguments marshalled only.

Every computation happens in the library's CUDA kernels.  Loading fails loudly when libvqd.so is
missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvqd.so")

VQD_F64, VQD_F32, VQD_F32_SPLIT = 0, 1, 2
VQD_T2_IS_TOTAL, VQD_NO_CHECK, VQD_HERMITIAN = 1, 2, 4
VQD_OK, VQD_EINVAL, VQD_ENOMEM, VQD_ENOTCP, VQD_EDEVICE, VQD_ENOTSUP = 0, -1, -2, -3, -4, -5
VQD_MAX_QUBITS = 16
VQD_MAX_FUSE = 6

# Native op codes, in the order of the header's vqd_op_code enum.
OP_CODES = ["rx", "ry", "rz", "sx", "h", "u", "r", "cz", "cph", "czphi", "zx", "zz", "xx", "zzphase", "zz_idle",
            "crz_xtalk", "exchange", "depol1", "depol2", "deph1", "deph2", "amp", "bitflip", "bitflip2", "gamp",
            "idle", "idle_depol", "stderr1", "stderr2", "ampdeph2", "leak_init", "leak_cz",
            "offres", "zz_static", "zy", "idle_t2s", "bitflip_asym"]
OP_CODE = {name: i for i, name in enumerate(OP_CODES)}

NATIVE_OP_DTYPE = np.dtype([("code", "<i4"), ("nq", "<i4"), ("q", "<i4", (2,)), ("par", "<f8", (4,))])
assert NATIVE_OP_DTYPE.itemsize == 48


class c128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class kstat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("alg_bytes", ctypes.c_double), ("amp_updates", ctypes.c_double), ("alg_fma", ctypes.c_double)]


class sc_device(ctypes.Structure):
    """vqd_sc_device: superconducting device table (pointers stay valid while the arrays live)."""
    _fields_ = [("n", ctypes.c_int32), ("ncouple", ctypes.c_int32),
                ("t1", ctypes.c_void_p), ("t2", ctypes.c_void_p), ("excited", ctypes.c_void_p),
                ("freq", ctypes.c_void_p), ("anharm", ctypes.c_void_p), ("couple", ctypes.c_void_p),
                ("coupling", ctypes.c_void_p), ("fid_read", ctypes.c_void_p),
                ("dur_rxy", ctypes.c_double), ("dur_zx", ctypes.c_double), ("dur_zz", ctypes.c_double),
                ("dur_meas", ctypes.c_double), ("flags", ctypes.c_uint32)]


VQD_SC_NO_PASSIVE = 1
VQD_SC_NO_STATIC_ZZ = 2


class si_device(ctypes.Structure):
    """vqd_si_device: silicon spin-qubit device table."""
    _fields_ = [("n", ctypes.c_int32), ("t1", ctypes.c_void_p), ("t2", ctypes.c_void_p), ("freq", ctypes.c_void_p),
                ("rabi", ctypes.c_void_p), ("fid_1q", ctypes.c_void_p), ("x_1q", ctypes.c_double),
                ("freq_cz", ctypes.c_void_p), ("fid_cz", ctypes.c_void_p), ("x_cz", ctypes.c_double),
                ("xtalk_on", ctypes.c_void_p), ("xtalk_off", ctypes.c_void_p), ("flags", ctypes.c_uint32)]


VQD_SI_NO_PASSIVE = 1
VQD_SI_NO_OFFRES = 2


class nv_device(ctypes.Structure):
    """vqd_nv_device: NV-centre device table (qubit 0 = electron spin)."""
    _fields_ = [("n", ctypes.c_int32), ("t1", ctypes.c_void_p), ("t2", ctypes.c_void_p),
                ("freq_xy", ctypes.c_void_p), ("freq_z", ctypes.c_void_p), ("fid_xy", ctypes.c_void_p),
                ("fid_z", ctypes.c_void_p), ("x_xy", ctypes.c_double), ("freq_crot", ctypes.c_void_p),
                ("fid_crot", ctypes.c_void_p), ("x_crot", ctypes.c_double), ("freq_zz", ctypes.c_double),
                ("fid_meas", ctypes.c_double), ("dur_meas", ctypes.c_double), ("flags", ctypes.c_uint32)]


VQD_NV_NO_PASSIVE = 1


class ion_device(ctypes.Structure):
    """vqd_ion_device: trapped-ion device table (every ion identical)."""
    _fields_ = [("n", ctypes.c_int32), ("t1", ctypes.c_double), ("t2s", ctypes.c_double), ("rabi", ctypes.c_double),
                ("fid_xy", ctypes.c_double), ("x_xy", ctypes.c_double), ("freq_cz", ctypes.c_double),
                ("fid_cz", ctypes.c_double), ("x_cz", ctypes.c_double), ("bf_read", ctypes.c_double),
                ("dur_read", ctypes.c_double), ("flags", ctypes.c_uint32)]


VQD_ION_NO_PASSIVE = 1


class na_device(ctypes.Structure):
    """vqd_na_device: neutral-atom device table (identical atoms at fixed sites)."""
    _fields_ = [("n", ctypes.c_int32), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("blockade", ctypes.c_double),
                ("t2", ctypes.c_double), ("t_vac", ctypes.c_double), ("p10", ctypes.c_double), ("p01", ctypes.c_double),
                ("leak_init", ctypes.c_double), ("leak_cz_a", ctypes.c_double), ("leak_cz_b", ctypes.c_double),
                ("dur_cz", ctypes.c_double), ("fid_meas", ctypes.c_double), ("flags", ctypes.c_uint32)]


VQD_NA_NO_PASSIVE = 1


VQD_TC_3XTF32 = 0
VQD_TC_BF16X3 = 1


class VQDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libvqd error {code}: {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libvqd.so not built at {LIB_PATH}; run paper_2306_07342_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, U, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint, ctypes.c_size_t
        sig = {
            "vqd_state_bytes": (S, [I, I]),
            "vqd_create": (I, [I, I, P, ctypes.POINTER(P)]),
            "vqd_create_batch": (I, [I, P, I, P, ctypes.POINTER(P)]),
            "vqd_create_on": (I, [I, I, P, S, P, ctypes.POINTER(P)]),
            "vqd_destroy": (None, [P]),
            "vqd_num_instances": (I, [P]),
            "vqd_num_qubits": (I, [P, I]),
            "vqd_state_ptr": (P, [P, I]),
            "vqd_sync": (I, [P]),
            "vqd_last_error": (ctypes.c_char_p, [P]),
            "vqd_set_flags": (I, [P, U]),
            "vqd_init_zero": (I, [P, I]),
            "vqd_init_classical": (I, [P, I, ctypes.c_uint64]),
            "vqd_init_product_diag": (I, [P, I, P]),
            "vqd_apply_unitary": (I, [P, I, I, P, P]),
            "vqd_apply_kraus": (I, [P, I, I, P, I, P]),
            "vqd_apply_superop": (I, [P, I, I, P, P]),
            "vqd_apply_native": (I, [P, I, I, P, U]),
            "vqd_run_program": (I, [P, I, I, P, I, U]),
            "vqd_run_batch": (I, [P, P, P, I, U]),
            "vqd_compile_op": (I, [P, U, P, P, P, P]),
            "vqd_stderr_params": (I, [I, D, D, P, P]),
            "vqd_prob": (I, [P, I, I, P, P]),
            "vqd_expect": (I, [P, I, I, P, P, P]),
            "vqd_trace": (I, [P, I, P, P]),
            "vqd_purity": (I, [P, I, P]),
            "vqd_get_state": (I, [P, I, P]),
            "vqd_set_state": (I, [P, I, P]),
            "vqd_profile": (I, [P, I]),
            "vqd_profile_reset": (I, [P]),
            "vqd_profile_read": (I, [P, I, P, P]),
            "vqd_prob_static": (I, [P, I, I, I, P, P, P]),
            "vqd_plan_info": (I, [I, I, I, P, I, I, I, U, P]),
            "vqd_set_tile_shape": (I, [P, I, I]),
            "vqd_measure": (I, [P, I, I, D, I, P, P]),
            "vqd_batch_reduce": (I, [P, P, P, P]),
            "vqd_measure_parity": (I, [P, I, I, I, D, I, I, P, P]),
            "vqd_schedule": (I, [I, I, P, P, I, P, P, I, P, P]),
            "vqd_sc_compile": (I, [P, I, P, I, I, P, P]),
            "vqd_si_compile": (I, [P, I, P, I, P, P]),
            "vqd_nv_compile": (I, [P, I, P, I, I, P, P]),
            "vqd_ion_compile": (I, [P, I, P, I, I, P, P]),
            "vqd_na_compile": (I, [P, I, P, I, I, I, P, P]),
            "vqd_traj_expect": (I, [I, I, I, P, U, I, ctypes.c_uint64, I, P, P, P, P, P, P]),
            "vqd_run_program_tc": (I, [P, I, I, P, I, I, U]),
            "vqd_measure_fma_rate": (I, [I, P, P]),
            "vqd_tc_plan_info": (I, [I, I, P, I, U, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, ctx=None):
    if rc != VQD_OK:
        msg = lib().vqd_last_error(ctx)
        raise VQDError(rc, msg.decode() if msg else "")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(m) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(m, dtype=np.complex128))


def _i32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def native_ops(ops: Iterable) -> np.ndarray:
    """Marshal NativeOp(name, qubits, params) records into the C struct array."""
    ops = list(ops)
    arr = np.zeros(len(ops), dtype=NATIVE_OP_DTYPE)
    if not ops:
        return arr
    arr["code"] = [OP_CODE[o.name] for o in ops]
    arr["nq"] = [len(o.qubits) for o in ops]
    arr["q"] = [(o.qubits + (0,))[:2] if len(o.qubits) == 1 else o.qubits for o in ops]
    arr["par"] = [tuple(o.params) + (0.0,) * (4 - len(o.params)) for o in ops]
    return arr


# ---------------------------------------------------------------- entry points (same names as the C ABI)
def vqd_state_bytes(n: int, prec: int) -> int:
    return lib().vqd_state_bytes(n, prec)


def vqd_create(n: int, prec: int = VQD_F64, stream: int = 0):
    h = ctypes.c_void_p()
    _check(lib().vqd_create(n, prec, ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def vqd_create_batch(ns: Sequence[int], prec: int = VQD_F64, stream: int = 0):
    a = _i32(ns)
    h = ctypes.c_void_p()
    _check(lib().vqd_create_batch(len(a), _ptr(a), prec, ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def vqd_create_on(n: int, prec: int, dev_ptr: int, nbytes: int, stream: int = 0):
    h = ctypes.c_void_p()
    _check(lib().vqd_create_on(n, prec, ctypes.c_void_p(dev_ptr), nbytes, ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def vqd_destroy(ctx):
    lib().vqd_destroy(ctx)


def vqd_num_qubits(ctx, inst: int = 0) -> int:
    return lib().vqd_num_qubits(ctx, inst)


def vqd_state_ptr(ctx, inst: int = 0) -> int:
    return lib().vqd_state_ptr(ctx, inst)


def vqd_sync(ctx):
    _check(lib().vqd_sync(ctx), ctx)


def vqd_set_tile_shape(ctx, tile_bits: int = 0, passenger_bits: int = -1):
    _check(lib().vqd_set_tile_shape(ctx, tile_bits, passenger_bits), ctx)


def vqd_set_flags(ctx, flags: int):
    _check(lib().vqd_set_flags(ctx, flags), ctx)


def vqd_init_zero(ctx, inst: int = 0):
    _check(lib().vqd_init_zero(ctx, inst), ctx)


def vqd_init_classical(ctx, inst: int, basis: int):
    _check(lib().vqd_init_classical(ctx, inst, basis), ctx)


def vqd_init_product_diag(ctx, inst: int, excited: Sequence[float]):
    e = np.ascontiguousarray(np.asarray(excited, dtype=np.float64))
    _check(lib().vqd_init_product_diag(ctx, inst, _ptr(e)), ctx)


def vqd_apply_unitary(ctx, inst: int, targets: Sequence[int], U):
    t, m = _i32(targets), _c128(U)
    _check(lib().vqd_apply_unitary(ctx, inst, len(t), _ptr(t), _ptr(m)), ctx)


def vqd_apply_kraus(ctx, inst: int, targets: Sequence[int], kraus):
    t = _i32(targets)
    m = _c128(np.stack([np.asarray(K) for K in kraus]))
    _check(lib().vqd_apply_kraus(ctx, inst, len(t), _ptr(t), len(m), _ptr(m)), ctx)


def vqd_apply_superop(ctx, inst: int, targets: Sequence[int], S):
    t, m = _i32(targets), _c128(S)
    _check(lib().vqd_apply_superop(ctx, inst, len(t), _ptr(t), _ptr(m)), ctx)


def vqd_apply_native(ctx, inst: int, ops, flags: int = 0):
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    _check(lib().vqd_apply_native(ctx, inst, len(a), _ptr(a), flags), ctx)


def vqd_run_program(ctx, inst: int, ops, fuse_qubits: int = 0, flags: int = 0):
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    _check(lib().vqd_run_program(ctx, inst, len(a), _ptr(a), fuse_qubits, flags), ctx)


def vqd_run_program_tc(ctx, inst: int, ops, k: int = 4, scheme: int = VQD_TC_3XTF32, flags: int = 0):
    """Fused k-qubit blocks applied as split-precision GEMMs on the tensor cores (complex64 contexts)."""
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    _check(lib().vqd_run_program_tc(ctx, inst, len(a), _ptr(a), k, scheme, flags), ctx)


def vqd_measure_fma_rate(which: int, stream: int = 0) -> float:
    """FMA instructions per second of this GPU: which = 0 for FP64, 1 for FP32 (synchronous)."""
    out = ctypes.c_double()
    _check(lib().vqd_measure_fma_rate(which, ctypes.c_void_p(stream), ctypes.byref(out)))
    return out.value


def vqd_tc_plan_info(n: int, ops, k: int = 4, flags: int = 0) -> dict:
    """Blocks of the tensor-core form for a program (host only, no GPU needed)."""
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    info = np.zeros(3, dtype=np.int64)
    _check(lib().vqd_tc_plan_info(n, len(a), _ptr(a), k, flags, _ptr(info)))
    return {"blocks": int(info[0]), "native_ops": int(info[1]), "max_block_ops": int(info[2])}


def vqd_run_batch(ctx, programs_ops: Sequence, fuse_qubits: int = 0, flags: int = 0):
    arrays = [p if isinstance(p, np.ndarray) else native_ops(p) for p in programs_ops]
    offsets = np.zeros(len(arrays) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([len(a) for a in arrays])
    allops = np.concatenate(arrays) if arrays else np.zeros(0, dtype=NATIVE_OP_DTYPE)
    allops = np.ascontiguousarray(allops)
    _check(lib().vqd_run_batch(ctx, _ptr(offsets), _ptr(allops), fuse_qubits, flags), ctx)


def vqd_compile_op(op, flags: int = 0):
    """Returns ("U", qubits, U) or ("S", qubits, S) from the library's device compiler (host only)."""
    a = native_ops([op])
    isu, k = ctypes.c_int(), ctypes.c_int()
    t = np.zeros(2, dtype=np.int32)
    m = np.zeros(256, dtype=np.complex128)
    _check(lib().vqd_compile_op(_ptr(a), flags, ctypes.byref(isu), ctypes.byref(k), _ptr(t), _ptr(m)))
    kk = k.value
    if isu.value:
        return "U", tuple(t[:kk]), m[: 4 ** kk].reshape(2 ** kk, 2 ** kk)
    return "S", tuple(t[:kk]), m[: 16 ** kk].reshape(4 ** kk, 4 ** kk)


def vqd_plan_info(n: int, prec: int, ops, fuse_qubits: int = 0, flags: int = 0, tile_bits: int = 0,
                  passenger_bits: int = -1) -> dict:
    """Fused-path plan statistics for a program (host only, no GPU needed)."""
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    info = np.zeros(8, dtype=np.int64)
    _check(lib().vqd_plan_info(n, prec, len(a), _ptr(a), fuse_qubits, tile_bits, passenger_bits, flags, _ptr(info)))
    keys = ["stages", "blocks", "diag", "sup1", "uni2", "sup2", "max_tile_bits", "native_ops"]
    return dict(zip(keys, (int(x) for x in info)))


def vqd_schedule(n: int, ops, durations, t1, t2, idle: str = "idle") -> np.ndarray:
    """Schedule gates (duration >= 0) and their trailing noise ops (duration < 0) into parallel layers with
    passive idle noise (host only).  Returns the scheduled native-op array."""
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    d = np.ascontiguousarray(np.asarray(durations, dtype=np.float64))
    t1a = np.ascontiguousarray(np.asarray(t1, dtype=np.float64))
    t2a = np.ascontiguousarray(np.asarray(t2, dtype=np.float64))
    cap = len(a) + n * max(1, len(a))
    out = np.zeros(cap, dtype=NATIVE_OP_DTYPE)
    cnt = ctypes.c_int()
    _check(lib().vqd_schedule(n, len(a), _ptr(a), _ptr(d), OP_CODE[idle], _ptr(t1a), _ptr(t2a), cap, _ptr(out),
                              ctypes.byref(cnt)))
    return out[: cnt.value].copy()


def vqd_sc_compile(dev: dict, ops, readout: bool = False) -> np.ndarray:
    """Compile a logical Rx/Ry/Rz/ZX/ZZ circuit for a superconducting device (host only).  ``dev`` holds
    n, t1, t2, excited, freq, anharm, couple (pairs), coupling, fid_read (or None), dur_rxy, dur_zx,
    dur_zz, dur_meas and optional flags.  Returns the native-op array."""
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    f64 = lambda key: np.ascontiguousarray(np.asarray(dev[key], dtype=np.float64))
    keep = {k: f64(k) for k in ("t1", "t2", "excited", "freq", "anharm", "coupling")}
    keep["couple"] = np.ascontiguousarray(np.asarray(dev["couple"], dtype=np.int32).reshape(-1))
    fr = dev.get("fid_read")
    keep["fid_read"] = None if fr is None else f64("fid_read")
    d = sc_device(int(dev["n"]), len(keep["coupling"]),
                  *[_ptr(keep[k]) if keep[k] is not None else None
                    for k in ("t1", "t2", "excited", "freq", "anharm", "couple", "coupling", "fid_read")],
                  float(dev["dur_rxy"]), float(dev["dur_zx"]), float(dev["dur_zz"]), float(dev["dur_meas"]),
                  int(dev.get("flags", 0)))
    cnt = ctypes.c_int()
    _check(lib().vqd_sc_compile(ctypes.byref(d), len(a), _ptr(a), int(bool(readout)), 0, None, ctypes.byref(cnt)))
    out = np.zeros(max(1, cnt.value), dtype=NATIVE_OP_DTYPE)
    _check(lib().vqd_sc_compile(ctypes.byref(d), len(a), _ptr(a), int(bool(readout)), cnt.value, _ptr(out),
                                ctypes.byref(cnt)))
    return out[: cnt.value].copy()


def vqd_si_compile(dev: dict, ops) -> np.ndarray:
    """Compile a logical Rx/Ry/Rz/CZ/CPh circuit for a silicon device (host only).  ``dev`` holds n, t1, t2,
    freq, rabi, fid_1q, x_1q, freq_cz, fid_cz, x_cz, xtalk_on ((n-1) x (n-1) or None), xtalk_off (or None)
    and optional flags.  Returns the native-op array."""
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    keep = {}
    for k in ("t1", "t2", "freq", "rabi", "fid_1q", "freq_cz", "fid_cz", "xtalk_on", "xtalk_off"):
        v = dev.get(k)
        keep[k] = None if v is None else np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1))
    p = lambda k: None if keep[k] is None else _ptr(keep[k])
    d = si_device(int(dev["n"]), p("t1"), p("t2"), p("freq"), p("rabi"), p("fid_1q"), float(dev["x_1q"]),
                  p("freq_cz"), p("fid_cz"), float(dev["x_cz"]), p("xtalk_on"), p("xtalk_off"),
                  int(dev.get("flags", 0)))
    cnt = ctypes.c_int()
    _check(lib().vqd_si_compile(ctypes.byref(d), len(a), _ptr(a), 0, None, ctypes.byref(cnt)))
    out = np.zeros(max(1, cnt.value), dtype=NATIVE_OP_DTYPE)
    _check(lib().vqd_si_compile(ctypes.byref(d), len(a), _ptr(a), cnt.value, _ptr(out), ctypes.byref(cnt)))
    return out[: cnt.value].copy()


def vqd_nv_compile(dev: dict, ops, readout: bool = False) -> np.ndarray:
    """Compile a logical Rx/Ry/Rz/CRx+-(zx)/CRy+-(zy) circuit for an NV-centre device (host only).  ``dev``
    holds n, t1, t2, freq_xy, freq_z, fid_xy, fid_z, x_xy, freq_crot, fid_crot, x_crot, freq_zz, fid_meas,
    dur_meas and optional flags.  Returns the native-op array."""
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    keep = {k: np.ascontiguousarray(np.asarray(dev[k], dtype=np.float64))
            for k in ("t1", "t2", "freq_xy", "freq_z", "fid_xy", "fid_z", "freq_crot", "fid_crot")}
    p = lambda k: _ptr(keep[k])
    d = nv_device(int(dev["n"]), p("t1"), p("t2"), p("freq_xy"), p("freq_z"), p("fid_xy"), p("fid_z"),
                  float(dev["x_xy"]), p("freq_crot"), p("fid_crot"), float(dev["x_crot"]), float(dev["freq_zz"]),
                  float(dev["fid_meas"]), float(dev["dur_meas"]), int(dev.get("flags", 0)))
    cnt = ctypes.c_int()
    _check(lib().vqd_nv_compile(ctypes.byref(d), len(a), _ptr(a), int(bool(readout)), 0, None, ctypes.byref(cnt)))
    out = np.zeros(max(1, cnt.value), dtype=NATIVE_OP_DTYPE)
    _check(lib().vqd_nv_compile(ctypes.byref(d), len(a), _ptr(a), int(bool(readout)), cnt.value, _ptr(out),
                                ctypes.byref(cnt)))
    return out[: cnt.value].copy()


def vqd_ion_compile(dev: dict, ops, readout: bool = False) -> np.ndarray:
    """Compile a logical Rx/Ry/Rz/CZ circuit for a trapped-ion device (host only).  ``dev`` holds n, t1, t2s,
    rabi, fid_xy, x_xy, freq_cz, fid_cz, x_cz, bf_read, dur_read and optional flags."""
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    d = ion_device(int(dev["n"]), *[float(dev[k]) for k in ("t1", "t2s", "rabi", "fid_xy", "x_xy", "freq_cz", "fid_cz",
                                                            "x_cz", "bf_read", "dur_read")], int(dev.get("flags", 0)))
    cnt = ctypes.c_int()
    _check(lib().vqd_ion_compile(ctypes.byref(d), len(a), _ptr(a), int(bool(readout)), 0, None, ctypes.byref(cnt)))
    out = np.zeros(max(1, cnt.value), dtype=NATIVE_OP_DTYPE)
    _check(lib().vqd_ion_compile(ctypes.byref(d), len(a), _ptr(a), int(bool(readout)), cnt.value, _ptr(out),
                                 ctypes.byref(cnt)))
    return out[: cnt.value].copy()


def vqd_na_compile(dev: dict, ops, init: bool = False, readout: bool = False) -> np.ndarray:
    """Compile a logical U / CZ(phi) circuit for a neutral-atom device (host only).  ``dev`` holds n, sites
    (list of (x, y)), blockade, t2, t_vac, p10, p01, leak_init, leak_cz (alpha, beta), dur_cz, fid_meas and
    optional flags."""
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    xs = np.ascontiguousarray(np.asarray([s[0] for s in dev["sites"]], dtype=np.float64))
    ys = np.ascontiguousarray(np.asarray([s[1] for s in dev["sites"]], dtype=np.float64))
    d = na_device(int(dev["n"]), _ptr(xs), _ptr(ys), float(dev["blockade"]), float(dev["t2"]), float(dev["t_vac"]),
                  float(dev["p10"]), float(dev["p01"]), float(dev["leak_init"]), float(dev["leak_cz"][0]),
                  float(dev["leak_cz"][1]), float(dev["dur_cz"]), float(dev["fid_meas"]), int(dev.get("flags", 0)))
    cnt = ctypes.c_int()
    args = (int(bool(init)), int(bool(readout)))
    _check(lib().vqd_na_compile(ctypes.byref(d), len(a), _ptr(a), *args, 0, None, ctypes.byref(cnt)))
    out = np.zeros(max(1, cnt.value), dtype=NATIVE_OP_DTYPE)
    _check(lib().vqd_na_compile(ctypes.byref(d), len(a), _ptr(a), *args, cnt.value, _ptr(out), ctypes.byref(cnt)))
    return out[: cnt.value].copy()


def vqd_stderr_params(nq: int, fbar: float, x: float):
    p, q = ctypes.c_double(), ctypes.c_double()
    _check(lib().vqd_stderr_params(nq, fbar, x, ctypes.byref(p), ctypes.byref(q)))
    return p.value, q.value


def vqd_prob(ctx, inst: int, qubits: Sequence[int]) -> np.ndarray:
    q = _i32(qubits)
    out = np.zeros(2 ** len(q), dtype=np.float64)
    _check(lib().vqd_prob(ctx, inst, len(q), _ptr(q), _ptr(out)), ctx)
    return out


def vqd_expect(ctx, inst: int, paulis, coeffs) -> float:
    p = np.ascontiguousarray(np.asarray(paulis, dtype=np.uint8))
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    out = ctypes.c_double()
    _check(lib().vqd_expect(ctx, inst, len(c), _ptr(p), _ptr(c), ctypes.byref(out)), ctx)
    return out.value


def vqd_traj_expect(n: int, prec: int, ops, ntraj: int, seed: int, paulis, coeffs, flags: int = 0, stream: int = 0):
    """Monte-Carlo trajectory estimate of Re sum_t c_t tr(P_t rho): (per-trajectory values, mean, standard error)."""
    a = ops if isinstance(ops, np.ndarray) else native_ops(ops)
    p = np.ascontiguousarray(np.asarray(paulis, dtype=np.uint8))
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    out = np.zeros(ntraj, dtype=np.float64)
    m, se = ctypes.c_double(), ctypes.c_double()
    _check(lib().vqd_traj_expect(n, prec, len(a), _ptr(a), flags, ntraj, seed, len(c), _ptr(p), _ptr(c),
                                 ctypes.c_void_p(stream), _ptr(out), ctypes.byref(m), ctypes.byref(se)))
    return out, m.value, se.value


def vqd_batch_reduce(ctx, ns):
    """Every instance's Z-basis probabilities (list of arrays), traces and purities in one batched reduction."""
    total = int(sum(2 ** n for n in ns))
    probs = np.zeros(total, dtype=np.float64)
    tr = np.zeros(len(ns), dtype=np.float64)
    pu = np.zeros(len(ns), dtype=np.float64)
    _check(lib().vqd_batch_reduce(ctx, _ptr(probs), _ptr(tr), _ptr(pu)), ctx)
    out, o = [], 0
    for n in ns:
        out.append(probs[o:o + 2 ** n])
        o += 2 ** n
    return out, tr, pu


def vqd_measure_parity(ctx, inst: int, qa: int, qb: int, u: float = 0.0, force: int = -1, decay: bool = True):
    """Parity measurement of (qa, qb) with collapse (Sec. 7): outcome 0 = odd, 1 = even; returns (outcome, prob)."""
    m, p = ctypes.c_int(), ctypes.c_double()
    _check(lib().vqd_measure_parity(ctx, inst, qa, qb, float(u), int(force), int(bool(decay)), ctypes.byref(m),
                                    ctypes.byref(p)), ctx)
    return m.value, p.value


def vqd_measure(ctx, inst: int, q: int, u: float = 0.0, force: int = -1):
    """Projective Z measurement of qubit q with collapse: (outcome, probability)."""
    m, pr = ctypes.c_int(), ctypes.c_double()
    _check(lib().vqd_measure(ctx, inst, q, u, force, ctypes.byref(m), ctypes.byref(pr)), ctx)
    return m.value, pr.value


def vqd_trace(ctx, inst: int = 0) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(lib().vqd_trace(ctx, inst, ctypes.byref(re), ctypes.byref(im)), ctx)
    return complex(re.value, im.value)


def vqd_purity(ctx, inst: int = 0) -> float:
    out = ctypes.c_double()
    _check(lib().vqd_purity(ctx, inst, ctypes.byref(out)), ctx)
    return out.value


def vqd_get_state(ctx, inst: int = 0) -> np.ndarray:
    """Flat 4^n complex128 vector v[r + (c << n)] = rho[r][c]."""
    n = vqd_num_qubits(ctx, inst)
    out = np.zeros(4 ** n, dtype=np.complex128)
    _check(lib().vqd_get_state(ctx, inst, _ptr(out)), ctx)
    return out


def vqd_set_state(ctx, inst: int, flat) -> None:
    a = _c128(flat).reshape(-1)
    _check(lib().vqd_set_state(ctx, inst, _ptr(a)), ctx)


VQD_PROB_STATIC_MAX_M = 14


def vqd_prob_static(dev_state: int, n: int, prec: int, qubits: Sequence[int], dev_out: int, stream: int = 0):
    """Allocation-free marginal probabilities into a caller-owned DEVICE array of 2^m doubles (asynchronous)."""
    q = _i32(qubits)
    _check(lib().vqd_prob_static(ctypes.c_void_p(dev_state), n, prec, len(q), _ptr(q), ctypes.c_void_p(dev_out),
                                 ctypes.c_void_p(stream)))


def vqd_profile(ctx, mode: int):
    _check(lib().vqd_profile(ctx, mode), ctx)


def vqd_profile_reset(ctx):
    _check(lib().vqd_profile_reset(ctx), ctx)


def vqd_profile_read(ctx) -> dict:
    arr = (kstat * 16)()
    n = ctypes.c_int()
    _check(lib().vqd_profile_read(ctx, 16, ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(n)), ctx)
    return {arr[i].name.decode(): {"launches": arr[i].launches, "total_ms": arr[i].total_ms,
                                   "alg_bytes": arr[i].alg_bytes, "amp_updates": arr[i].amp_updates,
                                   "alg_fma": arr[i].alg_fma}
            for i in range(min(n.value, 16))}


def rho_from_flat(flat: np.ndarray) -> np.ndarray:
    """Matrix rho[r, c] from the library's flat layout (a view conversion, no arithmetic)."""
    dim = int(round(np.sqrt(flat.size)))
    return np.ascontiguousarray(flat.reshape(dim, dim).T)
