/*
 * vqd.h - C ABI of libvqd: density-matrix emulation of a noisy quantum device on one GPU.
 *
 * The library evolves an n-qubit density matrix rho through a device's native gates
 * (rho <- U rho U^dagger) and noise processes (rho <- sum_k K_k rho K_k^dagger), as the
 * paper's Sec. 2 describes the emulation of a device specification: an ideal circuit is
 * turned into a sequence of unitary and decohering operators which are applied to the
 * density matrix.  It ends with Z-basis probabilities, Pauli expectation values, trace
 * and purity (the quantities reported in Sec. 4-8).
 *
 * Conventions (fixed here; the paper leaves them open)
 *   - Qubit q is bit q of a basis index (little-endian).
 *   - Matrices are row-major FP64 complex (vqd_c128).  For an operation on
 *     targets[0..k-1], the 2^k x 2^k matrix index is little-endian over targets:
 *     targets[0] is its least significant bit.
 *   - Superoperators are 4^k x 4^k, index s = r | (c << k) where r / c are the row /
 *     column indices of the k-qubit block; S = sum_k conj(K_k) (x) K_k (conj factor on
 *     the high, column part).
 *   - The state of an n-qubit instance is 4^n amplitudes, amplitude rho[r][c] at index
 *     r + (c << n) (column-major vectorisation).  vqd_get_state / vqd_set_state use this
 *     layout.
 *   - Rotations R_s(theta) = exp(-i theta s / 2); SX = Rx(pi/2).
 *
 * Precision: VQD_F64 stores complex128 and computes in FP64.  VQD_F32 stores complex64 and
 * computes in FP32.  VQD_F32_SPLIT stores every real and imaginary part as a float-float pair
 * hi + lo (|lo| <= ulp(hi)/2, about 48 significant bits; 16 bytes per amplitude, laid out as
 * re.hi, re.lo, im.hi, im.lo) and computes in float-float arithmetic on the FP32 pipes; its
 * operator coefficients are float-float roundings of the FP64 ones.  Operators are always composed
 * on the host in FP64; every reduction (probabilities, expectation values, trace, purity)
 * accumulates in FP64.  vqd_get_state / vqd_set_state convert to and from complex128 (hi + lo in
 * FP64; a double is split into its nearest float and the float of the remainder).
 *
 * Errors: every int-returning call returns 0 (VQD_OK) or a negative VQD_E* code and never
 * throws.  vqd_last_error(ctx) gives a human-readable message (ctx may be NULL for errors
 * raised before a context exists).  After VQD_EDEVICE the context should be destroyed.
 *
 * Ownership and streams: the caller owns every host array; each call copies what it needs
 * before returning.  Apply / init / run calls are asynchronous on the context's CUDA stream;
 * reductions and get_state synchronise that stream.  A context is not thread-safe.
 */
#ifndef VQD_H
#define VQD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VQD_OK 0
#define VQD_EINVAL (-1)  /* bad argument: k, target out of range or repeated, n too large, bad op code */
#define VQD_ENOMEM (-2)  /* device or host allocation failed */
#define VQD_ENOTCP (-3)  /* matrix is not unitary / Kraus set not trace non-increasing (tol 1e-10) */
#define VQD_EDEVICE (-4) /* CUDA error (message in vqd_last_error) */
#define VQD_ENOTSUP (-5) /* operation not supported in this configuration */

typedef enum { VQD_F64 = 0, VQD_F32 = 1, VQD_F32_SPLIT = 2 } vqd_prec;

typedef struct {
  double re, im;
} vqd_c128;

typedef struct vqd_ctx* vqd_t;

/* Largest qubit count of one instance (4^16 amplitudes: 68.7 GB complex128, 34.4 GB complex64). */
#define VQD_MAX_QUBITS 16

/* ------------------------------------------------------------------------------------------
 * Native operations: the device vocabulary compiled by the library's device compiler.
 * Parameters: angles in radians, durations in microseconds, frequencies in MHz.
 * The numeric codes are part of the ABI.
 * ---------------------------------------------------------------------------------------- */
typedef enum {
  /* native gates (unitaries) */
  VQD_OP_RX = 0,        /* q0; theta                                                          */
  VQD_OP_RY = 1,        /* q0; theta                                                          */
  VQD_OP_RZ = 2,        /* q0; theta (virtual Z of Sec. 8 is still a unitary here)            */
  VQD_OP_SX = 3,        /* q0; sqrt(X) := Rx(pi/2)                                            */
  VQD_OP_H = 4,         /* q0; Hadamard                                                       */
  VQD_OP_U = 5,         /* q0; phi, Omega, Delta, t: Raman U(phi, Delta, t), Sec. 6 Eq. (u)    */
  VQD_OP_R = 6,         /* q0; theta, phi: Eq. (u) with Delta = 0, Omega t = theta            */
  VQD_OP_CZ = 7,        /* q0,q1                                                              */
  VQD_OP_CPH = 8,       /* q0,q1; phi: diag(1,1,1,e^{i phi}), Sec. 7                          */
  VQD_OP_CZPHI = 9,     /* q0,q1; phi: Rydberg CZ(phi) = diag(1,e^{i phi},e^{i phi},e^{i(2phi-pi)}), Sec. 6 */
  VQD_OP_ZX = 10,       /* q0 = control, q1 = target; theta: exp(-i theta/2 Z X), Sec. 8      */
  VQD_OP_ZZ = 11,       /* q0,q1; theta: exp(-i theta/2 Z Z), Sec. 8                          */
  VQD_OP_XX = 12,       /* q0,q1; theta: Molmer-Sorensen exp(-i theta/2 X X), Sec. 4           */
  VQD_OP_ZZPHASE = 13,  /* q0,q1; alpha: exp(-i alpha Z Z), Sec. 3.4 Eq. (weak_dephasing_zz)   */
  VQD_OP_ZZ_IDLE = 14,  /* q0,q1; dt, xi: static ZZ crosstalk, alpha = pi xi dt / 2            */
  VQD_OP_CRZ_XTALK = 15,/* q0 = control, q1; alpha: conditional Rz, Eq. (weak_dephasing)       */
  VQD_OP_EXCHANGE = 16, /* q0,q1; theta: exp(-i (XX+YY+ZZ) theta/4), Eq. (exchange_pauli)      */
  /* noise processes (Kraus channels) */
  VQD_OP_DEPOL1 = 17,   /* q0; p in [0,3/4], Eq. (depol1)                                     */
  VQD_OP_DEPOL2 = 18,   /* q0,q1; p in [0,15/16], Eq. (depol2): p/15 on each of 15 Paulis      */
  VQD_OP_DEPH1 = 19,    /* q0; p in [0,1/2], Eq. (deph1)                                      */
  VQD_OP_DEPH2 = 20,    /* q0,q1; p in [0,3/4], Eq. (deph2)                                   */
  VQD_OP_AMP = 21,      /* q0; p in [0,1], Eq. (damp)                                         */
  VQD_OP_BITFLIP = 22,  /* q0; b in [0,1/2], Eq. (bf)                                         */
  VQD_OP_BITFLIP2 = 23, /* q0,q1; b in [0,3/4], Eq. (bf2)                                     */
  VQD_OP_GAMP = 24,     /* q0; dt, T1, p0: generalised damping, Eq. (gdamp)                   */
  VQD_OP_IDLE = 25,     /* q0; dt, T1, T2: amp(1-e^{-dt/T1}) then deph(1/2(1-e^{-dt/T2})), Eqs. (ampt1),(depht2) */
  VQD_OP_IDLE_DEPOL = 26,/* q0; dt, T1, T2: depol(3/4(1-e^{-dt/T1})) then the T2 dephasing, Eq. (depolt1) */
  VQD_OP_STDERR1 = 27,  /* q0; Fbar, x: deph(p) o depol(q) from the average fidelity, App. B   */
  VQD_OP_STDERR2 = 28,  /* q0,q1; Fbar, x: two-qubit standard error, App. B                   */
  VQD_OP_AMPDEPH2 = 29, /* q0,q1; dt, T1, T2: the T1/T2 decay of both qubits as one 2-qubit channel */
  VQD_OP_LEAK_INIT = 30,/* q0; gamma: CPTN L = diag(sqrt(1-gamma), 1), Sec. 6                 */
  VQD_OP_LEAK_CZ = 31,  /* q0,q1; alpha, beta: CPTN K of Eq. (czleak)                          */
  /* device-family crosstalk unitaries */
  VQD_OP_OFFRES = 32,   /* q0; Omega, Delta, t: off-resonant Rabi drive on a passive qubit, Sec. 3.3
                           Eq. (off_resonant) as printed: exp(i Omega_R t Z/2) exp(-i t (Omega X + Delta Z)/2),
                           Omega_R = sqrt(Omega^2 + Delta^2); near the identity for Delta >> Omega;
                           the identity when Omega = Delta = 0                                          */
  VQD_OP_ZZ_STATIC = 33,/* q0 = control, q1 = target; J dt, Delta_ct dt, alpha_t dt, alpha_c dt:
                           exp(-i beta Z Z), beta = J^2 (1/(Delta-alpha_t) - 1/(Delta+alpha_c)), Sec. 8;
                           the parameters are frequencies times the idle duration, so beta is the
                           accumulated phase; a zero denominator is VQD_EINVAL                       */
  VQD_OP_ZY = 34,       /* q0 = control, q1 = target; theta: NV conditional rotation CRy+-(theta) =
                           |0><0| (x) Ry(theta) + |1><1| (x) Ry(-theta) = exp(-i theta/2 Z Y), Sec. 5
                           Eq. (conditional_rots); CRx+- is VQD_OP_ZX                                   */
  VQD_OP_IDLE_T2S = 35, /* q0; dt, T1, T2*: depol(3/4(1-e^{-dt/T1})) then deph(1/2(1-e^{-(dt/T2*)^2})), Eqs. (depolt1),
                           (depht2s): passive decay with a Gaussian T2* (VQD_T2_IS_TOTAL does not apply)      */
  VQD_OP_BITFLIP_ASYM = 36,/* q0; p10, p01 in [0,1]: |1> -> |0> with p10, |0> -> |1> with p01 (the asymmetric
                           bit flip of Sec. 6): Kraus diag(sqrt(1-p01), sqrt(1-p10)), sqrt(p10)|0><1|,
                           sqrt(p01)|1><0|                                                             */
  VQD_OP_COUNT = 37
} vqd_op_code;

typedef struct {
  int32_t code;   /* vqd_op_code */
  int32_t nq;     /* number of qubits (must match the code) */
  int32_t q[2];   /* target qubits, q[0] = least significant bit of the matrix index */
  double par[4];  /* parameters in the order listed above; unused entries ignored */
} vqd_native_op;  /* 48 bytes */

/* Flags for compilation and run calls (bitwise or). */
#define VQD_T2_IS_TOTAL 1u  /* read T2 as the total coherence time: dephase with T_phi, 1/T2 = 1/(2T1) + 1/T_phi */
#define VQD_NO_CHECK 2u     /* skip the unitarity / CPTN checks of apply_unitary / apply_kraus */
/* vqd_run_program / vqd_run_batch / vqd_plan_info: the caller asserts that the state is Hermitian, as every
 * density matrix is (Sec. 2).  The fused path then updates only the tiles on or above the diagonal of
 * its tile grid and writes each one's conjugate transpose into the mirror tile, halving the arithmetic of a
 * stage; the state it leaves is exactly Hermitian (lower triangle = conjugate of the upper one, real
 * diagonal).  Ignored for programs with an operator that does not preserve Hermiticity (every native op
 * does).  Do not set it for other operators, such as |i><j| when propagating a process basis. */
#define VQD_HERMITIAN 4u

/* ------------------------------------------------------------------------------------------
 * Contexts and states
 * ---------------------------------------------------------------------------------------- */

/* Bytes of device memory one n-qubit state occupies in precision prec. */
size_t vqd_state_bytes(int n, int prec);

/* One n-qubit state (1 <= n <= VQD_MAX_QUBITS) in library-allocated device memory, initialised
 * to |0..0><0..0|: the density matrix on which Sec. 2 simulates the device's noisy channel (the
 * representation that captures noise completely, at quadratic cost over the statevector).  stream is a cudaStream_t (NULL = legacy default stream).  The library owns
 * the memory; vqd_destroy frees it. */
int vqd_create(int n, int prec, void* stream, vqd_t* out);

/* count independent instances (n[i] qubits each, 1..VQD_MAX_QUBITS) packed in one allocation;
 * every call that takes `inst` addresses one of them.  All start in |0..0><0..0|. */
int vqd_create_batch(int count, const int* n, int prec, void* stream, vqd_t* out);

/* One n-qubit state living in caller-owned device memory `dev_state` (>= vqd_state_bytes(n,prec)
 * bytes, 16-byte aligned), e.g. a torch tensor.  The state is NOT initialised; the caller keeps
 * the memory alive until vqd_destroy. */
int vqd_create_on(int n, int prec, void* dev_state, size_t bytes, void* stream, vqd_t* out);

void vqd_destroy(vqd_t ctx);
int vqd_num_instances(vqd_t ctx);
int vqd_num_qubits(vqd_t ctx, int inst);
/* Device address of instance inst's amplitudes (layout above). */
void* vqd_state_ptr(vqd_t ctx, int inst);
int vqd_sync(vqd_t ctx);
const char* vqd_last_error(vqd_t ctx);

/* Initial states (asynchronous). */
int vqd_init_zero(vqd_t ctx, int inst);                       /* |0..0><0..0|                    */
int vqd_init_classical(vqd_t ctx, int inst, uint64_t basis);  /* |x><x|, x < 2^n                 */
/* Thermal product state of Sec. 8 Eq. (thermalstate): (x)_j ((1-e_j)|0><0| + e_j|1><1|) where
 * e_j = excited[j] in [0,1] is qubit j's excited population. */
int vqd_init_product_diag(vqd_t ctx, int inst, const double* excited);

/* ------------------------------------------------------------------------------------------
 * Applying operators (asynchronous; one pass over the state per call)
 * ---------------------------------------------------------------------------------------- */

/* rho <- U rho U^dagger, U is 2^k x 2^k (k = 1 or 2) on distinct targets: one unitary operator of the
 * channel a device specification makes from a circuit (Sec. 2); the native gates of Sec. 4-8 are
 * such unitaries.  ENOTCP if U is not
 * unitary within 1e-10 (unless VQD_NO_CHECK is set with vqd_set_flags). */
int vqd_apply_unitary(vqd_t ctx, int inst, int k, const int* targets, const vqd_c128* U);

/* rho <- sum_j K_j rho K_j^dagger, nK operators of 2^k x 2^k stored one after another
 * (general Kraus map, Sec. 2).  ENOTCP if sum_j K_j^dagger K_j exceeds I by more than 1e-10
 * (CPTN maps such as the leakage operators of Sec. 6 are accepted). */
int vqd_apply_kraus(vqd_t ctx, int inst, int k, const int* targets, int nK, const vqd_c128* K);

/* vec-group <- S vec-group with the 4^k x 4^k superoperator S (index convention above);
 * no positivity check.  S is the matrix form of a general Kraus map of Sec. 2 acting on the density
 * matrix, S = sum_j conj(K_j) (x) K_j, so any channel of Sec. 3 can be passed in this form. */
int vqd_apply_superop(vqd_t ctx, int inst, int k, const int* targets, const vqd_c128* S);

/* Compile each native op with the device compiler and apply it with one pass over the state
 * (the plain, unfused path).  flags: VQD_T2_IS_TOTAL. */
int vqd_apply_native(vqd_t ctx, int inst, int nops, const vqd_native_op* ops, unsigned flags);

/* Same result as vqd_apply_native, through the fused path: consecutive ops are grouped into
 * stages acting on at most `fuse_qubits` qubits (2..VQD_MAX_FUSE); each stage is one pass over
 * the state in which the stage's tiles are staged in shared memory and all of its ops are
 * applied there.  fuse_qubits <= 0 picks the library default. */
#define VQD_MAX_FUSE 6
int vqd_run_program(vqd_t ctx, int inst, int nops, const vqd_native_op* ops, int fuse_qubits, unsigned flags);

/* Batched path: instance i of a batch context runs ops[offsets[i] .. offsets[i+1]) (native ops)
 * through the fused path.  Every instance's program is planned into stages; stage w of every instance
 * forms wave w, one persistent-kernel launch whose CTAs take (instance, stage, chunk of tiles) items
 * from an atomic queue, largest instances first, so that no CTA waits for another.  The waves of a
 * batch are captured into a CUDA graph on the context's stream (when it can capture) and the graph is
 * replayed when the same batch runs again.  offsets has count+1 entries.  The paper runs one device
 * at a time; batching many instances (parameter sweeps such as the noise-severity scans of Sec. 5) is
 * this library's addition. */
int vqd_run_batch(vqd_t ctx, const int64_t* offsets, const vqd_native_op* ops, int fuse_qubits, unsigned flags);

/* Tensor-core form of the fused path (Sec. 2's general Kraus map in its superoperator form, applied as a
 * dense matrix product).  The program's native ops are grouped, in program order with a commuting
 * lookahead (operators that share a qubit keep their order), into blocks on at most k qubits (k = 4, 5 or
 * 6; a block with fewer qubits is padded with identity qubits).  Each block is composed on the GPU in
 * FP64 into one 4^k x 4^k superoperator S, which is split into limbs and applied to every group of 4^k
 * amplitudes as a real GEMM on the tensor cores (tcgen05.mma with TMEM accumulators, TMA tile loads),
 * accumulating in FP32:
 *   VQD_TC_3XTF32: operands split as hi + lo TF32 parts, products lo*hi + hi*lo + hi*hi;
 *   VQD_TC_BF16X3: operands split into three BF16 parts, the six products of combined order <= 4.
 * Complex64 contexts only (VQD_ENOTSUP otherwise); needs n >= k.  The state is written out of place to a
 * second buffer of the context's state size (allocated on first use) and copied back at the end when an
 * odd number of blocks ran, so vqd_state_ptr stays valid.  The call synchronises the stream at the end
 * and returns VQD_EDEVICE if a kernel wait expired.  Results agree with vqd_run_program up to the FP32
 * rounding of the split products. */
#define VQD_TC_3XTF32 0
#define VQD_TC_BF16X3 1
int vqd_run_program_tc(vqd_t ctx, int inst, int nops, const vqd_native_op* ops, int k, int scheme, unsigned flags);

/* Blocks of the tensor-core form for an n-qubit program, without running it (host only):
 * info[0] = blocks (one GEMM pass over the state each), info[1] = original operators,
 * info[2] = the largest number of operators in one block. */
int vqd_tc_plan_info(int n, int nops, const vqd_native_op* ops, int k, unsigned flags, int64_t* info);

/* ------------------------------------------------------------------------------------------
 * Device compiler (host only, no GPU needed)
 * ---------------------------------------------------------------------------------------- */

/* Compile one native op.  On return *is_unitary says which form `mat` holds: the 2^k x 2^k
 * unitary (is_unitary = 1, 4^k entries used) or the 4^k x 4^k superoperator of the channel
 * (is_unitary = 0, 16^k entries used).  `mat` must hold 256 entries.  targets receives the k
 * qubits. */
int vqd_compile_op(const vqd_native_op* op, unsigned flags, int* is_unitary, int* k, int* targets,
                   vqd_c128* mat);

/* Tile shape of the fused and batched paths of a context: tile_bits index bits per shared-memory tile
 * (<= 13 for VQD_F32, <= 12 for VQD_F64 and VQD_F32_SPLIT: a 64 KB tile; 0 = that maximum) of which
 * passenger_bits (0..3; -1 = default 3 for VQD_F32, 2 otherwise; 2 and 1 for a VQD_HERMITIAN run) are the lowest
 * row bits, carried along so that every tile is made of contiguous DRAM runs (a VQD_HERMITIAN run carries their
 * column bits too and rounds tile_bits down to even).  Needs 4 + passenger_bits <= tile_bits.  Results do
 * not depend on the shape; speed does (the autotuner in the Python package picks it). */
int vqd_set_tile_shape(vqd_t ctx, int tile_bits, int passenger_bits);

/* Plan of the fused path for an n-qubit program, without running it (host only); tile_bits and
 * passenger_bits as in vqd_set_tile_shape, flags as in vqd_run_program (VQD_HERMITIAN plans the Hermitian
 * stages).  info[0..7] =
 * {stages (one pass over the state each), blocks (one shared-memory sweep each), operators after
 * composition that are diagonal / 1-qubit superoperators / 2-qubit unitaries / 2-qubit
 * superoperators, largest tile (index bits), original operators}. */
int vqd_plan_info(int n, int prec, int nops, const vqd_native_op* ops, int fuse_qubits, int tile_bits,
                  int passenger_bits, unsigned flags, int64_t* info);

/* Automatic scheduling (Sec. 2: idle qubits experience passive noise while waiting for the slowest
 * operation of their automatically scheduled parallel batch).  Input: `nin` native ops in program
 * order, where ops with dur[i] >= 0 are gates of that duration (us) and ops with dur[i] < 0 are the
 * noise that follows the previous gate on the same qubits (kept right after it).  Each gate goes to the
 * earliest layer after every earlier gate that shares a qubit; a layer lasts as long as its slowest
 * gate.  Output, layer by layer: the layer's gates, each followed by its noise ops, then for every
 * qubit j a passive-noise op of code idle_code (VQD_OP_IDLE, VQD_OP_IDLE_DEPOL or VQD_OP_IDLE_T2S, whose third
 * parameter is then T2*) with parameters
 * (dt, t1[j], t2[j]), dt = layer duration minus the time qubit j was busy in the layer (skipped when
 * dt = 0).  out has room for cap ops; *nout receives the count (VQD_EINVAL if cap is too small). */
int vqd_schedule(int n, int nin, const vqd_native_op* in, const double* dur, int idle_code, const double* t1,
                 const double* t2, int cap, vqd_native_op* out, int* nout);

/* ------------------------------------------------------------------------------------------
 * Device-family compilers (host only): a logical circuit in a family's native gates -> the
 * native op list with that family's noise, ready for vqd_apply_native / vqd_run_program.
 * ---------------------------------------------------------------------------------------- */

/* Superconducting transmon device of Sec. 8 with the parameters of its App. C table.  All arrays
 * are host arrays owned by the caller, read during the call only.  Frequencies in MHz, times in us. */
typedef struct {
  int32_t n;               /* qubits (1..32) */
  int32_t ncouple;         /* capacitively coupled pairs */
  const double* t1;        /* [n] T1 > 0 */
  const double* t2;        /* [n] T2 > 0, the dephasing time of Eq. (depht2) */
  const double* excited;   /* [n] thermal excited population p_j in [0,1] (Eq. thermalstate); gamp relaxes
                              towards it (gamp's ground population 1 - p_j) */
  const double* freq;      /* [n] qubit frequencies */
  const double* anharm;    /* [n] anharmonicities alpha_j, used with the sign given */
  const int32_t* couple;   /* [2*ncouple] pairs (c, t), distinct qubits */
  const double* coupling;  /* [ncouple] coupling strengths J */
  const double* fid_read;  /* [n] readout fidelities in [1/4,1], or NULL for no readout depolarisation */
  double dur_rxy;          /* duration of Rx, Ry; Rz is virtual and takes no time */
  double dur_zx;           /* duration of the cross-resonance ZX */
  double dur_zz;           /* duration of the siZZle ZZ */
  double dur_meas;         /* readout duration (the gamp(t_M) before the readout) */
  uint32_t flags;          /* VQD_SC_NO_PASSIVE | VQD_SC_NO_STATIC_ZZ */
} vqd_sc_device;
#define VQD_SC_NO_PASSIVE 1u    /* no T1/T2 decay (passive and readout gamp) */
#define VQD_SC_NO_STATIC_ZZ 2u  /* no static ZZ crosstalk */

/* Compile a logical circuit of Rx, Ry, Rz, ZX, ZZ ops (others: VQD_EINVAL) for the device.  Gates are
 * exact and run in parallel: each starts in the first layer where all its qubits are free; a layer
 * lasts as long as its longest gate.  Per layer with nonzero length L, in this order: its gates
 * (program order); for every coupled pair (c, t) with J != 0 not under a ZZ gate of the layer, a
 * VQD_OP_ZZ_STATIC with parameters 2 pi L (J, f_c - f_t, alpha_t, alpha_c); for every qubit j whose
 * gate in the layer (if any) is shorter than L, by dt = L - its gate's duration: gamp(dt, T1_j,
 * 1 - p_j) then deph1((1 - e^{-dt/T2_j})/2).  With readout != 0, for every qubit: gamp(t_M, T1_j,
 * 1 - p_j) (when t_M > 0), then depol1(1 - F_j) (when fid_read is given).  out == NULL only counts:
 * *nout receives the number of ops; otherwise out has room for cap ops (VQD_EINVAL if too few). */
int vqd_sc_compile(const vqd_sc_device* dev, int nin, const vqd_native_op* in, int readout, int cap,
                   vqd_native_op* out, int* nout);

/* Silicon spin-qubit device of Sec. 7 with the parameters of its App. C table: a line of n qubits,
 * controlled-phase gates between neighbours.  Host arrays owned by the caller.  MHz and us. */
typedef struct {
  int32_t n;               /* qubits (2..32) */
  const double* t1;        /* [n] T1 > 0 (passive decay as depolarising, Eq. depolt1) */
  const double* t2;        /* [n] T2 > 0 (Eq. depht2) */
  const double* freq;      /* [n] qubit (ESR) frequencies */
  const double* rabi;      /* [n] Rabi frequencies of the x/y rotations, > 0 */
  const double* fid_1q;    /* [n] average fidelities of x/y rotations, in (0,1] */
  double x_1q;             /* depolarising fraction of the single-qubit standard error, in [0,1] */
  const double* freq_cz;   /* [n-1] controlled-phase frequencies of the pairs (k, k+1), > 0 */
  const double* fid_cz;    /* [n-1] average fidelities of CZ/CPh on (k, k+1), in (0,1] */
  double x_cz;             /* depolarising fraction of the two-qubit standard error */
  const double* xtalk_on;  /* [(n-1)*(n-1)] row k = active pair, column j = passive pair; or NULL */
  const double* xtalk_off; /* [n-1] off-state crosstalk angles of the pairs (k, k+1); or NULL */
  uint32_t flags;          /* VQD_SI_NO_PASSIVE | VQD_SI_NO_OFFRES */
} vqd_si_device;
#define VQD_SI_NO_PASSIVE 1u  /* no passive T1/T2 decay */
#define VQD_SI_NO_OFFRES 2u   /* no off-resonant drive of bystanders */

/* Compile a logical circuit of Rx, Ry, Rz, CZ, CPh ops (CZ/CPh on neighbours; others: VQD_EINVAL) for
 * the device.  Gates run one at a time, in program order.  Rz: virtual, emitted alone.  Rx/Ry(theta) on
 * q, lasting t = |theta| / (2 pi rabi_q): the gate; its standard error (below) from fid_1q[q], x_1q; with t > 0, for every
 * j != q, offres(2 pi rabi_q, 2 pi |f_j - f_q|, t); for every j != q, idle_depol(t, T1_j, T2_j); for
 * every pair (k, k+1) not containing q, crz_xtalk(xtalk_off[k]) (when given and nonzero).  CZ or
 * CPh(theta) on (k, k+1) (CZ: theta = pi), lasting t = |theta| / (2 pi freq_cz[k]): the gate;
 * its standard error from fid_cz[k], x_cz on the gate's qubits; for every other pair j, crz_xtalk(xtalk_on[k][j]
 * theta / pi) on (j, j+1) (when given and nonzero); idle_depol(t, ...) on every qubit outside the pair.
 * A gate's standard error is App. B's deph(p) o depol(q) for its fidelity and depolarising fraction, with
 * App. C's angle rule (severities times |theta| / pi): depol(q |theta|/pi) then deph(p |theta|/pi), each
 * left out when zero.  out == NULL only counts; otherwise out has room for cap ops (VQD_EINVAL if too few). */
int vqd_si_compile(const vqd_si_device* dev, int nin, const vqd_native_op* in, int cap, vqd_native_op* out,
                   int* nout);

/* NV-centre device of Sec. 5 with the parameters of its App. C table: qubit 0 is the electron spin,
 * qubits 1..n-1 are nuclear spins coupled only to it (a star).  Host arrays owned by the caller.
 * Times and frequencies in any consistent units (the table's: seconds and Hz). */
typedef struct {
  int32_t n;               /* qubits (2..32) */
  const double* t1;        /* [n] T1 > 0 (passive decay as depolarising, Eq. depolt1) */
  const double* t2;        /* [n] T2 > 0 (Eq. depht2) */
  const double* freq_xy;   /* [n] Rabi frequencies of the x/y rotations, > 0 */
  const double* freq_z;    /* [n] frequencies of the z rotations, > 0 */
  const double* fid_xy;    /* [n] average fidelities of x/y rotations, in (0,1] */
  const double* fid_z;     /* [n] average fidelities of z rotations (1: noiseless virtual Z) */
  double x_xy;             /* depolarising fraction of the x/y rotations' standard error, in [0,1] */
  const double* freq_crot; /* [n-1] frequencies of the conditional rotations on nuclear spins 1..n-1, > 0 */
  const double* fid_crot;  /* [n-1] their average fidelities */
  double x_crot;           /* depolarising fraction of the conditional rotations' standard error */
  double freq_zz;          /* weak ZZ coupling frequency among passive nuclear spins (0: none) */
  double fid_meas;         /* electron readout fidelity (readout bias 1 - fid_meas), in [0,1] */
  double dur_meas;         /* electron readout duration */
  uint32_t flags;          /* VQD_NV_NO_PASSIVE */
} vqd_nv_device;
#define VQD_NV_NO_PASSIVE 1u  /* no passive T1/T2 decay or weak ZZ */

/* Compile a logical circuit of Rx, Ry, Rz on any qubit and the conditional rotations CRx+- (VQD_OP_ZX)
 * and CRy+- (VQD_OP_ZY) with control 0 and a nuclear target (others: VQD_EINVAL) for the device.  Gates
 * run one at a time, in program order.  Rx/Ry(theta) on q lasts t = |theta| / (2 pi freq_xy[q]) and is
 * followed by its standard error from fid_xy[q], x_xy; Rz(theta) lasts |theta| / (2 pi freq_z[q]) and is
 * followed by a dephasing standard error from fid_z[q] when fid_z[q] < 1; a conditional rotation theta on
 * (0, j) lasts |theta| / (2 pi freq_crot[j-1]) and is followed by its two-qubit standard error from
 * fid_crot[j-1], x_crot.  Standard errors are depol(q |theta|/pi) then deph(p |theta|/pi) (App. B's
 * severities with App. C's angle rule; zero ones left out).  During a gate of
 * length t > 0, on the qubits outside it: zz_idle(t, freq_zz) on every pair (i, k), 1 <= i < k, of
 * nuclear spins (when freq_zz != 0), then idle_depol(t, T1_j, T2_j) on every such qubit j.  With
 * readout != 0, the electron readout bias ends the program: rx(pi), amp(1 - fid_meas), rx(pi) on
 * qubit 0, then the passive noise of the other qubits over dur_meas.  out == NULL only counts;
 * otherwise out has room for cap ops (VQD_EINVAL if too few). */
int vqd_nv_compile(const vqd_nv_device* dev, int nin, const vqd_native_op* in, int readout, int cap,
                   vqd_native_op* out, int* nout);

/* Trapped-ion device of Sec. 4 with the parameters of its App. C table (every ion identical).  Zones,
 * shuttling, splitting and remote entanglement are not modelled: any two ions may take a CZ.  MHz, us. */
typedef struct {
  int32_t n;               /* ions (1..32) */
  double t1;               /* T1 > 0 (passive decay as depolarising, Eq. depolt1) */
  double t2s;              /* T2* > 0 (Gaussian dephasing, Eq. depht2s) */
  double rabi;             /* Rabi frequency of the x/y rotations, > 0 */
  double fid_xy, x_xy;     /* x/y rotation fidelity in (0,1] and depolarising fraction in [0,1] */
  double freq_cz;          /* CZ gate frequency, > 0 */
  double fid_cz, x_cz;     /* CZ fidelity in (0,1] and depolarising fraction in [0,1] */
  double bf_read;          /* readout bit-flip probability in [0,1/2] */
  double dur_read;         /* duration of one ion's readout, >= 0 */
  uint32_t flags;          /* VQD_ION_NO_PASSIVE */
} vqd_ion_device;
#define VQD_ION_NO_PASSIVE 1u  /* no passive T1/T2* decay */

/* Compile a logical circuit of Rx, Ry, Rz and CZ ops (others: VQD_EINVAL) for the ions.  Gates run one at
 * a time, in program order.  Rx/Ry(theta) lasts t = |theta| / (2 pi rabi) and is followed by depol1(q s)
 * then deph1(p s), s = |theta| / pi, (p, q) = App. B's severities for fid_xy, x_xy (zero ones left out);
 * Rz is virtual: instantaneous and exact; CZ lasts 1 / (2 freq_cz) and is followed by depol2(q) then
 * deph2(p) for fid_cz, x_cz.  During a gate of length t > 0, every other ion gets idle_t2s(t, t1, t2s).
 * With readout != 0 the ions are read one at a time, 0 first: bitflip(bf_read) on ion j, then
 * idle_t2s(dur_read, t1, t2s) on the ions not yet read.  out == NULL only counts; otherwise out has room
 * for cap ops (VQD_EINVAL if too few). */
int vqd_ion_compile(const vqd_ion_device* dev, int nin, const vqd_native_op* in, int readout, int cap,
                    vqd_native_op* out, int* nout);

/* Neutral-atom device of Sec. 6 with the parameters of its App. C table (identical atoms at fixed sites;
 * moves, atom loss and multi-qubit gates are not modelled).  Host arrays owned by the caller.  MHz, us. */
typedef struct {
  int32_t n;               /* atoms (1..32) */
  const double* x;         /* [n] site coordinates (lattice units) */
  const double* y;         /* [n] */
  double blockade;         /* CZ(phi) needs the two atoms within this distance */
  double t2;               /* T2 > 0 */
  double t_vac;            /* vacuum lifetime > 0; T1 = t_vac / n (collisional loss, Sec. 6) */
  double p10, p01;         /* asymmetric bit flip of a single rotation by pi: |1> -> |0> and |0> -> |1> */
  double leak_init;        /* initialisation leakage gamma in [0,1] (operator L of Sec. 6) */
  double leak_cz_a, leak_cz_b;  /* CZ leakage alpha, beta in [0,1] (Eq. czleak) */
  double dur_cz;           /* duration of a Rydberg CZ(phi), >= 0 (not tabulated: the caller's choice) */
  double fid_meas;         /* readout fidelity in [1/2,1] */
  uint32_t flags;          /* VQD_NA_NO_PASSIVE */
} vqd_na_device;
#define VQD_NA_NO_PASSIVE 1u  /* no passive T1/T2 decay */

/* Compile a logical circuit of Raman rotations U(phi, Omega, Delta, t) (VQD_OP_U) and Rydberg CZ(phi)
 * (VQD_OP_CZPHI) on atom pairs within the blockade radius (others: VQD_EINVAL) for the atoms.  Gates run
 * one at a time, in program order.  With init != 0 the program starts with leak_init(gamma) on every atom.
 * U on q (its duration is its own t) is followed by deph1(1 - e^{-t/(2 T2)}) (Sec. 6, with the sign of the
 * exponent read as decay) and bitflip_asym(p10 s, p01 s), s = Omega_R |t| / pi with
 * Omega_R = sqrt(Omega^2 + Delta^2) (App. C's angle rule); CZ(phi) on (a, b) lasts dur_cz and is followed
 * by leak_cz(alpha, beta).  During a gate of length t > 0 every other atom gets idle_depol(t, t_vac / n,
 * T2).  With readout != 0 every atom gets depol1(3 (1 - fid_meas) / 2), whose misclassification
 * probability is 1 - fid_meas.  out == NULL only counts; otherwise out has room for cap ops (VQD_EINVAL
 * if too few). */
int vqd_na_compile(const vqd_na_device* dev, int nin, const vqd_native_op* in, int init, int readout, int cap,
                   vqd_native_op* out, int* nout);

/* App. B: severities (p_deph, q_depol) of the standard error deph(p) o depol(q) whose average
 * gate fidelity is fbar, with depolarising fraction x in [0,1]; nq = 1 or 2. */
int vqd_stderr_params(int nq, double fbar, double x, double* p_deph, double* q_depol);

/* ------------------------------------------------------------------------------------------
 * Reductions (synchronous; FP64 accumulation, fixed summation order)
 * ---------------------------------------------------------------------------------------- */

/* Marginal Z-basis probabilities of qubits[0..m-1] (distinct; m <= n, 2^m outputs), the outcome
 * distribution of a projective measurement in the computational basis (Sec. 3.6 readout, and the
 * populations reported for the Bell states of Sec. 7):
 * out[v] = sum of Re rho[x][x] over basis states x whose bits on qubits spell v (qubits[0]
 * = least significant bit of v). */
int vqd_prob(vqd_t ctx, int inst, int m, const int* qubits, double* out);

/* *out = Re sum_t coeffs[t] tr(P_t rho); paulis is nterms x n bytes, paulis[t*n + q] in
 * {0=I, 1=X, 2=Y, 3=Z} is the factor on qubit q.  The expected value of a Pauli sum: the stabilisers
 * and logical operators of Sec. 6.4, the Hamiltonian terms of the VQE of Sec. 8.4, and the quantity
 * SampleExpecPauliString estimates by trajectories in Sec. 2. */
int vqd_expect(vqd_t ctx, int inst, int nterms, const uint8_t* paulis, const double* coeffs, double* out);

/* Reductions of every instance of a batch context in one batched launch (one CTA per chunk of 2^20
 * amplitudes of an instance), copied back once.  probs (host, sum_i 2^{n_i} doubles, instances in order)
 * receives each instance's full Z-basis distribution Re rho[x][x]; trace_re and purity (host, count
 * doubles) receive Re tr rho and sum |rho_ij|^2 per instance.  Any output may be NULL.  Synchronous. */
int vqd_batch_reduce(vqd_t ctx, double* probs, double* trace_re, double* purity);

/* Projective Z-basis measurement of qubit q with collapse (the readout of Sec. 3.6 / Sec. 6):
 * p_m = tr(P_m rho) / tr(rho) for P_m = |m><m|_q.  With force = -1 the outcome is 0 when
 * u tr(rho) < tr(P_0 rho), else 1 (u in [0,1) is the caller's uniform draw); force = 0 or 1
 * post-selects that outcome.  The state becomes P_m rho P_m / tr(P_m rho).  Returns the outcome and
 * its probability (either pointer may be NULL).  Synchronous.  EINVAL for a zero-probability
 * forced outcome. */
int vqd_measure(vqd_t ctx, int inst, int q, double u, int force, int* outcome, double* prob);

/* Parity measurement of the silicon device (Sec. 7, Eq. m) on qubits qa, qb with collapse.  Outcome 0 is
 * the odd subspace span{|01>, |10>} (a change of current is detected), outcome 1 the even subspace
 * span{|00>, |11>}; |ab> means qa = a, qb = b.  With force = -1 the outcome is 0 when u tr(rho) < tr(P_0 rho),
 * else 1; force = 0 or 1 post-selects.  The state becomes P_m rho P_m / tr(P_m rho); with decay != 0 the
 * Kraus map K = {|00><00|, |11><11|, |10><10|, |10><01|} of Sec. 7 follows, so that |01> ends in |10>.
 * Feedback is the caller's: branch on the returned outcome between calls.  Returns the outcome and its
 * probability (either pointer may be NULL).  Synchronous.  EINVAL for equal or out-of-range qubits or a
 * zero-probability forced outcome. */
int vqd_measure_parity(vqd_t ctx, int inst, int qa, int qb, double u, int force, int decay, int* outcome,
                       double* prob);

/* tr rho (not renormalised: the trace-decreasing leakage and loss maps of Sec. 3.7 and the CPTN
 * map of Sec. 6.3 leave it below 1). */
int vqd_trace(vqd_t ctx, int inst, double* re_out, double* im_out);

/* tr(rho^dagger rho) = sum |rho_ij|^2 (equals tr rho^2 for Hermitian rho).  The paper prints no purity;
 * it is the mixedness of the density matrix of Sec. 2, 1 for the pure output of a noiseless circuit and
 * lowered by every mixing channel of Sec. 3, so it tracks how much noise a program has applied. */
int vqd_purity(vqd_t ctx, int inst, double* out);

/* Copy instance inst to / from host, FP64 complex, layout above (4^n entries). */
int vqd_get_state(vqd_t ctx, int inst, vqd_c128* host_out);
int vqd_set_state(vqd_t ctx, int inst, const vqd_c128* host_in);

/* ------------------------------------------------------------------------------------------
 * Monte-Carlo trajectories (Sec. 2: the statevector alternative to the density matrix)
 *
 * Estimates Re sum_t coeffs[t] tr(P_t rho) for the state rho that the native program `ops` makes
 * from |0..0>, by ntraj statevector trajectories.  In every trajectory each channel is replaced by
 * one of its Kraus operators K_k, chosen with probability ||K_k psi||^2 (psi <- K_k psi / norm);
 * a trace-decreasing channel's missing probability ends the trajectory, which then contributes 0.
 * Kraus operators are enumerated in a fixed order: a composite process (step A then step B) has
 * operators B_j A_i with A's index i outer; Pauli channels list I, X, Y, Z (two-qubit: the first
 * qubit's Pauli outer).  The draw for native op o in trajectory t is the first two 32-bit words of
 * Philox4x32-10 (Salmon et al., SC 2011) at counter (o, t, 0, 0) with key (seed low, seed high),
 * as a 53-bit uniform u = (w0 >> 5) 2^-27 + (w1 >> 6) 2^-53; operator k is chosen when
 * sum_{j<k} p_j <= u < sum_{j<=k} p_j.
 *
 * prec is VQD_F32 or VQD_F64 (VQD_F32_SPLIT: VQD_EINVAL).
 * 1 <= n <= 16.  Every trajectory keeps its statevector in shared memory: in one CTA up to n = 14
 * (VQD_F32) or 13 (VQD_F64), beyond that split over a thread-block cluster of up to 8 CTAs (slices
 * of 64 KB, 128 KB for 16 qubits in VQD_F64) joined by distributed shared memory.
 * paulis is nterms x n codes (0=I,1=X,2=Y,3=Z) as in vqd_expect.  out (host, ntraj) receives each
 * trajectory's value; mean and stderr_out (either may be NULL) the sample mean and its standard
 * error.  Synchronous on `stream`.  Returns VQD_EINVAL for n outside 1..16, VQD_ENOTSUP for more
 * than 16 state-dependent Kraus operators in one channel; messages via vqd_last_error(NULL). */
int vqd_traj_expect(int n, int prec, int nops, const vqd_native_op* ops, unsigned flags, int ntraj, uint64_t seed,
                    int nterms, const uint8_t* paulis, const double* coeffs, void* stream, double* out,
                    double* mean, double* stderr_out);

/* ------------------------------------------------------------------------------------------
 * Allocation-free reduction (the paper has no counterpart: this serves callers of the library)
 *
 * vqd_prob_static computes the same marginal Z-basis probabilities as vqd_prob, for callers that
 * cannot allocate device memory: a host process whose framework's memory pool already owns all of
 * the GPU's memory, or a latency-critical loop that must not pay for the device-wide
 * synchronisation cudaMalloc / cudaFree can cause.  It needs no context and calls no cudaMalloc,
 * cudaFree or any other allocating routine.  Its partial sums live in a file-scope device array of
 * 2^14 doubles (128 KB), which every GPU that loads libvqd holds until the process exits.
 *
 *   dev_state  device address of an n-qubit state in the layout above (complex64 if prec ==
 *              VQD_F32, float-float pairs if VQD_F32_SPLIT, else complex128); read only.
 *   qubits     host array of m distinct qubits, 1 <= m <= VQD_PROB_STATIC_MAX_M (qubits[0] is the
 *              least significant bit of the output index, as in vqd_prob).
 *   dev_out    DEVICE array of 2^m doubles, written on `stream` (a cudaStream_t; NULL = legacy
 *              default stream).  The call is asynchronous: synchronise the stream before reading.
 *
 * Returns VQD_OK, VQD_EINVAL (bad argument; dev_state not aligned to its amplitude size, 8 bytes for
 * VQD_F32 and 16 otherwise, or dev_out not 8-byte aligned; or m above VQD_PROB_STATIC_MAX_M: the static
 * scratch holds at most 2^14 partial sums) or VQD_EDEVICE; the message is in vqd_last_error(NULL).
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and keeps it, keyed by the device ordinal; make that first call before any
 * stream capture.  The kept address belongs to the device's primary context, the one the CUDA runtime
 * uses: call it only with that context current, and not after cudaDeviceReset in the same process
 * (the reset destroys the context the address belongs to).  All calls
 * share the one array and each call overwrites what the previous one left there: calls that
 * overlap on the GPU (other streams, or other host threads) race, so serialise them.
 * ---------------------------------------------------------------------------------------- */
#define VQD_PROB_STATIC_MAX_M 14
int vqd_prob_static(const void* dev_state, int n, int prec, int m, const int* qubits, double* dev_out,
                    void* stream);

/* ------------------------------------------------------------------------------------------
 * Arithmetic peak of this GPU (the paper has no counterpart: it is the denominator of the roofline of
 * the kernels bound by FP64 or FP32 arithmetic rather than by memory).  which = 0: FP64 FMA, 1: FP32
 * FMA.  Times one launch of independent FMA chains on every SM (CUDA events on `stream`, a cudaStream_t)
 * and returns the FMA instructions per second (2 flops each).  Synchronous; allocates and frees 8 bytes.
 * ---------------------------------------------------------------------------------------- */
int vqd_measure_fma_rate(int which, void* stream, double* fma_per_s);

/* ------------------------------------------------------------------------------------------
 * Launch accounting: per kernel class, the number of launches, their summed device time
 * (CUDA events recorded on the context stream around every launch while enabled) and the
 * algorithmic bytes they move.  Used to report achieved bandwidth against the roofline.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
  char name[32];       /* kernel class */
  int64_t launches;
  double total_ms;     /* summed CUDA-event durations (0 unless timing was enabled) */
  double alg_bytes;    /* algorithmic bytes: 2 x state bytes per pass (read + write once) */
  double amp_updates;  /* sum over original (pre-fusion) ops of the amplitudes they update */
  double alg_fma;      /* real multiply-adds the class's arithmetic performs (plain passes and fused stages:
                          structured for VQD_F64 and VQD_F32_SPLIT, dense complex FMAs for fused VQD_F32;
                          a float-float multiply-add is one), for the roofline of arithmetic-bound kernels */
} vqd_kstat;

/* mode 0: off; 1: count launches only; 2: count and time every launch with CUDA events. */
int vqd_profile(vqd_t ctx, int mode);
int vqd_profile_reset(vqd_t ctx);
int vqd_profile_read(vqd_t ctx, int max, vqd_kstat* out, int* n_out);

/* Global flags for the checks of apply_unitary / apply_kraus (VQD_NO_CHECK). */
int vqd_set_flags(vqd_t ctx, unsigned flags);

#ifdef __cplusplus
}
#endif
#endif /* VQD_H */
