// Fused path of libvqd: stages of operators applied to shared-memory tiles of the state.
//
// A stage owns a set Q of at most `fuse_qubits` qubits.  Its tile holds the 2^m amplitudes that
// share one assignment of every index bit outside B = {q, q + n : q in Q} u {low row bits}; the
// low row bits are carried along so that each tile is made of runs of >= 64 contiguous bytes
// (full DRAM sectors).  A CTA loads a tile once, applies every operator of the stage to it, and
// stores it once: one pass over HBM per stage instead of one per operator.  Inside the tile the
// operators are grouped into blocks on one qubit or one pair of qubits; a thread holds the 4 or 16
// amplitudes of a block's group in registers and applies all of the block's operators to them, so
// that shared memory is swept once per block, not once per operator.
//
// Stages are formed greedily in program order with a commuting lookahead: an operator that does
// not fit the current stage is deferred, and later operators may still join the stage as long
// as they act on none of the deferred operators' qubits (so every pair of operators that share
// a qubit keeps its order).
//
// The batched kernel runs whole instances of a batch context, one instance per CTA at a time,
// taken from an atomic queue ordered largest first; each CTA walks its instance's stages and
// tiles on its own, so CTAs never wait for one another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "fused.h"
#include "kernels.h"
#include "numeric.h"

namespace vqd {

int tile_bits_budget(int prec) { return prec == VQD_F32 ? 13 : 12; }  // 64 KB tiles
// 64-byte runs; a Hermitian plan's tiles carry the passengers' column bits as well, so it takes 32-byte
// runs (one DRAM sector) to keep the same number of stage qubits.
int default_passengers(int prec, bool herm) {
  if (herm) return prec == VQD_F32 ? 2 : 1;
  return prec == VQD_F32 ? 3 : 2;
}
static int default_fuse(int prec) { (void)prec; return 6; }

static int popc(uint32_t x) { return __builtin_popcount(x); }

// Tile bits of a stage on qubits qmask with L passengers: both index bits of every stage qubit and the
// passengers' row bits (general plan), or both index bits of every stage or passenger qubit (Hermitian plan).
static int stage_bit_count(uint32_t qmask, int L, bool herm) {
  if (herm) return 2 * popc(qmask | ((1u << L) - 1u));
  int c = 2 * popc(qmask);
  for (int b = 0; b < L; b++)
    if (!(qmask >> b & 1)) c++;
  return c;
}

// A map preserves Hermiticity when its superoperator satisfies S[(c,r),(c',r')] = conj S[(r,c),(r',c')]
// (s = r | c << k): true of U rho U^dagger and of every Kraus map sum_i K_i rho K_i^dagger (Sec. 2).
bool preserves_hermiticity(const Op& op) {
  if (op.unitary) return true;
  const int d = 1 << op.k, D = d * d;
  double scale = 0;
  for (const cd& v : op.m) scale = std::max(scale, std::abs(v));
  const double tol = 1e-12 * std::max(1.0, scale);
  for (int s = 0; s < D; s++) {
    const int ts = (s >> op.k) | (s & (d - 1)) << op.k;
    for (int t = 0; t < D; t++) {
      const int tt = (t >> op.k) | (t & (d - 1)) << op.k;
      if (std::abs(op.m[(size_t)ts * D + tt] - std::conj(op.m[(size_t)s * D + t])) > tol) return false;
    }
  }
  return true;
}

// ---------------------------------------------------------------- operator algebra (FP64, host)
// Matrix of an operator on qubits `from` (k1) re-expressed on qubits `to` (k2, from within to),
// identity on the extra qubit.  Unitaries are 2^k square; superoperators 4^k with s = r | c << k.
static std::vector<cd> embed_on(const std::vector<cd>& m, bool unitary, int k1, const int* from, int k2,
                                const int* to) {
  int pos[2] = {0, 0};
  unsigned mask = 0;
  for (int j = 0; j < k1; j++) {
    for (int i = 0; i < k2; i++)
      if (to[i] == from[j]) pos[j] = i;
    mask |= 1u << pos[j];
  }
  auto sub = [&](int x) {
    int v = 0;
    for (int j = 0; j < k1; j++) v |= ((x >> pos[j]) & 1) << j;
    return v;
  };
  const int d2 = 1 << k2, d1 = 1 << k1;
  if (unitary) {
    std::vector<cd> o(d2 * d2, 0.0);
    for (int i = 0; i < d2; i++)
      for (int j = 0; j < d2; j++)
        if ((i & ~mask) == (j & ~mask)) o[i * d2 + j] = m[sub(i) * d1 + sub(j)];
    return o;
  }
  const int D2 = d2 * d2, D1 = d1 * d1;
  std::vector<cd> o(D2 * D2, 0.0);
  for (int a = 0; a < D2; a++)
    for (int b = 0; b < D2; b++) {
      int ra = a & (d2 - 1), ca = a >> k2, rb = b & (d2 - 1), cb = b >> k2;
      if ((ra & ~mask) != (rb & ~mask) || (ca & ~mask) != (cb & ~mask)) continue;
      o[a * D2 + b] = m[(sub(ra) | (sub(ca) << k1)) * D1 + (sub(rb) | (sub(cb) << k1))];
    }
  return o;
}

static std::vector<cd> matmul(const std::vector<cd>& a, const std::vector<cd>& b, int d) {
  std::vector<cd> c(d * d, 0.0);
  for (int i = 0; i < d; i++)
    for (int l = 0; l < d; l++) {
      const cd x = a[i * d + l];
      if (x == 0.0) continue;
      for (int j = 0; j < d; j++) c[i * d + j] += x * b[l * d + j];
    }
  return c;
}

static bool is_diag(const Op& op) {
  const int d = op.unitary ? (1 << op.k) : (1 << (2 * op.k));
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++)
      if (i != j && op.m[(size_t)i * d + j] != 0.0) return false;
  return true;
}
static bool is_dense2(const Op& op) { return op.k == 2 && !op.unitary && !is_diag(op); }

// second o first, on the union of their qubits (at most two).
static Op compose(const Op& first, const Op& second) {
  Op r;
  int u[2], nu = 0;
  for (int j = 0; j < first.k; j++) u[nu++] = first.q[j];
  for (int j = 0; j < second.k; j++) {
    bool seen = false;
    for (int i = 0; i < nu; i++) seen = seen || u[i] == second.q[j];
    if (!seen) u[nu++] = second.q[j];
  }
  r.k = nu;
  r.q[0] = u[0];
  r.q[1] = nu > 1 ? u[1] : 0;
  r.unitary = first.unitary && second.unitary;
  auto lift = [&](const Op& o) {
    std::vector<cd> m = (r.unitary || !o.unitary) ? o.m : superop_from_unitary(o.k, o.m.data());
    return embed_on(m, r.unitary, o.k, o.q, nu, r.q);
  };
  const int d = r.unitary ? (1 << nu) : (1 << (2 * nu));
  r.m = matmul(lift(second), lift(first), d);
  r.weight = first.weight + second.weight;
  return r;
}

// A two-qubit superoperator that is a tensor product A (x) B of one-qubit superoperators on q[0] and
// q[1] (the T1/T2 decay of both qubits of a pair, for instance) is applied as the two: 2 x 4 complex MACs
// per amplitude with coefficients in registers, against 16 MACs and 16 coefficient loads for the dense
// form.  S[so][si] = A[ao][ai] B[bo][bi] with s = r0 | r1 << 1 | c0 << 2 | c1 << 3, a = r0 | c0 << 1 and
// b = r1 | c1 << 1, so S realigned as M[(ao, ai)][(bo, bi)] has rank one; the factors are one column and
// one row of M through its largest entry, accepted when they reproduce every entry to 1e-15 of it (a
// few FP64 roundings of an exact product, as the kron of two one-qubit channels gives), so that a
// slightly entangling channel is never replaced by an approximation.
static bool split_product(const Op& op, Op& a, Op& b) {
  if (op.k != 2 || op.unitary || is_diag(op)) return false;
  auto a_of = [](int s) { return (s & 1) | (((s >> 2) & 1) << 1); };
  auto b_of = [](int s) { return ((s >> 1) & 1) | (((s >> 3) & 1) << 1); };
  std::vector<cd> M(256);
  for (int so = 0; so < 16; so++)
    for (int si = 0; si < 16; si++) M[(a_of(so) * 4 + a_of(si)) * 16 + b_of(so) * 4 + b_of(si)] = op.m[so * 16 + si];
  int pi = 0, pj = 0;
  for (int x = 0; x < 256; x++)
    if (std::abs(M[x]) > std::abs(M[pi * 16 + pj])) {
      pi = x / 16;
      pj = x % 16;
    }
  const double top = std::abs(M[pi * 16 + pj]);
  if (top == 0.0) return false;
  std::vector<cd> A(16), B(16);
  for (int x = 0; x < 16; x++) A[x] = M[x * 16 + pj];
  for (int y = 0; y < 16; y++) B[y] = M[pi * 16 + y] / M[pi * 16 + pj];
  for (int x = 0; x < 16; x++)
    for (int y = 0; y < 16; y++)
      if (std::abs(M[x * 16 + y] - A[x] * B[y]) > 1e-15 * top) return false;
  a = Op();
  a.unitary = false;
  a.k = 1;
  a.q[0] = op.q[0];
  a.m = A;
  a.weight = op.weight;
  b = Op();
  b.unitary = false;
  b.k = 1;
  b.q[0] = op.q[1];
  b.m = B;
  b.weight = 0.0;  // the pair stands for the original operation once
  return true;
}

// ---------------------------------------------------------------- composition inside a stage
// Arithmetic of one coefficient in a sweep that follows the coefficients' structure (zero: nothing;
// one: an add; real or imaginary: two real multiply-adds; complex: four), in real multiply-adds.
static double coef_cost(const cd& c) {
  if (c == 0.0) return 0.0;
  if (c == 1.0) return 1.0;
  if (c.imag() == 0.0 || c.real() == 0.0) return 2.0;
  return 4.0;
}

// Cost per amplitude of one sweep of an operator (k <= 2) whose arithmetic follows the structure of its
// coefficients, in real multiply-adds: a diagonal scales each member whose factor is not 1; a one-qubit
// operator is its 4 x 4 superoperator on the 4 members of a group; a two-qubit unitary is U A U^dagger
// on the 4 x 4 block A (each entry of U is used 8 times per 16 members); a two-qubit channel is its
// 16 x 16 superoperator, whose coefficients are read from shared memory for every group.  `branch` is
// the cost of examining one coefficient's structure (once per term and group).
static double sweep_cost(const Op& op, double branch) {
  const int d = 1 << op.k, D = d * d;
  double c = 0.0;
  if (is_diag(op)) {
    for (int s = 0; s < D; s++) {
      const int r = s & (d - 1), cc = s >> op.k;
      const cd f = op.unitary ? diag_unitary_factor(op.m[r * d + r], op.m[cc * d + cc]) : op.m[(size_t)s * D + s];
      c += f == 1.0 ? 0.0 : (f == 0.0 ? 1.0 : coef_cost(f)) + branch;
    }
    return c / D;
  }
  if (op.k == 2 && op.unitary) {
    for (const cd& u : op.m) c += coef_cost(u) + branch;
    return 8.0 * c / D;
  }
  const std::vector<cd> S = op.unitary ? superop_from_unitary(op.k, op.m.data()) : op.m;
  for (const cd& x : S) c += coef_cost(x) + (x == 0.0 ? branch : 2.0 * branch);
  return c / D;
}

// Real multiply-adds per amplitude of one complex64 sweep, which keeps straight-line complex FMAs: 4 per
// complex coefficient used (a diagonal: 4 per member it changes).
static double dense_cost(const Op& op) {
  const int d = 1 << op.k, D = d * d;
  if (is_diag(op)) {
    double c = 0.0;
    for (int s = 0; s < D; s++) {
      const int r = s & (d - 1), cc = s >> op.k;
      const cd f = op.unitary ? diag_unitary_factor(op.m[r * d + r], op.m[cc * d + cc]) : op.m[(size_t)s * D + s];
      if (f != 1.0) c += 4.0;
    }
    return c / D;
  }
  if (op.k == 2 && op.unitary) return 4.0 * 16.0 * 8.0 / 16.0;
  return 4.0 * (double)D;  // D x D coefficients per D members
}

// The stage's operators are merged into composites on at most two qubits, in FP64.  Open
// composites are kept on pairwise disjoint qubit sets; an operator merges with the composites it
// touches when their qubits and its own number at most two, otherwise it first emits them, so
// every qubit sees its operators in program order.
// Complex64 (FP32 arithmetic, where multiply-adds are cheap and every sweep costs shared-memory
// traffic and addressing): a merge is refused only when it would build a dense two-qubit
// superoperator out of cheaper pieces (16 complex MACs and 16 coefficient loads per amplitude).
// FP64 and float-float (where arithmetic dominates: FP64 runs at 1/58 of the FP32 rate on this GPU,
// and a float-float multiply-add takes about 15 FP32 instructions): the sweeps follow the
// coefficients' zero/one/real/imaginary structure, and a merge is taken only when the composite's
// structured arithmetic does not exceed that of its pieces plus the cost of the sweep it saves.
static std::vector<Op> compose_stage(const std::vector<Op>& ops, const std::vector<int>& idx, int prec) {
  const bool structured = prec != VQD_F32;
  // in real multiply-adds of the precision: a float-float one is about 15 FP32 instructions, an FP64 one
  // occupies the FP64 pipe for about as long as 30 FP32 instructions; a sweep's shared-memory traffic and
  // addressing take about 5 FP32 instructions per amplitude, a coefficient test about 2
  const double sweep_saved = prec == VQD_F64 ? 0.15 : 0.3;
  const double branch = prec == VQD_F64 ? 0.07 : 0.13;
  std::vector<Op> out, open;
  for (int i : idx) {
    const Op& op = ops[i];
    std::vector<int> hit;
    int uq[4], nu = 0;
    for (int j = 0; j < op.k; j++) uq[nu++] = op.q[j];
    for (size_t x = 0; x < open.size(); x++) {
      bool inter = false;
      for (int a = 0; a < open[x].k; a++)
        for (int j = 0; j < op.k; j++) inter = inter || open[x].q[a] == op.q[j];
      if (!inter) continue;
      hit.push_back((int)x);
      for (int a = 0; a < open[x].k; a++) {
        bool seen = false;
        for (int u = 0; u < nu; u++) seen = seen || uq[u] == open[x].q[a];
        if (!seen && nu < 4) uq[nu++] = open[x].q[a];
      }
    }
    bool merged = false;
    if (nu <= 2 && !hit.empty()) {
      Op c = open[hit[0]];
      bool dense_in = is_dense2(c) || is_dense2(op);
      double parts = structured ? sweep_cost(c, branch) + sweep_cost(op, branch) : 0.0;
      for (size_t h = 1; h < hit.size(); h++) {
        dense_in = dense_in || is_dense2(open[hit[h]]);
        if (structured) parts += sweep_cost(open[hit[h]], branch) + sweep_saved;
        c = compose(c, open[hit[h]]);  // disjoint composites commute
      }
      c = compose(c, op);
      const bool take = structured ? sweep_cost(c, branch) <= parts + sweep_saved : !(is_dense2(c) && !dense_in);
      if (take) {
        for (int h = (int)hit.size() - 1; h >= 0; h--) open.erase(open.begin() + hit[h]);
        open.push_back(std::move(c));
        merged = true;
      }
    }
    if (!merged) {
      for (int x : hit) out.push_back(open[x]);
      for (int h = (int)hit.size() - 1; h >= 0; h--) open.erase(open.begin() + hit[h]);
      open.push_back(op);
    }
  }
  for (Op& c : open) out.push_back(std::move(c));
  return out;
}

// Coefficients of one member inside a block on qubits bq (nq of them); returns the kind.
static int member_coefs(const Op& op, int nq, const int* bq, std::vector<cd>& out) {
  if (op.k == 1) {
    const bool on_b = nq == 2 && op.q[0] == bq[1];
    if (is_diag(op)) {  // factor of member t = r | c << 1
      for (int t = 0; t < 4; t++) {
        const int r = t & 1, c = t >> 1;
        out.push_back(op.unitary ? diag_unitary_factor(op.m[r * 2 + r], op.m[c * 2 + c]) : op.m[t * 5]);
      }
      return on_b ? BK_DIAG_B : BK_DIAG_A;
    }
    std::vector<cd> S = op.unitary ? superop_from_unitary(1, op.m.data()) : op.m;
    out.insert(out.end(), S.begin(), S.end());
    return on_b ? BK_SUP1_B : BK_SUP1_A;
  }
  std::vector<cd> m = embed_on(op.m, op.unitary, 2, op.q, 2, bq);  // qubit order of the block
  if (is_diag(op)) {  // factor of member t = r | c << 2
    for (int t = 0; t < 16; t++) {
      const int r = t & 3, c = t >> 2;
      out.push_back(op.unitary ? diag_unitary_factor(m[r * 4 + r], m[c * 4 + c]) : m[t * 17]);
    }
    return BK_DIAG2;
  }
  out.insert(out.end(), m.begin(), m.end());
  return op.unitary ? BK_UNI2 : BK_SUP2;
}

static void build_stage(FusedPlan& plan, const std::vector<Op>& ops, const std::vector<int>& idx, uint32_t qmask,
                        int n, int L, bool whole, int prec, bool herm) {
  // Blocks, members and their coefficients first: a stage whose coefficients overflow the shared
  // memory budget is split in two (each half is a valid stage on the same tile).
  const std::vector<Op> comp = compose_stage(ops, idx, prec);
  size_t ncoef = 0;
  for (const Op& o : comp) ncoef += is_diag(o) ? (o.k == 1 ? 4 : 16) : (o.k == 1 ? 16 : (o.unitary ? 16 : 256));
  if ((ncoef > (size_t)kCoefCap || comp.size() > (size_t)kOpCap || comp.size() > (size_t)kBlockCap) && idx.size() > 1) {
    std::vector<int> a(idx.begin(), idx.begin() + idx.size() / 2), b(idx.begin() + idx.size() / 2, idx.end());
    build_stage(plan, ops, a, qmask, n, L, whole, prec, herm);
    build_stage(plan, ops, b, qmask, n, L, whole, prec, herm);
    return;
  }
  StageDesc sd;
  std::memset(&sd, 0, sizeof(sd));
  bool in_tile[2 * VQD_MAX_QUBITS] = {false};
  if (whole) {
    for (int b = 0; b < 2 * n; b++) in_tile[b] = true;
  } else {
    for (int b = 0; b < std::min(L, n); b++) in_tile[b] = true;
    if (herm)
      for (int b = 0; b < std::min(L, n); b++) in_tile[b + n] = true;
    for (int q = 0; q < n; q++)
      if (qmask >> q & 1) in_tile[q] = in_tile[q + n] = true;
  }
  int local[2 * VQD_MAX_QUBITS];
  for (int b = 0; b < 2 * n; b++) {
    if (in_tile[b]) {
      local[b] = sd.nbits;
      sd.bits[sd.nbits++] = b;
    } else {
      local[b] = -1;
      sd.rest[sd.nrest++] = b;
    }
  }
  sd.herm = herm && !whole && sd.nrest > 0;
  if (sd.herm && (sd.nbits > 12 || sd.nbits % 2 != 0))
    throw Error(VQD_EINVAL, "internal: a Hermitian tile has an even number of bits, at most 12");
  sd.frac = 1.0;
  if (sd.herm) {
    const double K = std::ldexp(1.0, sd.nrest / 2);
    sd.frac = (K + 1.0) / (2.0 * K);
  }
  sd.block_begin = (int)plan.blocks.size();
  sd.coef_begin = (int)plan.coef.size();
  sd.op_begin = (int)plan.ops.size();
  for (const Op& o : comp) {
    TileBlock tb;
    std::memset(&tb, 0, sizeof(tb));
    tb.nq = o.k;
    for (int j = 0; j < tb.nq; j++) {
      tb.lbit[j] = local[o.q[j]];
      tb.lbit[j + tb.nq] = local[o.q[j] + n];
    }
    const int nb = 2 * tb.nq;
    for (int j = 0; j < nb; j++)
      if (tb.lbit[j] < 0) throw Error(VQD_EINVAL, "internal: operator outside its stage tile");
    for (int j = 0; j < nb; j++) tb.lsorted[j] = tb.lbit[j];
    std::sort(tb.lsorted, tb.lsorted + nb);
    tb.op_begin = (int)plan.ops.size();
    BlockOp bo;
    bo.coef = (int)plan.coef.size() - sd.coef_begin;
    bo.kind = member_coefs(o, o.k, o.q, plan.coef);
    bo.skip = 0;
    if (bo.kind == BK_DIAG_A || bo.kind == BK_DIAG_B || bo.kind == BK_DIAG2)
      for (size_t t = (size_t)bo.coef + sd.coef_begin; t < plan.coef.size(); t++)
        if (is_unit_factor(plan.coef[t])) bo.skip |= 1u << (t - bo.coef - sd.coef_begin);
    plan.ops.push_back(bo);
    sd.weight += o.weight;
    sd.fma_per_amp += prec == VQD_F32 ? dense_cost(o) : sweep_cost(o, 0.0);
    tb.op_end = (int)plan.ops.size();
    plan.blocks.push_back(tb);
  }
  while (plan.flag.size() < plan.coef.size()) plan.flag.push_back((uint8_t)flag_of(plan.coef[plan.flag.size()]));
  sd.block_end = (int)plan.blocks.size();
  sd.coef_end = (int)plan.coef.size();
  sd.op_end = (int)plan.ops.size();
  if (sd.coef_end - sd.coef_begin > kCoefCap || sd.op_end - sd.op_begin > kOpCap || sd.block_end - sd.block_begin > kBlockCap)
    throw Error(VQD_EINVAL, "internal: stage coefficients or blocks exceed budget");
  plan.max_bits = std::max(plan.max_bits, sd.nbits);
  plan.stages.push_back(sd);
}

FusedPlan plan_fused(const std::vector<Op>& ops_in, int n, int prec, int fuse_qubits, TileShape shape, bool herm) {
  FusedPlan plan;
  for (size_t i = 0; i < ops_in.size() && herm; i++) herm = preserves_hermiticity(ops_in[i]);
  plan.herm = herm;
  std::vector<Op> ops;
  ops.reserve(ops_in.size());
  for (const Op& o : ops_in) {
    Op a, b;
    if (split_product(o, a, b)) {
      ops.push_back(std::move(a));
      ops.push_back(std::move(b));
    } else {
      ops.push_back(o);
    }
  }
  const int tb = shape.tile_bits > 0 ? shape.tile_bits : tile_bits_budget(prec);
  const int Lset = shape.passengers >= 0 ? shape.passengers : default_passengers(prec, herm);
  if (tb > tile_bits_budget(prec) || Lset > 3 || tb < 4 + Lset)
    throw Error(VQD_EINVAL, "tile shape: need 4 + passengers <= tile bits <= the precision's maximum, passengers <= 3");
  // a Hermitian tile has an even number of bits and room for a two-qubit operator beside the passengers
  const int budget = herm ? tb & ~1 : tb;
  if (herm && budget < 2 * (Lset + 2))
    throw Error(VQD_EINVAL, "tile shape: a Hermitian plan needs 2 (passengers + 2) <= tile bits");
  const int L = std::min(Lset, n);
  int f = fuse_qubits <= 0 ? default_fuse(prec) : fuse_qubits;
  if (f < 2 || f > VQD_MAX_FUSE) throw Error(VQD_EINVAL, "fuse_qubits must be in 2..6");
  if (ops.empty()) return plan;
  if (2 * n <= budget) {  // the whole state is one tile: one stage holds every operator
    std::vector<int> all(ops.size());
    for (size_t i = 0; i < ops.size(); i++) all[i] = (int)i;
    build_stage(plan, ops, all, (1u << n) - 1, n, L, true, prec, herm);
    return plan;
  }
  const uint32_t full = (1u << n) - 1;
  const size_t kWindow = 1024;
  std::vector<int> remaining(ops.size());
  for (size_t i = 0; i < ops.size(); i++) remaining[i] = (int)i;
  std::vector<int> stage, deferred;
  while (!remaining.empty()) {
    stage.clear();
    deferred.clear();
    uint32_t q = 0, dmask = 0;
    size_t i = 0;
    for (; i < remaining.size() && i < kWindow; i++) {
      const Op& op = ops[remaining[i]];
      uint32_t m = 0;
      for (int j = 0; j < op.k; j++) m |= 1u << op.q[j];
      if (m & dmask) {
        deferred.push_back(remaining[i]);
        dmask |= m;
      } else {
        uint32_t q2 = q | m;
        if (popc(q2) <= f && stage_bit_count(q2, L, herm) <= budget) {
          q = q2;
          stage.push_back(remaining[i]);
        } else {
          deferred.push_back(remaining[i]);
          dmask |= m;
        }
      }
      if (dmask == full) {
        i++;
        break;
      }
    }
    build_stage(plan, ops, stage, q, n, L, false, prec, herm);
    std::vector<int> next;
    next.reserve(deferred.size() + remaining.size() - i);
    next.insert(next.end(), deferred.begin(), deferred.end());
    next.insert(next.end(), remaining.begin() + i, remaining.end());
    remaining.swap(next);
  }
  return plan;
}

BatchPlan merge_batch(const std::vector<FusedPlan>& plans, const std::vector<int>& n,
                      const std::vector<size_t>& byte_offsets, int prec) {
  BatchPlan bp;
  const size_t esz = prec == VQD_F32 ? 8 : 16;
  bp.passes.assign(plans.size(), 0);
  size_t max_stages = 0;
  for (size_t i = 0; i < plans.size(); i++) {
    const FusedPlan& p = plans[i];
    BatchInst bi;
    bi.offset_amps = byte_offsets[i] / esz;
    bi.n = n[i];
    bi.stage_begin = (int)bp.all.stages.size();
    const int b0 = (int)bp.all.blocks.size(), o0 = (int)bp.all.ops.size(), c0 = (int)bp.all.coef.size();
    for (StageDesc sd : p.stages) {
      sd.block_begin += b0;
      sd.block_end += b0;
      sd.op_begin += o0;
      sd.op_end += o0;
      sd.coef_begin += c0;
      sd.coef_end += c0;
      bp.all.stages.push_back(sd);
    }
    for (TileBlock t : p.blocks) {
      t.op_begin += o0;
      t.op_end += o0;
      bp.all.blocks.push_back(t);
    }
    bp.all.ops.insert(bp.all.ops.end(), p.ops.begin(), p.ops.end());
    bp.all.coef.insert(bp.all.coef.end(), p.coef.begin(), p.coef.end());
    bp.all.flag.insert(bp.all.flag.end(), p.flag.begin(), p.flag.end());
    bp.all.max_bits = std::max(bp.all.max_bits, p.max_bits);
    bi.stage_end = (int)bp.all.stages.size();
    bi.cost = std::ldexp(1.0, 2 * n[i]) * std::max<size_t>(1, p.stages.size());
    bp.passes[i] = (int)p.stages.size();
    max_stages = std::max(max_stages, p.stages.size());
    bp.inst.push_back(bi);
  }
  // Wave w: stage w of every instance that has one, split into chunks of at most kChunk tiles,
  // largest states first so that the long items start early.
  const uint32_t kChunk = 16;
  std::vector<int> order(plans.size());
  for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  for (size_t w = 0; w < max_stages; w++) {
    bp.wave_begin.push_back((int)bp.items.size());
    for (int i : order) {
      const BatchInst& bi = bp.inst[i];
      if ((int)w >= bi.stage_end - bi.stage_begin) continue;
      const int s = bi.stage_begin + (int)w;
      const uint32_t ntiles = (uint32_t)stage_work_tiles(bp.all.stages[s]);
      for (uint32_t t = 0; t < ntiles; t += kChunk) bp.items.push_back({i, s, t, std::min(kChunk, ntiles - t)});
    }
  }
  bp.wave_begin.push_back((int)bp.items.size());
  return bp;
}

// ================================================================== device side
namespace dev {


template <class T>
__device__ __forceinline__ void cmac(cx<T>& acc, const cx<T>& c, const cx<T>& x) {
  acc.x = fma(c.x, x.x, acc.x);
  acc.x = fma(-c.y, x.y, acc.x);
  acc.y = fma(c.x, x.y, acc.y);
  acc.y = fma(c.y, x.x, acc.y);
}
template <class T>
__device__ __forceinline__ cx<T> cmul(const cx<T>& a, const cx<T>& b) {
  cx<T> r;
  r.x = fma(a.x, b.x, -a.y * b.y);
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}

// Zero-bit insertion with precomputed masks: inserting a zero at bit p maps g to
// (g & low) | ((g & ~low) << 1) = g + (g & ~low), low = 2^p - 1.  hi[i] = ~(2^pos[i] - 1) for
// ascending positions, applied lowest first.
template <int NB>
struct Inserter {
  uint32_t hi[NB];
  __device__ __forceinline__ explicit Inserter(const int* pos) {
#pragma unroll
    for (int i = 0; i < NB; i++) hi[i] = ~((1u << pos[i]) - 1u);
  }
  __device__ __forceinline__ uint32_t operator()(uint32_t g) const {
#pragma unroll
    for (int i = 0; i < NB; i++) g += g & hi[i];
    return g;
  }
};

// Shared-memory position of tile element l: the low bits (one 128-byte row) are XORed with the
// row number, so that the strided member accesses of a block on a low tile bit spread over all
// banks.  A permutation within each row; identity for tiles of one row.
template <class T>
__device__ __forceinline__ uint32_t sw(uint32_t l) {
  return sizeof(T) == 4 ? l ^ ((l >> 4) & 15u) : l ^ ((l >> 3) & 7u);
}

constexpr uint32_t kThreads = 256;  // threads per CTA of the stage and wave kernels

// Deposit the low bits of t at the positions pos[0..cnt) (ascending).
__device__ __forceinline__ uint64_t deposit(uint64_t t, const int* pos, int cnt) {
  uint64_t r = 0;
  for (int j = 0; j < cnt; j++) r |= ((t >> j) & 1ull) << pos[j];
  return r;
}

// Amplitudes a thread moves per batch in the tile and mirror stores (loads from shared memory in flight before
// the global stores).  The stores follow the sweeps in the same kernel, and larger batches raise the register
// allocation of the whole stage kernel (spilling in the sweeps): these are the largest batches, per precision,
// that leave the float-float stage kernels without spills and the others with the fewest.
template <class T> struct StoreBatch { static constexpr int io = 8, mirror = 2; };
template <> struct StoreBatch<df> { static constexpr int io = 2, mirror = 2; };
template <> struct StoreBatch<float> { static constexpr int io = 2, mirror = 4; };

// Move one tile between HBM and shared memory.  Local index l = tid + it * 256; its global offset
// is deposit(l, bits) = deposit(tid) + deposit(it * 256), the second advanced with the
// masked-increment identity next = ((x | ~M) + 1) & M.  Each thread moves its amplitudes in
// batches of StoreBatch<T>::io independent accesses (that many loads per thread in flight at once).
template <class T, bool LOAD>
__device__ __forceinline__ void tile_io(cx<T>* __restrict__ st, cx<T>* __restrict__ sm, uint64_t base64, const int* bits,
                                        int nbits) {
  const uint32_t size = 1u << nbits;
  const int lowbits = min(nbits, 8);  // blockDim == 256
  if (threadIdx.x >= size) return;
  // element offsets fit 32 bits (4^16 amplitudes at most)
  cx<T>* __restrict__ sb = st + base64;
  uint32_t lo = 0;
  for (int j = 0; j < lowbits; j++) lo |= ((threadIdx.x >> j) & 1u) << bits[j];
  uint32_t M = 0;
  for (int j = 8; j < nbits; j++) M |= 1u << bits[j];
  const int iters = nbits > 8 ? 1 << (nbits - 8) : 1;
  const uint32_t swt = sw<T>(threadIdx.x);
  uint32_t hi = 0;
  constexpr int K = StoreBatch<T>::io;
  for (int it0 = 0; it0 < iters; it0 += K) {
    cx<T> v[K];
    uint32_t h = hi;
    if (LOAD) {
#pragma unroll
      for (int k = 0; k < K; k++) {
        if (it0 + k < iters) v[k] = sb[lo + h];
        h = ((h | ~M) + 1u) & M;
      }
#pragma unroll
      for (int k = 0; k < K; k++)
        if (it0 + k < iters) sm[swt + 256u * (uint32_t)(it0 + k)] = v[k];
    } else {
#pragma unroll
      for (int k = 0; k < K; k++)
        if (it0 + k < iters) v[k] = sm[swt + 256u * (uint32_t)(it0 + k)];
#pragma unroll
      for (int k = 0; k < K; k++) {
        if (it0 + k < iters) sb[lo + h] = v[k];
        h = ((h | ~M) + 1u) & M;
      }
    }
    hi = h;
  }
}

// Asynchronous tile load (cp.async): each thread issues all of its copies straight into shared memory
// (no register staging, so every copy of the tile is in flight at once), then waits for them.
template <class T>
__device__ __forceinline__ void tile_load_async(const cx<T>* __restrict__ st, cx<T>* __restrict__ sm, uint64_t base64,
                                                const int* bits, int nbits) {
  const uint32_t size = 1u << nbits;
  const int lowbits = min(nbits, 8);
  if (threadIdx.x >= size) return;
  const cx<T>* __restrict__ sb = st + base64;
  uint32_t lo = 0;
  for (int j = 0; j < lowbits; j++) lo |= ((threadIdx.x >> j) & 1u) << bits[j];
  uint32_t M = 0;
  for (int j = 8; j < nbits; j++) M |= 1u << bits[j];
  const int iters = nbits > 8 ? 1 << (nbits - 8) : 1;
  const uint32_t swt = sw<T>(threadIdx.x);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm) + swt * (uint32_t)sizeof(cx<T>);
  uint32_t hi = 0;
  for (int it = 0; it < iters; it++) {
    const uint32_t dst = sbase + 256u * (uint32_t)sizeof(cx<T>) * (uint32_t)it;
    const cx<T>* src = sb + (lo + hi);
    if (sizeof(T) == 4)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
    else
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    hi = ((hi | ~M) + 1u) & M;
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ---- Hermitian stages.  Tile u of a Hermitian stage is the u-th pair (R, C), R <= C, of row and column
// rest indices, ordered by C then R: C = floor((sqrt(8u + 1) - 1) / 2), R = u - C (C + 1) / 2.
__device__ __forceinline__ void tri_pair(uint64_t u, uint64_t& R, uint64_t& C) {
  uint64_t c = (uint64_t)((sqrt(8.0 * (double)u + 1.0) - 1.0) * 0.5);
  while (c > 0 && c * (c + 1) / 2 > u) c--;  // the FP64 root is off by at most one either way
  while ((c + 1) * (c + 2) / 2 <= u) c++;
  C = c;
  R = u - c * (c + 1) / 2;
}

// Tile-local bits of a Hermitian stage: l = i | j << h, i the row index and j the column index over the
// same h qubits.  The mirror store walks local bit order(k): row bits 0..r0-1 (distinct shared-memory banks
// across a quarter warp), then the column bits (the mirror's row bits, so contiguous DRAM runs), then the
// remaining row bits.
__device__ __forceinline__ int mirror_order(int k, int h, int r0) {
  return k < r0 ? k : (k < r0 + h ? h + (k - r0) : k - h);
}

// Offsets of the mirror store, computed once per stage from the stage's bits into shared memory: entries
// [0, 16) hold the tile-local offsets of the iteration bits (tile bits walked per iteration, beyond the 8 thread
// bits) and [16, 32) their mirror global offsets; entries 32 + t and 32 + 256 + t the tile-local and mirror global
// offsets of thread t's bits.  A Hermitian tile has at most 12 bits, so at most 16 iterations.  (Read from shared
// memory inside the tile loop, these offsets are not held in registers across the sweeps.)
constexpr int kMirrorIters = 16;
constexpr int kMirrorTable = 2 * kMirrorIters + 2 * 256;
__device__ __forceinline__ void mirror_table(uint32_t* s_mir, const int* bits, int nbits) {
  const int h = nbits >> 1, r0 = min(h, 3), lowbits = min(nbits, 8), hib = nbits - lowbits;
  const uint32_t t = threadIdx.x;
  if (t < (1u << hib) && t < (uint32_t)kMirrorIters) {
    uint32_t l = 0, g = 0;
    for (int e = 0; e < hib; e++)
      if (t >> e & 1u) {
        const int b = mirror_order(lowbits + e, h, r0);
        l |= 1u << b;
        g |= 1u << bits[b < h ? b + h : b - h];
      }
    s_mir[t] = l;
    s_mir[kMirrorIters + t] = g;
  }
  uint32_t l = 0, g = 0;
  for (int k = 0; k < lowbits; k++)
    if (t >> k & 1u) {
      const int b = mirror_order(k, h, r0);
      l |= 1u << b;
      g |= 1u << bits[b < h ? b + h : b - h];
    }
  s_mir[2 * kMirrorIters + t] = l;
  s_mir[2 * kMirrorIters + 256 + t] = g;
}

// Write the conjugate transpose of the tile in shared memory to its mirror tile at base64: element (i, j)
// goes to row j, column i.  A tile bit at local position b < h (row) is a column bit of the mirror,
// global position bits[b + h]; a column bit (b >= h) is a row bit of the mirror, bits[b - h].  Offsets from
// mirror_table.
template <class T>
__device__ __forceinline__ void tile_store_mirror(cx<T>* __restrict__ st, const cx<T>* __restrict__ sm, uint64_t base64,
                                                  int nbits, const uint32_t* __restrict__ s_mir) {
  const uint32_t size = 1u << nbits;
  if (threadIdx.x >= size) return;
  cx<T>* __restrict__ sb = st + base64;
  const uint32_t lt = s_mir[2 * kMirrorIters + threadIdx.x], gt = s_mir[2 * kMirrorIters + 256 + threadIdx.x];
  const int iters = 1 << (nbits - min(nbits, 8));
  constexpr int K = StoreBatch<T>::mirror;
  for (int it0 = 0; it0 < iters; it0 += K) {
    cx<T> v[K];
    uint32_t g[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (it0 + k < iters) {
        v[k] = sm[sw<T>(lt | s_mir[it0 + k])];
        v[k].y = -v[k].y;
        g[k] = gt | s_mir[kMirrorIters + it0 + k];
      }
    }
#pragma unroll
    for (int k = 0; k < K; k++)
      if (it0 + k < iters) sb[g[k]] = v[k];
  }
}

// Store a diagonal tile (R = C) of a Hermitian stage: the upper triangle (i < j) as computed, the lower one
// as its conjugate transpose and the diagonal with its imaginary part dropped, so that the stored state is
// exactly Hermitian (the mathematical result is; the two triangles differ only by rounding).
template <class T>
__device__ __forceinline__ void tile_store_diag(cx<T>* __restrict__ st, const cx<T>* __restrict__ sm, uint64_t base64,
                                                const int* bits, int nbits) {
  const uint32_t size = 1u << nbits, h = (uint32_t)nbits >> 1, hm = (1u << h) - 1u;
  cx<T>* __restrict__ sb = st + base64;
  for (uint32_t l = threadIdx.x; l < size; l += kThreads) {
    const uint32_t i = l & hm, j = l >> h;
    cx<T> v;
    if (i > j) {
      v = sm[sw<T>(j | i << h)];
      v.y = -v.y;
    } else {
      v = sm[sw<T>(l)];
      if (i == j) v.y = T(0.0);
    }
    uint32_t g = 0;
    for (int b = 0; b < nbits; b++) g |= ((l >> b) & 1u) << bits[b];
    sb[g] = v;
  }
}

// Structured arithmetic (coefficient flags, see compose_stage) for FP64 and float-float; complex64
// keeps straight-line FMAs.
// FP64 structured sweeps test a coefficient's complex case first (numeric.h, cmac_flag)
template <class T> constexpr bool kCplxFirst = std::is_same<T, double>::value;
template <class T> struct Structured { static constexpr bool value = true; };
template <> struct Structured<float> { static constexpr bool value = false; };

template <class T>
__device__ __forceinline__ void mac_s(cx<T>& acc, const cx<T>& c, int fl, const cx<T>& x) {
  if (Structured<T>::value) cmac_flag<T>(acc, c, fl, x);
  else cmac<T>(acc, c, x);
}
template <class T>
__device__ __forceinline__ cx<T> scale_s(cx<T> x, const cx<T>& f, int fl) {
  if (Structured<T>::value) {
    cscale_flag<T>(x, f, fl);
    return x;
  }
  return cmul<T>(x, f);
}

// ---- one operator, one sweep over the tile.  Each kind has its own loop with the operator's
// coefficients in registers (loaded once per sweep from shared memory); member s of a group is
// r | c << k over the operator's tile bits.  The XOR swizzle is linear: sw(base | off) =
// sw(base) ^ sw(off), so a member address costs one XOR.
template <class T, bool DIAG>
__device__ __forceinline__ void sweep1(cx<T>* __restrict__ sm, int nbits, const TileBlock& B,
                                       const cx<T>* __restrict__ c, const uint8_t* __restrict__ fl, uint32_t skip) {
  const uint32_t m1 = sw<T>(1u << B.lbit[0]), m2 = sw<T>(1u << B.lbit[1]);
  const uint32_t ng = 1u << (nbits - 2);
  cx<T> S[DIAG ? 4 : 16];
  int F[DIAG ? 4 : 16];
#pragma unroll
  for (int i = 0; i < (DIAG ? 4 : 16); i++) {
    S[i] = c[i];
    F[i] = Structured<T>::value ? (int)fl[i] : FL_CPLX;
  }
  const Inserter<2> ins(B.lsorted);
  #pragma unroll 2
  for (uint32_t g = threadIdx.x; g < ng; g += kThreads) {
    const uint32_t b = sw<T>(ins(g));
    const uint32_t a[4] = {b, b ^ m1, b ^ m2, b ^ m1 ^ m2};
    cx<T> x[4];
    if (DIAG) {  // members with factor 1 are left as they are
#pragma unroll
      for (int t = 0; t < 4; t++)
        if (!(skip >> t & 1u)) x[t] = sm[a[t]];
#pragma unroll
      for (int t = 0; t < 4; t++)
        if (!(skip >> t & 1u)) sm[a[t]] = scale_s<T>(x[t], S[t], F[t]);
    } else {
#pragma unroll
      for (int t = 0; t < 4; t++) x[t] = sm[a[t]];
#pragma unroll
      for (int t = 0; t < 4; t++) {
        cx<T> y;
        y.x = 0; y.y = 0;
#pragma unroll
        for (int u = 0; u < 4; u++) mac_s<T>(y, S[t * 4 + u], F[t * 4 + u], x[u]);
        sm[a[t]] = y;
      }
    }
  }
}

// kind: BK_DIAG2, BK_UNI2 (U A U^dagger on the 4x4 block A[r][c] = member r | c << 2) or BK_SUP2
template <class T, int KIND>
__device__ __forceinline__ void sweep2(cx<T>* __restrict__ sm, int nbits, const TileBlock& B,
                                       const cx<T>* __restrict__ c, const uint8_t* __restrict__ fl, uint32_t skip) {
  uint32_t soff[16];
#pragma unroll
  for (int s = 0; s < 16; s++) {
    uint32_t o = 0;
#pragma unroll
    for (int j = 0; j < 4; j++)
      if (s >> j & 1) o |= 1u << B.lbit[j];
    soff[s] = sw<T>(o);
  }
  const uint32_t ng = 1u << (nbits - 4);
  cx<T> u[KIND == BK_SUP2 ? 1 : 16];
  int F[KIND == BK_SUP2 ? 1 : 16];
  if (KIND != BK_SUP2) {
#pragma unroll
    for (int i = 0; i < 16; i++) {
      u[i] = c[i];
      F[i] = Structured<T>::value ? (int)fl[i] : FL_CPLX;
    }
  }
  const Inserter<4> ins(B.lsorted);
  if constexpr (KIND == BK_DIAG2) {  // members with factor 1 are left as they are
  #pragma unroll 1
    for (uint32_t g = threadIdx.x; g < ng; g += kThreads) {
      const uint32_t b = sw<T>(ins(g));
#pragma unroll
      for (int s = 0; s < 16; s++)
        if (!(skip >> s & 1u)) sm[b ^ soff[s]] = scale_s<T>(sm[b ^ soff[s]], u[s], F[s]);
    }
  } else {
  #pragma unroll 1
  for (uint32_t g = threadIdx.x; g < ng; g += kThreads) {
    const uint32_t b = sw<T>(ins(g));
    cx<T> x[16];
#pragma unroll
    for (int s = 0; s < 16; s++) x[s] = sm[b ^ soff[s]];
    if (KIND == BK_UNI2) {
#pragma unroll
      for (int cc = 0; cc < 4; cc++) {  // columns: A[:,c] <- U A[:,c]
        cx<T> t[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
          t[r].x = 0; t[r].y = 0;
#pragma unroll
          for (int m = 0; m < 4; m++) mac_s<T>(t[r], u[r * 4 + m], F[r * 4 + m], x[m | (cc << 2)]);
        }
#pragma unroll
        for (int r = 0; r < 4; r++) x[r | (cc << 2)] = t[r];
      }
#pragma unroll
      for (int r = 0; r < 4; r++) {  // rows: A[r,:] <- A[r,:] U^dagger
        cx<T> t[4];
#pragma unroll
        for (int cc = 0; cc < 4; cc++) {
          t[cc].x = 0; t[cc].y = 0;
#pragma unroll
          for (int m = 0; m < 4; m++) {
            cx<T> uc = u[cc * 4 + m];
            uc.y = -uc.y;
            mac_s<T>(t[cc], uc, F[cc * 4 + m], x[r | (m << 2)]);
          }
        }
#pragma unroll
        for (int cc = 0; cc < 4; cc++) sm[b ^ soff[r | (cc << 2)]] = t[cc];
      }
    } else {
#pragma unroll 1
      for (int i = 0; i < 16; i++) {
        cx<T> y;
        y.x = 0; y.y = 0;
#pragma unroll
        for (int j = 0; j < 16; j++) mac_s<T>(y, c[i * 16 + j], Structured<T>::value ? (int)fl[i * 16 + j] : FL_CPLX, x[j]);
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < 4; j++)
          if (i >> j & 1) o |= 1u << B.lbit[j];
        sm[b ^ sw<T>(o)] = y;
      }
    }
  }
}  // KIND != BK_DIAG2
}

// ---- FP64 and float-float sweeps.  Their arithmetic (FP64 at 1/58 of the FP32 rate; a float-float
// multiply-add is about 15 FP32 instructions) dwarfs a shared-memory read, so each term reads its
// coefficient and structure flag from shared memory (a broadcast: every thread reads the same word)
// instead of holding all of them in registers, and a two-qubit unitary U A U^dagger is applied as a
// column pass and a row pass over 4-member vectors.  This keeps the live state to a few amplitudes per
// thread, so that two CTAs (16 warps) fit on an SM to hide the long dependency chains.  A one-qubit sweep
// takes two groups per iteration when the tile has at least two per thread: two independent chains per
// coefficient, and one coefficient read for both.
template <class T>
__device__ __forceinline__ void sweep1_s(cx<T>* __restrict__ sm, int nbits, const TileBlock& B, const cx<T>* __restrict__ c,
                                         const uint8_t* __restrict__ fl, uint32_t skip, bool diag) {
  const uint32_t m1 = sw<T>(1u << B.lbit[0]), m2 = sw<T>(1u << B.lbit[1]);
  const uint32_t ng = 1u << (nbits - 2);
  const Inserter<2> ins(B.lsorted);
  if (ng >= 2 * kThreads) {  // two groups per iteration: each coefficient read serves both
    for (uint32_t g = threadIdx.x; g < ng; g += 2 * kThreads) {
      const uint32_t b0 = sw<T>(ins(g)), b1 = sw<T>(ins(g + kThreads));
      const uint32_t a0[4] = {b0, b0 ^ m1, b0 ^ m2, b0 ^ m1 ^ m2};
      const uint32_t a1[4] = {b1, b1 ^ m1, b1 ^ m2, b1 ^ m1 ^ m2};
      if (diag) {
#pragma unroll
        for (int t = 0; t < 4; t++)
          if (!(skip >> t & 1u)) {
            cx<T> x0 = sm[a0[t]], x1 = sm[a1[t]];
            const cx<T> ct = c[t];
            const int ft = fl[t];
            cscale_flag<T, kCplxFirst<T>>(x0, ct, ft);
            cscale_flag<T, kCplxFirst<T>>(x1, ct, ft);
            sm[a0[t]] = x0;
            sm[a1[t]] = x1;
          }
      } else {
        cx<T> x0[4], x1[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
          x0[t] = sm[a0[t]];
          x1[t] = sm[a1[t]];
        }
#pragma unroll 1
        for (int t = 0; t < 4; t++) {
          CAcc<T> y0, y1;
          y0.zero();
          y1.zero();
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const cx<T> cu = c[t * 4 + u];
            const int fu = fl[t * 4 + u];
            y0.mac(cu, fu, x0[u]);
            y1.mac(cu, fu, x1[u]);
          }
          const uint32_t o = ((t & 1) ? m1 : 0u) ^ ((t & 2) ? m2 : 0u);
          sm[b0 ^ o] = y0.get();
          sm[b1 ^ o] = y1.get();
        }
      }
    }
    return;
  }
  for (uint32_t g = threadIdx.x; g < ng; g += kThreads) {
    const uint32_t b = sw<T>(ins(g));
    const uint32_t a[4] = {b, b ^ m1, b ^ m2, b ^ m1 ^ m2};
    if (diag) {
#pragma unroll
      for (int t = 0; t < 4; t++)
        if (!(skip >> t & 1u)) {
          cx<T> x = sm[a[t]];
          cscale_flag<T, kCplxFirst<T>>(x, c[t], fl[t]);
          sm[a[t]] = x;
        }
    } else {
      cx<T> x[4];
#pragma unroll
      for (int t = 0; t < 4; t++) x[t] = sm[a[t]];
#pragma unroll
      for (int t = 0; t < 4; t++) {
        CAcc<T> y;
        y.zero();
#pragma unroll
        for (int u = 0; u < 4; u++) y.mac(c[t * 4 + u], fl[t * 4 + u], x[u]);
        sm[a[t]] = y.get();
      }
    }
  }
}

template <class T, bool SUP2>
__device__ __forceinline__ void sweep2_s(cx<T>* __restrict__ sm, int nbits, const TileBlock& B, const cx<T>* __restrict__ c,
                                         const uint8_t* __restrict__ fl, uint32_t skip, int kind) {
  uint32_t soff[16];
#pragma unroll
  for (int s = 0; s < 16; s++) {
    uint32_t o = 0;
#pragma unroll
    for (int j = 0; j < 4; j++)
      if (s >> j & 1) o |= 1u << B.lbit[j];
    soff[s] = sw<T>(o);
  }
  const uint32_t ng = 1u << (nbits - 4);
  const Inserter<4> ins(B.lsorted);
  for (uint32_t g = threadIdx.x; g < ng; g += kThreads) {
    const uint32_t b = sw<T>(ins(g));
    if (kind == BK_DIAG2) {  // rolled, as the unitary's loops below
#pragma unroll 1
      for (int s = 0; s < 16; s++)
        if (!(skip >> s & 1u)) {
          const uint32_t o = ((s & 1) ? soff[1] : 0u) ^ ((s & 2) ? soff[2] : 0u) ^ ((s & 4) ? soff[4] : 0u) ^
                             ((s & 8) ? soff[8] : 0u);
          cx<T> x = sm[b ^ o];
          cscale_flag<T, kCplxFirst<T>>(x, c[s], fl[s]);
          sm[b ^ o] = x;
        }
    } else if (kind == BK_UNI2) {
      // columns: A[:, cc] <- U A[:, cc]; then rows: A[r, :] <- A[r, :] U^dagger (A[r][cc] = member r | cc << 2).
      // The loops stay rolled (one copy of a 4-term body instead of 32 terms): the stage kernel holds every
      // sweep inline, and its leading stall was instruction fetch.  The swizzle is XOR-linear, so a member's
      // offset is the XOR of its bits' offsets: soff[r | cc << 2] = soff[r] ^ soff[cc << 2].
#pragma unroll 1
      for (int cc = 0; cc < 4; cc += 2) {  // two columns per iteration
        const uint32_t oc0 = (cc & 2) ? soff[8] : 0u, oc1 = oc0 ^ soff[4];
        cx<T> x0[4], x1[4];
#pragma unroll
        for (int m = 0; m < 4; m++) {
          x0[m] = sm[b ^ soff[m] ^ oc0];
          x1[m] = sm[b ^ soff[m] ^ oc1];
        }
#pragma unroll 1
        for (int r = 0; r < 4; r++) {
          CAcc<T> t0, t1;
          t0.zero();
          t1.zero();
#pragma unroll
          for (int m = 0; m < 4; m++) {
            const cx<T> cu = c[r * 4 + m];
            const int fu = fl[r * 4 + m];
            t0.mac(cu, fu, x0[m]);
            t1.mac(cu, fu, x1[m]);
          }
          const uint32_t orr = ((r & 1) ? soff[1] : 0u) ^ ((r & 2) ? soff[2] : 0u);
          sm[b ^ orr ^ oc0] = t0.get();
          sm[b ^ orr ^ oc1] = t1.get();
        }
      }
#pragma unroll 1
      for (int r = 0; r < 4; r += 2) {  // two rows per iteration
        const uint32_t or0 = (r & 2) ? soff[2] : 0u, or1 = or0 ^ soff[1];
        cx<T> x0[4], x1[4];
#pragma unroll
        for (int m = 0; m < 4; m++) {
          x0[m] = sm[b ^ or0 ^ soff[m << 2]];
          x1[m] = sm[b ^ or1 ^ soff[m << 2]];
        }
#pragma unroll 1
        for (int cc = 0; cc < 4; cc++) {
          CAcc<T> t0, t1;
          t0.zero();
          t1.zero();
#pragma unroll
          for (int m = 0; m < 4; m++) {
            cx<T> uc = c[cc * 4 + m];
            uc.y = -uc.y;
            const int fu = fl[cc * 4 + m];
            t0.mac(uc, fu, x0[m]);
            t1.mac(uc, fu, x1[m]);
          }
          const uint32_t oc = ((cc & 1) ? soff[4] : 0u) ^ ((cc & 2) ? soff[8] : 0u);
          sm[b ^ or0 ^ oc] = t0.get();
          sm[b ^ or1 ^ oc] = t1.get();
        }
      }
    } else if constexpr (SUP2) {
      cx<T> x[16];
#pragma unroll
      for (int s = 0; s < 16; s++) x[s] = sm[b ^ soff[s]];
#pragma unroll 1
      for (int i = 0; i < 16; i++) {
        CAcc<T> y;
        y.zero();
#pragma unroll
        for (int j = 0; j < 16; j++) y.mac(c[i * 16 + j], fl[i * 16 + j], x[j]);
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < 4; j++)
          if (i >> j & 1) o |= 1u << B.lbit[j];
        sm[b ^ sw<T>(o)] = y.get();
      }
    }
  }
}

// Apply the stage's operators (one block each) to the tile, one sweep per operator.  SUP2 = false leaves
// out the dense two-qubit superoperator sweep, whose 16 amplitudes in registers would otherwise set the
// register allocation (and the spills) of the whole stage kernel in FP64 and float-float; the host picks
// that instantiation for stages without such a block.
// blocks[0 .. be - bb) are the stage's block descriptors (in shared memory).
template <class T, bool SUP2 = true>
__device__ __forceinline__ void tile_blocks(cx<T>* __restrict__ sm, const cx<T>* __restrict__ csm,
                                            const uint8_t* __restrict__ fsm, int nbits,
                                            const TileBlock* __restrict__ blocks, int bb, int be,
                                            const BlockOp* __restrict__ sops, int op0) {
  for (int b = bb; b < be; b++) {
    const TileBlock B = blocks[b - bb];
    const BlockOp bo = sops[B.op_begin - op0];
    const cx<T>* c = csm + bo.coef;
    const uint8_t* f = fsm + bo.coef;
    if constexpr (Structured<T>::value) {
      if (bo.kind == BK_DIAG_A || bo.kind == BK_SUP1_A) sweep1_s<T>(sm, nbits, B, c, f, bo.skip, bo.kind == BK_DIAG_A);
      else sweep2_s<T, SUP2>(sm, nbits, B, c, f, bo.skip, bo.kind);
      __syncthreads();
      continue;
    }
    switch (bo.kind) {
      case BK_DIAG_A: sweep1<T, true>(sm, nbits, B, c, f, bo.skip); break;
      case BK_SUP1_A: sweep1<T, false>(sm, nbits, B, c, f, 0u); break;
      case BK_DIAG2: sweep2<T, BK_DIAG2>(sm, nbits, B, c, f, bo.skip); break;
      case BK_UNI2: sweep2<T, BK_UNI2>(sm, nbits, B, c, f, 0u); break;
      default: sweep2<T, BK_SUP2>(sm, nbits, B, c, f, 0u); break;
    }
    __syncthreads();
  }
}

// Tile index of work item u: u itself, or in a Hermitian stage the tile (R, C), t = R | C << m, of group
// u >> 2b (the pair (R_h, C_h) of tri_pair) and item u & (4^b - 1) (R_l | C_l << b), R = R_l | R_h << b and
// C = C_l | C_h << b.  Returns 0 for a general tile, 1 for a diagonal tile of a Hermitian stage, 2 for an
// off-diagonal one (whose mirror tile index C | R << m goes to *tm), -1 for an item with nothing to do.
__device__ __forceinline__ int tile_of(uint64_t u, bool herm, int nrest, uint64_t* t, uint64_t* tm) {
  if (!herm) {
    *t = u;
    return 0;
  }
  const int m = nrest >> 1, b = herm_group_bits(nrest);
  uint64_t Rh, Ch;
  tri_pair(u >> (2 * b), Rh, Ch);
  const uint64_t w = u & ((1ull << (2 * b)) - 1), Rl = w & ((1ull << b) - 1), Cl = w >> b;
  if (Rh == Ch && Rl > Cl) return -1;
  const uint64_t R = Rl | Rh << b, C = Cl | Ch << b;
  *t = R | C << m;
  *tm = C | R << m;
  return R == C ? 1 : 2;
}

// One tile of a stage: load, apply the stage's blocks, store (and, in a Hermitian stage, the mirror tile or the
// symmetrised diagonal tile).  The tile's offsets and kind pass from before the sweeps to the store phase through
// shared memory (s_io, written by thread 0 and read after the load's barrier), so that nothing besides the
// sweeps' own values is held in registers across them.
template <class T, bool SUP2>
__device__ __forceinline__ void stage_tile(cx<T>* __restrict__ st, cx<T>* __restrict__ sm, const cx<T>* __restrict__ csm,
                                           const uint8_t* __restrict__ fsm, const int* s_bits, int nbits,
                                           const int* s_rest, int nrest, bool herm, uint64_t u,
                                           const TileBlock* __restrict__ blocks, int bb, int be,
                                           const BlockOp* __restrict__ sops, int op0, const uint32_t* s_mir,
                                           uint64_t* s_io) {
  {
    uint64_t t = 0, tm = 0;
    const int kind = tile_of(u, herm, nrest, &t, &tm);
    if (kind < 0) return;  // uniform across the CTA
    const uint64_t base = deposit(t, s_rest, nrest);
    if (threadIdx.x == 0) {
      s_io[0] = base;
      s_io[1] = kind == 2 ? deposit(tm, s_rest, nrest) : 0;
      s_io[2] = (uint64_t)kind;
    }
    tile_load_async<T>(st, sm, base, s_bits, nbits);
  }
  __syncthreads();
  tile_blocks<T, SUP2>(sm, csm, fsm, nbits, blocks, bb, be, sops, op0);
  const uint64_t base = s_io[0];
  const int kind = (int)s_io[2];
  if (kind == 1) {
    tile_store_diag<T>(st, sm, base, s_bits, nbits);
  } else {
    tile_io<T, false>(st, sm, base, s_bits, nbits);
    if (kind == 2) tile_store_mirror<T>(st, sm, s_io[1], nbits, s_mir);
  }
  __syncthreads();
}

template <class T>
__device__ __forceinline__ void stage_coefs(cx<T>* __restrict__ csm, const cx<T>* __restrict__ coef,
                                            uint8_t* __restrict__ fsm, const uint8_t* __restrict__ flag, int cb, int ce,
                                            BlockOp* __restrict__ sops, const BlockOp* __restrict__ bops, int ob,
                                            int oe) {
  for (int i = threadIdx.x; i < ce - cb; i += kThreads) {
    csm[i] = coef[cb + i];
    fsm[i] = flag[cb + i];
  }
  for (int i = threadIdx.x; i < oe - ob; i += kThreads) sops[i] = bops[ob + i];
}

template <class T, bool SUP2>
__global__ void __launch_bounds__(256, 2) k_stage(cx<T>* __restrict__ st, const StageDesc S,
                                                                       const TileBlock* __restrict__ blocks,
                                                                       const BlockOp* __restrict__ bops,
                                                                       const cx<T>* __restrict__ coef,
                                                                       const uint8_t* __restrict__ flag) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<T>* csm = reinterpret_cast<cx<T>*>(smraw);
  cx<T>* sm = csm + kCoefCap;
  __shared__ int s_bits[kMaxTileBits];
  __shared__ int s_rest[2 * VQD_MAX_QUBITS];
  if (threadIdx.x < kMaxTileBits) s_bits[threadIdx.x] = S.bits[threadIdx.x];
  if (threadIdx.x < 2 * VQD_MAX_QUBITS) s_rest[threadIdx.x] = S.rest[threadIdx.x];
  const int nbits = S.nbits, nrest = S.nrest, bb = S.block_begin, be = S.block_end;
  BlockOp* sops = reinterpret_cast<BlockOp*>(sm + (1u << nbits));
  uint8_t* fsm = reinterpret_cast<uint8_t*>(sops + kOpCap);
  __shared__ uint32_t s_mir[kMirrorTable];
  __shared__ uint64_t s_io[3];
  __shared__ TileBlock s_blk[kBlockCap];  // the stage's block descriptors, read by every thread for every tile
  stage_coefs<T>(csm, coef, fsm, flag, S.coef_begin, S.coef_end, sops, bops, S.op_begin, S.op_end);
  for (int i = threadIdx.x; i < be - bb && i < kBlockCap; i += kThreads) s_blk[i] = blocks[bb + i];
  __syncthreads();
  if (S.herm) {
    mirror_table(s_mir, s_bits, nbits);
    __syncthreads();
  }
  const uint64_t ntiles = stage_work_tiles(S);
  for (uint64_t u = blockIdx.x; u < ntiles; u += gridDim.x)
    stage_tile<T, SUP2>(st, sm, csm, fsm, s_bits, nbits, s_rest, nrest, S.herm != 0, u, s_blk, bb, be, sops,
                        S.op_begin, s_mir, s_io);
}

// One wave of the batched path: CTAs take (instance, stage, tile chunk) items from an atomic
// queue; a CTA restages coefficients and operator descriptors only when its next item belongs to
// another stage.  Items of one wave never depend on each other, so no CTA waits for another.
template <class T>
__global__ void __launch_bounds__(256, 2) k_wave(cx<T>* __restrict__ all,
                                                                      const BatchInst* __restrict__ inst,
                                                                      const StageDesc* __restrict__ stages,
                                                                      const TileBlock* __restrict__ blocks,
                                                                      const BlockOp* __restrict__ bops,
                                                                      const cx<T>* __restrict__ coef,
                                                                      const uint8_t* __restrict__ flag,
                                                                      const WaveItem* __restrict__ items, int nitems,
                                                                      int* __restrict__ counter, int max_bits) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<T>* csm = reinterpret_cast<cx<T>*>(smraw);
  cx<T>* sm = csm + kCoefCap;
  BlockOp* sops = reinterpret_cast<BlockOp*>(sm + (1u << max_bits));
  uint8_t* fsm = reinterpret_cast<uint8_t*>(sops + kOpCap);
  __shared__ int item;
  __shared__ int s_bits[kMaxTileBits];
  __shared__ int s_rest[2 * VQD_MAX_QUBITS];
  __shared__ uint32_t s_mir[kMirrorTable];
  __shared__ uint64_t s_io[3];
  __shared__ TileBlock s_blk[kBlockCap];
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int i = item;
    __syncthreads();  // every thread has read `item` before thread 0 may overwrite it
    if (i >= nitems) break;
    const WaveItem W = items[i];
    const StageDesc& S = stages[W.stage];
    if (W.stage != cur) {
      if (threadIdx.x < kMaxTileBits) s_bits[threadIdx.x] = S.bits[threadIdx.x];
      if (threadIdx.x < 2 * VQD_MAX_QUBITS) s_rest[threadIdx.x] = S.rest[threadIdx.x];
      stage_coefs<T>(csm, coef, fsm, flag, S.coef_begin, S.coef_end, sops, bops, S.op_begin, S.op_end);
      for (int i = threadIdx.x; i < S.block_end - S.block_begin && i < kBlockCap; i += kThreads)
        s_blk[i] = blocks[S.block_begin + i];
      __syncthreads();
      if (S.herm) {
        mirror_table(s_mir, s_bits, S.nbits);
        __syncthreads();
      }
      cur = W.stage;
    }
    cx<T>* st = all + inst[W.inst].offset_amps;
    const int nbits = S.nbits, nrest = S.nrest, op0 = S.op_begin;
    const bool herm = S.herm != 0;
    for (uint32_t t = W.tile_begin; t < W.tile_begin + W.tile_count; t++)
      stage_tile<T, true>(st, sm, csm, fsm, s_bits, nbits, s_rest, nrest, herm, t, s_blk, S.block_begin,
                          S.block_end, sops, op0, s_mir, s_io);
  }
}

}  // namespace dev

// ================================================================== host side
using namespace dev;

static void grow(void** p, size_t* cap, size_t need) {
  if (need <= *cap) return;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(p, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(VQD_ENOMEM, std::string("fused plan allocation: ") + cudaGetErrorString(e));
  }
  *cap = need;
}

static void check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(VQD_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

void fused_cache_free(FusedCache& c) {
  for (void* p : {c.d_blocks, c.d_ops, c.d_coef, c.d_flag, c.d_stages, c.d_inst, c.d_items, (void*)c.d_counter})
    if (p) cudaFree(p);
  c = FusedCache();
}

template <class T>
static void upload_common(FusedCache& c, const FusedPlan& p, cudaStream_t s) {
  // The host vectors are converted into a temporary buffer; the copy is synchronised before the
  // buffer goes out of scope.
  std::vector<cx<T>> cf(p.coef.size());
  for (size_t i = 0; i < p.coef.size(); i++) {
    cf[i].x = (T)p.coef[i].real();
    cf[i].y = (T)p.coef[i].imag();
  }
  grow(&c.d_blocks, &c.blocks_cap, std::max<size_t>(1, p.blocks.size()) * sizeof(TileBlock));
  grow(&c.d_ops, &c.ops_cap, std::max<size_t>(1, p.ops.size()) * sizeof(BlockOp));
  grow(&c.d_coef, &c.coef_cap, std::max<size_t>(1, cf.size()) * sizeof(cx<T>));
  grow(&c.d_flag, &c.flag_cap, std::max<size_t>(1, p.flag.size()));
  grow(&c.d_stages, &c.stages_cap, std::max<size_t>(1, p.stages.size()) * sizeof(StageDesc));
  if (!p.blocks.empty())
    check(cudaMemcpyAsync(c.d_blocks, p.blocks.data(), p.blocks.size() * sizeof(TileBlock), cudaMemcpyHostToDevice, s),
          "upload blocks");
  if (!p.ops.empty())
    check(cudaMemcpyAsync(c.d_ops, p.ops.data(), p.ops.size() * sizeof(BlockOp), cudaMemcpyHostToDevice, s), "upload ops");
  if (!cf.empty())
    check(cudaMemcpyAsync(c.d_coef, cf.data(), cf.size() * sizeof(cx<T>), cudaMemcpyHostToDevice, s), "upload coefficients");
  if (!p.flag.empty())
    check(cudaMemcpyAsync(c.d_flag, p.flag.data(), p.flag.size(), cudaMemcpyHostToDevice, s), "upload coefficient flags");
  if (!p.stages.empty())
    check(cudaMemcpyAsync(c.d_stages, p.stages.data(), p.stages.size() * sizeof(StageDesc), cudaMemcpyHostToDevice, s),
          "upload stages");
  check(cudaStreamSynchronize(s), "upload plan");
}

void upload_plan(FusedCache& c, const FusedPlan& p, int prec, cudaStream_t s) {
  if (prec == VQD_F32) upload_common<float>(c, p, s);
  else if (prec == VQD_F32_SPLIT) upload_common<df>(c, p, s);
  else upload_common<double>(c, p, s);
}

template <class K>
static unsigned persistent_grid(K kernel, size_t smem, uint64_t work) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess || per_sm <= 0) per_sm = 1;
  uint64_t full = (uint64_t)per_sm * num_sms();
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(full, work));
}

template <class T>
static size_t stage_smem(int nbits) {
  return ((size_t)kCoefCap + ((size_t)1 << nbits)) * sizeof(cx<T>) + (size_t)kOpCap * sizeof(BlockOp) + (size_t)kCoefCap;
}

template <class T, bool SUP2>
static cudaError_t stage_kt(FusedCache& c, const StageDesc& S, void* state, cudaStream_t s) {
  const size_t smem = stage_smem<T>(S.nbits);
  cudaError_t e = cudaFuncSetAttribute(k_stage<T, SUP2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  unsigned grid = persistent_grid(k_stage<T, SUP2>, smem, stage_work_tiles(S));
  k_stage<T, SUP2><<<grid, 256, smem, s>>>((cx<T>*)state, S, (const TileBlock*)c.d_blocks, (const BlockOp*)c.d_ops,
                                           (const cx<T>*)c.d_coef, (const uint8_t*)c.d_flag);
  return cudaGetLastError();
}

template <class T>
static cudaError_t stage_t(FusedCache& c, const FusedPlan& p, int stage, void* state, cudaStream_t s) {
  const StageDesc& S = p.stages[stage];
  bool sup2 = !Structured<T>::value;  // complex64 keeps one instantiation
  for (int o = S.op_begin; o < S.op_end && !sup2; o++) sup2 = p.ops[o].kind == BK_SUP2;
  return sup2 ? stage_kt<T, true>(c, S, state, s) : stage_kt<T, false>(c, S, state, s);
}

cudaError_t launch_stage(FusedCache& c, const FusedPlan& p, int stage, int prec, void* state, int n, cudaStream_t s) {
  (void)n;
  if (prec == VQD_F32) return stage_t<float>(c, p, stage, state, s);
  if (prec == VQD_F32_SPLIT) return stage_t<df>(c, p, stage, state, s);
  return stage_t<double>(c, p, stage, state, s);
}

void upload_batch(FusedCache& c, const BatchPlan& p, int prec, cudaStream_t s) {
  upload_plan(c, p.all, prec, s);
  grow(&c.d_inst, &c.inst_cap, std::max<size_t>(1, p.inst.size()) * sizeof(BatchInst));
  grow(&c.d_items, &c.items_cap, std::max<size_t>(1, p.items.size()) * sizeof(WaveItem));
  grow((void**)&c.d_counter, &c.counter_cap, std::max<size_t>(1, p.wave_begin.size()) * sizeof(int));
  check(cudaMemcpyAsync(c.d_inst, p.inst.data(), p.inst.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, s),
        "upload instances");
  if (!p.items.empty())
    check(cudaMemcpyAsync(c.d_items, p.items.data(), p.items.size() * sizeof(WaveItem), cudaMemcpyHostToDevice, s),
          "upload wave items");
  check(cudaStreamSynchronize(s), "upload batch");
}

template <class T>
static cudaError_t batch_t(FusedCache& c, const BatchPlan& p, void* base, cudaStream_t s) {
  const int mb = std::max(1, p.all.max_bits);
  const size_t smem = stage_smem<T>(mb);
  cudaError_t e = cudaFuncSetAttribute(k_wave<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nw = (int)p.wave_begin.size() - 1;
  if (nw <= 0) return cudaSuccess;
  e = cudaMemsetAsync(c.d_counter, 0, sizeof(int) * nw, s);
  if (e != cudaSuccess) return e;
  for (int w = 0; w < nw; w++) {
    const int b = p.wave_begin[w], cnt = p.wave_begin[w + 1] - b;
    unsigned grid = persistent_grid(k_wave<T>, smem, (uint64_t)cnt);
    k_wave<T><<<grid, 256, smem, s>>>((cx<T>*)base, (const BatchInst*)c.d_inst, (const StageDesc*)c.d_stages,
                                      (const TileBlock*)c.d_blocks, (const BlockOp*)c.d_ops, (const cx<T>*)c.d_coef,
                                      (const uint8_t*)c.d_flag, (const WaveItem*)c.d_items + b, cnt, c.d_counter + w, mb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_batch(FusedCache& c, const BatchPlan& p, int prec, void* base, cudaStream_t s) {
  if (prec == VQD_F32) return batch_t<float>(c, p, base, s);
  if (prec == VQD_F32_SPLIT) return batch_t<df>(c, p, base, s);
  return batch_t<double>(c, p, base, s);
}

}  // namespace vqd
