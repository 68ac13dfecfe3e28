// Fused path of libvqd: stages of operators applied to shared-memory tiles of the state.
//
// A stage owns a set Q of at most `fuse_qubits` qubits.  Its tile holds the 2^m amplitudes that
// share one assignment of every index bit outside B = {q, q + n : q in Q} u {low row bits}; the
// low row bits are carried along so that each tile is made of runs of >= 64 contiguous bytes
// (full DRAM sectors).  A CTA loads a tile once, applies every operator of the stage to it in
// shared memory, and stores it once: one pass over HBM per stage instead of one per operator.
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

namespace vqd {

int tile_bits_budget(int prec) { return prec == VQD_F32 ? 13 : 12; }  // 64 KB tiles
static int passenger_bits(int prec) { return prec == VQD_F32 ? 3 : 2; }  // 64-byte runs
static int default_fuse(int prec) { (void)prec; return 5; }

static int popc(uint32_t x) { return __builtin_popcount(x); }

static int stage_bit_count(uint32_t qmask, int L) {
  int c = 2 * popc(qmask);
  for (int b = 0; b < L; b++)
    if (!(qmask >> b & 1)) c++;
  return c;
}

// ---------------------------------------------------------------- composition inside a stage
// Operators of one stage are merged into composites acting on at most two qubits, in FP64: a run of
// operators whose qubits stay within one pair becomes a single 4^k x 4^k superoperator (or a
// 2^k x 2^k unitary when every member is unitary).  Open composites are kept on pairwise disjoint
// qubit sets; an operator that would join qubits of composites into more than two qubits first
// emits them.  Every qubit therefore sees its operators in program order.
struct Composite {
  int k = 0;
  int q[2] = {0, 0};
  bool unitary = true;
  std::vector<cd> m;
  double weight = 0;
};

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

static Op composite_to_op(const Composite& c) {
  Op o;
  o.k = c.k;
  o.q[0] = c.q[0];
  o.q[1] = c.q[1];
  o.unitary = c.unitary;
  o.m = c.m;
  o.weight = c.weight;
  return o;
}

static std::vector<Op> compose_stage(const std::vector<Op>& ops, const std::vector<int>& idx) {
  std::vector<Op> out;
  std::vector<Composite> open;
  for (int i : idx) {
    const Op& op = ops[i];
    std::vector<int> hit;
    int uq[4], nu = 0;
    for (int j = 0; j < op.k; j++) uq[nu++] = op.q[j];
    for (size_t x = 0; x < open.size(); x++) {
      bool inter = false;
      for (int a = 0; a < open[x].k; a++)
        for (int j = 0; j < op.k; j++)
          if (open[x].q[a] == op.q[j]) inter = true;
      if (!inter) continue;
      hit.push_back((int)x);
      for (int a = 0; a < open[x].k; a++) {
        bool seen = false;
        for (int u = 0; u < nu; u++)
          if (uq[u] == open[x].q[a]) seen = true;
        if (!seen && nu < 4) uq[nu++] = open[x].q[a];
      }
    }
    Composite c;
    if (nu <= 2) {  // merge the operator with every composite it touches
      c.k = nu;
      for (int u = 0; u < nu; u++) c.q[u] = uq[u];
      c.unitary = op.unitary;
      for (int x : hit) c.unitary = c.unitary && open[x].unitary;
      const int d = c.unitary ? (1 << nu) : (1 << (2 * nu));
      c.m.assign((size_t)d * d, 0.0);
      for (int a = 0; a < d; a++) c.m[a * d + a] = 1.0;
      for (int x : hit) {  // disjoint composites commute: their product in any order
        const Composite& h = open[x];
        std::vector<cd> hm = (c.unitary || !h.unitary) ? h.m : superop_from_unitary(h.k, h.m.data());
        c.m = matmul(embed_on(hm, c.unitary, h.k, h.q, nu, c.q), c.m, d);
        c.weight += h.weight;
      }
      std::vector<cd> om = (c.unitary || !op.unitary) ? op.m : superop_from_unitary(op.k, op.m.data());
      c.m = matmul(embed_on(om, c.unitary, op.k, op.q, nu, c.q), c.m, d);
      c.weight += op.weight;
    } else {  // emit what it touches and start afresh
      for (int x : hit) out.push_back(composite_to_op(open[x]));
      c.k = op.k;
      c.q[0] = op.q[0];
      c.q[1] = op.q[1];
      c.unitary = op.unitary;
      c.m = op.m;
      c.weight = op.weight;
    }
    for (int h = (int)hit.size() - 1; h >= 0; h--) open.erase(open.begin() + hit[h]);
    open.push_back(std::move(c));
  }
  for (const Composite& c : open) out.push_back(composite_to_op(c));
  return out;
}

static void build_stage(FusedPlan& plan, const std::vector<Op>& ops, const std::vector<int>& idx, uint32_t qmask,
                        int n, int prec, bool whole) {
  StageDesc sd;
  std::memset(&sd, 0, sizeof(sd));
  bool in_tile[2 * VQD_MAX_QUBITS] = {false};
  if (whole) {
    for (int b = 0; b < 2 * n; b++) in_tile[b] = true;
  } else {
    const int L = std::min(passenger_bits(prec), n);
    for (int b = 0; b < L; b++) in_tile[b] = true;
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
  sd.op_begin = (int)plan.ops.size();
  const std::vector<Op> merged = compose_stage(ops, idx);
  for (const Op& op : merged) {
    Pass p = classify(op);
    TileOp t;
    std::memset(&t, 0, sizeof(t));
    t.kind = p.kind;
    t.nb = 2 * op.k;
    for (int j = 0; j < op.k; j++) {
      t.lbit[j] = local[op.q[j]];
      t.lbit[j + op.k] = local[op.q[j] + n];
    }
    for (int j = 0; j < t.nb; j++)
      if (t.lbit[j] < 0) throw Error(VQD_EINVAL, "internal: operator outside its stage tile");
    for (int j = 0; j < t.nb; j++) t.lsorted[j] = t.lbit[j];
    std::sort(t.lsorted, t.lsorted + t.nb);
    t.coef = (int)plan.coef.size();
    t.ncoef = (int)p.coef.size();
    t.real = 1;
    for (const cd& c : p.coef)
      if (c.imag() != 0.0) t.real = 0;
    plan.coef.insert(plan.coef.end(), p.coef.begin(), p.coef.end());
    plan.ops.push_back(t);
    sd.weight += op.weight;
  }
  sd.op_end = (int)plan.ops.size();
  plan.max_bits = std::max(plan.max_bits, sd.nbits);
  plan.stages.push_back(sd);
}

FusedPlan plan_fused(const std::vector<Op>& ops, int n, int prec, int fuse_qubits) {
  FusedPlan plan;
  const int budget = tile_bits_budget(prec);
  const int L = std::min(passenger_bits(prec), n);
  int f = fuse_qubits <= 0 ? default_fuse(prec) : fuse_qubits;
  if (f < 2 || f > VQD_MAX_FUSE) throw Error(VQD_EINVAL, "fuse_qubits must be in 2..6");
  if (ops.empty()) return plan;
  if (2 * n <= budget) {  // the whole state is one tile: one stage holds every operator
    std::vector<int> all(ops.size());
    for (size_t i = 0; i < ops.size(); i++) all[i] = (int)i;
    build_stage(plan, ops, all, (1u << n) - 1, n, prec, true);
    return plan;
  }
  const uint32_t full = (1u << n) - 1;
  const size_t kWindow = 1024;
  std::vector<int> remaining(ops.size());
  for (size_t i = 0; i < ops.size(); i++) remaining[i] = (int)i;
  size_t head = 0;  // remaining[head..] is the unplanned suffix
  std::vector<int> stage, deferred;
  while (head < remaining.size()) {
    stage.clear();
    deferred.clear();
    uint32_t q = 0, dmask = 0;
    size_t i = head;
    for (; i < remaining.size() && i - head < kWindow; i++) {
      const Op& op = ops[remaining[i]];
      uint32_t m = 0;
      for (int j = 0; j < op.k; j++) m |= 1u << op.q[j];
      if (m & dmask) {
        deferred.push_back(remaining[i]);
        dmask |= m;
      } else {
        uint32_t q2 = q | m;
        if (popc(q2) <= f && stage_bit_count(q2, L) <= budget) {
          q = q2;
          stage.push_back(remaining[i]);
        } else {
          deferred.push_back(remaining[i]);
          dmask |= m;
        }
      }
      if ((dmask | q) == full && dmask == full) {
        i++;
        break;
      }
    }
    build_stage(plan, ops, stage, q, n, prec, false);
    // new suffix: deferred operators (in order) followed by the unscanned rest
    size_t rest = remaining.size() - i;
    std::vector<int> next;
    next.reserve(deferred.size() + rest);
    next.insert(next.end(), deferred.begin(), deferred.end());
    next.insert(next.end(), remaining.begin() + i, remaining.end());
    remaining.swap(next);
    head = 0;
  }
  return plan;
}

BatchPlan plan_batch(const std::vector<std::vector<Op>>& lists, const std::vector<int>& n,
                     const std::vector<size_t>& byte_offsets, int prec, int fuse_qubits) {
  BatchPlan bp;
  const size_t esz = prec == VQD_F32 ? 8 : 16;
  bp.passes.assign(lists.size(), 0);
  for (size_t i = 0; i < lists.size(); i++) {
    FusedPlan p = plan_fused(lists[i], n[i], prec, fuse_qubits);
    BatchInst bi;
    bi.offset_amps = byte_offsets[i] / esz;
    bi.n = n[i];
    bi.stage_begin = (int)bp.all.stages.size();
    const int op0 = (int)bp.all.ops.size(), c0 = (int)bp.all.coef.size();
    for (StageDesc sd : p.stages) {
      sd.op_begin += op0;
      sd.op_end += op0;
      bp.all.stages.push_back(sd);
    }
    for (TileOp t : p.ops) {
      t.coef += c0;
      bp.all.ops.push_back(t);
    }
    bp.all.coef.insert(bp.all.coef.end(), p.coef.begin(), p.coef.end());
    bp.all.max_bits = std::max(bp.all.max_bits, p.max_bits);
    bi.stage_end = (int)bp.all.stages.size();
    bi.cost = std::ldexp(1.0, 2 * n[i]) * std::max<size_t>(1, p.stages.size());
    bp.passes[i] = (int)p.stages.size();
    bp.inst.push_back(bi);
  }
  std::stable_sort(bp.inst.begin(), bp.inst.end(), [](const BatchInst& a, const BatchInst& b) { return a.cost > b.cost; });
  return bp;
}

// ================================================================== device side
namespace dev {

template <class T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };
template <class T> using cx = typename V2<T>::t;

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

template <int NB>
__device__ __forceinline__ uint32_t insert_zeros32(uint32_t g, const int* pos) {
#pragma unroll
  for (int i = 0; i < NB; i++) {
    const uint32_t lo = g & ((1u << pos[i]) - 1u);
    g = ((g >> pos[i]) << (pos[i] + 1)) | lo;
  }
  return g;
}

// Shared-memory position of tile element l: the low bits (one 128-byte row) are XORed with the
// row number, so that the strided member accesses of an operator on a low tile bit spread over
// all banks.  A permutation within each row; identity for tiles of one row.
template <class T>
__device__ __forceinline__ uint32_t sw(uint32_t l) {
  return sizeof(T) == 4 ? l ^ ((l >> 4) & 15u) : l ^ ((l >> 3) & 7u);
}

// Deposit the low bits of t at the positions pos[0..cnt) (ascending).
__device__ __forceinline__ uint64_t deposit(uint64_t t, const int* pos, int cnt) {
  uint64_t r = 0;
  for (int j = 0; j < cnt; j++) r |= ((t >> j) & 1ull) << pos[j];
  return r;
}

// Move one tile between HBM and shared memory.  Local index l = tid + it * blockDim; its global
// offset is deposit(l, bits) = deposit(tid) + deposit(it * blockDim), the second advanced with
// the masked-increment identity next = ((x | ~M) + 1) & M.
template <class T, bool LOAD>
__device__ __forceinline__ void tile_io(cx<T>* __restrict__ st, cx<T>* __restrict__ sm, uint64_t base, const int* bits,
                                        int nbits) {
  const uint32_t size = 1u << nbits;
  const int lowbits = min(nbits, 8);  // blockDim == 256
  if (threadIdx.x >= size) return;
  uint64_t lo = 0;
  for (int j = 0; j < lowbits; j++) lo |= (uint64_t)((threadIdx.x >> j) & 1u) << bits[j];
  uint64_t M = 0;
  for (int j = 8; j < nbits; j++) M |= 1ull << bits[j];
  uint64_t hi = 0;
  for (uint32_t l = threadIdx.x; l < size; l += 256) {
    if (LOAD) sm[sw<T>(l)] = st[base + lo + hi];
    else st[base + lo + hi] = sm[sw<T>(l)];
    hi = ((hi | ~M) + 1ull) & M;
  }
}

// Apply one operator to the tile in shared memory; csm holds its coefficients.
template <class T>
__device__ __forceinline__ void tile_apply(cx<T>* __restrict__ sm, int nbits, const TileOp& op,
                                           const cx<T>* __restrict__ csm) {
  if (op.nb == 2) {
    uint32_t moff[4];
#pragma unroll
    for (int s = 0; s < 4; s++) moff[s] = ((s & 1) ? 1u << op.lbit[0] : 0u) | ((s & 2) ? 1u << op.lbit[1] : 0u);
    const uint32_t ng = 1u << (nbits - 2);
    if (op.kind == KK_ELEM) {
      cx<T> f[4];
#pragma unroll
      for (int s = 0; s < 4; s++) f[s] = csm[s];
      for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) {
        const uint32_t b = insert_zeros32<2>(g, op.lsorted);
#pragma unroll
        for (int s = 0; s < 4; s++) sm[sw<T>(b | moff[s])] = cmul<T>(sm[sw<T>(b | moff[s])], f[s]);
      }
    } else {  // KK_SUP1
      cx<T> a[16];
#pragma unroll
      for (int i = 0; i < 16; i++) a[i] = csm[i];
      for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) {
        const uint32_t b = insert_zeros32<2>(g, op.lsorted);
        cx<T> x[4];
#pragma unroll
        for (int s = 0; s < 4; s++) x[s] = sm[sw<T>(b | moff[s])];
#pragma unroll
        for (int i = 0; i < 4; i++) {
          cx<T> y;
          y.x = 0; y.y = 0;
#pragma unroll
          for (int j = 0; j < 4; j++) cmac<T>(y, a[i * 4 + j], x[j]);
          sm[sw<T>(b | moff[i])] = y;
        }
      }
    }
    return;
  }
  // two-qubit operators: 16-member groups, member s = r | c << 2
  uint32_t moff[16];
#pragma unroll
  for (int s = 0; s < 16; s++) {
    uint32_t o = 0;
#pragma unroll
    for (int j = 0; j < 4; j++)
      if (s >> j & 1) o |= 1u << op.lbit[j];
    moff[s] = o;
  }
  const uint32_t ng = 1u << (nbits - 4);
  if (op.kind == KK_ELEM) {
    for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) {
      const uint32_t b = insert_zeros32<4>(g, op.lsorted);
#pragma unroll
      for (int s = 0; s < 16; s++) sm[sw<T>(b | moff[s])] = cmul<T>(sm[sw<T>(b | moff[s])], csm[s]);
    }
  } else if (op.kind == KK_UNI2) {
    cx<T> u[16];
#pragma unroll
    for (int i = 0; i < 16; i++) u[i] = csm[i];
    for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) {
      const uint32_t b = insert_zeros32<4>(g, op.lsorted);
      cx<T> A[16], B[16];
#pragma unroll
      for (int s = 0; s < 16; s++) A[s] = sm[sw<T>(b | moff[s])];
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
          cx<T> acc;
          acc.x = 0; acc.y = 0;
#pragma unroll
          for (int m = 0; m < 4; m++) cmac<T>(acc, u[r * 4 + m], A[m | (c << 2)]);
          B[r | (c << 2)] = acc;
        }
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
          cx<T> acc;
          acc.x = 0; acc.y = 0;
#pragma unroll
          for (int m = 0; m < 4; m++) {
            cx<T> uc = u[c * 4 + m];
            uc.y = -uc.y;
            cmac<T>(acc, uc, B[r | (m << 2)]);
          }
          sm[sw<T>(b | moff[r | (c << 2)])] = acc;
        }
    }
  } else {  // KK_SUP2: coefficients read from shared memory (broadcast), one output row at a time
    for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) {
      const uint32_t b = insert_zeros32<4>(g, op.lsorted);
      cx<T> x[16];
#pragma unroll
      for (int s = 0; s < 16; s++) x[s] = sm[sw<T>(b | moff[s])];
#pragma unroll 1
      for (int i = 0; i < 16; i++) {
        cx<T> y;
        y.x = 0; y.y = 0;
#pragma unroll
        for (int j = 0; j < 16; j++) cmac<T>(y, csm[i * 16 + j], x[j]);
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < 4; j++)
          if (i >> j & 1) o |= 1u << op.lbit[j];
        sm[sw<T>(b | o)] = y;
      }
    }
  }
}

// Run ops [ob, oe) on the tile.  Coefficients are staged in csm (256 entries) per operator.
template <class T>
__device__ __forceinline__ void tile_ops(cx<T>* __restrict__ sm, cx<T>* __restrict__ csm, int nbits,
                                         const TileOp* __restrict__ ops, int ob, int oe,
                                         const cx<T>* __restrict__ coef) {
  for (int o = ob; o < oe; o++) {
    const TileOp op = ops[o];
    for (int i = threadIdx.x; i < op.ncoef; i += blockDim.x) csm[i] = coef[op.coef + i];
    __syncthreads();
    tile_apply<T>(sm, nbits, op, csm);
    __syncthreads();
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_stage(cx<T>* __restrict__ st, const StageDesc S,
                                               const TileOp* __restrict__ ops, const cx<T>* __restrict__ coef) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smraw);
  cx<T>* csm = sm + (1u << S.nbits);
  const uint64_t ntiles = 1ull << S.nrest;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = deposit(t, S.rest, S.nrest);
    tile_io<T, true>(st, sm, base, S.bits, S.nbits);
    __syncthreads();
    tile_ops<T>(sm, csm, S.nbits, ops, S.op_begin, S.op_end, coef);
    tile_io<T, false>(st, sm, base, S.bits, S.nbits);
    __syncthreads();
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_batch(cx<T>* __restrict__ all, const BatchInst* __restrict__ inst, int ninst,
                                               const StageDesc* __restrict__ stages, const TileOp* __restrict__ ops,
                                               const cx<T>* __restrict__ coef, int* __restrict__ counter,
                                               int max_bits) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smraw);
  cx<T>* csm = sm + (1u << max_bits);
  __shared__ int item;
  __shared__ int s_bits[kMaxTileBits];
  __shared__ int s_rest[2 * VQD_MAX_QUBITS];
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int i = item;
    __syncthreads();  // every thread has read `item` before thread 0 may overwrite it
    if (i >= ninst) break;
    const BatchInst I = inst[i];
    cx<T>* st = all + I.offset_amps;
    for (int s = I.stage_begin; s < I.stage_end; s++) {
      const int nbits = stages[s].nbits, nrest = stages[s].nrest;
      const int ob = stages[s].op_begin, oe = stages[s].op_end;
      if (threadIdx.x < kMaxTileBits) s_bits[threadIdx.x] = stages[s].bits[threadIdx.x];
      if (threadIdx.x < 2 * VQD_MAX_QUBITS) s_rest[threadIdx.x] = stages[s].rest[threadIdx.x];
      __syncthreads();
      const uint64_t ntiles = 1ull << nrest;
      for (uint64_t t = 0; t < ntiles; t++) {
        const uint64_t base = deposit(t, s_rest, nrest);
        tile_io<T, true>(st, sm, base, s_bits, nbits);
        __syncthreads();
        tile_ops<T>(sm, csm, nbits, ops, ob, oe, coef);
        tile_io<T, false>(st, sm, base, s_bits, nbits);
        __syncthreads();
      }
    }
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
  if (c.d_ops) cudaFree(c.d_ops);
  if (c.d_coef) cudaFree(c.d_coef);
  if (c.d_stages) cudaFree(c.d_stages);
  if (c.d_inst) cudaFree(c.d_inst);
  if (c.d_counter) cudaFree(c.d_counter);
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
  grow(&c.d_ops, &c.ops_cap, std::max<size_t>(1, p.ops.size()) * sizeof(TileOp));
  grow(&c.d_coef, &c.coef_cap, std::max<size_t>(1, cf.size()) * sizeof(cx<T>));
  grow(&c.d_stages, &c.stages_cap, std::max<size_t>(1, p.stages.size()) * sizeof(StageDesc));
  if (!p.ops.empty())
    check(cudaMemcpyAsync(c.d_ops, p.ops.data(), p.ops.size() * sizeof(TileOp), cudaMemcpyHostToDevice, s), "upload ops");
  if (!cf.empty())
    check(cudaMemcpyAsync(c.d_coef, cf.data(), cf.size() * sizeof(cx<T>), cudaMemcpyHostToDevice, s), "upload coefficients");
  if (!p.stages.empty())
    check(cudaMemcpyAsync(c.d_stages, p.stages.data(), p.stages.size() * sizeof(StageDesc), cudaMemcpyHostToDevice, s),
          "upload stages");
  check(cudaStreamSynchronize(s), "upload plan");
}

void upload_plan(FusedCache& c, const FusedPlan& p, int prec, cudaStream_t s) {
  if (prec == VQD_F32) upload_common<float>(c, p, s);
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
static cudaError_t stage_t(FusedCache& c, const FusedPlan& p, int stage, void* state, cudaStream_t s) {
  const StageDesc& S = p.stages[stage];
  const size_t smem = ((size_t)1 << S.nbits) * sizeof(cx<T>) + 256 * sizeof(cx<T>);
  cudaError_t e = cudaFuncSetAttribute(k_stage<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  unsigned grid = persistent_grid(k_stage<T>, smem, 1ull << S.nrest);
  k_stage<T><<<grid, 256, smem, s>>>((cx<T>*)state, S, (const TileOp*)c.d_ops, (const cx<T>*)c.d_coef);
  return cudaGetLastError();
}

cudaError_t launch_stage(FusedCache& c, const FusedPlan& p, int stage, int prec, void* state, int n, cudaStream_t s) {
  (void)n;
  if (prec == VQD_F32) return stage_t<float>(c, p, stage, state, s);
  return stage_t<double>(c, p, stage, state, s);
}

void upload_batch(FusedCache& c, const BatchPlan& p, int prec, cudaStream_t s) {
  upload_plan(c, p.all, prec, s);
  grow(&c.d_inst, &c.inst_cap, std::max<size_t>(1, p.inst.size()) * sizeof(BatchInst));
  check(cudaMemcpyAsync(c.d_inst, p.inst.data(), p.inst.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, s),
        "upload instances");
  if (!c.d_counter) check(cudaMalloc(&c.d_counter, sizeof(int)), "queue counter");
  check(cudaStreamSynchronize(s), "upload batch");
  c.n_inst = (int)p.inst.size();
  c.max_bits = p.all.max_bits;
}

template <class T>
static cudaError_t batch_t(FusedCache& c, const BatchPlan& p, void* base, cudaStream_t s) {
  const int mb = std::max(1, p.all.max_bits);
  const size_t smem = ((size_t)1 << mb) * sizeof(cx<T>) + 256 * sizeof(cx<T>);
  cudaError_t e = cudaFuncSetAttribute(k_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(c.d_counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  unsigned grid = persistent_grid(k_batch<T>, smem, p.inst.size());
  k_batch<T><<<grid, 256, smem, s>>>((cx<T>*)base, (const BatchInst*)c.d_inst, (int)p.inst.size(),
                                     (const StageDesc*)c.d_stages, (const TileOp*)c.d_ops, (const cx<T>*)c.d_coef,
                                     c.d_counter, mb);
  return cudaGetLastError();
}

cudaError_t launch_batch(FusedCache& c, const BatchPlan& p, int prec, void* base, cudaStream_t s) {
  if (prec == VQD_F32) return batch_t<float>(c, p, base, s);
  return batch_t<double>(c, p, base, s);
}

cudaError_t batch_status(FusedCache& c, cudaStream_t s) {
  (void)c;
  (void)s;
  return cudaGetLastError();
}

}  // namespace vqd
