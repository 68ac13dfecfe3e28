// Monte-Carlo trajectory path of libvqd: Pauli-sum expectation values from statevector trajectories.
//
// Sec. 2 describes the unravelling that replaces the density matrix: every decoherence channel is
// replaced, in each trajectory, by one of its Kraus operators chosen at random, the chosen operator
// acts on a statevector, and the expectation value is averaged over trajectories.  Here operator k
// of a channel {K_k} is chosen with probability p_k = ||K_k psi||^2 and psi <- K_k psi / sqrt(p_k).
// When sum_k p_k < 1 (trace-decreasing leakage) the missing probability is a branch in which the
// trajectory is lost and contributes 0, so the mean still estimates Re tr(H rho).
//
// One CTA runs one trajectory at a time with the whole statevector in shared memory (2^n
// amplitudes: n <= 14 for complex64, n <= 13 for complex128).  Larger statevectors (up to 16 qubits)
// are spread over the CTAs of a thread-block cluster, 2^c CTAs with one slice each, and reached
// across CTAs through distributed shared memory; every operator's groups are split evenly over the
// cluster, each group read and written by one thread, with a cluster barrier between operators.  The random number of channel o in
// trajectory t is the first Philox4x32-10 output for counter (o, t, 0, 0) and key = the seed
// (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011); the same
// draws can therefore be reproduced anywhere.  Channels whose Kraus operators are all multiples
// of unitaries have state-independent probabilities and skip the norm computation.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "vqd_internal.h"

namespace vqd {
namespace dev {

template <class T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };
template <class T> using cx = typename V2<T>::t;

enum { TJ_UNITARY = 0, TJ_MIXTURE = 1, TJ_KRAUS = 2 };
constexpr int kTrajThreads = 256;
constexpr int kMaxKraus = 16;  // state-dependent channels (mixtures may have more operators)

struct TrajOp {
  int kind;
  int k;
  int q[2];
  int nK;
  int coef;  // offset (complex) of operator 0; operator j at coef + j d^2
  int wofs;  // mixtures: offset of the weights
  int pad;
};

struct PauliTerm {
  uint32_t xm, zy;
  int ny;
  int pad;
  double c;
};

// Philox4x32 with 10 rounds: round (x0,x1,x2,x3) -> (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1,
// lo(M0 x0)), key bumped by the Weyl constants after each round.
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; r++) {
    const uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

// Uniform double in [0, 1) with 53 random bits from the first two output words.
__host__ __device__ inline double draw_uniform(uint64_t seed, uint32_t op, uint32_t traj) {
  uint32_t c[4] = {op, traj, 0u, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6)) * (1.0 / 9007199254740992.0);
}

template <class T>
__device__ __forceinline__ cx<T> cmadd(cx<T> acc, const cx<T>& c, const cx<T>& x) {
  acc.x = fma(c.x, x.x, acc.x);
  acc.x = fma(-c.y, x.y, acc.x);
  acc.y = fma(c.x, x.y, acc.y);
  acc.y = fma(c.y, x.x, acc.y);
  return acc;
}

__device__ __forceinline__ uint32_t ins0(uint32_t g, int p) { return g + (g & ~((1u << p) - 1u)); }

// The statevector in this CTA's shared memory.
template <class T>
struct LocalPsi {
  cx<T>* p;
  __device__ __forceinline__ cx<T>& operator[](uint32_t i) const { return p[i]; }
};

// The statevector spread over a cluster: amplitude i is at offset i & mask of the slice of CTA rank
// i >> shift (distributed shared memory for the other ranks).
template <class T>
struct ClusterPsi {
  cx<T>* p;
  int shift;
  uint32_t mask;
  __device__ __forceinline__ cx<T>& operator[](uint32_t i) const {
    return *cooperative_groups::this_cluster().map_shared_rank(p + (i & mask), i >> shift);
  }
};

// psi <- scale * K psi on the op's qubits (K is d x d, row-major, index little-endian over q), for the
// groups g0 <= g < g1 (a group: the d amplitudes that differ only on the op's qubits)
template <class T, class Psi>
__device__ void apply_op(const Psi& psi, const TrajOp& op, const cx<T>* __restrict__ K, T scale, uint32_t g0,
                         uint32_t g1) {
  if (op.k == 1) {
    const uint32_t m = 1u << op.q[0];
    const cx<T> a = K[0], b = K[1], c = K[2], d = K[3];
    for (uint32_t g = g0 + threadIdx.x; g < g1; g += kTrajThreads) {
      const uint32_t i0 = ins0(g, op.q[0]);
      const cx<T> x0 = psi[i0], x1 = psi[i0 | m];
      cx<T> y0, y1;
      y0.x = 0; y0.y = 0; y1 = y0;
      y0 = cmadd<T>(cmadd<T>(y0, a, x0), b, x1);
      y1 = cmadd<T>(cmadd<T>(y1, c, x0), d, x1);
      y0.x *= scale; y0.y *= scale; y1.x *= scale; y1.y *= scale;
      psi[i0] = y0;
      psi[i0 | m] = y1;
    }
  } else {
    const int lo = min(op.q[0], op.q[1]), hi = max(op.q[0], op.q[1]);
    const uint32_t m0 = 1u << op.q[0], m1 = 1u << op.q[1];
    cx<T> U[16];
#pragma unroll
    for (int i = 0; i < 16; i++) U[i] = K[i];
    for (uint32_t g = g0 + threadIdx.x; g < g1; g += kTrajThreads) {
      const uint32_t b = ins0(ins0(g, lo), hi);
      const uint32_t idx[4] = {b, b | m0, b | m1, b | m0 | m1};
      cx<T> x[4];
#pragma unroll
      for (int s = 0; s < 4; s++) x[s] = psi[idx[s]];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        cx<T> y;
        y.x = 0; y.y = 0;
#pragma unroll
        for (int s = 0; s < 4; s++) y = cmadd<T>(y, U[r * 4 + s], x[s]);
        y.x *= scale;
        y.y *= scale;
        psi[idx[r]] = y;
      }
    }
  }
}

// p[k] = ||K_k psi||^2 restricted to the groups g0 <= g < g1, for k < nK (FP64 accumulation, fixed
// order); this CTA's sums in red[0..nK)
template <class T, class Psi>
__device__ void kraus_norms(const Psi& psi, const TrajOp& op, const cx<T>* __restrict__ Ks, uint32_t g0, uint32_t g1,
                            double* __restrict__ red) {
  double acc[kMaxKraus];
#pragma unroll
  for (int j = 0; j < kMaxKraus; j++) acc[j] = 0.0;
  if (op.k == 1) {
    const uint32_t m = 1u << op.q[0];
    for (uint32_t g = g0 + threadIdx.x; g < g1; g += kTrajThreads) {
      const uint32_t i0 = ins0(g, op.q[0]);
      const cx<T> x0 = psi[i0], x1 = psi[i0 | m];
#pragma unroll
      for (int j = 0; j < kMaxKraus; j++) {
        if (j >= op.nK) break;
        const cx<T>* K = Ks + 4 * j;
        cx<T> y0, y1;
        y0.x = 0; y0.y = 0; y1 = y0;
        y0 = cmadd<T>(cmadd<T>(y0, K[0], x0), K[1], x1);
        y1 = cmadd<T>(cmadd<T>(y1, K[2], x0), K[3], x1);
        acc[j] += (double)y0.x * y0.x + (double)y0.y * y0.y + (double)y1.x * y1.x + (double)y1.y * y1.y;
      }
    }
  } else {
    const int lo = min(op.q[0], op.q[1]), hi = max(op.q[0], op.q[1]);
    const uint32_t m0 = 1u << op.q[0], m1 = 1u << op.q[1];
    for (uint32_t g = g0 + threadIdx.x; g < g1; g += kTrajThreads) {
      const uint32_t b = ins0(ins0(g, lo), hi);
      const cx<T> x[4] = {psi[b], psi[b | m0], psi[b | m1], psi[b | m0 | m1]};
#pragma unroll
      for (int j = 0; j < kMaxKraus; j++) {
        if (j >= op.nK) break;
        const cx<T>* K = Ks + 16 * j;
#pragma unroll
        for (int r = 0; r < 4; r++) {
          cx<T> y;
          y.x = 0; y.y = 0;
#pragma unroll
          for (int s = 0; s < 4; s++) y = cmadd<T>(y, K[r * 4 + s], x[s]);
          acc[j] += (double)y.x * y.x + (double)y.y * y.y;
        }
      }
    }
  }
  // block reduction of the nK sums in fixed order: warps, then over warps
  __shared__ double wsum[kTrajThreads / 32][kMaxKraus];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kMaxKraus; j++) {
    double v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (l == 0) wsum[w][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < kMaxKraus) {
    double v = 0;
    for (int i = 0; i < kTrajThreads / 32; i++) v += wsum[i][threadIdx.x];
    red[threadIdx.x] = v;
  }
  __syncthreads();
}

// One CTA (CtaTeam) or the CTAs of a cluster (ClusterTeam) working on one statevector.  combine()
// turns each CTA's block sums v[0..cnt) into the team's totals, summed in rank order so that every
// CTA holds bit-identical values (and so takes the same random branch).
struct CtaTeam {
  int rank, c;
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ void combine(double*, int) const {}
};
struct ClusterTeam {
  double* part;  // [8][kMaxKraus] partial sums; rank 0's copy gathers them
  int rank, c;
  __device__ __forceinline__ void sync() const { cooperative_groups::this_cluster().sync(); }
  __device__ void combine(double* v, int cnt) const {
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    if (threadIdx.x < (unsigned)cnt) *cl.map_shared_rank(part + rank * kMaxKraus + threadIdx.x, 0) = v[threadIdx.x];
    cl.sync();
    if (threadIdx.x < (unsigned)cnt) {
      double acc = 0.0;
      for (int r = 0; r < (1 << c); r++) acc += *cl.map_shared_rank(part + r * kMaxKraus + threadIdx.x, 0);
      v[threadIdx.x] = acc;
    }
    cl.sync();  // rank 0's gather area is reused only after every CTA has read it
  }
};

struct TrajShared {
  double red[kMaxKraus];
  double part[8 * kMaxKraus];
  double warp[kTrajThreads / 32][2];
  double scale;
  int choice;
};

// One trajectory from |0...0>; returns Re <psi|H|psi> (0 if the trajectory was lost), valid in thread
// 0 of every CTA of the team.  This CTA holds amplitudes [rank * len, (rank + 1) * len) in `slice`.
template <class T, class Psi, class Team>
__device__ double one_trajectory(const Psi& psi, const Team& team, cx<T>* __restrict__ slice, uint32_t len, int n,
                                 const TrajOp* __restrict__ ops, int nops, const cx<T>* __restrict__ coef,
                                 const double* __restrict__ wts, uint64_t seed, int t,
                                 const PauliTerm* __restrict__ terms, int nterms, TrajShared& sh) {
  for (uint32_t i = threadIdx.x; i < len; i += kTrajThreads) {
    cx<T> z;
    z.x = (team.rank == 0 && i == 0) ? (T)1 : (T)0;
    z.y = 0;
    slice[i] = z;
  }
  team.sync();
  for (int o = 0; o < nops; o++) {
    const TrajOp op = ops[o];
    const int dd = op.k == 1 ? 4 : 16;
    const uint32_t per = (1u << (n - op.k)) >> team.c, g0 = team.rank * per, g1 = g0 + per;
    if (op.kind == TJ_UNITARY) {
      apply_op<T>(psi, op, coef + op.coef, (T)1, g0, g1);
      team.sync();
      continue;
    }
    if (op.kind == TJ_KRAUS) {
      kraus_norms<T>(psi, op, coef + op.coef, g0, g1, sh.red);
      team.combine(sh.red, op.nK);
    }
    if (threadIdx.x == 0) {
      const double u = draw_uniform(seed, (uint32_t)o, (uint32_t)t);
      double cum = 0.0, pk = 0.0;
      int choice = -1;
      for (int j = 0; j < op.nK; j++) {
        const double p = op.kind == TJ_MIXTURE ? wts[op.wofs + j] : sh.red[j];
        cum += p;
        if (u < cum) {
          choice = j;
          pk = p;
          break;
        }
      }
      sh.choice = choice;
      sh.scale = (op.kind == TJ_KRAUS && choice >= 0) ? 1.0 / sqrt(pk) : 1.0;
    }
    __syncthreads();
    const int choice = sh.choice;
    if (choice < 0) return 0.0;  // the trajectory left the computational space (trace-decreasing branch)
    apply_op<T>(psi, op, coef + op.coef + dd * choice, (T)sh.scale, g0, g1);
    team.sync();
  }
  // <psi|H|psi> = sum_t c_t i^{ny} sum_x (-1)^{popc(x & zy)} conj(psi[x ^ xm]) psi[x], x over this CTA's slice
  double total = 0.0;
  const uint32_t x0 = team.rank * len;
  for (int j = 0; j < nterms; j++) {
    const PauliTerm P = terms[j];
    double re = 0.0, im = 0.0;
    for (uint32_t x = x0 + threadIdx.x; x < x0 + len; x += kTrajThreads) {
      const cx<T> a = psi[x ^ P.xm], b = slice[x - x0];
      const double sg = (__popc(x & P.zy) & 1) ? -1.0 : 1.0;
      re += sg * ((double)a.x * b.x + (double)a.y * b.y);
      im += sg * ((double)a.x * b.y - (double)a.y * b.x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) {
      sh.warp[threadIdx.x >> 5][0] = re;
      sh.warp[threadIdx.x >> 5][1] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0, si = 0;
      for (int w = 0; w < kTrajThreads / 32; w++) {
        sr += sh.warp[w][0];
        si += sh.warp[w][1];
      }
      sh.red[0] = sr;
      sh.red[1] = si;
    }
    __syncthreads();
    team.combine(sh.red, 2);
    if (threadIdx.x == 0) {
      // times i^{ny}: real part of (sr + i si) i^ny
      const double sr = sh.red[0], si = sh.red[1];
      const int r = P.ny & 3;
      const double v = r == 0 ? sr : r == 1 ? -si : r == 2 ? -sr : si;
      total += P.c * v;
    }
    __syncthreads();
  }
  return total;
}

// Whole statevector in this CTA's shared memory.
template <class T>
__global__ void __launch_bounds__(kTrajThreads) k_traj(const TrajOp* __restrict__ ops, int nops,
                                                      const cx<T>* __restrict__ coef, const double* __restrict__ wts,
                                                      uint64_t seed, int ntraj, int n,
                                                      const PauliTerm* __restrict__ terms, int nterms,
                                                      double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<T>* psi = reinterpret_cast<cx<T>*>(smraw);
  __shared__ TrajShared sh;
  const CtaTeam team{0, 0};
  const LocalPsi<T> P{psi};
  for (int t = blockIdx.x; t < ntraj; t += gridDim.x) {
    const double v = one_trajectory<T>(P, team, psi, 1u << n, n, ops, nops, coef, wts, seed, t, terms, nterms, sh);
    if (threadIdx.x == 0) out[t] = v;
    __syncthreads();
  }
}

// Statevector spread over a cluster of 2^c CTAs (launched with that cluster shape): CTA rank r of
// cluster k holds amplitudes [r 2^{n-c}, (r+1) 2^{n-c}) of trajectory k, k + clusters, ...
template <class T>
__global__ void __launch_bounds__(kTrajThreads) k_traj_cluster(const TrajOp* __restrict__ ops, int nops,
                                                              const cx<T>* __restrict__ coef,
                                                              const double* __restrict__ wts, uint64_t seed, int ntraj,
                                                              int n, const PauliTerm* __restrict__ terms, int nterms,
                                                              double* __restrict__ out, int c) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<T>* slice = reinterpret_cast<cx<T>*>(smraw);
  __shared__ TrajShared sh;
  const ClusterTeam team{sh.part, (int)cooperative_groups::this_cluster().block_rank(), c};
  const uint32_t len = 1u << (n - c);
  const ClusterPsi<T> P{slice, n - c, len - 1};
  const int nclusters = gridDim.x >> c;
  for (int t = blockIdx.x >> c; t < ntraj; t += nclusters) {
    const double v = one_trajectory<T>(P, team, slice, len, n, ops, nops, coef, wts, seed, t, terms, nterms, sh);
    if (team.rank == 0 && threadIdx.x == 0) out[t] = v;
    team.sync();
  }
}

}  // namespace dev

static int max_traj_qubits(int) { return VQD_MAX_QUBITS; }

// Cluster size (log2) for an n-qubit statevector: 0 while it fits one CTA (n <= 14 complex64, <= 13
// complex128), else slices of at most 64 KB (128 KB for 16 qubits in complex128) on up to 8 CTAs.
static int traj_cluster_log(int n, size_t amp_bytes) {
  const int single = amp_bytes == 8 ? 14 : 13;
  if (n <= single) return 0;
  return std::min(3, n - (single - 1));
}

template <class T>
static cudaError_t traj_run(const std::vector<dev::TrajOp>& ops, const std::vector<cd>& coef,
                            const std::vector<double>& wts, uint64_t seed, int ntraj, int n,
                            const std::vector<dev::PauliTerm>& terms, cudaStream_t s, double* host_out) {
  using namespace dev;
  std::vector<cx<T>> cf(coef.size());
  for (size_t i = 0; i < coef.size(); i++) {
    cf[i].x = (T)coef[i].real();
    cf[i].y = (T)coef[i].imag();
  }
  void *d_ops = nullptr, *d_coef = nullptr, *d_w = nullptr, *d_terms = nullptr, *d_out = nullptr;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b > 0 ? b : 16);
  };
  al(&d_ops, ops.size() * sizeof(TrajOp));
  al(&d_coef, cf.size() * sizeof(cx<T>));
  al(&d_w, wts.size() * sizeof(double));
  al(&d_terms, terms.size() * sizeof(PauliTerm));
  al(&d_out, (size_t)ntraj * sizeof(double));
  if (e == cudaSuccess && !ops.empty())
    e = cudaMemcpyAsync(d_ops, ops.data(), ops.size() * sizeof(TrajOp), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !cf.empty())
    e = cudaMemcpyAsync(d_coef, cf.data(), cf.size() * sizeof(cx<T>), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !wts.empty())
    e = cudaMemcpyAsync(d_w, wts.data(), wts.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !terms.empty())
    e = cudaMemcpyAsync(d_terms, terms.data(), terms.size() * sizeof(PauliTerm), cudaMemcpyHostToDevice, s);
  const int c = traj_cluster_log(n, sizeof(cx<T>));
  const size_t smem = ((size_t)1 << (n - c)) * sizeof(cx<T>);
  if (c == 0) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_traj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traj<T>, kTrajThreads, smem) != cudaSuccess ||
          per_sm < 1)
        per_sm = 1;
      const int grid = std::max(1, std::min(ntraj, per_sm * num_sms()));
      k_traj<T><<<grid, kTrajThreads, smem, s>>>((const TrajOp*)d_ops, (int)ops.size(), (const cx<T>*)d_coef,
                                                 (const double*)d_w, seed, ntraj, n, (const PauliTerm*)d_terms,
                                                 (int)terms.size(), (double*)d_out);
      e = cudaGetLastError();
    }
  } else {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_traj_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 1u << c;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.blockDim = dim3(kTrajThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cfg.gridDim = dim3((unsigned)(1 << c));
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, k_traj_cluster<T>, &cfg) != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        clusters = 1;
      }
      clusters = std::max(1, std::min(ntraj, clusters));
      cfg.gridDim = dim3((unsigned)(clusters << c));
      e = cudaLaunchKernelEx(&cfg, k_traj_cluster<T>, (const TrajOp*)d_ops, (int)ops.size(), (const cx<T>*)d_coef,
                             (const double*)d_w, seed, ntraj, n, (const PauliTerm*)d_terms, (int)terms.size(),
                             (double*)d_out, c);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, d_out, (size_t)ntraj * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (void* p : {d_ops, d_coef, d_w, d_terms, d_out})
    if (p) cudaFree(p);
  return e;
}

}  // namespace vqd

extern "C" int vqd_traj_expect(int n, int prec, int nops, const vqd_native_op* ops, unsigned flags, int ntraj,
                               uint64_t seed, int nterms, const uint8_t* paulis, const double* coeffs, void* stream,
                               double* out, double* mean, double* stderr_out) {
  using namespace vqd;
  try {
    if (prec != VQD_F32 && prec != VQD_F64) throw Error(VQD_EINVAL, "bad precision");
    if (n < 1 || n > max_traj_qubits(prec))
      throw Error(VQD_EINVAL, "trajectories: n must be in 1.." + std::to_string(max_traj_qubits(prec)));
    if (ntraj < 1 || nops < 0 || (nops > 0 && !ops) || nterms < 1 || !paulis || !coeffs || !out)
      throw Error(VQD_EINVAL, "bad argument");
    std::vector<dev::TrajOp> top;
    std::vector<cd> coef;
    std::vector<double> wts;
    for (int i = 0; i < nops; i++) {
      const int ar = native_arity(ops[i].code);
      if (ar < 1 || ops[i].nq != ar) throw Error(VQD_EINVAL, "bad native op at index " + std::to_string(i));
      for (int j = 0; j < ar; j++)
        if (ops[i].q[j] < 0 || ops[i].q[j] >= n || (j == 1 && ops[i].q[1] == ops[i].q[0]))
          throw Error(VQD_EINVAL, "bad target qubit at index " + std::to_string(i));
      KrausForm f = compile_kraus_form(ops[i], flags);
      dev::TrajOp t;
      std::memset(&t, 0, sizeof(t));
      t.k = f.k;
      t.q[0] = f.q[0];
      t.q[1] = f.q[1];
      t.nK = (int)f.K.size();
      t.coef = (int)coef.size();
      t.wofs = -1;
      t.kind = f.unitary ? dev::TJ_UNITARY : f.mixture ? dev::TJ_MIXTURE : dev::TJ_KRAUS;
      if (t.kind == dev::TJ_KRAUS && t.nK > dev::kMaxKraus)
        throw Error(VQD_ENOTSUP, "more than 16 state-dependent Kraus operators");
      for (size_t j = 0; j < f.K.size(); j++) {
        const double inv = t.kind == dev::TJ_MIXTURE ? 1.0 / std::sqrt(f.w[j]) : 1.0;
        for (const cd& x : f.K[j]) coef.push_back(x * inv);
      }
      if (t.kind == dev::TJ_MIXTURE) {
        t.wofs = (int)wts.size();
        wts.insert(wts.end(), f.w.begin(), f.w.end());
      }
      top.push_back(t);
    }
    std::vector<dev::PauliTerm> terms(nterms);
    for (int t = 0; t < nterms; t++) {
      uint32_t x = 0, z = 0;
      int y = 0;
      for (int q = 0; q < n; q++) {
        const uint8_t s = paulis[(size_t)t * n + q];
        if (s > 3) throw Error(VQD_EINVAL, "Pauli code must be 0..3");
        if (s == 1 || s == 2) x |= 1u << q;
        if (s == 2 || s == 3) z |= 1u << q;
        if (s == 2) y++;
      }
      terms[t] = {x, z, y, 0, coeffs[t]};
    }
    cudaError_t e = prec == VQD_F32
                        ? traj_run<float>(top, coef, wts, seed, ntraj, n, terms, (cudaStream_t)stream, out)
                        : traj_run<double>(top, coef, wts, seed, ntraj, n, terms, (cudaStream_t)stream, out);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error(e == cudaErrorMemoryAllocation ? VQD_ENOMEM : VQD_EDEVICE, cudaGetErrorString(e));
    }
    // two passes (mean, then squared deviations): the one-pass E[x^2] - E[x]^2 loses the spread of
    // nearly equal values to cancellation
    double s1 = 0, s2 = 0;
    for (int t = 0; t < ntraj; t++) s1 += out[t];
    const double m = s1 / ntraj;
    for (int t = 0; t < ntraj; t++) s2 += (out[t] - m) * (out[t] - m);
    if (mean) *mean = m;
    if (stderr_out) *stderr_out = ntraj > 1 ? std::sqrt(s2 / (ntraj - 1) / ntraj) : 0.0;
    return VQD_OK;
  } catch (const Error& e) {
    return report_static_error(e.code, e.what());
  } catch (const std::exception& e) {
    return report_static_error(VQD_EINVAL, e.what());
  }
}
