// Plain-path kernels of libvqd: one pass over the state per operator, FP64 reductions, init.
//
// State layout: amplitude rho[r][c] of an n-qubit instance at index r + (c << n).  An operator
// on k qubits q touches, for every assignment of the other 2n - 2k index bits, the group of 4^k
// amplitudes spanned by the row bits q and the column bits q + n.  Each thread owns whole groups,
// loads them once from HBM, applies the operator in registers and stores them once: 2 x state
// bytes of DRAM traffic per pass, the algorithmic minimum for one operator.
//
// Coefficients arrive as kernel parameters (constant bank, broadcast to the warp).  Each
// coefficient carries a type flag (zero / one / real / imaginary / complex) that is uniform
// across the grid; the SPARSE instantiations branch on it so that structured operators (Pauli
// and damping channels, rotations whose entries are real or imaginary) issue only the
// multiply-adds they need.  That matters for FP64, whose FMA rate on this GPU is about 1/58 of
// FP32; the dense instantiations keep straight-line FMA code for FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "numeric.h"

namespace vqd {
namespace dev {

template <class T>
__device__ __forceinline__ void cmac(cx<T>& acc, const cx<T>& c, const cx<T>& x) {
  acc.x = fma(c.x, x.x, acc.x);
  acc.x = fma(-c.y, x.y, acc.x);
  acc.y = fma(c.x, x.y, acc.y);
  acc.y = fma(c.y, x.x, acc.y);
}

template <bool SPARSE, class T>
__device__ __forceinline__ void mac(cx<T>& acc, const cx<T>& c, int fl, const cx<T>& x) {
  if (SPARSE) cmac_flag<T>(acc, c, fl, x);
  else cmac<T>(acc, c, x);
}

// Insert a zero bit at each of the NB ascending positions pos[] into g.
template <int NB>
__device__ __forceinline__ uint64_t insert_zeros(uint64_t g, const int* pos) {
#pragma unroll
  for (int i = 0; i < NB; i++) {
    const uint64_t lo = g & ((1ull << pos[i]) - 1ull);
    g = ((g >> pos[i]) << (pos[i] + 1)) | lo;
  }
  return g;
}

template <int G>
struct Group {
  uint64_t off[G];  // member offsets, member index s = r | c << k
  int pos[4];       // ascending positions of the 2k group bits
};

template <class T> struct Sup1P { Group<4> g; cx<T> s[16]; unsigned char fl[16]; };
template <class T> struct Uni2P { Group<16> g; cx<T> u[16]; cx<T> uc[16]; unsigned char fl[16]; };
template <class T> struct Sup2P { Group<16> g; cx<T> s[256]; unsigned char fl[256]; };

#define GRID_STRIDE_LOOP(i, count)                                                         \
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, _st = (uint64_t)gridDim.x * blockDim.x; \
       i < (count); i += _st)

// ---- one-qubit operator as a 4x4 superoperator
template <class T, bool SPARSE>
__global__ void __launch_bounds__(256) k_sup1(cx<T>* __restrict__ st, uint64_t ngroups, const Sup1P<T> P) {
  GRID_STRIDE_LOOP(g, ngroups) {
    const uint64_t base = insert_zeros<2>(g, P.g.pos);
    cx<T> x[4], y[4];
#pragma unroll
    for (int s = 0; s < 4; s++) x[s] = st[base + P.g.off[s]];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      y[i].x = 0; y[i].y = 0;
#pragma unroll
      for (int j = 0; j < 4; j++) mac<SPARSE, T>(y[i], P.s[i * 4 + j], P.fl[i * 4 + j], x[j]);
    }
#pragma unroll
    for (int s = 0; s < 4; s++) st[base + P.g.off[s]] = y[s];
  }
}

// ---- two-qubit unitary: A <- U A U^dagger on the 4x4 block A[r][c] = amplitude r | c << 2.
// k_uni2_pair (FP32): two neighbouring threads share a group; thread h holds columns 2h and 2h+1
// (8 amplitudes), so all of its loads are in flight at once with few registers.  B = U A needs only a
// thread's own columns; U A U^dagger needs every column of B, so the partner's half of B comes over
// one warp shuffle per value.  Member offsets and coefficients that depend on h are chosen between
// two static parameter entries, never indexed by h.  The grid-stride step is even, so partners run
// the same iterations.
// k_uni2_whole (FP64): one thread per group, with the zero/real/imaginary coefficient flags, since
// FP64 is bound by its FMA rate rather than by memory.
template <class T>
__global__ void __launch_bounds__(256) k_uni2_pair(cx<T>* __restrict__ st, uint64_t ngroups, const Uni2P<T> P) {
  GRID_STRIDE_LOOP(t, 2 * ngroups) {
    const unsigned mask = __activemask();
    const uint64_t g = t >> 1;
    const bool h = (t & 1) != 0;
    const uint64_t base = insert_zeros<4>(g, P.g.pos);
    cx<T> B[2][4];  // B[j][r] = (U A)[r][2h + j]
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const uint64_t cofs = h ? P.g.off[(2 + j) << 2] : P.g.off[j << 2];
      cx<T> a[4];
#pragma unroll
      for (int m = 0; m < 4; m++) a[m] = st[base + P.g.off[m] + cofs];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        cx<T> acc; acc.x = 0; acc.y = 0;
#pragma unroll
        for (int m = 0; m < 4; m++) cmac<T>(acc, P.u[r * 4 + m], a[m]);
        B[j][r] = acc;
      }
    }
    cx<T> O[2][4];  // the partner's columns 2(1-h) + j
#pragma unroll
    for (int j = 0; j < 2; j++)
#pragma unroll
      for (int r = 0; r < 4; r++) {
        O[j][r].x = __shfl_xor_sync(mask, B[j][r].x, 1);
        O[j][r].y = __shfl_xor_sync(mask, B[j][r].y, 1);
      }
    // A'[r][c] = sum_m B[r][m] conj(U[c][m]) for this thread's columns c = 2h + j; B[r][m] is the
    // thread's own value when m's half equals h
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const uint64_t cofs = h ? P.g.off[(2 + j) << 2] : P.g.off[j << 2];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        cx<T> acc; acc.x = 0; acc.y = 0;
#pragma unroll
        for (int m = 0; m < 4; m++) {
          const cx<T> bm = (((m >> 1) != 0) == h) ? B[m & 1][r] : O[m & 1][r];
          cx<T> uc;
          uc.x = h ? P.uc[(2 + j) * 4 + m].x : P.uc[j * 4 + m].x;
          uc.y = h ? P.uc[(2 + j) * 4 + m].y : P.uc[j * 4 + m].y;
          cmac<T>(acc, uc, bm);
        }
        st[base + P.g.off[r] + cofs] = acc;
      }
    }
  }
}

template <class T, bool SPARSE>
__global__ void __launch_bounds__(256) k_uni2_whole(cx<T>* __restrict__ st, uint64_t ngroups, const Uni2P<T> P) {
  GRID_STRIDE_LOOP(g, ngroups) {
    const uint64_t base = insert_zeros<4>(g, P.g.pos);
    cx<T> B[16];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      cx<T> a[4];
#pragma unroll
      for (int m = 0; m < 4; m++) a[m] = st[base + P.g.off[m | (c << 2)]];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        cx<T> acc; acc.x = 0; acc.y = 0;
#pragma unroll
        for (int m = 0; m < 4; m++) mac<SPARSE, T>(acc, P.u[r * 4 + m], P.fl[r * 4 + m], a[m]);
        B[r | (c << 2)] = acc;
      }
    }
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int c = 0; c < 4; c++) {
        cx<T> acc; acc.x = 0; acc.y = 0;
#pragma unroll
        for (int m = 0; m < 4; m++) mac<SPARSE, T>(acc, P.uc[c * 4 + m], P.fl[c * 4 + m], B[r | (m << 2)]);
        st[base + P.g.off[r | (c << 2)]] = acc;
      }
  }
}

// ---- two-qubit channel as a 16x16 superoperator
template <class T, bool SPARSE>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && SPARSE) ? 2 : 1) k_sup2(cx<T>* __restrict__ st, uint64_t ngroups, const Sup2P<T> P) {
  GRID_STRIDE_LOOP(g, ngroups) {
    const uint64_t base = insert_zeros<4>(g, P.g.pos);
    cx<T> x[16];
#pragma unroll
    for (int s = 0; s < 16; s++) x[s] = st[base + P.g.off[s]];
#pragma unroll
    for (int i = 0; i < 16; i++) {
      cx<T> acc; acc.x = 0; acc.y = 0;
#pragma unroll
      for (int j = 0; j < 16; j++) mac<SPARSE, T>(acc, P.s[i * 16 + j], P.fl[i * 16 + j], x[j]);
      st[base + P.g.off[i]] = acc;
    }
  }
}

// ---- diagonal superoperator: every member s of a group is scaled by its own factor f[s].
// Same group walk as the dense kernels, so the factor index is static and the factors stay in
// registers; REAL when every factor is real (dephasing-type channels).
template <class T, bool REAL>
__device__ __forceinline__ void scale(cx<T>& v, const cx<T>& f) {
  if (REAL) { v.x *= f.x; v.y *= f.x; }
  else { const T re = fma(v.x, f.x, -v.y * f.y); v.y = fma(v.x, f.y, v.y * f.x); v.x = re; }
}
// skip: members whose factor is exactly 1 (bit s for member s).  They are neither read nor written:
// a diagonal phase or dephasing leaves half of the amplitudes unchanged (those whose row and column
// bits agree on the targets, or have equal parity), so the pass moves half the bytes.
template <class T> struct Diag1P { Group<4> g; cx<T> f[4]; uint32_t skip; };
template <class T> struct Diag2P { Group<16> g; cx<T> f[16]; uint32_t skip; };
template <class T, bool REAL>
__global__ void __launch_bounds__(256) k_diag1(cx<T>* __restrict__ st, uint64_t ngroups, const Diag1P<T> P) {
  GRID_STRIDE_LOOP(g, ngroups) {
    const uint64_t base = insert_zeros<2>(g, P.g.pos);
    cx<T> x[4];
#pragma unroll
    for (int s = 0; s < 4; s++)
      if (!(P.skip >> s & 1u)) x[s] = st[base + P.g.off[s]];
#pragma unroll
    for (int s = 0; s < 4; s++)
      if (!(P.skip >> s & 1u)) { scale<T, REAL>(x[s], P.f[s]); st[base + P.g.off[s]] = x[s]; }
  }
}
template <class T, bool REAL>
__global__ void __launch_bounds__(256) k_diag2(cx<T>* __restrict__ st, uint64_t ngroups, const Diag2P<T> P) {
  GRID_STRIDE_LOOP(g, ngroups) {
    const uint64_t base = insert_zeros<4>(g, P.g.pos);
    cx<T> x[16];
#pragma unroll
    for (int s = 0; s < 16; s++)
      if (!(P.skip >> s & 1u)) x[s] = st[base + P.g.off[s]];
#pragma unroll
    for (int s = 0; s < 16; s++)
      if (!(P.skip >> s & 1u)) { scale<T, REAL>(x[s], P.f[s]); st[base + P.g.off[s]] = x[s]; }
  }
}

// ---- initial states
struct DiagProductP { double e[VQD_MAX_QUBITS]; };
template <class T>
__global__ void k_set_diag_product(cx<T>* __restrict__ st, int n, const DiagProductP P) {
  const uint64_t dim = 1ull << n;
  GRID_STRIDE_LOOP(x, dim) {
    double p = 1.0;
#pragma unroll
    for (int q = 0; q < VQD_MAX_QUBITS; q++)
      if (q < n) p *= ((x >> q) & 1ull) ? P.e[q] : 1.0 - P.e[q];
    cx<T> v; v.x = (T)p; v.y = 0;
    st[x * (dim + 1)] = v;
  }
}
template <class T>
__global__ void k_set_one(cx<T>* __restrict__ st, uint64_t idx) {
  cx<T> v; v.x = 1; v.y = 0;
  st[idx] = v;
}

// ---- reductions (FP64 accumulation, fixed order: grid-stride per thread, then a block tree)
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0;
  if (w == 0) {
    v = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

template <class T>
__global__ void __launch_bounds__(256) k_purity(const cx<T>* __restrict__ st, uint64_t N, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0;
  GRID_STRIDE_LOOP(i, N) {
    const cx<T> v = st[i];
    const double re = (double)v.x, im = (double)v.y;
    acc = fma(re, re, fma(im, im, acc));
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

template <class T>
__global__ void __launch_bounds__(256) k_trace(const cx<T>* __restrict__ st, int n, double* __restrict__ part) {
  __shared__ double sh[32];
  const uint64_t dim = 1ull << n;
  double re = 0, im = 0;
  GRID_STRIDE_LOOP(x, dim) {
    const cx<T> v = st[x * (dim + 1)];
    re += (double)v.x;
    im += (double)v.y;
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = re; part[2 * blockIdx.x + 1] = im; }
}

struct ProbP { int meas[16]; int rest[16]; int m, nr; };
// thread (v, ch) sums chunk ch of bin v: basis states x = deposit(v -> measured) | deposit(u -> rest)
template <class T>
__global__ void __launch_bounds__(256) k_prob(const cx<T>* __restrict__ st, int n, ProbP P, uint64_t chunks,
                                              uint64_t chunk_len, double* __restrict__ part) {
  const uint64_t dim = 1ull << n;
  const uint64_t nbins = 1ull << P.m;
  GRID_STRIDE_LOOP(t, nbins * chunks) {
    const uint64_t v = t / chunks, ch = t % chunks;
    uint64_t xv = 0;
    for (int j = 0; j < P.m; j++) xv |= ((v >> j) & 1ull) << P.meas[j];
    double acc = 0;
    for (uint64_t u = ch * chunk_len; u < (ch + 1) * chunk_len; u++) {
      uint64_t x = xv;
      for (int j = 0; j < P.nr; j++) x |= ((u >> j) & 1ull) << P.rest[j];
      acc += (double)st[x * (dim + 1)].x;
    }
    part[t] = acc;
  }
}

struct ExpectP { uint32_t xm[kExpectTermsPerLaunch]; uint32_t zy[kExpectTermsPerLaunch]; };
// block (b, t): partial of sum_c (-1)^popc(c & zy_t) rho[c][c ^ x_t]
template <class T>
__global__ void __launch_bounds__(256) k_expect(const cx<T>* __restrict__ st, int n, const ExpectP P,
                                                double* __restrict__ part) {
  __shared__ double sh[32];
  const uint64_t dim = 1ull << n;
  const int t = blockIdx.y;
  const uint32_t xm = P.xm[t], zy = P.zy[t];
  double re = 0, im = 0;
  GRID_STRIDE_LOOP(c, dim) {
    const cx<T> v = st[c + ((c ^ xm) << n)];
    const double sg = (__popcll(c & zy) & 1) ? -1.0 : 1.0;
    re = fma(sg, (double)v.x, re);
    im = fma(sg, (double)v.y, im);
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  if (threadIdx.x == 0) {
    part[(size_t)(t * gridDim.x + blockIdx.x) * 2] = re;
    part[(size_t)(t * gridDim.x + blockIdx.x) * 2 + 1] = im;
  }
}

// out[v] = sum_j part[v * nparts + j], one block per value.
__global__ void __launch_bounds__(256) k_sum_rows(const double* __restrict__ part, uint64_t nparts, int stride_v,
                                                  int stride_j, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0;
  for (uint64_t j = threadIdx.x; j < nparts; j += blockDim.x) acc += part[(uint64_t)blockIdx.x * stride_v + j * stride_j];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

}  // namespace dev

// ================================================================== host launchers
using namespace dev;

static int g_nsm = 0;
int num_sms() {
  if (!g_nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    if (g_nsm <= 0) g_nsm = 1;
  }
  return g_nsm;
}

template <class K>
static unsigned grid_for(K kernel, uint64_t work, int block = 256) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm <= 0) per_sm = 1;
  uint64_t full = (uint64_t)per_sm * num_sms();
  uint64_t need = (work + block - 1) / block;
  return (unsigned)std::max<uint64_t>(1, std::min(full, need));
}


template <class T>
static cx<T> to_cx(cd c) {
  cx<T> v;
  v.x = (T)c.real();
  v.y = (T)c.imag();
  return v;
}

// Group geometry for k targets q on an n-qubit state: member s = r | c << k at offset
// sum_j r_j 2^{q_j} + c_j 2^{q_j + n}; the 2k bits sorted ascending for zero insertion.
template <int G>
static Group<G> make_group(int n, int k, const int* q) {
  Group<G> g;
  int nb = 2 * k;
  int bits[4];
  for (int j = 0; j < k; j++) { bits[j] = q[j]; bits[j + k] = q[j] + n; }
  for (int s = 0; s < G; s++) {
    uint64_t o = 0;
    for (int b = 0; b < nb; b++)
      if ((s >> b) & 1) o |= 1ull << bits[b];
    g.off[s] = o;
  }
  std::sort(bits, bits + nb);
  for (int b = 0; b < 4; b++) g.pos[b] = b < nb ? bits[b] : 0;
  return g;
}

// Does the sparse instantiation pay off?  Count multiply-adds it would issue vs the dense one.
static bool use_sparse(const std::vector<cd>& c, bool fp64) {
  int dense = 4 * (int)c.size(), sparse = 0;
  for (const cd& x : c) {
    int f = flag_of(x);
    sparse += f == FL_ZERO ? 0 : f == FL_ONE ? 2 : f == FL_CPLX ? 4 : 2;
  }
  return fp64 ? sparse < dense : 2 * sparse < dense;
}

template <class T>
static cudaError_t launch_pass_t(cx<T>* st, int n, const Pass& p, cudaStream_t s) {
  const uint64_t N = 1ull << (2 * n);
  const bool fp64 = sizeof(T) == 8;
  if (p.kind == KK_ELEM) {
    bool real = true;
    for (const cd& c : p.coef)
      if (c.imag() != 0.0) real = false;
    if (p.k == 1) {
      Diag1P<T> P;
      P.g = make_group<4>(n, 1, p.q);
      P.skip = 0;
      for (int i = 0; i < 4; i++) {
        P.f[i] = to_cx<T>(p.coef[i]);
        if (is_unit_factor(p.coef[i])) P.skip |= 1u << i;
      }
      const uint64_t ng = N / 4;
      if (real) k_diag1<T, true><<<grid_for(k_diag1<T, true>, ng), 256, 0, s>>>(st, ng, P);
      else k_diag1<T, false><<<grid_for(k_diag1<T, false>, ng), 256, 0, s>>>(st, ng, P);
    } else {
      Diag2P<T> P;
      P.g = make_group<16>(n, 2, p.q);
      P.skip = 0;
      for (int i = 0; i < 16; i++) {
        P.f[i] = to_cx<T>(p.coef[i]);
        if (is_unit_factor(p.coef[i])) P.skip |= 1u << i;
      }
      const uint64_t ng = N / 16;
      if (real) k_diag2<T, true><<<grid_for(k_diag2<T, true>, ng), 256, 0, s>>>(st, ng, P);
      else k_diag2<T, false><<<grid_for(k_diag2<T, false>, ng), 256, 0, s>>>(st, ng, P);
    }
    return cudaGetLastError();
  }
  if (p.kind == KK_SUP1) {
    Sup1P<T> P;
    P.g = make_group<4>(n, 1, p.q);
    for (int i = 0; i < 16; i++) { P.s[i] = to_cx<T>(p.coef[i]); P.fl[i] = (unsigned char)flag_of(p.coef[i]); }
    const uint64_t ng = N / 4;
    if (use_sparse(p.coef, fp64)) k_sup1<T, true><<<grid_for(k_sup1<T, true>, ng), 256, 0, s>>>(st, ng, P);
    else k_sup1<T, false><<<grid_for(k_sup1<T, false>, ng), 256, 0, s>>>(st, ng, P);
    return cudaGetLastError();
  }
  if (p.kind == KK_UNI2) {
    Uni2P<T> P;
    P.g = make_group<16>(n, 2, p.q);
    for (int i = 0; i < 16; i++) {
      P.u[i] = to_cx<T>(p.coef[i]);
      P.uc[i] = to_cx<T>(std::conj(p.coef[i]));
      P.fl[i] = (unsigned char)flag_of(p.coef[i]);
    }
    // conj keeps the flag class except ONE stays ONE; an entry equal to 1 has conj 1 as well.
    const uint64_t ng = N / 16;
    if constexpr (sizeof(T) == 4) {
      k_uni2_pair<T><<<grid_for(k_uni2_pair<T>, 2 * ng), 256, 0, s>>>(st, ng, P);
    } else {
      if (use_sparse(p.coef, fp64)) k_uni2_whole<T, true><<<grid_for(k_uni2_whole<T, true>, ng), 256, 0, s>>>(st, ng, P);
      else k_uni2_whole<T, false><<<grid_for(k_uni2_whole<T, false>, ng), 256, 0, s>>>(st, ng, P);
    }
    return cudaGetLastError();
  }
  if (p.kind == KK_SUP2) {
    Sup2P<T> P;
    P.g = make_group<16>(n, 2, p.q);
    for (int i = 0; i < 256; i++) { P.s[i] = to_cx<T>(p.coef[i]); P.fl[i] = (unsigned char)flag_of(p.coef[i]); }
    const uint64_t ng = N / 16;
    if (use_sparse(p.coef, fp64)) k_sup2<T, true><<<grid_for(k_sup2<T, true>, ng), 256, 0, s>>>(st, ng, P);
    else k_sup2<T, false><<<grid_for(k_sup2<T, false>, ng), 256, 0, s>>>(st, ng, P);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

double pass_touched_fraction(const Pass& p) {
  if (p.kind != KK_ELEM) return 1.0;
  int touched = 0;
  for (const cd& c : p.coef)
    if (!is_unit_factor(c)) touched++;
  return p.coef.empty() ? 1.0 : (double)touched / (double)p.coef.size();
}

static double flag_cost(const cd& c) {
  const int f = flag_of(c);
  return f == FL_ZERO ? 0.0 : f == FL_CPLX ? 4.0 : 2.0;
}

double pass_fma_per_amp(const Pass& p, bool fp64) {
  double sparse = 0.0;
  const double dense = 4.0 * (double)p.coef.size();
  for (const cd& c : p.coef) sparse += flag_cost(c);
  const double used = use_sparse(p.coef, fp64) ? sparse : dense;
  switch (p.kind) {
    case KK_ELEM: {  // one multiply per changed amplitude: 2 (real or imaginary factor) or 4 (complex)
      double t = 0.0;
      for (const cd& c : p.coef)
        if (!is_unit_factor(c)) t += flag_cost(c);
      return t / (double)p.coef.size();
    }
    case KK_SUP1: return used / 4.0;                         // 16 coefficients per 4 members
    case KK_UNI2: return (fp64 ? used : dense) * 8.0 / 16.0;  // each of U's 16 entries used 8 times per 16 members
    default: return used / 16.0;                              // 256 coefficients per 16 members
  }
}

cudaError_t launch_pass(int prec, void* state, int n, const Pass& p, cudaStream_t s) {
  if (prec == VQD_F32) return launch_pass_t<float>((cx<float>*)state, n, p, s);
  if (prec == VQD_F32_SPLIT) return launch_pass_t<df>((cx<df>*)state, n, p, s);
  return launch_pass_t<double>((cx<double>*)state, n, p, s);
}

template <class T>
static cudaError_t init_classical_t(cx<T>* st, int n, uint64_t basis, cudaStream_t s) {
  const uint64_t dim = 1ull << n;
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(cx<T>) * dim * dim, s);
  if (e != cudaSuccess) return e;
  k_set_one<T><<<1, 1, 0, s>>>(st, basis * (dim + 1));
  return cudaGetLastError();
}
cudaError_t launch_init_classical(int prec, void* state, int n, uint64_t basis, cudaStream_t s) {
  if (prec == VQD_F32) return init_classical_t<float>((cx<float>*)state, n, basis, s);
  if (prec == VQD_F32_SPLIT) return init_classical_t<df>((cx<df>*)state, n, basis, s);
  return init_classical_t<double>((cx<double>*)state, n, basis, s);
}

template <class T>
static cudaError_t init_product_t(cx<T>* st, int n, const double* e, cudaStream_t s) {
  const uint64_t dim = 1ull << n;
  cudaError_t err = cudaMemsetAsync(st, 0, sizeof(cx<T>) * dim * dim, s);
  if (err != cudaSuccess) return err;
  DiagProductP P;
  for (int q = 0; q < VQD_MAX_QUBITS; q++) P.e[q] = q < n ? e[q] : 0.0;
  k_set_diag_product<T><<<grid_for(k_set_diag_product<T>, dim), 256, 0, s>>>(st, n, P);
  return cudaGetLastError();
}
cudaError_t launch_init_product_diag(int prec, void* state, int n, const double* excited, cudaStream_t s) {
  if (prec == VQD_F32) return init_product_t<float>((cx<float>*)state, n, excited, s);
  if (prec == VQD_F32_SPLIT) return init_product_t<df>((cx<df>*)state, n, excited, s);
  return init_product_t<double>((cx<double>*)state, n, excited, s);
}

// Scratch: reduction partials.  kMaxParts bounds the blocks of one reduction launch.
static const uint64_t kMaxParts = 2048;
static const uint64_t kProbThreads = 1ull << 16;
size_t reduce_scratch_doubles() {
  return std::max<size_t>(2 * kMaxParts * kExpectTermsPerLaunch, kProbThreads);
}
size_t reduce_out_doubles() { return (1u << VQD_MAX_QUBITS) + 2 * kExpectTermsPerLaunch; }

static unsigned reduce_blocks(uint64_t work) {
  uint64_t b = (work + 255) / 256;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, std::min<uint64_t>(kMaxParts, 8ull * num_sms())));
}

template <class T>
static cudaError_t purity_t(const cx<T>* st, int n, double* scratch, double* out, cudaStream_t s) {
  const uint64_t N = 1ull << (2 * n);
  unsigned nb = reduce_blocks(N);
  k_purity<T><<<nb, 256, 0, s>>>(st, N, scratch);
  k_sum_rows<<<1, 256, 0, s>>>(scratch, nb, 0, 1, out);
  return cudaGetLastError();
}
cudaError_t launch_purity(int prec, const void* state, int n, double* scratch, double* out, cudaStream_t s) {
  if (prec == VQD_F32) return purity_t<float>((const cx<float>*)state, n, scratch, out, s);
  if (prec == VQD_F32_SPLIT) return purity_t<df>((const cx<df>*)state, n, scratch, out, s);
  return purity_t<double>((const cx<double>*)state, n, scratch, out, s);
}

template <class T>
static cudaError_t trace_t(const cx<T>* st, int n, double* scratch, double* out, cudaStream_t s) {
  unsigned nb = reduce_blocks(1ull << n);
  k_trace<T><<<nb, 256, 0, s>>>(st, n, scratch);
  k_sum_rows<<<2, 256, 0, s>>>(scratch, nb, 1, 2, out);
  return cudaGetLastError();
}
cudaError_t launch_trace(int prec, const void* state, int n, double* scratch, double* out, cudaStream_t s) {
  if (prec == VQD_F32) return trace_t<float>((const cx<float>*)state, n, scratch, out, s);
  if (prec == VQD_F32_SPLIT) return trace_t<df>((const cx<df>*)state, n, scratch, out, s);
  return trace_t<double>((const cx<double>*)state, n, scratch, out, s);
}

template <class T>
static cudaError_t prob_t(const cx<T>* st, int n, int m, const int* qubits, double* scratch, double* out,
                          cudaStream_t s) {
  ProbP P;
  std::memset(&P, 0, sizeof(P));
  P.m = m;
  unsigned used = 0;
  for (int j = 0; j < m; j++) { P.meas[j] = qubits[j]; used |= 1u << qubits[j]; }
  P.nr = 0;
  for (int q = 0; q < n; q++)
    if (!(used >> q & 1)) P.rest[P.nr++] = q;
  const uint64_t bins = 1ull << m, per_bin = 1ull << P.nr;
  uint64_t chunks = std::min<uint64_t>(per_bin, std::max<uint64_t>(1, kProbThreads / bins));
  const uint64_t len = per_bin / chunks;
  k_prob<T><<<grid_for(k_prob<T>, bins * chunks), 256, 0, s>>>(st, n, P, chunks, len, scratch);
  k_sum_rows<<<(unsigned)bins, 256, 0, s>>>(scratch, chunks, (int)chunks, 1, out);
  return cudaGetLastError();
}
cudaError_t launch_prob(int prec, const void* state, int n, int m, const int* qubits, double* scratch, double* out,
                        cudaStream_t s) {
  if (prec == VQD_F32) return prob_t<float>((const cx<float>*)state, n, m, qubits, scratch, out, s);
  if (prec == VQD_F32_SPLIT) return prob_t<df>((const cx<df>*)state, n, m, qubits, scratch, out, s);
  return prob_t<double>((const cx<double>*)state, n, m, qubits, scratch, out, s);
}

template <class T>
static cudaError_t expect_t(const cx<T>* st, int n, int nterms, const uint32_t* xm, const uint32_t* zy,
                            double* scratch, double* out, cudaStream_t s) {
  ExpectP P;
  std::memset(&P, 0, sizeof(P));
  for (int t = 0; t < nterms; t++) { P.xm[t] = xm[t]; P.zy[t] = zy[t]; }
  unsigned nb = std::min<unsigned>(reduce_blocks(1ull << n), (unsigned)(kMaxParts));
  dim3 grid(nb, nterms);
  k_expect<T><<<grid, 256, 0, s>>>(st, n, P, scratch);
  // value 2t + j sums part[(t * nb + b) * 2 + j] over b: row stride 2 nb for t, but j interleaves;
  // launch one row-sum per (t, j) with base offset (t * nb) * 2 + j and element stride 2.
  for (int j = 0; j < 2; j++) {
    // out[2t + j]: use a strided view: part + j, row stride 2 nb, element stride 2
    k_sum_rows<<<nterms, 256, 0, s>>>(scratch + j, nb, (int)(2 * nb), 2, out + (size_t)j * nterms);
  }
  return cudaGetLastError();
}
cudaError_t launch_expect(int prec, const void* state, int n, int nterms, const uint32_t* xmask, const uint32_t* zymask,
                          double* scratch, double* out, cudaStream_t s) {
  if (prec == VQD_F32) return expect_t<float>((const cx<float>*)state, n, nterms, xmask, zymask, scratch, out, s);
  if (prec == VQD_F32_SPLIT) return expect_t<df>((const cx<df>*)state, n, nterms, xmask, zymask, scratch, out, s);
  return expect_t<double>((const cx<double>*)state, n, nterms, xmask, zymask, scratch, out, s);
}

// ================================================================== batched reductions
namespace dev {
// One CTA per (instance, chunk of its amplitudes): diagonal -> probabilities (written directly),
// and FP64 partial sums of Re tr, Im tr and sum |rho_ij|^2 for the chunk.
struct BatchRedItem {
  uint64_t offset_amps;  // instance start in the batch allocation
  uint64_t begin, end;   // amplitude range of this chunk
  uint64_t prob_offset;  // where the instance's 2^n probabilities go
  int n;
  int inst;
};
template <class T>
__global__ void __launch_bounds__(256) k_batch_reduce(const cx<T>* __restrict__ all, const BatchRedItem* __restrict__ items,
                                                      double* __restrict__ probs, double* __restrict__ part) {
  __shared__ double sh[32];
  const BatchRedItem it = items[blockIdx.x];
  const cx<T>* st = all + it.offset_amps;
  const uint64_t dim = 1ull << it.n;
  double tr_re = 0, tr_im = 0, pur = 0;
  for (uint64_t i = it.begin + threadIdx.x; i < it.end; i += blockDim.x) {
    const cx<T> v = st[i];
    pur = fma((double)v.x, (double)v.x, fma((double)v.y, (double)v.y, pur));
    const uint64_t r = i & (dim - 1), c = i >> it.n;
    if (r == c) {
      tr_re += (double)v.x;
      tr_im += (double)v.y;
      probs[it.prob_offset + r] = (double)v.x;
    }
  }
  tr_re = block_sum(tr_re, sh);
  tr_im = block_sum(tr_im, sh);
  pur = block_sum(pur, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = tr_re;
    part[3 * blockIdx.x + 1] = tr_im;
    part[3 * blockIdx.x + 2] = pur;
  }
}
}  // namespace dev

cudaError_t launch_batch_reduce(int prec, const void* base, const std::vector<int>& n, const std::vector<size_t>& off_bytes,
                                double* d_probs, double* d_part, void* d_items, size_t nitems, cudaStream_t s) {
  if (prec == VQD_F32)
    dev::k_batch_reduce<float><<<(unsigned)nitems, 256, 0, s>>>((const cx<float>*)base, (const dev::BatchRedItem*)d_items,
                                                                d_probs, d_part);
  else if (prec == VQD_F32_SPLIT)
    dev::k_batch_reduce<dev::df><<<(unsigned)nitems, 256, 0, s>>>((const cx<dev::df>*)base,
                                                                  (const dev::BatchRedItem*)d_items, d_probs, d_part);
  else
    dev::k_batch_reduce<double><<<(unsigned)nitems, 256, 0, s>>>((const cx<double>*)base, (const dev::BatchRedItem*)d_items,
                                                                 d_probs, d_part);
  (void)n;
  (void)off_bytes;
  return cudaGetLastError();
}

size_t batch_reduce_item_bytes() { return sizeof(dev::BatchRedItem); }

void batch_reduce_items(const std::vector<int>& n, const std::vector<size_t>& off_bytes, size_t esize,
                        std::vector<unsigned char>& items, std::vector<int>& item_inst) {
  const uint64_t chunk = 1ull << 20;  // amplitudes per CTA
  uint64_t prob_off = 0;
  items.clear();
  item_inst.clear();
  for (size_t i = 0; i < n.size(); i++) {
    const uint64_t N = 1ull << (2 * n[i]);
    for (uint64_t b = 0; b < N; b += chunk) {
      dev::BatchRedItem it;
      it.offset_amps = off_bytes[i] / esize;
      it.begin = b;
      it.end = std::min(N, b + chunk);
      it.prob_offset = prob_off;
      it.n = n[i];
      it.inst = (int)i;
      const unsigned char* p = (const unsigned char*)&it;
      items.insert(items.end(), p, p + sizeof(it));
      item_inst.push_back((int)i);
    }
    prob_off += 1ull << n[i];
  }
}

// ================================================================== arithmetic peak probe
namespace dev {
// Eight independent FMA chains per thread (enough to cover the pipe latency), many warps per SM.
template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(T* __restrict__ sink, int iters, T seed) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; i++) a[i] = seed + (T)(i + threadIdx.x) * (T)1e-3;
  const T m = (T)0.9999999, c = (T)1e-7;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = fma(a[i], m, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) s += a[i];
  if (s == (T)-1) sink[0] = s;  // never true; keeps the chains live
}
}  // namespace dev

template <class T>
static cudaError_t fma_probe_t(cudaStream_t s, double* out) {
  T* sink = nullptr;  // never written (the kernel's condition is false); a valid address is still passed
  cudaError_t e = cudaMalloc(&sink, sizeof(T));
  if (e != cudaSuccess) return e;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int iters = sizeof(T) == 8 ? 4096 : 65536;
  const unsigned grid = 8u * num_sms();
  dev::k_fma_probe<T><<<grid, 256, 0, s>>>(sink, 256, (T)1);  // warm-up
  cudaEventRecord(a, s);
  dev::k_fma_probe<T><<<grid, 256, 0, s>>>(sink, iters, (T)1);
  cudaEventRecord(b, s);
  e = cudaEventSynchronize(b);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e == cudaSuccess) *out = (double)grid * 256.0 * iters * 8.0 / (ms * 1e-3);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  return e;
}

// ================================================================== allocation-free probabilities
// vqd_prob_static: the marginal-probability reduction with its partial sums in a file-scope device
// array instead of memory from cudaMalloc.  Every GPU that loads the library holds this array
// (128 KB) until the process exits.  Host code must not use the array's name as a device address;
// the address comes from cudaGetSymbolAddress, taken once per device with that device current.
static const int kStaticPartials = 1 << 14;
static __device__ __align__(256) double g_static_partials[kStaticPartials];

static std::mutex g_static_mu;
static double* g_static_ptr[64] = {nullptr};

static cudaError_t static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_partials);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = (double*)p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

template <class T>
static cudaError_t prob_static_t(const cx<T>* st, int n, int m, const int* qubits, double* scratch, double* out,
                                 cudaStream_t s) {
  ProbP P;
  std::memset(&P, 0, sizeof(P));
  P.m = m;
  unsigned used = 0;
  for (int j = 0; j < m; j++) { P.meas[j] = qubits[j]; used |= 1u << qubits[j]; }
  for (int q = 0; q < n; q++)
    if (!(used >> q & 1)) P.rest[P.nr++] = q;
  const uint64_t bins = 1ull << m, per_bin = 1ull << P.nr;
  // bins * chunks <= kStaticPartials (bins <= kStaticPartials is checked by the caller)
  const uint64_t chunks = std::min<uint64_t>(per_bin, (uint64_t)kStaticPartials / bins);
  k_prob<T><<<grid_for(k_prob<T>, bins * chunks), 256, 0, s>>>(st, n, P, chunks, per_bin / chunks, scratch);
  k_sum_rows<<<(unsigned)bins, 256, 0, s>>>(scratch, chunks, (int)chunks, 1, out);
  return cudaGetLastError();
}

}  // namespace vqd

extern "C" int vqd_measure_fma_rate(int which, void* stream, double* fma_per_s) {
  using namespace vqd;
  if (!fma_per_s || (which != 0 && which != 1)) return report_static_error(VQD_EINVAL, "vqd_measure_fma_rate: bad argument");
  cudaError_t e = which == 0 ? fma_probe_t<double>((cudaStream_t)stream, fma_per_s)
                             : fma_probe_t<float>((cudaStream_t)stream, fma_per_s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return report_static_error(VQD_EDEVICE, cudaGetErrorString(e));
  }
  return VQD_OK;
}

extern "C" int vqd_prob_static(const void* dev_state, int n, int prec, int m, const int* qubits, double* dev_out,
                               void* stream) {
  using namespace vqd;
  if (!dev_state || !qubits || !dev_out) return report_static_error(VQD_EINVAL, "vqd_prob_static: NULL argument");
  if (n < 1 || n > VQD_MAX_QUBITS) return report_static_error(VQD_EINVAL, "vqd_prob_static: n outside 1..16");
  if (prec != VQD_F64 && prec != VQD_F32 && prec != VQD_F32_SPLIT)
    return report_static_error(VQD_EINVAL, "vqd_prob_static: bad precision");
  if (m < 1 || m > n) return report_static_error(VQD_EINVAL, "vqd_prob_static: need 1 <= m <= n measured qubits");
  if (m > VQD_PROB_STATIC_MAX_M)
    return report_static_error(VQD_EINVAL,
                               "vqd_prob_static: more than 14 measured qubits; its static scratch holds 2^14 partial sums");
  unsigned used = 0;
  for (int j = 0; j < m; j++) {
    if (qubits[j] < 0 || qubits[j] >= n || (used >> qubits[j] & 1))
      return report_static_error(VQD_EINVAL, "vqd_prob_static: measured qubit out of range or repeated");
    used |= 1u << qubits[j];
  }
  // The kernels read whole amplitudes (8 bytes for complex64, 16 for complex128 and float-float) and
  // write doubles: a misaligned address would fault on the GPU, so it is refused here.
  const uintptr_t align = prec == VQD_F32 ? 8 : 16;
  if ((uintptr_t)dev_state % align != 0 || (uintptr_t)dev_out % 8 != 0)
    return report_static_error(VQD_EINVAL,
                               "vqd_prob_static: dev_state must be 8-byte (VQD_F32) or 16-byte aligned and dev_out 8-byte aligned");
  double* scratch = nullptr;
  cudaError_t e = static_scratch(&scratch);
  if (e == cudaSuccess) {
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == VQD_F32) e = prob_static_t<float>((const cx<float>*)dev_state, n, m, qubits, scratch, dev_out, s);
    else if (prec == VQD_F32_SPLIT) e = prob_static_t<df>((const cx<df>*)dev_state, n, m, qubits, scratch, dev_out, s);
    else e = prob_static_t<double>((const cx<double>*)dev_state, n, m, qubits, scratch, dev_out, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return report_static_error(VQD_EDEVICE, cudaGetErrorString(e));
  }
  return VQD_OK;
}
