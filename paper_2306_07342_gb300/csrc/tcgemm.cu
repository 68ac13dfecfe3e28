// Tensor-core path of libvqd: fused k-qubit blocks (k = 4, 5, 6) applied as dense GEMMs on the
// fifth-generation tensor cores of sm_103a (tcgen05.mma with TMEM accumulators, TMA tile loads).
//
// A block's operators are composed in FP64 into one 4^k x 4^k superoperator S (the matrix form of the
// block's Kraus map, Sec. 2).  For every assignment g of the 2n - 2k index bits outside the block, the
// 4^k amplitudes x_g at the block's row and column bits are replaced by S x_g.  In real arithmetic,
// with complex numbers interleaved (re, im), this is Y = X R^T over all groups: X has one row per group
// and 2 * 4^k columns, R = [[Re S, -Im S], [Im S, Re S]] interleaved the same way.  The GEMM runs with
//   M = 128 groups per tile (one TMEM lane each),
//   N = 256 output reals per work item (one TMEM accumulator slot of 256 columns; two slots per CTA),
//   K = 2 * 4^k input reals, in chunks of 16, each chunk accumulated in its own slot and the chunks
//   summed in FP32 registers.
// Split precision: the FP32 operands are split into limbs and the limb products accumulate in FP32:
//   3xTF32: x = hi + lo (hi = tf32(x), lo = tf32(x - hi)), products lo*hi + hi*lo + hi*hi;
//   BF16x3: x = b1 + b2 + b3 (each the bf16 rounding of the remainder), the six products b_i*b_j with
//   i + j <= 4, smallest first.
// The state (complex64) is read by the CTA's threads: thread m gathers group m's members (consecutive
// groups are consecutive amplitudes when the block's bits are not the lowest, so a warp's loads
// coalesce), splits them and stores them in the tensor core's K-major shared-memory layout.  R is split
// and laid out on the device in exactly that layout once per block, so each chunk of R is one TMA tile
// load (cp.async.bulk.tensor) per limb, completing on an mbarrier.  The result goes to a second state
// buffer (out of place), so n-tiles of the same groups may run on different CTAs.
//
// Every wait is bounded (about 2 s of the global timer): on expiry the kernel records an error, waits
// (bounded again) for its own copies and tensor-core operations, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "tcgemm.h"

namespace vqd {
namespace tc {

constexpr int kM = 128;       // groups per tile (MMA M, TMEM lanes)
constexpr int kNT = 256;      // output reals per work item (TMEM columns of one accumulator slot)
constexpr int kKc = 16;       // input reals per K chunk
constexpr int kThreads = 704;  // 4 gather warps, 16 readout warps, a TMA warp and an MMA warp
constexpr int kStages = 3;

// Limb schemes: element size, limbs, MMA K per instruction, products (pairs of limbs, smallest first).
template <int SCHEME> struct Scheme;
template <> struct Scheme<VQD_TC_3XTF32> {
  static constexpr int esz = 4, limbs = 2, kper = 8, nprod = 3;
  // products lo*hi, hi*lo, hi*hi (limb of A, limb of B)
  __host__ __device__ static constexpr int pa(int p) { return p == 0 ? 1 : 0; }
  __host__ __device__ static constexpr int pb(int p) { return p == 1 ? 1 : 0; }
};
template <> struct Scheme<VQD_TC_BF16X3> {
  static constexpr int esz = 2, limbs = 3, kper = 16, nprod = 6;
  // products b3*b1, b2*b2, b1*b3, b2*b1, b1*b2, b1*b1 (limb of A, limb of B)
  __host__ __device__ static constexpr int pa(int p) { return p == 0 ? 2 : p == 1 ? 1 : p == 3 ? 1 : 0; }
  __host__ __device__ static constexpr int pb(int p) { return p == 1 ? 1 : p == 2 ? 2 : p == 4 ? 1 : 0; }
};

// Bytes of one limb's chunk in shared memory: A (kM rows) and B (kNT rows), kKc elements per row.
template <int SCHEME> __host__ __device__ constexpr int a_bytes() { return kM * kKc * Scheme<SCHEME>::esz; }
template <int SCHEME> __host__ __device__ constexpr int b_bytes() { return kNT * kKc * Scheme<SCHEME>::esz; }
template <int SCHEME> __host__ __device__ constexpr int stage_bytes() {
  return Scheme<SCHEME>::limbs * (a_bytes<SCHEME>() + b_bytes<SCHEME>());
}
constexpr int kMaxMembers = 4096;  // 4^6
constexpr int kBarBytes = 8 * (3 * kStages + 8) + 16;  // mbarriers, TMEM address, failure flag
constexpr int kRingBytes = 4 * 16 / 2 * 128 * 8;         // 4 chunks x 8 members x 128 groups x float2
template <int SCHEME> __host__ __device__ constexpr size_t smem_bytes() {
  return 1024 + (size_t)kStages * stage_bytes<SCHEME>() + kMaxMembers * 4 + kBarBytes + kRingBytes;
}

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete; false after about 2 s.
__device__ __noinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  if (mbar_try(a, parity)) return true;
  const uint64_t t0 = gtimer();
  for (;;) {
    for (int i = 0; i < 64; i++)
      if (mbar_try(a, parity)) return true;
    if (gtimer() - t0 > 2000000000ull) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand without swizzle: 8-row x 16-byte core matrices; lbo = byte stride between core
// matrices along K, sbo = byte stride between 8-row groups; descriptor version 1 (sm_100 family).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor: FP32 accumulator, A and B of format fmt (TF32 = 2 for kind::tf32, BF16 = 1 for
// kind::f16), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, uint32_t M, uint32_t N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <int SCHEME>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (SCHEME == VQD_TC_3XTF32)
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                 "l"(a), "l"(b), "r"(id), "r"(acc)
                 : "memory");
  else
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                 "l"(a), "l"(b), "r"(id), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 32 lanes x 16 columns of 32 bits: thread i of the warp receives lane (base lane + i), 16 columns.  The
// registers are valid after tmem_wait().
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Limbs of one FP32 value packed for shared memory.
template <int SCHEME> struct Limbs;
template <> struct Limbs<VQD_TC_3XTF32> {
  float l[2];
  __device__ __forceinline__ explicit Limbs(float x) {
    l[0] = tf32r(x);
    l[1] = tf32r(x - l[0]);
  }
};
template <> struct Limbs<VQD_TC_BF16X3> {
  __nv_bfloat16 l[3];
  __device__ __forceinline__ explicit Limbs(float x) {
    l[0] = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(l[0]);
    l[1] = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(l[1]);
    l[2] = __float2bfloat16_rn(r2);
  }
};

// ------------------------------------------------------------------ the block kernel
// Warp-specialised and persistent: every role walks the same sequence of (work item, K chunk) pairs and
// the roles hand chunks to one another through mbarriers.
//   warps 0-3, gather: one thread per group row loads the row's 8 members of the chunk (three chunks
//     ahead, cp.async into a shared-memory ring), splits them into limbs and stores them into the K-major
//     A tile of a shared-memory stage;
//   warp 20 (one lane), TMA: loads the chunk's limbs of R into the stage (cp.async.bulk.tensor);
//   warp 21 (one lane), MMA: when both halves of a stage are full and one of two TMEM slots is free, issues the
//     chunk's tcgen05.mma (accumulating into the slot from zero) and commits to the stage's "empty" and the
//     slot's "full" barriers;
//   warps 4-19, readout: four threads per group row read a quarter of the row's lane of the slot each
//     (tcgen05.ld), add it into FP32 registers and free the slot; after the item's last chunk they write
//     the group's outputs.
// The tensor core's accumulation rounds toward zero, so summing all 2 * 4^k inputs in TMEM would shrink
// every output by roughly (number of additions) x 2^-25 (measured: a trace 3.6e-5 low after 17 blocks of
// k = 4); summing one chunk's 16 inputs there and the chunks in registers (round to nearest) keeps the
// result unbiased.
constexpr int kGatherThreads = 128, kReadThreads = 512;  // one gather thread and four readout threads per group row
constexpr int kTmaWarp = 20, kMmaWarp = 21;
constexpr int kGatherWarps = kGatherThreads / 32, kMemPerThread = 8 * kM / kGatherThreads;
constexpr int kAhead = 3, kRing = kAhead + 1;  // chunks of the state in flight ahead of the one being split
constexpr int kSlots = 2;                       // TMEM accumulator slots of kNT columns: all 512 columns

template <int SCHEME>
__global__ void __launch_bounds__(kThreads, 1) k_tc_block(const __grid_constant__ CUtensorMap tmB, const TcParams P) {
  using Sc = Scheme<SCHEME>;
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint32_t* s_off = (uint32_t*)(sm + kStages * stage_bytes<SCHEME>());
  uint64_t* full_a = (uint64_t*)(s_off + kMaxMembers);
  uint64_t* full_b = full_a + kStages;
  uint64_t* empty = full_b + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + kSlots;
  uint32_t* s_tmem = (uint32_t*)(tempty + kSlots);
  volatile int* s_flag = (volatile int*)(s_tmem + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto a_tile = [&](int st, int limb) { return sm + st * stage_bytes<SCHEME>() + limb * a_bytes<SCHEME>(); };
  auto b_tile = [&](int st, int limb) {
    return sm + st * stage_bytes<SCHEME>() + Sc::limbs * a_bytes<SCHEME>() + limb * b_bytes<SCHEME>();
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(s_tmem)), "r"(kSlots * kNT)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kStages; i++) {
      mbar_init(su32(&full_a[i]), kGatherThreads / 32);  // one arrival per gather warp
      mbar_init(su32(&full_b[i]), 1);
      mbar_init(su32(&empty[i]), 1);
    }
    for (int i = 0; i < kSlots; i++) {
      mbar_init(su32(&tfull[i]), 1);
      mbar_init(su32(&tempty[i]), kReadThreads / 32);  // one arrival per readout warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_flag = 0;
  }
  // member offsets: bit j of member s sits at index bit P.mbit[j]
  for (int s = tid; s < P.nmem; s += kThreads) {
    uint32_t o = 0;
    for (int j = 0; j < P.mb; j++)
      if (s >> j & 1) o |= 1u << P.mbit[j];
    s_off[s] = o;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  const uint64_t items = (uint64_t)P.n_gtiles * P.n_ntiles;
  const int nk = P.n_kchunks;
  auto group_base = [&](uint32_t g) {  // zero bits inserted at the block's (ascending) bit positions
    uint32_t b = g;
    for (int j = 0; j < P.mb; j++) {
      const uint32_t low = (1u << P.pos[j]) - 1u;
      b = (b & low) | ((b & ~low) << 1);
    }
    return b;
  };
  // a wait that gave up marks the CTA failed; every role then leaves its loop
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    if (mbar_wait(su32(bar), parity)) return true;
    *s_flag = 1;
    return false;
  };

  if (warp < kGatherWarps) {
    // ---------------------------------------------------------------- gather
    // Thread (row, half) handles members 4 half .. 4 half + 3 of each chunk of group row `row`.  The
    // members of chunk c + kAhead are copied into a ring of raw FP32 values in shared memory (cp.async,
    // [slot][member][row] so that a warp's copies and reads are conflict-free) while chunk c is split; each
    // thread reads back only what it copied itself.
    const int row = tid & (kM - 1), half = tid >> 7;  // half = 0 with one gather thread per row
    const float2* __restrict__ X = P.X;
    float2* ring = (float2*)(sm + kStages * stage_bytes<SCHEME>() + kMaxMembers * 4 + kBarBytes);
    constexpr uint32_t kAslice = kM * 16;
    constexpr int kElemPer16 = 16 / Sc::esz;
    const uint64_t my_items = items > blockIdx.x ? (items - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const uint64_t total = my_items * nk;
    // cursor of the chunk whose copies are issued next: (item, chunk), advanced without divisions
    uint64_t p_item = blockIdx.x;
    int p_kc = 0, p_slot = 0;
    uint32_t p_base = 0;
    bool p_valid = false, p_new = true;
    uint64_t issued = 0;
    auto issue = [&]() {  // copies of the next chunk (if any), one commit group per chunk
      if (issued < total) {
        if (p_new) {
          const uint32_t g = (uint32_t)(p_item / P.n_ntiles) * kM + row;
          p_valid = g < P.groups;
          p_base = p_valid ? group_base(g) : 0u;
          p_new = false;
        }
        float2* dst = ring + ((size_t)p_slot * (kKc / 2) + kMemPerThread * half) * kM + row;
        const uint32_t* off = s_off + p_kc * (kKc / 2) + kMemPerThread * half;
        if (p_valid) {
#pragma unroll
          for (int e = 0; e < kMemPerThread; e++)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(su32(dst + e * kM)), "l"(X + p_base + off[e])
                         : "memory");
        } else {
#pragma unroll
          for (int e = 0; e < kMemPerThread; e++) dst[e * kM] = make_float2(0.f, 0.f);
        }
        issued++;
        p_slot = p_slot + 1 == kRing ? 0 : p_slot + 1;
        if (++p_kc == nk) {
          p_kc = 0;
          p_item += gridDim.x;
          p_new = true;
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int a = 0; a < kAhead; a++) issue();
    int r_slot = 0, st = 0;
    uint32_t ph = 0;
    for (uint64_t c = 0; c < total; c++) {
      issue();
      asm volatile("cp.async.wait_group %0;" ::"n"(kAhead) : "memory");
      const float2* src = ring + ((size_t)r_slot * (kKc / 2) + kMemPerThread * half) * kM + row;
      r_slot = r_slot + 1 == kRing ? 0 : r_slot + 1;
      float2 vcur[kMemPerThread];
#pragma unroll
      for (int e = 0; e < kMemPerThread; e++) vcur[e] = src[e * kM];
      if (!wait(&empty[st], ph ^ 1u) || *s_flag) break;
#pragma unroll
      for (int l = 0; l < Sc::limbs; l++) {
        unsigned char* at = a_tile(st, l);
        // K slice q holds reals [q * kElemPer16, (q + 1) * kElemPer16) of the chunk, row r at 16 r; this
        // thread's members start at slice kMemPerThread * half * 2 / kElemPer16
        constexpr int kPairsPerSlice = kElemPer16 / 2;  // complex members per 16-byte slice
        const int q0 = kMemPerThread * half / kPairsPerSlice;
#pragma unroll
        for (int q = 0; q < kMemPerThread / kPairsPerSlice; q++) {
          if constexpr (SCHEME == VQD_TC_3XTF32) {
            float4 w;
            w.x = Limbs<SCHEME>(vcur[2 * q].x).l[l];
            w.y = Limbs<SCHEME>(vcur[2 * q].y).l[l];
            w.z = Limbs<SCHEME>(vcur[2 * q + 1].x).l[l];
            w.w = Limbs<SCHEME>(vcur[2 * q + 1].y).l[l];
            *(float4*)(at + (q0 + q) * kAslice + 16 * row) = w;
          } else {
            __nv_bfloat16 h[8];
#pragma unroll
            for (int e = 0; e < 4; e++) {
              h[2 * e] = Limbs<SCHEME>(vcur[4 * q + e].x).l[l];
              h[2 * e + 1] = Limbs<SCHEME>(vcur[4 * q + e].y).l[l];
            }
            *(uint4*)(at + (q0 + q) * kAslice + 16 * row) = *(const uint4*)h;
          }
        }
      }
      // every lane's stores are made visible to the tensor core's (async) proxy, then one lane per warp
      // arrives: same-address shared-memory arrivals serialise, so 8 per chunk instead of 256
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&full_a[st])) : "memory");
      if (++st == kStages) {
        st = 0;
        ph ^= 1u;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp < kGatherWarps + kReadThreads / 32) {
    // ---------------------------------------------------------------- readout
    // TMEM lane = group row; warp w reads lanes 32 (w % 4) .. 32 (w % 4) + 31 and one of the column quarters
    float2* __restrict__ Y = P.Y;
    constexpr int kCols = kNT * kM / kReadThreads;
    const int row = (warp & 3) * 32 + lane, ch = (warp - kGatherWarps) >> 2;
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + ch * kCols;
    uint32_t c = 0;
    bool ok = true;
    float sum[kCols];
    for (uint64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
      const uint32_t gt = (uint32_t)(item / P.n_ntiles), nt = (uint32_t)(item % P.n_ntiles);
      const uint32_t g = gt * kM + row;
#pragma unroll
      for (int i = 0; i < kCols; i++) sum[i] = 0.f;
      for (int kc = 0; kc < nk; kc++, c++) {
        const int slot = c % kSlots;
        if (!wait(&tfull[slot], (c / kSlots) & 1u) || *s_flag) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < kCols; c0 += 16) {
          uint32_t v[16];
          tmem_ld16(lane_addr + slot * kNT + c0, v);
          tmem_wait();
#pragma unroll
          for (int i = 0; i < 16; i++) sum[c0 + i] += __uint_as_float(v[i]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tempty[slot])) : "memory");
      }
      if (!ok) break;
      if (g < P.groups) {
        const uint32_t base = group_base(g);
        const uint32_t out0 = nt * (kNT / 2) + ch * (kCols / 2);
#pragma unroll
        for (int e = 0; e < kCols / 2; e++) Y[base + s_off[out0 + e]] = make_float2(sum[2 * e], sum[2 * e + 1]);
      }
    }
  } else if (warp == kTmaWarp) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      const uint32_t stage_tx = (uint32_t)(Sc::limbs * b_bytes<SCHEME>());
      uint32_t c = 0;
      bool ok = true;
      for (uint64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const uint32_t nt = (uint32_t)(item % P.n_ntiles);
        for (int kc = 0; kc < nk; kc++, c++) {
          const int st = c % kStages;
          if (!wait(&empty[st], ((c / kStages) & 1u) ^ 1u) || *s_flag) { ok = false; break; }
          mbar_expect_tx(su32(&full_b[st]), stage_tx);
          for (int l = 0; l < Sc::limbs; l++) {
            const int blk = (nt * nk + kc) * Sc::limbs + l;
            tma_load_2d(su32(b_tile(st, l)), &tmB, 0, blk * (kNT * kKc / 256), su32(&full_b[st]));
          }
        }
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t id = idesc(SCHEME == VQD_TC_3XTF32 ? 2u : 1u, kM, kNT);
      constexpr uint32_t kAslice = kM * 16, kBslice = kNT * 16;  // bytes per 16-byte K slice of A and B
      constexpr int kSteps = kKc / Sc::kper;                       // MMAs along K per chunk and product
      uint32_t c = 0;
      bool ok = true;
      for (uint64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
        for (int kc = 0; kc < nk; kc++, c++) {
          const int st = c % kStages, slot = c % kSlots;
          const uint32_t ph = (c / kStages) & 1u;
          if (!wait(&full_b[st], ph) || !wait(&full_a[st], ph) || !wait(&tempty[slot], ((c / kSlots) & 1u) ^ 1u) ||
              *s_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + slot * kNT;
#pragma unroll
          for (int ks = 0; ks < kSteps; ks++)
#pragma unroll
            for (int p = 0; p < Sc::nprod; p++) {
              const uint64_t ad = sdesc(su32(a_tile(st, Sc::pa(p))) + ks * 2 * kAslice, kAslice, 128);
              const uint64_t bd = sdesc(su32(b_tile(st, Sc::pb(p))) + ks * 2 * kBslice, kBslice, 128);
              mma<SCHEME>(d, ad, bd, id, (ks > 0 || p > 0) ? 1u : 0u);
            }
          mma_commit(su32(&empty[st]));
          mma_commit(su32(&tfull[slot]));
        }
      }
      // leave with no tensor-core operation of this CTA in flight (bounded), whatever happened
      if (c > 0) mbar_wait(su32(&tfull[(c - 1) % kSlots]), ((c - 1) / kSlots) & 1u);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && *s_flag) atomicExch(P.err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kSlots * kNT) : "memory");
}

// ------------------------------------------------------------------ R: limbs in the tiled K-major layout
// S is read from the composition buffer (complex128, layout of compose_index); block (nt, kc, limb) of
// the output holds rows n in [nt * kNT, (nt + 1) * kNT) and reals k in [kc * kKc, (kc + 1) * kKc) as
// [k slice][row][16 bytes].
template <int SCHEME>
__global__ void k_tc_build_r(const double2* __restrict__ S, int k, int n_kchunks, unsigned char* __restrict__ out) {
  using Sc = Scheme<SCHEME>;
  const uint32_t D = 1u << (2 * k), NR = 2 * D;  // members and reals
  const uint64_t total = (uint64_t)NR * NR;
  constexpr int E = 16 / Sc::esz;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t row = (uint32_t)(t / NR), col = (uint32_t)(t % NR);  // output real, input real
    const uint32_t i = row >> 1, a = row & 1, j = col >> 1, b = col & 1;
    // S[i][j] sits at compose_index(i, j)
    const uint32_t mk = (1u << k) - 1u;
    const uint32_t r = i & mk, c = i >> k, jl = j & mk, jh = j >> k;
    const uint64_t idx = (uint64_t)r | ((uint64_t)jl << k) | ((uint64_t)c << (2 * k)) | ((uint64_t)jh << (3 * k));
    const double2 s = S[idx];
    const double v = a == 0 ? (b == 0 ? s.x : -s.y) : (b == 0 ? s.y : s.x);
    const uint32_t nt = row / kNT, nl = row % kNT, kc = col / kKc, kl = col % kKc;
    const uint32_t q = kl / E, ke = kl % E;
    const size_t within = ((size_t)q * kNT + nl) * E + ke;
    if constexpr (SCHEME == VQD_TC_3XTF32) {
      const float hi = tf32r((float)v);
      const float lo = tf32r((float)(v - (double)hi));
      const size_t b0 = ((size_t)(nt * n_kchunks + kc) * 2) * (kNT * kKc);
      ((float*)out)[b0 + within] = hi;
      ((float*)out)[b0 + kNT * kKc + within] = lo;
    } else {
      const float x = (float)v;
      const __nv_bfloat16 h1 = __float2bfloat16_rn(x);
      const double r1 = v - (double)__bfloat162float(h1);
      const __nv_bfloat16 h2 = __float2bfloat16_rn((float)r1);
      const double r2 = r1 - (double)__bfloat162float(h2);
      const __nv_bfloat16 h3 = __float2bfloat16_rn((float)r2);
      const size_t b0 = ((size_t)(nt * n_kchunks + kc) * 3) * (kNT * kKc);
      __nv_bfloat16* o = (__nv_bfloat16*)out;
      o[b0 + within] = h1;
      o[b0 + kNT * kKc + within] = h2;
      o[b0 + 2 * kNT * kKc + within] = h3;
    }
  }
}

// The identity superoperator in the composition layout (see compose_index).
__global__ void k_tc_identity(double2* __restrict__ S, int k) {
  const uint32_t D = 1u << (2 * k);
  const uint32_t mk = (1u << k) - 1u;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < D; j += gridDim.x * blockDim.x) {
    const uint32_t r = j & mk, c = j >> k;
    const uint64_t idx = (uint64_t)r | ((uint64_t)r << k) | ((uint64_t)c << (2 * k)) | ((uint64_t)c << (3 * k));
    S[idx] = make_double2(1.0, 0.0);
  }
}

}  // namespace tc

// ================================================================== host side
using namespace tc;

std::vector<TcBlock> plan_tc_blocks(const std::vector<Op>& ops, int n, int k) {
  std::vector<TcBlock> blocks;
  const uint32_t full = n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const size_t kWindow = 1024;
  std::vector<int> remaining(ops.size());
  for (size_t i = 0; i < ops.size(); i++) remaining[i] = (int)i;
  std::vector<int> deferred;
  while (!remaining.empty()) {
    TcBlock b;
    deferred.clear();
    uint32_t dmask = 0;
    size_t i = 0;
    for (; i < remaining.size() && i < kWindow; i++) {
      const Op& op = ops[remaining[i]];
      uint32_t m = 0;
      for (int j = 0; j < op.k; j++) m |= 1u << op.q[j];
      if (!(m & dmask) && __builtin_popcount(b.qmask | m) <= k) {
        b.qmask |= m;
        b.ops.push_back(remaining[i]);
        b.weight += op.weight;
      } else {
        deferred.push_back(remaining[i]);
        dmask |= m;
      }
      if (dmask == full) {
        i++;
        break;
      }
    }
    blocks.push_back(std::move(b));
    std::vector<int> next(deferred);
    next.insert(next.end(), remaining.begin() + i, remaining.end());
    remaining.swap(next);
  }
  return blocks;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

size_t tc_r_bytes(int k, int scheme) {
  const size_t NR = (size_t)2 << (2 * k);
  return NR * NR * (scheme == VQD_TC_3XTF32 ? 8 : 6);
}
size_t tc_compose_bytes(int k) { return sizeof(double2) << (4 * k); }

cudaError_t tc_compose_init(void* S, int k, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(S, 0, tc_compose_bytes(k), s);
  if (e != cudaSuccess) return e;
  const uint32_t D = 1u << (2 * k);
  k_tc_identity<<<(D + 255) / 256, 256, 0, s>>>((double2*)S, k);
  return cudaGetLastError();
}

cudaError_t tc_build_r(const void* S, int k, int scheme, void* R, cudaStream_t s) {
  const int n_kchunks = (2 << (2 * k)) / kKc;
  const uint64_t total = (uint64_t)(2u << (2 * k)) * (2u << (2 * k));
  const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, 8ull * num_sms());
  if (scheme == VQD_TC_3XTF32)
    k_tc_build_r<VQD_TC_3XTF32><<<grid, 256, 0, s>>>((const double2*)S, k, n_kchunks, (unsigned char*)R);
  else
    k_tc_build_r<VQD_TC_BF16X3><<<grid, 256, 0, s>>>((const double2*)S, k, n_kchunks, (unsigned char*)R);
  return cudaGetLastError();
}

template <int SCHEME>
static cudaError_t launch_t(const TcParams& P, const void* R, int k, cudaStream_t s) {
  using Sc = Scheme<SCHEME>;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // R as a 2-D tensor of rows of 256 elements; one limb's chunk is kNT * kKc / 256 rows
  const uint64_t elems = (uint64_t)(2u << (2 * k)) * (2u << (2 * k)) * Sc::limbs;
  CUtensorMap tm;
  cuuint64_t gdim[2] = {256, (cuuint64_t)(elems / 256)};
  cuuint64_t gstride[1] = {(cuuint64_t)256 * Sc::esz};
  cuuint32_t box[2] = {256, (cuuint32_t)(kNT * kKc / 256)};
  cuuint32_t estride[2] = {1, 1};
  CUresult cr = enc(&tm, SCHEME == VQD_TC_3XTF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void*>(R), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const size_t smem = smem_bytes<SCHEME>();
  cudaError_t e = cudaFuncSetAttribute(k_tc_block<SCHEME>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const uint64_t items = (uint64_t)P.n_gtiles * P.n_ntiles;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_block<SCHEME>, kThreads, smem) != cudaSuccess ||
      per_sm <= 0)
    per_sm = 1;
  per_sm = std::min(per_sm, 2);  // at most two CTAs of 256 TMEM columns fill an SM's 512
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(items, (uint64_t)per_sm * num_sms()));
  k_tc_block<SCHEME><<<grid, kThreads, smem, s>>>(tm, P);
  return cudaGetLastError();
}

cudaError_t tc_apply(const void* X, void* Y, int n, int k, const int* q, int scheme, const void* R, int* d_err,
                     cudaStream_t s) {
  TcParams P;
  std::memset(&P, 0, sizeof(P));
  P.X = (const float2*)X;
  P.Y = (float2*)Y;
  P.R = R;
  P.groups = (uint32_t)(1ull << (2 * (n - k)));
  P.n_gtiles = (P.groups + kM - 1) / kM;
  P.n_ntiles = (2 << (2 * k)) / kNT;
  P.n_kchunks = (2 << (2 * k)) / kKc;
  P.nmem = 1 << (2 * k);
  P.mb = 2 * k;
  int bits[12];
  for (int j = 0; j < k; j++) {
    bits[j] = q[j];
    bits[j + k] = q[j] + n;
    P.mbit[j] = (uint32_t)q[j];
    P.mbit[j + k] = (uint32_t)(q[j] + n);
  }
  std::sort(bits, bits + 2 * k);
  for (int j = 0; j < 2 * k; j++) P.pos[j] = bits[j];
  P.err = d_err;
  if (scheme == VQD_TC_3XTF32) return launch_t<VQD_TC_3XTF32>(P, R, k, s);
  return launch_t<VQD_TC_BF16X3>(P, R, k, s);
}

}  // namespace vqd
