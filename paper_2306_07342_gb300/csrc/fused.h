// Fused path of libvqd: stage planning (host) and the shared-memory tiled stage kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "vqd_internal.h"

namespace vqd {

constexpr int kMaxTileBits = 16;
constexpr int kCoefCap = 2048;  // complex coefficients of one stage, staged in shared memory
constexpr int kOpCap = 512;     // operator descriptors of one stage, staged in shared memory
constexpr int kBlockCap = 64;   // blocks (shared-memory sweeps) of one stage, their descriptors staged in shared memory

// Operator kinds inside a block on qubits (a, b); member index s = ra | rb << 1 | ca << 2 | cb << 3.
enum BlockOpKind { BK_DIAG_A = 0, BK_SUP1_A, BK_DIAG_B, BK_SUP1_B, BK_DIAG2, BK_UNI2, BK_SUP2 };

struct BlockOp {
  int kind;
  int coef;       // offset within the stage's coefficients
  uint32_t skip;  // diagonal kinds: members whose factor is 1 (left untouched)
};

// A block: operators acting within one qubit (nq = 1) or one pair (nq = 2), applied back to back
// to amplitudes held in registers (one shared-memory sweep per block).
struct TileBlock {
  int nq;
  int lbit[4];     // tile-local bits: a_row, b_row, a_col, b_col (nq = 2) or a_row, a_col (nq = 1)
  int lsorted[4];  // the same bits ascending (zero insertion)
  int op_begin, op_end;
};

// One stage: a set of index bits held in a shared-memory tile and the blocks applied to it.
struct StageDesc {
  int nbits;                 // tile-local bits (ascending global positions in bits[])
  int bits[kMaxTileBits];
  int nrest;                 // remaining global bit positions (ascending), deposited from the tile index
  int rest[2 * VQD_MAX_QUBITS];
  int block_begin, block_end;
  int coef_begin, coef_end;  // this stage's coefficients in the plan's array (<= kCoefCap of them)
  int op_begin, op_end;      // this stage's operator descriptors (<= kOpCap of them)
  double weight;             // original operations applied by this stage
  double fma_per_amp;        // real multiply-adds of the stage's sweeps per amplitude of the state (arithmetic as
                             // the kernel performs it: dense for complex64, structured for FP64 and float-float)
  int herm;                  // 1: Hermitian stage (see plan_fused): rows and columns of the tile on the same qubits,
                             // rest[] = the m row rest bits then the same qubits' m column rest bits (nrest = 2m),
                             // and only the tiles whose row rest index is <= their column rest index run
  double frac;               // fraction of the state's amplitudes this stage reads (1, or (K + 1) / 2K for K = 2^m)
};

// Work items of a Hermitian stage come in groups of 2^b x 2^b tiles (b = kHermGroupBits, at most m) that share
// the high bits of their row and column rest indices: the groups on or above the diagonal of the grid of groups,
// K_h (K_h + 1) / 2 of them for K_h = K / 2^b, each with every (low row bits, low column bits) pair.  Tiles
// processed together then fill whole DRAM lines with both their own stores and their mirror stores (the lowest
// rest bits are the lowest qubits outside the tile).  In a diagonal group the items below the diagonal do
// nothing.
constexpr int kHermGroupBits = 2;
__host__ __device__ inline int herm_group_bits(int nrest) {
  return nrest / 2 < kHermGroupBits ? nrest / 2 : kHermGroupBits;
}
// Work items of one pass of the stage: 2^nrest tiles, or the Hermitian stage's groups of tiles.
__host__ __device__ inline uint64_t stage_work_tiles(const StageDesc& s) {
  if (!s.herm) return 1ull << s.nrest;
  const int b = herm_group_bits(s.nrest);
  const uint64_t Kh = 1ull << (s.nrest / 2 - b);
  return (Kh * (Kh + 1) / 2) << (2 * b);
}

struct FusedPlan {
  bool herm = false;  // planned on symmetric tiles (Hermitian stages)
  std::vector<StageDesc> stages;
  std::vector<TileBlock> blocks;
  std::vector<BlockOp> ops;
  std::vector<cd> coef;
  std::vector<uint8_t> flag;  // structure of each coefficient (FL_* of numeric.h), used by FP64 and float-float
  int max_bits = 0;
};

// Tile shape of the fused path: index bits held in a tile (0 = default for the precision) and
// low row bits carried along in every tile for contiguous DRAM runs (-1 = default).
struct TileShape {
  int tile_bits = 0;
  int passengers = -1;
};

// Group the compiled operators of one n-qubit instance into stages of at most `fuse_qubits`
// qubits (0 = default) whose tiles have the given shape.
// herm: the state is Hermitian (a density matrix).  If every operator also preserves Hermiticity
// (S[(c,r),(c',r')] = conj S[(r,c),(r',c')], true of every Kraus map), the stages are planned on symmetric
// tiles (the passenger qubits' column bits join the tile) and each stage runs only the tiles on or above
// the diagonal of the tile grid; an off-diagonal tile also writes its conjugate transpose into its mirror
// tile, a diagonal tile writes its upper triangle's conjugate into its lower one (and a real diagonal),
// so that the whole state stays exactly Hermitian.  Otherwise the plan is the general one.
FusedPlan plan_fused(const std::vector<Op>& ops, int n, int prec, int fuse_qubits, TileShape shape = TileShape(),
                     bool herm = false);
bool preserves_hermiticity(const Op& op);

// Per-instance description used by the batched kernel.
struct BatchInst {
  uint64_t offset_amps;  // first amplitude of the instance in the batch allocation
  int n;
  int stage_begin, stage_end;
  double cost;
};
// One work item of a wave: a chunk of tiles of one stage of one instance.
struct WaveItem {
  int inst;
  int stage;
  uint32_t tile_begin, tile_count;
};
struct BatchPlan {
  FusedPlan all;                 // stages of every instance, concatenated (offsets global)
  std::vector<BatchInst> inst;   // indexed by instance id
  std::vector<int> passes;       // passes over the state per instance
  std::vector<WaveItem> items;   // wave w holds items [wave_begin[w], wave_begin[w+1]), largest first
  std::vector<int> wave_begin;
};
// Concatenate per-instance plans (planned independently, e.g. on several host threads).
BatchPlan merge_batch(const std::vector<FusedPlan>& plans, const std::vector<int>& n,
                      const std::vector<size_t>& byte_offsets, int prec);
// Device buffers reused across calls (grown on demand; freed with the context).
struct FusedCache {
  void* d_blocks = nullptr;
  size_t blocks_cap = 0;
  void* d_ops = nullptr;
  size_t ops_cap = 0;
  void* d_coef = nullptr;
  size_t coef_cap = 0;
  void* d_flag = nullptr;
  size_t flag_cap = 0;
  void* d_stages = nullptr;
  size_t stages_cap = 0;
  void* d_inst = nullptr;
  size_t inst_cap = 0;
  void* d_items = nullptr;
  size_t items_cap = 0;
  int* d_counter = nullptr;  // one work counter per wave
  size_t counter_cap = 0;
};
void fused_cache_free(FusedCache& c);
void upload_plan(FusedCache& c, const FusedPlan& p, int prec, cudaStream_t s);
cudaError_t launch_stage(FusedCache& c, const FusedPlan& p, int stage, int prec, void* state, int n, cudaStream_t s);
void upload_batch(FusedCache& c, const BatchPlan& p, int prec, cudaStream_t s);
cudaError_t launch_batch(FusedCache& c, const BatchPlan& p, int prec, void* base, cudaStream_t s);

// Largest tile (index bits) the shared-memory budget allows for a precision, and the defaults.
int tile_bits_budget(int prec);
int default_passengers(int prec, bool herm = false);

}  // namespace vqd
