// Fused path of libvqd: stage planning (host) and the shared-memory tiled stage kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "vqd_internal.h"

namespace vqd {

constexpr int kMaxTileBits = 16;

// One operator inside a stage, addressed by tile-local bit positions (device record).
struct TileOp {
  int kind;        // KK_ELEM / KK_SUP1 / KK_UNI2 / KK_SUP2
  int nb;          // 2k member bits
  int lbit[4];     // tile-local bit of member bit j (row bits of q0, q1, then column bits)
  int lsorted[4];  // the same bits ascending (zero insertion)
  int coef;        // offset of the coefficients in the plan's coefficient array
  int ncoef;
  int real;        // ELEM: every factor real
  int pad;
};

// One stage: a set of index bits held in a shared-memory tile and the operators applied to it.
struct StageDesc {
  int nbits;                 // tile-local bits (ascending global positions in bits[])
  int bits[kMaxTileBits];
  int nrest;                 // remaining global bit positions (ascending), deposited from the tile index
  int rest[2 * VQD_MAX_QUBITS];
  int op_begin, op_end;      // range in the plan's TileOp array
  double weight;             // original operations applied by this stage
};

struct FusedPlan {
  std::vector<StageDesc> stages;
  std::vector<TileOp> ops;
  std::vector<cd> coef;
  int max_bits = 0;
};

// Group the compiled operators of one n-qubit instance into stages of at most `fuse_qubits`
// qubits (0 = default) whose tiles fit the shared-memory budget of precision `prec`.
FusedPlan plan_fused(const std::vector<Op>& ops, int n, int prec, int fuse_qubits);

// Per-instance description used by the batched kernel.
struct BatchInst {
  uint64_t offset_amps;  // first amplitude of the instance in the batch allocation
  int n;
  int stage_begin, stage_end;
  double cost;           // 4^n x stages, for largest-first ordering
};
struct BatchPlan {
  FusedPlan all;                 // stages of every instance, concatenated (op/coef offsets global)
  std::vector<BatchInst> inst;   // in queue order (largest first)
  std::vector<int> passes;       // passes over the state per instance (indexed by instance id)
};
BatchPlan plan_batch(const std::vector<std::vector<Op>>& lists, const std::vector<int>& n,
                     const std::vector<size_t>& byte_offsets, int prec, int fuse_qubits);

// Device buffers reused across calls (grown on demand; freed with the context).
struct FusedCache {
  void* d_ops = nullptr;
  size_t ops_cap = 0;
  void* d_coef = nullptr;
  size_t coef_cap = 0;
  void* d_stages = nullptr;
  size_t stages_cap = 0;
  void* d_inst = nullptr;
  size_t inst_cap = 0;
  int* d_counter = nullptr;
  int n_inst = 0;
  int max_bits = 0;
};
void fused_cache_free(FusedCache& c);
void upload_plan(FusedCache& c, const FusedPlan& p, int prec, cudaStream_t s);
cudaError_t launch_stage(FusedCache& c, const FusedPlan& p, int stage, int prec, void* state, int n, cudaStream_t s);
void upload_batch(FusedCache& c, const BatchPlan& p, int prec, cudaStream_t s);
cudaError_t launch_batch(FusedCache& c, const BatchPlan& p, int prec, void* base, cudaStream_t s);
cudaError_t batch_status(FusedCache& c, cudaStream_t s);

// Shared-memory tile budget (index bits) for a precision.
int tile_bits_budget(int prec);

}  // namespace vqd
