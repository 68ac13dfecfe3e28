// Tensor-core path of libvqd (implemented in tcgemm.cu): fused k-qubit blocks applied as split-precision
// GEMMs with tcgen05.mma.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "vqd_internal.h"

namespace vqd {

struct TcParams {
  const float2* X;  // input state (complex64)
  float2* Y;        // output state (complex64), a different buffer
  const void* R;    // the operator's limbs in the tiled layout (read by TMA)
  uint32_t groups;  // 4^(n-k)
  uint32_t n_gtiles;
  uint32_t n_ntiles;
  int n_kchunks;
  int nmem;          // 4^k members of a group
  int mb;            // 2k index bits of a group
  int pos[12];       // the 2k bits, ascending (zero insertion)
  uint32_t mbit[12]; // index bit of member bit j: q_j (row) for j < k, q_{j-k} + n (column)
  int* err;          // set to 1 when a bounded wait expired
};

// Bytes of the composition buffer (a 4^k x 4^k complex128 superoperator) and of the tiled limbs of R.
size_t tc_compose_bytes(int k);
size_t tc_r_bytes(int k, int scheme);
// The composition buffer holds S[i][j] (i = r | c << k, j = jl | jh << k) at index
// r | jl << k | c << 2k | jh << 3k: a 2k-qubit "state" on which an operator of the block acting on block
// qubit b touches bits b and b + 2k, so the plain FP64 kernels compose operators into S column by column.
cudaError_t tc_compose_init(void* S, int k, cudaStream_t s);
// Split S into the limbs of the real embedding R = [[Re S, -Im S], [Im S, Re S]], in the tiled layout.
cudaError_t tc_build_r(const void* S, int k, int scheme, void* R, cudaStream_t s);
// Y <- the block applied to X for every group (n-qubit complex64 states; q = the block's k qubits in
// the order of S's index bits).
cudaError_t tc_apply(const void* X, void* Y, int n, int k, const int* q, int scheme, const void* R, int* d_err,
                     cudaStream_t s);

// Blocks of at most k qubits, in program order with the commuting lookahead of the fused path.
struct TcBlock {
  std::vector<int> ops;  // indices into the compiled program
  uint32_t qmask = 0;
  double weight = 0.0;   // original operations
};
std::vector<TcBlock> plan_tc_blocks(const std::vector<Op>& ops, int n, int k);

}  // namespace vqd
