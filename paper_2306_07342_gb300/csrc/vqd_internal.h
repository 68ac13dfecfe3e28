// Internal declarations shared by the host-side translation units of libvqd.
#pragma once
#include <complex>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/vqd.h"

namespace vqd {

using cd = std::complex<double>;

// Exception carrying a VQD_E* code; caught at the C boundary.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// One operator of the compiled program: a unitary (2^k x 2^k) or a channel given by its
// superoperator (4^k x 4^k, index s = r | c << k).  Row-major FP64.
struct Op {
  bool unitary = true;
  int k = 1;
  int q[2] = {0, 0};
  std::vector<cd> m;
  double weight = 1.0;  // number of original (pre-fusion) operations this operator stands for
};

// ---- device compiler (devcomp.cpp)
Op compile_native(const vqd_native_op& op, unsigned flags);
void stderr_params(int nq, double fbar, double x, double* p_deph, double* q_depol);
std::vector<cd> superop_from_kraus(int k, int nK, const cd* K);   // sum conj(K) (x) K
std::vector<cd> superop_from_unitary(int k, const cd* U);            // |U_rr|^2 of a diagonal U set to 1
// Factor U_rr conj(U_cc) of a diagonal unitary's superoperator: exactly 1 when the two entries are the
// same number (|U_rr| = 1), else their product.
inline cd diag_unitary_factor(const cd& ur, const cd& uc) { return ur == uc ? cd(1.0) : ur * std::conj(uc); }
bool is_diagonal_matrix(int d, const cd* M);
void check_unitary(int k, const cd* U);                           // throws VQD_ENOTCP
void check_cptn(int k, int nK, const cd* K);                      // throws VQD_ENOTCP
int native_arity(int code);

// Kraus form of one native op for the trajectory path: a unitary (K = {U}) or the channel's Kraus
// operators in a fixed order.  For a composite process (first step A, then step B) the operators
// are B_j A_i with the first step's index i outer.  `mixture` marks channels whose operators are
// all sqrt(w_k) times a unitary: their branch probabilities w_k do not depend on the state.
struct KrausForm {
  bool unitary = true;
  int k = 1;
  int q[2] = {0, 0};
  std::vector<std::vector<cd>> K;
  bool mixture = false;
  std::vector<double> w;
};
KrausForm compile_kraus_form(const vqd_native_op& op, unsigned flags);

// ---- kernel classes of the plain path
enum KernelKind { KK_ELEM = 0, KK_SUP1 = 1, KK_UNI2 = 2, KK_SUP2 = 3, KK_COUNT_PLAIN = 4 };

// A plain-path pass, ready to launch: kind, bit positions of the targets and FP64 coefficients.
struct Pass {
  int kind = KK_ELEM;
  int k = 1;
  int q[2] = {0, 0};
  std::vector<cd> coef;  // ELEM: 4^k factors; SUP1: 16; UNI2: 16 (U); SUP2: 256
  double weight = 1.0;
};
Pass classify(const Op& op);

}  // namespace vqd
