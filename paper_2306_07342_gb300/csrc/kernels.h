// Host-callable launchers of the libvqd kernels (implemented in kernels.cu / fused.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <complex>
#include <cstdint>
#include <vector>

#include "vqd_internal.h"

namespace vqd {

// A diagonal factor equal to 1: elementwise passes (plain and fused) leave the amplitudes with this
// factor untouched.  The comparison is exact.  The device compiler and the fused composer write the
// factors U_rr conj(U_cc) of diagonal unitaries as exactly 1 when U_rr and U_cc are the same number
// (see diag_unitary_factor), so a phase or a dephasing skips the members it leaves unchanged; a factor
// of a caller's superoperator is skipped only when it is exactly 1.
inline bool is_unit_factor(const std::complex<double>& c) { return c.real() == 1.0 && c.imag() == 0.0; }
// Fraction of the state's amplitudes a plain pass reads and writes: elementwise passes skip the
// amplitudes whose factor is 1; every other pass touches all of them.
double pass_touched_fraction(const Pass& p);
// Real multiply-adds per amplitude of the state that a plain pass issues, counting the structure of its
// coefficients as the kernels use it (a zero costs nothing, a one two adds, a real or imaginary
// coefficient two multiply-adds and a complex one four; an elementwise pass only on the amplitudes it
// changes; the dense form where it is cheaper).  For FP64 these are FP64 instructions.
double pass_fma_per_amp(const Pass& p, bool fp64);
cudaError_t launch_pass(int prec, void* state, int n, const Pass& p, cudaStream_t s);

// Initialisation.
cudaError_t launch_init_classical(int prec, void* state, int n, uint64_t basis, cudaStream_t s);
cudaError_t launch_init_product_diag(int prec, void* state, int n, const double* excited, cudaStream_t s);

// Reductions: each writes its partial sums to `scratch` (device, >= scratch_need(...) doubles)
// and its final values to `out` (device).  Deterministic summation order.
size_t reduce_scratch_doubles();
size_t reduce_out_doubles();
cudaError_t launch_trace(int prec, const void* state, int n, double* scratch, double* out, cudaStream_t s);      // out[0..1]
cudaError_t launch_purity(int prec, const void* state, int n, double* scratch, double* out, cudaStream_t s);     // out[0]
cudaError_t launch_prob(int prec, const void* state, int n, int m, const int* qubits, double* scratch, double* out,
                        cudaStream_t s);                                                                          // out[0..2^m)
// Up to kExpectTermsPerLaunch terms: xmask / zymask per term; out[2t], out[2t+1] = sum of
// (-1)^popc(c & zymask) rho[c][c ^ xmask] (re, im) for term t.
constexpr int kExpectTermsPerLaunch = 64;
cudaError_t launch_expect(int prec, const void* state, int n, int nterms, const uint32_t* xmask,
                          const uint32_t* zymask, double* scratch, double* out, cudaStream_t s);

int num_sms();

// Batched reductions of a batch context: per-CTA items over (instance, chunk of amplitudes).
size_t batch_reduce_item_bytes();
void batch_reduce_items(const std::vector<int>& n, const std::vector<size_t>& off_bytes, size_t esize,
                        std::vector<unsigned char>& items, std::vector<int>& item_inst);
cudaError_t launch_batch_reduce(int prec, const void* base, const std::vector<int>& n, const std::vector<size_t>& off_bytes,
                                double* d_probs, double* d_part, void* d_items, size_t nitems, cudaStream_t s);

// Records the message of a failed vqd_prob_static call for vqd_last_error(NULL); returns code.
int report_static_error(int code, const char* msg);

}  // namespace vqd
