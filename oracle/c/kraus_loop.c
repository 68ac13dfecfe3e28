/*
 * Oracle (test infrastructure only): the density-matrix update rho <- sum_j K_j rho K_j^dagger of
 * Sec. 2 (a general Kraus map acting on the density matrix; a unitary is the one-operator case), written
 * as plain FP64 loops over explicit (row, column) indices.  It computes exactly what
 * oracle/evolve.apply_kraus computes with tensor contractions; it exists so that the oracle can run
 * the full-size (14- to 16-qubit) programs in minutes rather than hours.  Nothing here is shared with
 * the library: this file is compiled on its own and only the oracle's Python wrapper loads it.
 *
 * Layout: rho is the 2^n x 2^n matrix rho[r][c] stored row by row (rho[r * 2^n + c]), qubit q is bit q
 * of r and of c.  The k target qubits t[0..k-1] index a Kraus operator little-endian: t[0] is the least
 * significant bit of its 2^k x 2^k row-major index.
 *
 * For every row base rb and column base cb (the indices with all target bits zero) the 2^k x 2^k block
 * B[a][b] = rho[rb + off(a)][cb + off(b)], off(a) = sum_j a_j 2^{t_j}, is replaced by
 * sum_j K_j B K_j^dagger.  Blocks are disjoint, so they may be processed in any order; OpenMP spreads
 * the row bases over the threads and every block is computed the same way whatever the thread count.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

void oracle_set_threads(int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Returns 0, or -1 for bad arguments (k outside 1..4, a target outside 0..n-1 or repeated). */
int oracle_apply_kraus(cplx* rho, int n, int k, const int* t, int nK, const cplx* K) {
  if (n < 1 || n > 16 || k < 1 || k > 4 || nK < 1) return -1;
  uint64_t mask = 0;
  for (int j = 0; j < k; j++) {
    if (t[j] < 0 || t[j] >= n || (mask >> t[j] & 1u)) return -1;
    mask |= 1ull << t[j];
  }
  const uint64_t dim = 1ull << n;
  const int d = 1 << k;
  uint64_t off[16];
  for (int a = 0; a < d; a++) {
    off[a] = 0;
    for (int j = 0; j < k; j++)
      if (a >> j & 1) off[a] |= 1ull << t[j];
  }
  /* the row (or column) bases, in increasing order: indices with every target bit zero */
  const uint64_t nb = dim >> k;
  uint64_t* base = (uint64_t*)malloc(nb * sizeof(uint64_t));
  if (!base) return -1;
  uint64_t cnt = 0;
  for (uint64_t x = 0; x < dim; x++)
    if (!(x & mask)) base[cnt++] = x;

#pragma omp parallel for schedule(static)
  for (int64_t ir = 0; ir < (int64_t)nb; ir++) {
    const uint64_t rb = base[ir];
    cplx B[16][16], KB[16][16], O[16][16];
    for (uint64_t ic = 0; ic < nb; ic++) {
      const uint64_t cb = base[ic];
      for (int a = 0; a < d; a++)
        for (int b = 0; b < d; b++) B[a][b] = rho[(rb + off[a]) * dim + cb + off[b]];
      for (int a = 0; a < d; a++)
        for (int b = 0; b < d; b++) O[a][b] = 0;
      for (int m = 0; m < nK; m++) {
        const cplx* Km = K + (size_t)m * d * d;
        /* KB = K_m B */
        for (int a = 0; a < d; a++)
          for (int b = 0; b < d; b++) {
            cplx s = 0;
            for (int l = 0; l < d; l++) s += Km[a * d + l] * B[l][b];
            KB[a][b] = s;
          }
        /* O += (K_m B) K_m^dagger: O[a][b] += sum_l KB[a][l] conj(K_m[b][l]) */
        for (int a = 0; a < d; a++)
          for (int b = 0; b < d; b++) {
            cplx s = 0;
            for (int l = 0; l < d; l++) s += KB[a][l] * conj(Km[b * d + l]);
            O[a][b] += s;
          }
      }
      for (int a = 0; a < d; a++)
        for (int b = 0; b < d; b++) rho[(rb + off[a]) * dim + cb + off[b]] = O[a][b];
    }
  }
  free(base);
  return 0;
}
