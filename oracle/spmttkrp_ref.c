/*
 * spmttkrp_ref.c - FP64 CPU oracle of mode-n spMTTKRP, multi-threaded, for timing.
 *
 * TEST INFRASTRUCTURE ONLY.  It is the plain definition of Eq. 1 (Section
 * 2.1.5, elementwise form), written for the host cores so that the CPU
 * baseline and the reference arm of the benchmark time a fair CPU program.
 * Only tests, the smoke check and the benchmark's CPU legs load it; it shares
 * no code with the CUDA engine.
 *
 * Definition: M[i_n, r] = sum over nonzeros e with coordinate i_n of
 *             v_e * prod_{k != n} A_k[i_k(e), r].
 * Order of arithmetic (so that results equal the NumPy oracle bit for bit when
 * built without floating-point contraction): the product is formed as
 * ((v * A_{k1}) * A_{k2}) ... with k ascending, and each output entry adds its
 * nonzeros' products in input order.  The nonzeros are first grouped by output
 * row with one stable counting pass (input order kept inside a row), so rows can
 * be summed by different threads without sharing an output entry.
 *
 * Returns 0, or -1 on a bad argument (including a coordinate outside dims) or an
 * allocation failure.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int spm_oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int spm_oracle_mttkrp(const int64_t* coo, const double* vals, int64_t nnz, int nmodes,
                      const int64_t* dims, const double* const* factors, int rank, int mode,
                      double* out, int threads) {
  if (!coo || !vals || !dims || !factors || !out || nmodes < 2 || rank < 1 || mode < 0 ||
      mode >= nmodes || nnz < 0)
    return -1;
  for (int64_t e = 0; e < nnz; ++e)
    for (int k = 0; k < nmodes; ++k)
      if (coo[e * nmodes + k] < 0 || coo[e * nmodes + k] >= dims[k]) return -1;
  const int64_t rows = dims[mode];
  int64_t* start = (int64_t*)calloc((size_t)rows + 1, sizeof(int64_t));
  int64_t* fill = (int64_t*)malloc(((size_t)rows + 1) * sizeof(int64_t));
  int64_t* order = (int64_t*)malloc(((size_t)nnz + 1) * sizeof(int64_t));
  if (!start || !fill || !order) {
    free(start);
    free(fill);
    free(order);
    return -1;
  }
  /* stable grouping by output row: counts, prefix sums, placement in input order */
  for (int64_t e = 0; e < nnz; ++e) start[coo[e * nmodes + mode] + 1] += 1;
  for (int64_t i = 0; i < rows; ++i) start[i + 1] += start[i];
  memcpy(fill, start, ((size_t)rows + 1) * sizeof(int64_t));
  for (int64_t e = 0; e < nnz; ++e) order[fill[coo[e * nmodes + mode]]++] = e;

  const int R = rank;
#ifdef _OPENMP
  if (threads < 1) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 256) num_threads(threads)
#endif
  for (int64_t i = 0; i < rows; ++i) {
    double* m = out + i * R;
    for (int r = 0; r < R; ++r) m[r] = 0.0;
    for (int64_t p = start[i]; p < start[i + 1]; ++p) {
      const int64_t e = order[p];
      for (int r = 0; r < R; ++r) {
        double prod = vals[e];
        for (int k = 0; k < nmodes; ++k)
          if (k != mode) prod = prod * factors[k][coo[e * nmodes + k] * R + r];
        m[r] = m[r] + prod;
      }
    }
  }
  free(start);
  free(fill);
  free(order);
  return 0;
}
