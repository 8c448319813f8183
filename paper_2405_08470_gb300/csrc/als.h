// als.h - launchers of the CP-ALS and CP-loss kernels.
#pragma once

#include "engine.h"

namespace spm {

struct FactorPtrs {
  const void* p[kMaxModes];
};

int launch_gram(const void* A, int dtype, int64_t I, int R, double* part, int max_chunks,
                double* G, cudaStream_t s);
int launch_als_prep(const double* grams, int N, int n, int R, double* work, float* vinv,
                    int* status, cudaStream_t s);
int launch_als_solve(const float* M, float* U, const float* vinv, int64_t I, int R,
                     double* colsq, const int* status, int nb, cudaStream_t s);
int launch_als_lambda(const double* colsq, int nb, int R, double* lam64, float* lam_out,
                      const int* status, cudaStream_t s);
// R <= 64: U is not read (nor written by launch_als_solve, which then leaves the
// column norms only); the scale pass forms M V^-1 again from M and vinv.
int launch_als_scale(const float* U, const float* M, const float* vinv, void* A, int dtype,
                     const double* lam64, int64_t I, int R, double* mdot, const int* status,
                     int nb, cudaStream_t s);
int launch_fill_f64(double* p, int n, double v, cudaStream_t s);
// The end of a column-scale-folded loop: lambda_r = prod_k sqrt(G_k[r, r]) and
// every factor divided by its column norms (the Grams must be the stored factors').
int launch_als_fold_finish(void* const* factors, int dtype, const int64_t* dims, int N, int R,
                           const double* grams, double* lam64, float* lam_out, const int* status,
                           int nb, cudaStream_t s);
int launch_als_fit(const double* grams, int N, int R, const double* lam64, const double* mdot,
                   int nb, double normx2, double* fit_out, const int* status, cudaStream_t s);
int launch_cp_fwd(const uint8_t* elems, uint8_t* res, int64_t nnz, int es, int N,
                  const FactorPtrs& fp, const PackInfo& pk, int R, int dtype, double* part,
                  int nb, float* loss, double* loss64, cudaStream_t s);

int launch_als_converge(const double* fit, const int* status, double* fits, int* iters, int t,
                        double tol, cudaGraphConditionalHandle next, int has_next,
                        cudaStream_t s);

// api.cu
int run_mode(spmttkrp_plan* p, int mode, const void* const* factors, float* out,
             const uint8_t* ein, uint8_t* eout, const float* scale,
             double* loss_part = nullptr);
int compute_mode(spmttkrp_plan* p, int mode, const void* const* factors, float* out,
                 bool keep_order);
int upload_mode_tables(spmttkrp_plan* p, int n);
int plan_dalloc(spmttkrp_plan* p, void** ptr, size_t bytes);

}  // namespace spm
