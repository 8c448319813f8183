// check.cu - device-side consistency check of a working copy (the engine's
// stand-in for a memory sanitizer, which this platform does not run): every
// index of every nonzero is inside its mode's dimension, every remap id is in
// [0, nnz), the remap ids of one pass form a permutation (each target position
// is hit exactly once: the scatter of Algorithm 3 writes every element once),
// and remap ids carried inside the nonzeros agree with the next_pos array.
// Violations are counted and the first offending position is recorded; nothing
// is written outside the check's own counters and nothing traps.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "engine.h"
#include "mttkrp_common.cuh"

namespace spm {
namespace {

struct CheckState {
  unsigned long long bad_index;   // count, first position in first_*
  unsigned long long bad_target;
  unsigned long long bad_alpha;
  unsigned long long first_index, first_target, first_alpha;
};

struct Dims16 {
  int64_t d[kMaxModes];
};

__global__ void check_elements_kernel(const uint8_t* __restrict__ elems, int64_t nnz, int N,
                                      Dims16 dims, int es, const int32_t* __restrict__ next_pos,
                                      int alpha_word, PackInfo pk,
                                      unsigned int* __restrict__ hits, CheckState* st) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nnz) return;
  const int32_t* el = reinterpret_cast<const int32_t*>(elems + q * es);
  bool ok = true;
  for (int k = 0; k < N; ++k) {
    const int ik = elem_index(elems + q * es, k, pk);
    ok = ok && ik >= 0 && (int64_t)ik < dims.d[k];
  }
  if (!ok) {
    atomicAdd(&st->bad_index, 1ull);
    atomicMin(&st->first_index, (unsigned long long)q);
  }
  if (next_pos) {
    const int32_t t = next_pos[q];
    if (t < 0 || (int64_t)t >= nnz) {
      atomicAdd(&st->bad_target, 1ull);
      atomicMin(&st->first_target, (unsigned long long)q);
    } else {
      atomicAdd(&hits[t], 1u);
      if (alpha_word > 0 && (el[alpha_word] & 0x7fffffff) != t) {  // bit 31: hot-row flag
        atomicAdd(&st->bad_alpha, 1ull);
        atomicMin(&st->first_alpha, (unsigned long long)q);
      }
    }
  }
}

// Targets hit zero or several times: the remap ids are not a permutation.
__global__ void check_hits_kernel(const unsigned int* __restrict__ hits, int64_t nnz,
                                  CheckState* st) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nnz && hits[q] != 1u) {
    atomicAdd(&st->bad_target, 1ull);
    atomicMin(&st->first_target, (unsigned long long)q);
  }
}

int run_check(const uint8_t* elems, int64_t nnz, int N, const int64_t* dims, int es,
              const int32_t* next_pos, int alpha_word, const PackInfo& pk, cudaStream_t s) {
  if (nnz <= 0) return SPM_OK;
  Dims16 d{};
  for (int k = 0; k < N; ++k) d.d[k] = dims[k];
  CheckState h{0, 0, 0, ~0ull, ~0ull, ~0ull};
  CheckState* dst = nullptr;
  unsigned int* hits = nullptr;
  SPM_CUDA(cudaMalloc(&dst, sizeof(CheckState)));
  cudaError_t e = next_pos ? cudaMalloc(&hits, (size_t)nnz * sizeof(unsigned int)) : cudaSuccess;
  if (e == cudaSuccess && hits) e = cudaMemsetAsync(hits, 0, (size_t)nnz * 4, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, &h, sizeof(h), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    const unsigned grid = (unsigned)((nnz + 255) / 256);
    check_elements_kernel<<<grid, 256, 0, s>>>(elems, nnz, N, d, es, next_pos, alpha_word, pk,
                                                hits, dst);
    if (next_pos) check_hits_kernel<<<grid, 256, 0, s>>>(hits, nnz, dst);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, dst, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dst);
  if (hits) cudaFree(hits);
  if (e != cudaSuccess) return cuda_fail(e, "working-copy check");
  if (h.bad_index)
    return fail(SPM_ERR_INDEX_RANGE, std::to_string(h.bad_index) +
                                         " nonzeros with an index outside dims, first at " +
                                         std::to_string(h.first_index));
  if (h.bad_target)
    return fail(SPM_ERR_STATE, std::to_string(h.bad_target) +
                                   " remap ids out of range or not a permutation, first at " +
                                   std::to_string(h.first_target));
  if (h.bad_alpha)
    return fail(SPM_ERR_STATE, std::to_string(h.bad_alpha) +
                                   " remap ids in the nonzeros differ from next_pos, first at " +
                                   std::to_string(h.first_alpha));
  return SPM_OK;
}

}  // namespace
}  // namespace spm

using namespace spm;

extern "C" {

int spmttkrp_check_elements(const void* elems, int64_t nnz, int nmodes, const int64_t* dims,
                            int elem_bytes, const int32_t* next_pos, int alpha_word,
                            void* stream) {
  if (nnz < 0 || nmodes < 2 || nmodes > kMaxModes || !dims || (nnz > 0 && !elems))
    return fail(SPM_ERR_INVALID_ARG, "check: bad arguments");
  if (elem_bytes < 4 * nmodes + 4 || elem_bytes % 16)
    return fail(SPM_ERR_INVALID_ARG, "check: elem_bytes must hold the nonzero, multiple of 16");
  if (alpha_word && (alpha_word <= nmodes || 4 * alpha_word >= elem_bytes))
    return fail(SPM_ERR_INVALID_ARG, "check: alpha_word outside the padding");
  return run_check(static_cast<const uint8_t*>(elems), nnz, nmodes, dims, elem_bytes, next_pos,
                   alpha_word, PackInfo(), static_cast<cudaStream_t>(stream));
}

int spmttkrp_plan_check(spmttkrp_plan_t p) {
  if (!p || p->destroyed) return fail(SPM_ERR_INVALID_ARG, "null or destroyed plan");
  if (p->host_only) return fail(SPM_ERR_STATE, "plan was built host-only");
  const int m = p->cur_mode;
  const int aw = p->alpha ? 4 + (m + 1) % p->N : 0;
  return run_check(cur_elems(p), p->nnz, p->N, p->dims.data(), p->es, p->md[(size_t)m].next_pos,
                   aw, p->pack, p->stream);
}

}  // extern "C"
