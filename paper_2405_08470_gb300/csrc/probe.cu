// probe.cu - spmttkrp_memprobe: memory-system ceilings for the access patterns
// of the dynamic remap (sequential copy, scattered and gathered 32-byte
// records), timed by the caller.  The paper has no counterpart; the engine's
// roofline is stated against these measured ceilings as well as against the
// copy bandwidth.
#include "engine.h"
#include "mttkrp_common.cuh"

namespace spm {

// Record r of run q goes to run pi(q) = (A q + C) mod m of the destination
// (m = n / run runs), keeping its place inside the run; A is a prime that does
// not divide m, so pi is a permutation.
__device__ __forceinline__ int64_t probe_dst(int64_t i, int run, int64_t m, uint64_t A) {
  const int64_t q = i / run;
  return (int64_t)((A * (uint64_t)q + 12345ull) % (uint64_t)m) * run + (i - q * run);
}

__global__ void memprobe_kernel(const uint4* __restrict__ a, uint4* __restrict__ b, int64_t n,
                                int kind, int run, int64_t m, uint64_t A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (kind == 0) {  // copy
    st_hint_v8(b + 2 * i, __ldg(a + 2 * i), __ldg(a + 2 * i + 1), make_policy(0));
  } else if (kind == 1) {  // scatter
    const int64_t d = probe_dst(i, run, m, A);
    st_hint_v8(b + 2 * d, __ldg(a + 2 * i), __ldg(a + 2 * i + 1), make_policy(0));
  } else {  // gather
    const int64_t s = probe_dst(i, run, m, A);
    st_hint_v8(b + 2 * i, __ldg(a + 2 * s), __ldg(a + 2 * s + 1), make_policy(0));
  }
}

}  // namespace spm

using namespace spm;

extern "C" int spmttkrp_memprobe(int kind, const void* src, void* dst, int64_t n, int run,
                                 void* stream) {
  if (kind < 0 || kind > 2) return fail(SPM_ERR_INVALID_ARG, "memprobe: kind must be 0, 1 or 2");
  if (n < 1 || n >= (int64_t(1) << 40)) return fail(SPM_ERR_INVALID_ARG, "memprobe: n out of range");
  if (run < 1 || n % run) return fail(SPM_ERR_INVALID_ARG, "memprobe: run must divide n");
  if (!src || !dst || (((uintptr_t)src | (uintptr_t)dst) & 31u))
    return fail(SPM_ERR_INVALID_ARG, "memprobe: buffers must be 32-byte aligned device memory");
  const int64_t m = n / run;
  const uint64_t primes[] = {2654435761ull, 2246822519ull, 3266489917ull, 668265263ull,
                             374761393ull};
  uint64_t A = 1;
  for (uint64_t p : primes)
    if ((uint64_t)m % p != 0) {
      A = p;
      break;
    }
  const int64_t blocks = (n + 255) / 256;
  memprobe_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      static_cast<const uint4*>(src), static_cast<uint4*>(dst), n, kind, run, m, A % (uint64_t)m);
  SPM_CUDA(cudaGetLastError());
  return SPM_OK;
}
