// noalloc.cu - spmttkrp_compute_noalloc: one mode of the fused spMTTKRP +
// remap for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a
// framework's allocator-free region, a process whose device memory is fully
// owned by another pool, or a library call made where an allocation would
// break an outer stream capture or a memory budget.  Such callers cannot
// create a plan (plan creation allocates), so this entry point takes every
// input and output as caller-owned device memory and keeps its own scratch
// (block descriptors, split-row table and split-row partial sums) in one
// file-scope __device__ array of fixed size instead of allocating it.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "engine.h"
#include "mttkrp_kernel.cuh"

namespace spm {

constexpr int kNaMaxBlocks = 4096;  // blocks per call
constexpr int kNaMaxDevices = 64;

// 2 x 4096 x 256 floats of partial sums (8 MiB) + 4096 block descriptors
// (64 KiB) + 4096 split-row entries (128 KiB).  Every device that loads this
// library holds it until the process exits.
struct NoallocScratch {
  float part[(size_t)2 * kNaMaxBlocks * kMaxRank];
  int4 blkinfo[kNaMaxBlocks];
  SplitRow splits[kNaMaxBlocks];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

static std::mutex g_na_mu;
static NoallocScratch* g_na_ptr[kNaMaxDevices] = {};

__device__ __forceinline__ int na_row(const uint8_t* elems, int es, int mode, int64_t p) {
  return __ldg(reinterpret_cast<const int*>(elems + p * es) + mode);
}

// Even split: block b holds positions [b*T, min((b+1)*T, nnz)).
__global__ void na_blocks_kernel(const uint8_t* __restrict__ elems, int es, int64_t nnz,
                                 int mode, int nblk, int64_t T, int4* __restrict__ blkinfo) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  const int64_t lo = min((int64_t)b * T, nnz), hi = min(lo + T, nnz);
  int4 bi = make_int4((int)lo, (int)hi, -1, 0);
  if (lo < hi) {
    if (lo > 0) {
      bi.z = na_row(elems, es, mode, lo - 1);
      if (bi.z == na_row(elems, es, mode, lo)) bi.w |= BLK_HEAD_SPLIT;
    }
    if (hi < nnz && na_row(elems, es, mode, hi) == na_row(elems, es, mode, hi - 1))
      bi.w |= BLK_TAIL_SPLIT;
  }
  blkinfo[b] = bi;
}

// One entry per block: the row that starts in block b and continues past it
// (row = -1 when there is none).  Every entry is rewritten on every call.
__global__ void na_splits_kernel(const uint8_t* __restrict__ elems, int es, int64_t nnz,
                                 int mode, int nblk, int64_t T, const int4* __restrict__ blkinfo,
                                 SplitRow* __restrict__ splits) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  SplitRow sr;
  sr.row = -1;
  sr.first_blk = sr.last_blk = b;
  sr.first_slot = 0;
  sr.prev_row = -1;
  sr.is_last = 0;  // rows after the last nonempty row are zeroed by na_tail_kernel
  sr.chunk0 = sr.pad1 = 0;
  const int4 bi = blkinfo[b];
  const int64_t lo = bi.x, hi = bi.y;
  if (lo < hi && (bi.w & BLK_TAIL_SPLIT)) {
    const int r = na_row(elems, es, mode, hi - 1);
    const bool single = (bi.w & BLK_HEAD_SPLIT) && na_row(elems, es, mode, lo) == r;
    if (!single) {  // the row starts inside this block
      int64_t a = lo, c = hi - 1;  // first position of row r in [lo, hi)
      while (a < c) {
        const int64_t m = (a + c) / 2;
        if (na_row(elems, es, mode, m) < r) a = m + 1; else c = m;
      }
      int64_t e0 = hi, e1 = nnz;  // one past the last position of row r
      while (e0 < e1) {
        const int64_t m = (e0 + e1) / 2;
        if (na_row(elems, es, mode, m) <= r) e0 = m + 1; else e1 = m;
      }
      sr.row = r;
      sr.first_slot = (a == lo) ? 0 : 1;
      sr.last_blk = (int)((e0 - 1) / T);
      sr.prev_row = a > 0 ? na_row(elems, es, mode, a - 1) : -1;
    }
  }
  splits[b] = sr;
}

// Sum of each split row's block partials, one CTA per split-row entry (most
// entries are empty and return at once).  Warp w adds the partials of blocks
// first_blk + w, first_blk + w + 8, ... in ascending order; the eight warp sums
// are then added in warp order, so the result is the same on every call.  A
// head row spread over thousands of blocks is thus summed by eight warps with
// several loads in flight each, instead of one warp walking every block.
__global__ void __launch_bounds__(256) na_fixup_kernel(const float* __restrict__ part,
                                                       const SplitRow* __restrict__ splits,
                                                       float* __restrict__ out, int R) {
  __shared__ float wsum[8][kMaxRank];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const SplitRow sr = splits[blockIdx.x];
  if (sr.row < 0) return;
  for (int r = lane; r < R; r += 32) {
    float acc = 0.f;
    for (int b = sr.first_blk + w; b <= sr.last_blk; b += 8)
      acc += part[((size_t)b * 2 + ((b == sr.first_blk) ? sr.first_slot : 0)) * R + r];
    wsum[w][r] = acc;
  }
  __syncthreads();
  if (w == 0) {
    for (int64_t z = (int64_t)sr.prev_row + 1; z < sr.row; ++z)
      for (int r = lane; r < R; r += 32) out[z * R + r] = 0.f;
  }
  for (int r = threadIdx.x; r < R; r += 256) {
    float acc = wsum[0][r];
#pragma unroll
    for (int q = 1; q < 8; ++q) acc += wsum[q][r];
    out[(int64_t)sr.row * R + r] = acc;
  }
}

// Rows after the last nonempty row.
__global__ void na_tail_kernel(const uint8_t* __restrict__ elems, int es, int64_t nnz, int mode,
                               float* __restrict__ out, int64_t out_rows, int R) {
  const int64_t first = (int64_t)na_row(elems, es, mode, nnz - 1) + 1;
  const int64_t n = (out_rows - first) * R;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[first * R + i] = 0.f;
}

}  // namespace spm

using namespace spm;

extern "C" int spmttkrp_compute_noalloc(const void* elems, int64_t nnz, int nmodes, int mode,
                                        const int64_t* dims, int rank, int factor_dtype,
                                        const void* const* factors, float* out, void* elems_out,
                                        const int32_t* next_pos, int nblk, void* stream) {
  if (nmodes < 2 || nmodes > kMaxModes)
    return fail(SPM_ERR_UNSUPPORTED, "noalloc: nmodes must be in [2, 16]");
  if (mode < 0 || mode >= nmodes) return fail(SPM_ERR_INVALID_ARG, "noalloc: mode out of range");
  if (rank < 1) return fail(SPM_ERR_INVALID_ARG, "noalloc: rank must be >= 1");
  if (rank > kMaxRank)
    return fail(SPM_ERR_UNSUPPORTED, "noalloc: rank > 256 exceeds the static scratch");
  if (nnz < 0 || nnz >= (int64_t(1) << 31) - 4)
    return fail(SPM_ERR_UNSUPPORTED, "noalloc: nnz must be in [0, 2^31 - 4)");
  if (nblk < 0) return fail(SPM_ERR_INVALID_ARG, "noalloc: nblk must be >= 0");
  if (nblk > kNaMaxBlocks)
    return fail(SPM_ERR_UNSUPPORTED,
                "noalloc: nblk > 4096 exceeds the static scratch (4096 blocks of 2 x 256 floats)");
  if (factor_dtype != SPM_DTYPE_F32 && factor_dtype != SPM_DTYPE_BF16)
    return fail(SPM_ERR_INVALID_ARG, "noalloc: factor_dtype must be F32 or BF16");
  if (!dims || !out || !factors || (nnz > 0 && !elems))
    return fail(SPM_ERR_INVALID_ARG, "noalloc: null argument");
  if ((elems_out == nullptr) != (next_pos == nullptr))
    return fail(SPM_ERR_INVALID_ARG, "noalloc: elems_out and next_pos go together");
  for (int k = 0; k < nmodes; ++k)
    if (k != mode && !factors[k]) return fail(SPM_ERR_INVALID_ARG, "noalloc: null factor");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t out_rows = dims[mode];
  if (nnz == 0) return launch_zero_rows(out, out_rows, rank, s);

  // one-time set-up per device: the device address of the static scratch
  int dev = 0;
  SPM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return fail(SPM_ERR_UNSUPPORTED, "noalloc: device id");
  NoallocScratch* sp;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaGetSymbolAddress");
      g_na_ptr[dev] = static_cast<NoallocScratch*>(ptr);
    }
    sp = g_na_ptr[dev];
  }

  const int es = ((4 * nmodes + 4) + 15) & ~15;
  if (nblk == 0) nblk = (int)std::min<int64_t>(kNaMaxBlocks, std::max<int64_t>(1, (nnz + 8191) / 8192));
  const int64_t T = (nnz + nblk - 1) / nblk;
  const uint8_t* ein = static_cast<const uint8_t*>(elems);
  na_blocks_kernel<<<(nblk + 255) / 256, 256, 0, s>>>(ein, es, nnz, mode, nblk, T, sp->blkinfo);
  na_splits_kernel<<<(nblk + 255) / 256, 256, 0, s>>>(ein, es, nnz, mode, nblk, T, sp->blkinfo,
                                                      sp->splits);
  SPM_CUDA(cudaGetLastError());
  MttkrpArgs a;
  std::memset(&a, 0, sizeof(a));
  a.elems_in = ein;
  a.elems_out = static_cast<uint8_t*>(elems_out);
  a.next_pos = next_pos;
  a.blkinfo = sp->blkinfo;
  a.nblk = nblk;
  for (int k = 0; k < nmodes; ++k) a.factors[k] = factors[k];
  a.out = out;
  a.out_rows = out_rows;
  a.R = rank;
  a.mode = mode;
  a.nmodes = nmodes;
  a.es = es;
  a.tile = 512;
  a.part = sp->part;
  a.last_row = -1;  // the tail kernel below zeroes the rows after the last nonempty row
  a.err = nullptr;
  a.scale = nullptr;
  a.dtype = factor_dtype;
  a.variant = 1;  // CTA blocks, direct runs: no bulk-copy staging (next_pos needs no
                  // padding) and no device error word
  int st = launch_mttkrp(a, s);
  if (st) return st;
  na_fixup_kernel<<<nblk, 256, 0, s>>>(sp->part, sp->splits, out, rank);
  na_tail_kernel<<<64, 256, 0, s>>>(ein, es, nnz, mode, out, out_rows, rank);
  SPM_CUDA(cudaGetLastError());
  return SPM_OK;
}
