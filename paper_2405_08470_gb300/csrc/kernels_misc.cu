// kernels_misc.cu - split-row fix-up, zero fill, remap-only pass, and the
// dispatcher of the fused spMTTKRP + remap kernel.
#include "mttkrp_kernel.cuh"
#include "mttkrp_tile.cuh"

namespace spm {

int launch_mttkrp_f32(const MttkrpArgs& a, const LaneCfg& c, cudaStream_t s);
int launch_mttkrp_bf16(const MttkrpArgs& a, const LaneCfg& c, cudaStream_t s);
int launch_mttkrp_tile(const MttkrpArgs& a, cudaStream_t s);

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static LaneCfg cfg_for(const MttkrpArgs& a) {
  bool al = aligned16(a.out);
  for (int k = 0; k < a.nmodes; ++k)
    if (k != a.mode) al = al && aligned16(a.factors[k]);
  return lane_config(a.R, a.dtype, al, a.variant == 0 || a.variant == 3);  // form 0's lanes
}

size_t mttkrp_smem_bytes(int es, int tile, int R, int dtype, int stages) {
  size_t m = 0;
  for (bool al : {true, false}) {
    const LaneCfg c = lane_config(R, dtype, al, true);
    const int G = 32 / c.L;
    m = std::max(m, (size_t)kWarps * warp_layout(es, warp_tile_for(tile, G), R, G, stages).total);
  }
  return m;
}

int launch_mttkrp(const MttkrpArgs& a, cudaStream_t s) {
  if (a.nblk <= 0) return SPM_OK;
  LaneCfg c = cfg_for(a);
  if (a.loss_part)  // the fused CP-loss pass runs in the warp-block form
    return a.dtype == SPM_DTYPE_BF16 ? launch_mttkrp_bf16(a, c, s) : launch_mttkrp_f32(a, c, s);
  if (a.variant == 2) {
    // the tile form needs 16-byte aligned factors and output; otherwise form 0
    bool al = aligned16(a.out);
    for (int k = 0; k < a.nmodes; ++k)
      if (k != a.mode) al = al && aligned16(a.factors[k]);
    if (al && tile_form_supported(a.nmodes, a.es, a.alpha_word, a.R) && a.no_fill == 0)
      return launch_mttkrp_tile(a, s);
    MttkrpArgs b = a;
    b.variant = 0;
    return a.dtype == SPM_DTYPE_BF16 ? launch_mttkrp_bf16(b, c, s) : launch_mttkrp_f32(b, c, s);
  }
  if (a.variant == 3 &&
      !(c.vec && a.nmodes == 3 && a.es == 32 && a.alpha_word && a.no_fill == 0 && a.elems_out)) {
    // form 3 needs 32-byte 3-mode nonzeros with their ids and write orders, the
    // contiguous split, and a remap to do; otherwise form 0
    MttkrpArgs b = a;
    b.variant = 0;
    return a.dtype == SPM_DTYPE_BF16 ? launch_mttkrp_bf16(b, c, s) : launch_mttkrp_f32(b, c, s);
  }
  return a.dtype == SPM_DTYPE_BF16 ? launch_mttkrp_bf16(a, c, s) : launch_mttkrp_f32(a, c, s);
}

// Split-row fix-up in two launches, both in a fixed order (results are
// bit-identical run to run).  Pass 1: one CTA per chunk of up to kFixChunk
// consecutive blocks of a split row; warp w sums the chunk's blocks w, w+8, ...
// (lanes over R) and the 8 warp sums are added in warp order.  Pass 2: one CTA
// per split row adds its chunk sums in chunk order, writes the row once and
// zeroes the empty rows before it (and after it, for the last nonempty row).  A
// row spread over thousands of blocks (a Zipf head row) is summed by many CTAs.
__global__ void __launch_bounds__(256) splitrow_chunk_kernel(const float* __restrict__ part,
                                                             const SplitRow* __restrict__ splits,
                                                             int nsplit, int nchunk, int R,
                                                             float* __restrict__ chunk_sums) {
  __shared__ float red[8][kMaxRank];
  const int c = blockIdx.x;
  if (c >= nchunk) return;
  int lo = 0, hi = nsplit - 1;  // the split row holding chunk c: last chunk0 <= c
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (splits[mid].chunk0 <= c) lo = mid; else hi = mid - 1;
  }
  const SplitRow sr = splits[lo];
  const int j = c - sr.chunk0;
  const int b0 = sr.first_blk + j * kFixChunk;
  const int nb = min(kFixChunk, sr.last_blk + 1 - b0);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = lane; r < R; r += 32) {
    float acc = 0.f;
    for (int i = w; i < nb; i += 8) {
      const int b = b0 + i;
      const int slot = (b == sr.first_blk) ? sr.first_slot : 0;
      acc += __ldg(part + ((size_t)b * 2 + slot) * R + r);
    }
    red[w][r] = acc;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc += red[q][r];
    chunk_sums[(size_t)c * R + r] = acc;
  }
}

__global__ void __launch_bounds__(256) splitrow_fixup_kernel(const float* __restrict__ chunk_sums,
                                                             const SplitRow* __restrict__ splits,
                                                             int nsplit, float* __restrict__ out,
                                                             int64_t out_rows, int R,
                                                             const float* scale) {
  if ((int)blockIdx.x >= nsplit) return;
  const SplitRow sr = splits[blockIdx.x];
  const float sc = scale ? __ldg(scale) : 1.0f;
  const int nc = (sr.last_blk - sr.first_blk + kFixChunk) / kFixChunk;
  const int64_t gap0 = (int64_t)sr.prev_row + 1, ngap = ((int64_t)sr.row - gap0) * R;
  for (int64_t i = threadIdx.x; i < ngap; i += blockDim.x) out[gap0 * R + i] = 0.f;
  if (sr.is_last) {
    const int64_t t0 = (int64_t)sr.row + 1, nt = (out_rows - t0) * R;
    for (int64_t i = threadIdx.x; i < nt; i += blockDim.x) out[t0 * R + i] = 0.f;
  }
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    float acc = 0.f;
    for (int q = 0; q < nc; ++q) acc += chunk_sums[(size_t)(sr.chunk0 + q) * R + r];
    out[(int64_t)sr.row * R + r] = acc * sc;
  }
}

int launch_fixup(const float* part, const SplitRow* splits, int nsplit, int nchunk,
                 float* chunk_sums, float* out, int64_t out_rows, int R, const float* scale,
                 cudaStream_t s) {
  if (nsplit <= 0) return SPM_OK;
  splitrow_chunk_kernel<<<nchunk, 256, 0, s>>>(part, splits, nsplit, nchunk, R, chunk_sums);
  splitrow_fixup_kernel<<<nsplit, 256, 0, s>>>(chunk_sums, splits, nsplit, out, out_rows, R,
                                               scale);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "split-row fix-up launch");
}

__global__ void zero_kernel(float4* __restrict__ out4, float* __restrict__ out, int64_t n4,
                            int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
    out4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = 0.f;
}

// Zeroes the listed output rows (rows of the mode with no nonzero when blocks
// own non-contiguous row sets): one warp per row.
__global__ void zero_listed_rows_kernel(float* __restrict__ out, const int32_t* __restrict__ rows,
                                        int nrows, int R) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= nrows) return;
  float* d = out + (int64_t)rows[w] * R;
  for (int r = lane; r < R; r += 32) d[r] = 0.f;
}

int launch_zero_listed_rows(float* out, const int32_t* rows, int nrows, int R, cudaStream_t s) {
  if (nrows <= 0) return SPM_OK;
  const int64_t threads = (int64_t)nrows * 32;
  zero_listed_rows_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(out, rows, nrows, R);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "zero_listed_rows_kernel launch");
}

int launch_zero_rows(float* out, int64_t rows, int R, cudaStream_t s) {
  const int64_t n = rows * R;
  if (n <= 0) return SPM_OK;
  const int64_t n4 = ((uintptr_t)out & 15u) ? 0 : n / 4;
  int64_t blocks = std::min<int64_t>((n / 4 + 255) / 256 + 1, 152 * 8);
  zero_kernel<<<(int)blocks, 256, 0, s>>>(reinterpret_cast<float4*>(out), out, n4, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "zero_kernel launch");
}

// Remap without compute (Algorithm 3 alone): T_out[next_pos[p]] = T_in[p].
// Elements whose stride is a multiple of 32 bytes move in whole 32-byte
// sectors (one 256-bit store each), others in 16-byte pieces.
// Remap-only pass: element p to its place next_pos[p] of the next order.  One
// thread per element (per 32-byte sector of it, or per 16-byte vector when the
// stride is not a multiple of 32) on a full grid: measured 1.6 ms for 100M
// scattered 32-byte elements, where a grid-stride loop over the same stores
// took 2.4-2.8 ms (its warps wait on each element's loads before the next).
__global__ void remap_only_kernel(const uint4* __restrict__ in, uint4* __restrict__ out,
                                  const int32_t* __restrict__ next_pos, int64_t nnz, int nv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((nv & 1) == 0) {  // one whole 32-byte sector per thread
    const int nw = nv / 2;
    if (i >= nnz * nw) return;
    const int64_t p = nw == 1 ? i : i / nw;
    const int c = (int)(i - p * nw);
    const uint4 lo = __ldg(in + p * nv + 2 * c), hi = __ldg(in + p * nv + 2 * c + 1);
    st_hint_v8(out + (int64_t)__ldg(next_pos + p) * nv + 2 * c, lo, hi, make_policy(1));
    return;
  }
  if (i >= nnz * nv) return;
  const int64_t p = nv == 1 ? i : i / nv;
  const int c = (int)(i - p * nv);
  out[(int64_t)__ldg(next_pos + p) * nv + c] = __ldg(in + i);
}

// dst = scale * src over n floats (the CP-loss gradient of the fused pass's mode).
__global__ void scale_copy_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                  int64_t n, const float* __restrict__ scale) {
  const float sc = scale ? __ldg(scale) : 1.0f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = __ldg(src + i) * sc;
}

int launch_scale_copy(const float* src, float* dst, int64_t n, const float* scale,
                      cudaStream_t s) {
  if (n <= 0) return SPM_OK;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  scale_copy_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, n, scale);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "scale_copy_kernel launch");
}

// 1/2 sum of n FP64 partials in a fixed order: thread t adds a contiguous chunk,
// then the 256 chunk sums are added in a fixed tree; loss = that half-sum.
__global__ void __launch_bounds__(256) loss_reduce_kernel(const double* __restrict__ part,
                                                          int64_t n, float* __restrict__ loss,
                                                          double* __restrict__ loss64) {
  __shared__ double red[256];
  const int64_t chunk = (n + 255) / 256;
  const int64_t b = (int64_t)threadIdx.x * chunk, e = min(n, b + chunk);
  double acc = 0.0;
  for (int64_t i = b; i < e; ++i) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loss64[0] = 0.5 * red[0];
    loss[0] = (float)(0.5 * red[0]);
  }
}

int launch_loss_reduce(const double* part, int64_t n, float* loss, double* loss64,
                       cudaStream_t s) {
  loss_reduce_kernel<<<1, 256, 0, s>>>(part, n, loss, loss64);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "loss_reduce_kernel launch");
}

// Remap-only pass in destination order, for 3-mode nonzeros in 32-byte sectors
// that carry their remap ids and write orders: thread j takes slot j of its
// tile of kTileNnz positions, reads there the tile-local index of the nonzero
// whose destination is the tile's j-th smallest, and stores that nonzero.
// Consecutive threads then store consecutive sectors wherever destinations are
// consecutive (the stable partition of Observation 1).
__global__ void remap_ordered_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                     int64_t nnz, int mode, int* err) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nnz) return;
  const int64_t base = j - j % kTileNnz;
  const uint32_t wo = __ldg(reinterpret_cast<const uint32_t*>(in + j * 32) + kTileWordW);
  const int64_t src = base + ((wo >> (10 * mode)) & 1023u);
  if (src >= nnz) {
    if (err) atomicOr(err, 2);
    return;
  }
  const uint4* sp = reinterpret_cast<const uint4*>(in + src * 32);
  const uint4 lo = __ldg(sp), hi = __ldg(sp + 1);
  const int nx = (mode + 1) % 3;
  const uint32_t dst = (nx == 0 ? hi.x : (nx == 1 ? hi.y : hi.z)) & kAlphaMask;
  if ((int64_t)dst >= nnz) {
    if (err) atomicOr(err, 2);
    return;
  }
  st_hint_v8(out + (int64_t)dst * 32, lo, hi, make_policy(1));
}

int launch_remap_ordered(const uint8_t* in, uint8_t* out, int64_t nnz, int mode, int* err,
                         cudaStream_t s) {
  if (nnz <= 0) return SPM_OK;
  const int64_t blocks = (nnz + 255) / 256;
  remap_ordered_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, nnz, mode, err);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "remap_ordered_kernel launch");
}

int launch_remap_only(const uint8_t* in, uint8_t* out, const int32_t* next_pos, int64_t nnz,
                      int es, cudaStream_t s) {
  if (nnz <= 0) return SPM_OK;
  const int nv = es / 16;
  const int64_t units = (nv & 1) == 0 ? nnz * (nv / 2) : nnz * nv;
  const int64_t blocks = (units + 255) / 256;
  if (blocks > 0x7fffffffLL) return fail(SPM_ERR_UNSUPPORTED, "remap pass too large");
  remap_only_kernel<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const uint4*>(in),
                                                     reinterpret_cast<uint4*>(out), next_pos,
                                                     nnz, nv);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "remap_only_kernel launch");
}

}  // namespace spm
