// kernels_misc.cu - split-row fix-up, zero fill, remap-only pass, and the
// dispatcher of the fused spMTTKRP + remap kernel.
#include "mttkrp_kernel.cuh"

namespace spm {

int launch_mttkrp_f32(const MttkrpArgs& a, const LaneCfg& c, cudaStream_t s);
int launch_mttkrp_bf16(const MttkrpArgs& a, const LaneCfg& c, cudaStream_t s);

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static LaneCfg cfg_for(const MttkrpArgs& a) {
  bool al = aligned16(a.out);
  for (int k = 0; k < a.nmodes; ++k)
    if (k != a.mode) al = al && aligned16(a.factors[k]);
  return lane_config(a.R, a.dtype, al);
}

size_t mttkrp_smem_bytes(int es, int tile, int R, int dtype) {
  size_t m = 0;
  for (bool al : {true, false}) {
    const LaneCfg c = lane_config(R, dtype, al);
    m = std::max(m, (size_t)kWarps * warp_layout(es, tile, R, 32 / c.L).total);
  }
  return m;
}

int launch_mttkrp(const MttkrpArgs& a, cudaStream_t s) {
  if (a.nblk <= 0) return SPM_OK;
  LaneCfg c = cfg_for(a);
  return a.dtype == SPM_DTYPE_BF16 ? launch_mttkrp_bf16(a, c, s) : launch_mttkrp_f32(a, c, s);
}

// One warp per split row: sum the block partials in ascending block order,
// zero the empty rows before it (and after it, for the last nonempty row),
// write the row once.
__global__ void __launch_bounds__(256) splitrow_fixup_kernel(const float* __restrict__ part,
                                                             const SplitRow* __restrict__ splits,
                                                             int nsplit, float* __restrict__ out,
                                                             int64_t out_rows, int R,
                                                             const float* scale) {
  const int w = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= nsplit) return;
  const SplitRow sr = splits[w];
  const float sc = scale ? __ldg(scale) : 1.0f;
  for (int64_t z = (int64_t)sr.prev_row + 1; z < sr.row; ++z)
    for (int r = lane; r < R; r += 32) out[z * R + r] = 0.f;
  for (int r = lane; r < R; r += 32) {
    float acc = 0.f;
    for (int b = sr.first_blk; b <= sr.last_blk; ++b) {
      const int slot = (b == sr.first_blk) ? sr.first_slot : 0;
      acc += part[((size_t)b * 2 + slot) * R + r];
    }
    out[(int64_t)sr.row * R + r] = acc * sc;
  }
  if (sr.is_last)
    for (int64_t z = (int64_t)sr.row + 1; z < out_rows; ++z)
      for (int r = lane; r < R; r += 32) out[z * R + r] = 0.f;
}

int launch_fixup(const float* part, const SplitRow* splits, int nsplit, float* out,
                 int64_t out_rows, int R, const float* scale, cudaStream_t s) {
  if (nsplit <= 0) return SPM_OK;
  splitrow_fixup_kernel<<<(nsplit + 7) / 8, 256, 0, s>>>(part, splits, nsplit, out, out_rows, R,
                                                         scale);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "splitrow_fixup_kernel launch");
}

__global__ void zero_kernel(float4* __restrict__ out4, float* __restrict__ out, int64_t n4,
                            int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
    out4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = 0.f;
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
__global__ void remap_only_kernel(const uint4* __restrict__ in, uint4* __restrict__ out,
                                  const int32_t* __restrict__ next_pos, int64_t nnz, int nv) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz * nv; i += stride) {
    const int64_t p = i / nv;
    const int c = (int)(i - p * nv);
    out[(int64_t)__ldg(next_pos + p) * nv + c] = __ldg(in + i);
  }
}

int launch_remap_only(const uint8_t* in, uint8_t* out, const int32_t* next_pos, int64_t nnz,
                      int es, cudaStream_t s) {
  if (nnz <= 0) return SPM_OK;
  const int nv = es / 16;
  int64_t blocks = std::min<int64_t>((nnz * nv + 255) / 256, 152 * 16);
  remap_only_kernel<<<(int)blocks, 256, 0, s>>>(reinterpret_cast<const uint4*>(in),
                                                reinterpret_cast<uint4*>(out), next_pos, nnz, nv);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "remap_only_kernel launch");
}

}  // namespace spm
