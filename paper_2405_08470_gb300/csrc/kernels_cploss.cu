// kernels_cploss.cu - CP loss on the observed entries (completion form):
//   m_e = sum_r prod_k A_k[i_k(e), r],   e_e = m_e - x_e,   L = 1/2 sum_e e_e^2.
// One pass over the working copy in whatever mode order it is in: groups of L
// lanes own one nonzero at a time (16-byte factor-row slices per lane, as in
// the spMTTKRP kernel), the model value is summed across the group with
// shuffles, and the nonzero is written to the residual copy with its value
// replaced by e_e.  The gradient is then one all-mode spMTTKRP sweep of the
// residual copy.  The loss is reduced in a fixed order: each lane adds short
// runs of squared residuals in FP32 to its FP64 total, then the lanes, CTAs and
// partial sums are added in FP64 in index order.
#include "als.h"
#include "mttkrp_kernel.cuh"

namespace spm {

template <int NT, typename T, int VW, int RC>
__global__ void __launch_bounds__(256) cp_fwd_kernel(const uint8_t* __restrict__ elems,
                                                     uint8_t* __restrict__ res, int64_t nnz,
                                                     int es, int nmodes, FactorPtrs fp,
                                                     PackInfo pk, int R,
                                                     int L, double* __restrict__ loss_part) {
  constexpr int NV = VW * RC;
  const int N = NT > 0 ? NT : nmodes;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int sub = lane % L, gw = lane / L, G = 32 / L;
  const int64_t gid = ((int64_t)blockIdx.x * 8 + w) * G + gw;
  const int64_t ngroups = (int64_t)gridDim.x * 8 * G;
  double sq = 0.0;
  float run = 0.f;  // FP32 sum of up to 8 squared residuals, then added to sq
  int nrun = 0;
  // the loop bound is uniform across the warp so that the shuffles below see
  // every lane; groups past the end carry an inactive flag
  for (int64_t eb = gid - gw; eb < nnz; eb += ngroups) {
    const int64_t e = eb + gw;
    const bool active = e < nnz;
    const int* el = reinterpret_cast<const int*>(elems + (active ? e : 0) * es);
    const uint8_t* ep = reinterpret_cast<const uint8_t*>(el);
    float p[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) p[j] = active ? 1.f : 0.f;
    for (int k = 0; k < N && active; ++k) {
      const int64_t idx = elem_index(ep, k, pk);
      float x[NV];
      if constexpr (VW > 1) {
        if (sub * VW < R) {
          Slice<T, VW>::load(fp.p[k], idx, R, sub, x);
        } else {
#pragma unroll
          for (int j = 0; j < NV; ++j) x[j] = 0.f;
        }
      } else {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          const int r = sub + L * j;
          x[j] = r < R ? load_scalar<T>(fp.p[k], idx * R + r) : 0.f;
        }
      }
#pragma unroll
      for (int j = 0; j < NV; ++j) p[j] *= x[j];
    }
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < NV; ++j) m += p[j];
    for (int off = L / 2; off > 0; off >>= 1) m += __shfl_xor_sync(0xffffffffu, m, off);
    if (active && sub == 0) {
      const float x = elem_value(ep, N, pk);
      const float r = m - x;
      run = fmaf(r, r, run);
      const int nv = es / 16;
      const uint4* src = reinterpret_cast<const uint4*>(el);
      uint4* dst = reinterpret_cast<uint4*>(res + e * es);
      for (int c = 0; c < nv; ++c) {
        uint4 v = __ldg(src + c);
        const int word = (pk.packed ? 3 : N) - 4 * c;  // the value field's word
        if (word == 0) v.x = __float_as_uint(r);
        else if (word == 1) v.y = __float_as_uint(r);
        else if (word == 2) v.z = __float_as_uint(r);
        else if (word == 3) v.w = __float_as_uint(r);
        dst[c] = v;
      }
    }
    if (++nrun == 8) {  // warp-uniform count of iterations
      sq += (double)run;
      run = 0.f;
      nrun = 0;
    }
  }
  sq += (double)run;
  __shared__ double red[256];
  red[threadIdx.x] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < 256; ++q) s += red[q];
    loss_part[blockIdx.x] = s;
  }
}

// Starts a bulk copy of `bytes` (a multiple of 16, 16-byte aligned source) into
// L2 without waiting for it; nothing lands in shared memory or registers.
__device__ __forceinline__ void prefetch_l2_bulk(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Batched form for 3 and 4 modes on the 16-byte-slice path: each lane group takes
// U consecutive nonzeros at a time, issues all their factor-row slice loads before
// using any (U * N 16-byte loads in flight per lane), reduces the U model values
// with interleaved shuffles, and writes the U residual nonzeros with one 16-byte
// chunk per lane.  Same products and sums per nonzero as cp_fwd_kernel; the loss is
// accumulated per lane in a fixed order.  The warp's nonzeros of the next
// iteration are prefetched into L2 while this one waits on its factor rows, so
// only the gather latency stays on the loop's critical path.
template <int NT, typename T, int VW, int U>
__global__ void __launch_bounds__(256, 4) cp_fwd_batched_kernel(const uint8_t* __restrict__ elems,
                                                             uint8_t* __restrict__ res,
                                                             int64_t nnz, int es, FactorPtrs fp,
                                                             PackInfo pk, int R, int L,
                                                             double* __restrict__ loss_part) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int sub = lane % L, gw = lane / L, G = 32 / L;
  const int64_t per_warp = (int64_t)G * U;
  const int64_t wid = (int64_t)blockIdx.x * 8 + w, nw = (int64_t)gridDim.x * 8;
  const bool lane_on = sub * VW < R;
  const int nv = es / 16;
  const uint64_t pol = make_policy(2);  // factor rows are reused: evict last in L2
  double sq = 0.0;
  const int64_t stride = nw * per_warp;
  for (int64_t base = wid * per_warp; base < nnz; base += stride) {  // warp-uniform
    if (lane == 0 && base + stride < nnz) {
      const int64_t next = base + stride, cnt = min(per_warp, nnz - next);
      prefetch_l2_bulk(elems + next * es, (uint32_t)(cnt * es));
    }
    int idx[U][NT];
    float val[U];
    bool act[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = base + (int64_t)gw * U + u;
      act[u] = e < nnz;
      const int* el = reinterpret_cast<const int*>(elems + (act[u] ? e : 0) * es);
      const int4 w0 = __ldg(reinterpret_cast<const int4*>(el));
      const int f[4] = {w0.x, w0.y, w0.z, w0.w};
#pragma unroll
      for (int k = 0; k < NT; ++k) idx[u][k] = k < 4 ? f[k < 4 ? k : 0] : 0;
      if (NT < 4)
        val[u] = __int_as_float(f[NT < 4 ? NT : 0]);
      else if (!pk.packed)  // (a packed nonzero has no word NT: 16 bytes)
        val[u] = __int_as_float(__ldg(el + NT));
      if (pk.packed) {  // bit fields in words 0..2, the value in word 3
        const uint32_t pw[3] = {(uint32_t)w0.x, (uint32_t)w0.y, (uint32_t)w0.z};
#pragma unroll
        for (int k = 0; k < NT; ++k) idx[u][k] = (int)pk_field(pw, pk.off[k], pk.bits[k]);
        val[u] = __int_as_float(w0.w);
      }
    }
    uint4 raw[U][NT];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < NT; ++k)
        raw[u][k] = (act[u] && lane_on)
                        ? ld_nc_hint_v4(reinterpret_cast<const uint4*>(
                                            static_cast<const T*>(fp.p[k]) + (int64_t)idx[u][k] * R) +
                                            sub,
                                        pol)
                        : make_uint4(0u, 0u, 0u, 0u);
    float m[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float p[VW], x[VW];
      Landing<T, VW, 1>::unpack(raw[u][0], p);
#pragma unroll
      for (int k = 1; k < NT; ++k) {
        Landing<T, VW, 1>::unpack(raw[u][k], x);
#pragma unroll
        for (int j = 0; j < VW; ++j) p[j] *= x[j];
      }
      float t = 0.f;
#pragma unroll
      for (int j = 0; j < VW; ++j) t += p[j];
      m[u] = t;
    }
    for (int off = L / 2; off > 0; off >>= 1)
#pragma unroll
      for (int u = 0; u < U; ++u) m[u] += __shfl_xor_sync(0xffffffffu, m[u], off);
    // the U squared residuals are summed in FP32 and added to the FP64 total once
    // per iteration: FP64 issues slowly on this part, once per nonzero it bounds
    // the loop
    float r[U], s4 = 0.f;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      r[u] = m[u] - val[u];
      if (act[u]) s4 = fmaf(r[u], r[u], s4);
    }
    if (sub == 0) sq += (double)s4;
    // residual copy: chunk c of nonzero u per lane, the value word replaced by e_e
    for (int j = sub; j < U * nv; j += L) {
      const int u = j / nv, c = j - u * nv;
      bool on = false;
      float ru = 0.f;
#pragma unroll
      for (int q = 0; q < U; ++q)
        if (q == u) {
          on = act[q];
          ru = r[q];
        }
      if (!on) continue;
      const int64_t e = base + (int64_t)gw * U + u;
      uint4 v = __ldg(reinterpret_cast<const uint4*>(elems + e * es) + c);
      const int word = (pk.packed ? 3 : NT) - 4 * c;
      if (word == 0) v.x = __float_as_uint(ru);
      else if (word == 1) v.y = __float_as_uint(ru);
      else if (word == 2) v.z = __float_as_uint(ru);
      else if (word == 3) v.w = __float_as_uint(ru);
      reinterpret_cast<uint4*>(res + e * es)[c] = v;
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < 256; ++q) s += red[q];
    loss_part[blockIdx.x] = s;
  }
}

__global__ void cp_loss_final_kernel(const double* __restrict__ part, int nb,
                                     float* __restrict__ loss, double* __restrict__ loss64) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[b];
  loss64[0] = 0.5 * s;
  loss[0] = (float)(0.5 * s);
}

// Grid of the forward: the CTAs that are resident at once (a multiple of the SM
// count), capped by the partial-sum slots; every CTA strides over the whole copy.
template <typename K>
static int resident_grid(K kernel, int cap) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0) != cudaSuccess ||
      occ < 1)
    return cap;
  return std::max(1, std::min(cap, occ * sms));
}

template <typename T>
static int fwd_dispatch(const uint8_t* elems, uint8_t* res, int64_t nnz, int es, int N,
                        const FactorPtrs& fp, const PackInfo& pk, int R, bool aligned,
                        double* part, int cap, cudaStream_t s) {
  const int dtype = std::is_same<T, float>::value ? SPM_DTYPE_F32 : SPM_DTYPE_BF16;
  const LaneCfg c = lane_config(R, dtype, aligned);
  constexpr int VWV = std::is_same<T, float>::value ? 4 : 8;
  int nb = cap;
  if (c.vec) {
    if (N == 3) {
      nb = resident_grid(cp_fwd_batched_kernel<3, T, VWV, 4>, cap);
      cp_fwd_batched_kernel<3, T, VWV, 4><<<nb, 256, 0, s>>>(elems, res, nnz, es, fp, pk, R, c.L,
                                                             part);
    } else if (N == 4) {
      nb = resident_grid(cp_fwd_batched_kernel<4, T, VWV, 4>, cap);
      cp_fwd_batched_kernel<4, T, VWV, 4><<<nb, 256, 0, s>>>(elems, res, nnz, es, fp, pk, R, c.L,
                                                             part);
    } else {
      cp_fwd_kernel<0, T, VWV, 1><<<nb, 256, 0, s>>>(elems, res, nnz, es, N, fp, pk, R, c.L, part);
    }
  } else {
    switch (c.RC) {
      case 1: cp_fwd_kernel<0, T, 1, 1><<<nb, 256, 0, s>>>(elems, res, nnz, es, N, fp, pk, R, c.L, part); break;
      case 2: cp_fwd_kernel<0, T, 1, 2><<<nb, 256, 0, s>>>(elems, res, nnz, es, N, fp, pk, R, c.L, part); break;
      case 4: cp_fwd_kernel<0, T, 1, 4><<<nb, 256, 0, s>>>(elems, res, nnz, es, N, fp, pk, R, c.L, part); break;
      default: cp_fwd_kernel<0, T, 1, 8><<<nb, 256, 0, s>>>(elems, res, nnz, es, N, fp, pk, R, c.L, part); break;
    }
  }
  return nb;
}

int launch_cp_fwd(const uint8_t* elems, uint8_t* res, int64_t nnz, int es, int N,
                  const FactorPtrs& fp, const PackInfo& pk, int R, int dtype, double* part,
                  int nb, float* loss, double* loss64, cudaStream_t s) {
  bool aligned = true;
  for (int k = 0; k < N; ++k) aligned = aligned && (((uintptr_t)fp.p[k] & 15u) == 0);
  const int used = dtype == SPM_DTYPE_BF16
                       ? fwd_dispatch<__nv_bfloat16>(elems, res, nnz, es, N, fp, pk, R, aligned,
                                                     part, nb, s)
                       : fwd_dispatch<float>(elems, res, nnz, es, N, fp, pk, R, aligned, part, nb,
                                             s);
  cp_loss_final_kernel<<<1, 32, 0, s>>>(part, used, loss, loss64);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "cp_fwd kernels");
}

}  // namespace spm
