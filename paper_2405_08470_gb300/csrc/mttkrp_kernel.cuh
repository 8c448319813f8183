// mttkrp_kernel.cuh - the fused mode-n spMTTKRP + dynamic remap kernel.
//
// One CTA owns one block [lo, hi) of the mode-n ordered working copy (the
// paper's thread block over a tensor partition, Algorithm 4).  Its nonzeros
// are streamed through shared memory in tiles by 1D bulk-async copies
// (cp.async.bulk, completion on an mbarrier, three buffers, two tiles in
// flight).  For every tile:
//   * remap (Algorithm 3): every thread copies elements to their place in
//     the next mode's order, T_out[next_pos[p]] = x_p;
//   * elementwise computation (Algorithm 2): the CTA is cut into groups of L
//     lanes, each lane owning a 16-byte slice of a rank-R row; a group walks
//     a contiguous run of the tile, gathers A_k[i_k, slice] for k != n with
//     16-byte read-only loads, forms val * Hadamard product, and accumulates
//     it in registers while the output row stays the same;
//   * rows that start and end inside one run are written straight to M_n;
//     a run's first and last rows leave partial sums in shared-memory slots
//     that one warp adds in run order on the next tile (carrying the row
//     that continues into the following tile).
// A row that continues past the block's end is written as a partial to
// `part` and summed by the fix-up kernel in block order.  Nothing is added
// atomically, so results are bit-identical from run to run, and every output
// row is written exactly once (rows without nonzeros are zero-filled by the
// writer of the next nonempty row, or of the last one).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "engine.h"

namespace spm {

constexpr int kNBuf = 3;  // element tile buffers (two tiles in flight)

struct LaneCfg {
  int L;    // lanes per nonzero (power of two <= 32)
  int VW;   // elements per lane per load (4 fp32 / 8 bf16 for 16-byte loads, else 1)
  int RC;   // rank chunks per lane for the scalar path
  bool vec;
};

__host__ __device__ inline int pow2ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

inline LaneCfg lane_config(int R, int dtype, bool aligned16) {
  LaneCfg c;
  int vw = dtype == SPM_DTYPE_BF16 ? 8 : 4;
  if (aligned16 && R % vw == 0 && R / vw <= 32) {
    c.vec = true;
    c.VW = vw;
    c.L = pow2ceil(R / vw);
    c.RC = 1;
  } else {
    c.vec = false;
    c.VW = 1;
    if (R <= 32) {
      c.L = pow2ceil(R);
      c.RC = 1;
    } else {
      c.L = 32;
      c.RC = pow2ceil((R + 31) / 32);
    }
  }
  return c;
}

// Shared-memory layout of the fused kernel (bytes, in order).
struct SmemLayout {
  size_t ebuf, npbuf, sacc, srow, sprev, cacc, cmeta, mbar, total;
};

__host__ __device__ inline SmemLayout smem_layout(int es, int tile, int R, int NG) {
  SmemLayout l;
  size_t o = 0;
  l.ebuf = o;
  o += (size_t)kNBuf * tile * es;
  l.npbuf = o;
  o += (size_t)kNBuf * (tile + 8) * 4;
  l.sacc = o;
  o += (size_t)2 * 2 * NG * R * 4;
  l.srow = o;
  o += (size_t)2 * 2 * NG * 4;
  l.sprev = o;
  o += (size_t)2 * 2 * NG * 4;
  l.cacc = o;
  o += (size_t)R * 4;
  l.cmeta = o;
  o += 16;
  o = (o + 7) & ~(size_t)7;
  l.mbar = o;
  o += (size_t)kNBuf * 8;
  l.total = (o + 127) & ~(size_t)127;
  return l;
}

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// 1D bulk async copy global -> shared, completes `bytes` on the mbarrier.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: gives up after ~2 s and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const uint64_t t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > 2000000000ull) return false;
  }
}

// ------------------------------------------------------------ factor slices

template <typename T, int VW>
struct Slice;

template <>
struct Slice<float, 4> {
  __device__ __forceinline__ static void load(const void* base, int64_t row, int R, int sub,
                                              float* x) {
    const float4 v =
        __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(base) + row * R) + sub);
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
  }
};

template <>
struct Slice<__nv_bfloat16, 8> {
  __device__ __forceinline__ static void load(const void* base, int64_t row, int R, int sub,
                                              float* x) {
    const uint4 v = __ldg(
        reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(base) + row * R) + sub);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[2 * j] = __uint_as_float(w[j] << 16);
      x[2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
    }
  }
};

template <typename T>
__device__ __forceinline__ float load_scalar(const void* base, int64_t idx);
template <>
__device__ __forceinline__ float load_scalar<float>(const void* base, int64_t idx) {
  return __ldg(static_cast<const float*>(base) + idx);
}
template <>
__device__ __forceinline__ float load_scalar<__nv_bfloat16>(const void* base, int64_t idx) {
  const unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(base) + idx);
  return __uint_as_float((uint32_t)u << 16);
}

// ------------------------------------------------------------ the kernel

// NT: number of modes at compile time (0 = runtime).  T: factor type.
// VW: values per lane per load (vector path) or 1 (scalar path).
// RC: rank chunks per lane (scalar path; 1 on the vector path).
template <int NT, typename T, int VW, int RC>
__global__ void __launch_bounds__(kThreads) mttkrp_remap_kernel(const MttkrpArgs a, const int L) {
  constexpr int NV = VW * RC;  // accumulator values per lane
  constexpr int U = (VW > 1) ? 4 : 2;  // nonzeros in flight per group
  const int N = NT > 0 ? NT : a.nmodes;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = 32 / L, NG = (kThreads / 32) * G;
  const int tile = a.tile, K = tile / NG, es = a.es, R = a.R, mode = a.mode;
  const int sub = lane % L, gw = lane / L, gi = warp * G + gw;

  extern __shared__ __align__(128) uint8_t smem[];
  const SmemLayout lay = smem_layout(es, tile, R, NG);
  uint8_t* ebuf = smem + lay.ebuf;
  int32_t* npbuf = reinterpret_cast<int32_t*>(smem + lay.npbuf);
  float* sacc = reinterpret_cast<float*>(smem + lay.sacc);
  int* srow = reinterpret_cast<int*>(smem + lay.srow);
  int* sprev = reinterpret_cast<int*>(smem + lay.sprev);
  float* cacc = reinterpret_cast<float*>(smem + lay.cacc);
  int* cmeta = reinterpret_cast<int*>(smem + lay.cmeta);  // carry row, carry prev, emitted, status
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + lay.mbar);

  const int4 bi = a.blkinfo[blockIdx.x];
  const int lo = bi.x, hi = bi.y;
  if (lo >= hi) return;
  const int ntiles = (hi - lo + tile - 1) / tile;
  const bool remap = a.elems_out != nullptr;
  const float sc = a.scale ? __ldg(a.scale) : 1.0f;
  const int64_t out_rows = a.out_rows;
  float* __restrict__ out = a.out;

  auto issue = [&](int t) {
    const int buf = t % kNBuf;
    const int tlo = lo + t * tile;
    const int n = min(tile, hi - tlo);
    const uint32_t ebytes = (uint32_t)n * es;
    uint32_t npbytes = 0;
    int np0 = 0;
    if (remap) {
      np0 = tlo & ~3;
      npbytes = ((uint32_t)(tlo + n - np0) * 4u + 15u) & ~15u;
    }
    fence_proxy_async_smem();
    mbar_expect_tx(&mbar[buf], ebytes + npbytes);
    bulk_g2s(ebuf + (size_t)buf * tile * es, a.elems_in + (size_t)tlo * es, ebytes, &mbar[buf]);
    if (remap) bulk_g2s(npbuf + buf * (tile + 8), a.next_pos + np0, npbytes, &mbar[buf]);
  };

  if (tid == 0) {
    for (int b = 0; b < kNBuf; ++b) mbar_init(&mbar[b], 1);
    fence_mbar_init();
    cmeta[0] = -1;    // carry row: none yet
    cmeta[1] = bi.z;  // row before the carry row (row before the block)
    cmeta[2] = 0;     // no row emitted yet
    cmeta[3] = 0;     // status
  }
  for (int r = tid; r < R; r += kThreads) cacc[r] = 0.f;
  __syncthreads();
  if (tid == 0) {
    issue(0);
    if (ntiles > 1) issue(1);
  }

  // ---- helpers: rank slices owned by a lane of a group
  auto rank_of = [&](int j) -> int {  // j in [0, NV): rank index of accumulator slot j
    if constexpr (VW > 1) return sub * VW + j;
    return sub + L * j;
  };
  auto zero_rows_group = [&](int64_t from, int64_t to) {  // rows [from, to)
    for (int64_t z = from; z < to; ++z) {
      if constexpr (VW > 1) {
        if (sub * VW < R) {
          float4* d = reinterpret_cast<float4*>(out + z * R + sub * VW);
#pragma unroll
          for (int q = 0; q < VW / 4; ++q) d[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      } else {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          const int r = rank_of(j);
          if (r < R) out[z * R + r] = 0.f;
        }
      }
    }
  };
  auto write_row_group = [&](int row, const float* acc, int prev) {
    zero_rows_group((int64_t)prev + 1, row);
    if constexpr (VW > 1) {
      if (sub * VW < R) {
        float4* d = reinterpret_cast<float4*>(out + (int64_t)row * R + sub * VW);
#pragma unroll
        for (int q = 0; q < VW / 4; ++q)
          d[q] = make_float4(acc[4 * q] * sc, acc[4 * q + 1] * sc, acc[4 * q + 2] * sc,
                             acc[4 * q + 3] * sc);
      }
    } else {
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const int r = rank_of(j);
        if (r < R) out[(int64_t)row * R + r] = acc[j] * sc;
      }
    }
    if (row == a.last_row) zero_rows_group((int64_t)row + 1, out_rows);
  };
  auto store_slot = [&](int sb, int s, int row, int prev, const float* acc) {
    const int so = sb * 2 * NG + s;
    if (sub == 0) {
      srow[so] = row;
      sprev[so] = prev;
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      const int r = rank_of(j);
      if (r < R) sacc[(size_t)so * R + r] = acc[j];
    }
  };

  // ---- combine (one warp): slots of tile tt in run order, then the block's last row
  constexpr int CC = (kMaxRank + 31) / 32;
  auto combine = [&](int tt) {
    const int sb = tt & 1;
    int crow = cmeta[0], cprev = cmeta[1], emitted = cmeta[2];
    const int ncc = (R + 31) / 32;
    float ca[CC];
#pragma unroll
    for (int c = 0; c < CC; ++c) ca[c] = (c < ncc && lane + 32 * c < R) ? cacc[lane + 32 * c] : 0.f;

    auto emit = [&](int row, int prev, bool first, bool last) {
      const bool split = (first && (bi.w & BLK_HEAD_SPLIT)) || (last && (bi.w & BLK_TAIL_SPLIT));
      if (split) {
        float* d = a.part + ((size_t)blockIdx.x * 2 + (first ? 0 : 1)) * R;
#pragma unroll
        for (int c = 0; c < CC; ++c)
          if (c < ncc && lane + 32 * c < R) d[lane + 32 * c] = ca[c];
        return;
      }
      for (int64_t z = (int64_t)prev + 1; z < row; ++z)
#pragma unroll
        for (int c = 0; c < CC; ++c)
          if (c < ncc && lane + 32 * c < R) out[z * R + lane + 32 * c] = 0.f;
#pragma unroll
      for (int c = 0; c < CC; ++c)
        if (c < ncc && lane + 32 * c < R) out[(int64_t)row * R + lane + 32 * c] = ca[c] * sc;
      if (row == a.last_row)
        for (int64_t z = (int64_t)row + 1; z < out_rows; ++z)
#pragma unroll
          for (int c = 0; c < CC; ++c)
            if (c < ncc && lane + 32 * c < R) out[z * R + lane + 32 * c] = 0.f;
    };

    for (int s = 0; s < 2 * NG; ++s) {
      const int so = sb * 2 * NG + s;
      const int row = srow[so];
      if (row < 0) continue;
      const float* sa = sacc + (size_t)so * R;
      if (row == crow) {
#pragma unroll
        for (int c = 0; c < CC; ++c)
          if (c < ncc && lane + 32 * c < R) ca[c] += sa[lane + 32 * c];
      } else {
        if (crow >= 0) {
          emit(crow, cprev, emitted == 0, false);
          emitted = 1;
        }
        const int pv = sprev[so];
        cprev = (pv != -2) ? pv : (crow >= 0 ? crow : cprev);
        crow = row;
#pragma unroll
        for (int c = 0; c < CC; ++c)
          if (c < ncc && lane + 32 * c < R) ca[c] = sa[lane + 32 * c];
      }
    }
    if (tt == ntiles - 1) {
      if (crow >= 0) emit(crow, cprev, emitted == 0, true);
    } else {
#pragma unroll
      for (int c = 0; c < CC; ++c)
        if (c < ncc && lane + 32 * c < R) cacc[lane + 32 * c] = ca[c];
      __syncwarp();
      if (lane == 0) {
        cmeta[0] = crow;
        cmeta[1] = cprev;
        cmeta[2] = emitted;
      }
    }
  };

  int issued = min(ntiles, 2);
  for (int t = 0; t <= ntiles; ++t) {
    if (tid == 0 && t < ntiles) {
      if (!mbar_wait_bounded(&mbar[t % kNBuf], (uint32_t)((t / kNBuf) & 1))) cmeta[3] = 1;
    }
    __syncthreads();
    if (cmeta[3]) {
      // a bulk copy did not complete in time: record it, wait (bounded) for
      // the copies still in flight, and leave without touching the outputs
      if (tid == 0) {
        atomicOr(a.err, 1);
        for (int q = t; q < issued; ++q)
          (void)mbar_wait_bounded(&mbar[q % kNBuf], (uint32_t)((q / kNBuf) & 1));
      }
      return;
    }
    if (tid == 0 && t + 2 < ntiles) {
      issue(t + 2);
      issued = t + 3;
    }
    if (t >= 1 && warp == (t - 1) % (kThreads / 32)) combine(t - 1);
    if (t == ntiles) break;

    // ---- tile t
    const int buf = t % kNBuf, sb = t & 1;
    const int tlo = lo + t * tile;
    const int n = min(tile, hi - tlo);
    const uint8_t* eb = ebuf + (size_t)buf * tile * es;

    if (remap) {  // Algorithm 3: every element to its place in the next mode's order
      const int32_t* np = npbuf + buf * (tile + 8) + (tlo & 3);
      const int nv = es / 16;
      for (int i = tid; i < n * nv; i += kThreads) {
        const int e = i / nv, c = i - e * nv;
        const uint4 v = reinterpret_cast<const uint4*>(eb + (size_t)e * es)[c];
        reinterpret_cast<uint4*>(a.elems_out + (size_t)np[e] * es)[c] = v;
      }
    }

    // Algorithm 2 over this group's run [a0, b0) of the tile
    const int a0 = gi * K, b0 = min(a0 + K, n);
    if (a0 >= b0) {
      if (sub == 0) {
        srow[sb * 2 * NG + 2 * gi] = -1;
        srow[sb * 2 * NG + 2 * gi + 1] = -1;
      }
      continue;
    }
    float acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = 0.f;
    int cur = reinterpret_cast<const int*>(eb + (size_t)a0 * es)[mode];
    bool head = true;
    int prev_in_run = -1;
    for (int e = a0; e < b0; e += U) {
      float prod[U][NV];
      int rows[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (e + u < b0) {
          const int* el = reinterpret_cast<const int*>(eb + (size_t)(e + u) * es);
          rows[u] = el[mode];
          const float v = __int_as_float(el[N]);
#pragma unroll
          for (int j = 0; j < NV; ++j) prod[u][j] = v;
        }
      }
      for (int k = 0; k < N; ++k) {
        if (k == mode) continue;
        const void* Ak = a.factors[k];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (e + u < b0) {
            const int64_t idx = reinterpret_cast<const int*>(eb + (size_t)(e + u) * es)[k];
            float x[NV];
            if constexpr (VW > 1) {
              if (sub * VW < R) {
                Slice<T, VW>::load(Ak, idx, R, sub, x);
              } else {
#pragma unroll
                for (int j = 0; j < NV; ++j) x[j] = 0.f;
              }
            } else {
#pragma unroll
              for (int j = 0; j < NV; ++j) {
                const int r = rank_of(j);
                x[j] = (r < R) ? load_scalar<T>(Ak, idx * R + r) : 0.f;
              }
            }
#pragma unroll
            for (int j = 0; j < NV; ++j) prod[u][j] *= x[j];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (e + u < b0) {
          if (rows[u] != cur) {
            if (head) {
              store_slot(sb, 2 * gi, cur, -2, acc);
              head = false;
            } else {
              write_row_group(cur, acc, prev_in_run);
            }
            prev_in_run = cur;
            cur = rows[u];
#pragma unroll
            for (int j = 0; j < NV; ++j) acc[j] = 0.f;
          }
#pragma unroll
          for (int j = 0; j < NV; ++j) acc[j] += prod[u][j];
        }
      }
    }
    if (head) {
      store_slot(sb, 2 * gi, cur, -2, acc);
      if (sub == 0) srow[sb * 2 * NG + 2 * gi + 1] = -1;
    } else {
      store_slot(sb, 2 * gi + 1, cur, prev_in_run, acc);
    }
  }
}

// ------------------------------------------------------------ launcher

template <int NT, typename T, int VW, int RC>
int launch_variant(const MttkrpArgs& a, int L, cudaStream_t s) {
  const int NG = (kThreads / 32) * (32 / L);
  const SmemLayout lay = smem_layout(a.es, a.tile, a.R, NG);
  auto kfn = mttkrp_remap_kernel<NT, T, VW, RC>;
  static int configured = 0;  // per instantiation: raise the dynamic smem limit once
  if (configured < (int)lay.total) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max<size_t>(lay.total, 48 * 1024));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(mttkrp)");
    configured = (int)std::max<size_t>(lay.total, 48 * 1024);
  }
  kfn<<<a.nblk, kThreads, lay.total, s>>>(a, L);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mttkrp_remap_kernel launch");
  return SPM_OK;
}

}  // namespace spm
