// mttkrp_common.cuh - helpers shared by the fused spMTTKRP + remap kernels:
// lane layout of a rank-R row over a group of lanes, bulk-async copy and
// mbarrier PTX wrappers with bounded waits, and 16-byte factor-row loads.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "engine.h"

namespace spm {


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

// narrow_bf16: BF16 rows of R <= 32 values use 8-byte lane slices (4 values), so
// that a rank-32 row takes 8 lanes, as an FP32 one does (the warp-block form).
inline LaneCfg lane_config(int R, int dtype, bool aligned16, bool narrow_bf16 = false) {
  LaneCfg c;
  int vw = dtype == SPM_DTYPE_BF16 ? ((narrow_bf16 && R <= 32) ? 4 : 8) : 4;
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

// ------------------------------------------------------------ stored nonzeros

// Index k of a stored nonzeros (plain: word k; packed: its bit field).
__device__ __forceinline__ uint32_t pk_field(const uint32_t* w, int off, int b) {
  uint64_t x;
  if (off < 32)
    x = (((uint64_t)w[1] << 32) | w[0]) >> off;
  else if (off < 64)
    x = (((uint64_t)w[2] << 32) | w[1]) >> (off - 32);
  else
    x = (uint64_t)(w[2] >> (off - 64));
  return (uint32_t)x & ((1u << b) - 1u);
}
__device__ __forceinline__ int elem_index(const uint8_t* ep, int k, const PackInfo& pk) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(ep);
  return pk.packed ? (int)pk_field(w, pk.off[k], pk.bits[k]) : (int)w[k];
}
__device__ __forceinline__ float elem_value(const uint8_t* ep, int N, const PackInfo& pk) {
  return reinterpret_cast<const float*>(ep)[pk.packed ? 3 : N];
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

// 1D bulk async copy with an L2 cache policy (e.g. evict_first for streams).
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// L2 cache policies: 0 = evict_normal, 1 = evict_first, 2 = evict_last.
__device__ __forceinline__ uint64_t make_policy(int kind) {
  uint64_t p;
  if (kind == 1)
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  else if (kind == 2)
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  else
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 16-byte global store with an L2 cache policy, not allocated in L1.
__device__ __forceinline__ void st_hint_v4(void* ptr, uint4 v, uint64_t policy) {
  asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(
                   ptr),
               "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "l"(policy)
               : "memory");
}

// 32-byte global store (a whole DRAM sector) with an L2 cache policy; the
// address must be 32-byte aligned.  A full-sector write needs no read of the
// sector's old contents, unlike a 16-byte write into it.
__device__ __forceinline__ void st_hint_v8(void* ptr, uint4 lo, uint4 hi, uint64_t policy) {
  asm volatile(
      "st.global.L1::no_allocate.L2::cache_hint.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8}, "
      "%9;" ::"l"(ptr),
      "r"(lo.x), "r"(lo.y), "r"(lo.z), "r"(lo.w), "r"(hi.x), "r"(hi.y), "r"(hi.z), "r"(hi.w),
      "l"(policy)
      : "memory");
}

// 16-byte read-only global load with an L2 cache policy.
__device__ __forceinline__ uint4 ld_nc_hint_v4(const void* ptr, uint64_t policy) {
  uint4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(ptr), "l"(policy));
  return v;
}

// 8-byte read-only global load with an L2 cache policy, and with an L1 choice.
__device__ __forceinline__ uint2 ld_nc_hint_v2(const void* ptr, uint64_t policy) {
  uint2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
               : "=r"(v.x), "=r"(v.y)
               : "l"(ptr), "l"(policy));
  return v;
}
__device__ __forceinline__ uint2 ld_nc_l1_v2(const void* ptr, uint64_t policy, bool keep) {
  uint2 v;
  if (keep)
    asm volatile("ld.global.nc.L1::evict_last.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(ptr), "l"(policy));
  else
    asm volatile("ld.global.nc.L1::evict_first.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(ptr), "l"(policy));
  return v;
}

// 16-byte read-only global load with an L1 choice and an L2 cache policy: rows
// marked hot are kept in L1 longest (evict_last), the others leave it first
// (evict_first), so that L1 favours the most frequently gathered factor rows.
__device__ __forceinline__ uint4 ld_nc_l1_v4(const void* ptr, uint64_t policy, bool keep) {
  uint4 v;
  if (keep)
    asm volatile("ld.global.nc.L1::evict_last.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(ptr), "l"(policy));
  else
    asm volatile("ld.global.nc.L1::evict_first.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(ptr), "l"(policy));
  return v;
}

// Paired FP32 arithmetic (two lanes of IEEE round-to-nearest per instruction;
// the same result as two scalar operations).
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)),
        "l"(*reinterpret_cast<unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(r)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)),
        "l"(*reinterpret_cast<unsigned long long*>(&b)),
        "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return *reinterpret_cast<float2*>(&r);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // default bounded-wait limit

// Bounded wait on an mbarrier phase: gives up after limit_ns and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
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
    if (global_ns() - t0 > limit_ns) return false;
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
  __device__ __forceinline__ static void load_hint(const void* base, int64_t row, int R, int sub,
                                                   uint64_t pol, float* x) {
    const uint4 v = ld_nc_hint_v4(
        reinterpret_cast<const float4*>(static_cast<const float*>(base) + row * R) + sub, pol);
    x[0] = __uint_as_float(v.x);
    x[1] = __uint_as_float(v.y);
    x[2] = __uint_as_float(v.z);
    x[3] = __uint_as_float(v.w);
  }
};

template <>
struct Slice<__nv_bfloat16, 8> {
  __device__ __forceinline__ static void unpack(uint4 v, float* x) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[2 * j] = __uint_as_float(w[j] << 16);
      x[2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
    }
  }
  __device__ __forceinline__ static void load(const void* base, int64_t row, int R, int sub,
                                              float* x) {
    unpack(__ldg(reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(base) + row * R) +
                 sub),
           x);
  }
  __device__ __forceinline__ static void load_hint(const void* base, int64_t row, int R, int sub,
                                                   uint64_t pol, float* x) {
    unpack(ld_nc_hint_v4(
               reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(base) + row * R) +
                   sub,
               pol),
           x);
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

}  // namespace spm
