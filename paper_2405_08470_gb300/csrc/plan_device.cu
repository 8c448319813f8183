// plan_device.cu - the plan's orders built on the GPU (the preprocessing of
// Sections 3.1 and 3.4, whose cost the evaluation reports in Section 5.7):
// the canonical orders K_n by a stable LSD radix sort, the duplicate check, the
// mode-0 working copy, every mode's next_pos and the row starts the host
// partition reads.  With distinct coordinates every K_n order is total, so the
// result equals the host build's bit for bit.
//
// Radix sort: (key, element) pairs, 8-bit digits, three kernels per pass —
// digit counts per tile of 4096, an exclusive scan of the digit-major count
// table, and a stable scatter in which each warp places its 512-element
// sub-tile chunk by chunk (ranks inside a chunk from __match_any_sync).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "engine.h"
#include "mttkrp_tile.cuh"

namespace spm {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 elements per block
constexpr int kSubTile = kSortTile / kSortWarps;      // 512 per warp
constexpr int kDigits = 256;

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;  // 8192

// Exclusive prefix of v over a block of kScanThreads threads; *total = block sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_sums[lane] = t;
  }
  __syncthreads();
  const uint32_t before = w ? warp_sums[w - 1] : 0u;
  *total = warp_sums[31];
  __syncthreads();
  return before + x - v;
}

__global__ void scan_partials_kernel(const uint32_t* __restrict__ in, int64_t m,
                                     uint32_t* __restrict__ partial) {
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j)
    if (base + j < m) s += in[base + j];
  uint32_t tot;
  (void)block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void scan_top_kernel(uint32_t* __restrict__ partial, int np) {
  uint32_t carry = 0;
  for (int base = 0; base < np; base += kScanThreads) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < np ? partial[i] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(v, &tot);
    if (i < np) partial[i] = carry + ex;
    carry += tot;
  }
}

// in and out may be the same array: each element is read and written by one thread.
__global__ void scan_apply_kernel(const uint32_t* in, uint32_t* out, int64_t m,
                                  const uint32_t* __restrict__ partial) {
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < m ? in[base + j] : 0u;
    s += v[j];
  }
  uint32_t tot;
  uint32_t ex = block_exclusive_scan(s, &tot) + partial[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < m) out[base + j] = ex;
    ex += v[j];
  }
}

// Digit counts of one tile, stored digit-major: counts[d * nb + tile].
__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                  uint32_t mask, uint32_t* __restrict__ counts, int nb) {
  __shared__ uint32_t h[kDigits];
  for (int d = threadIdx.x; d < kDigits; d += kSortThreads) h[d] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int j = 0; j < kSortItems; ++j) {
    const int64_t i = t0 + threadIdx.x + (int64_t)j * kSortThreads;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kDigits; d += kSortThreads)
    counts[(int64_t)d * nb + blockIdx.x] = h[d];
}

// Stable placement of one tile by digit; offsets = exclusive scan of counts.
__global__ void radix_scatter_kernel(const uint32_t* __restrict__ kin,
                                     const int32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                                     int32_t* __restrict__ vout, int64_t n, int shift,
                                     uint32_t mask, const uint32_t* __restrict__ offsets, int nb) {
  __shared__ uint32_t wpos[kSortWarps][kDigits];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (int d = lane; d < kDigits; d += 32) wpos[w][d] = 0;
  __syncwarp();
  const int64_t s0 = (int64_t)blockIdx.x * kSortTile + (int64_t)w * kSubTile;
  // 1) digit counts of this warp's sub-tile (the lowest lane of each digit group adds)
  for (int c = 0; c < kSubTile; c += 32) {
    const int64_t i = s0 + c + lane;
    const uint32_t d = i < n ? (kin[i] >> shift) & mask : (uint32_t)kDigits;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (d < (uint32_t)kDigits && (peers & below) == 0) wpos[w][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // 2) each warp's first position per digit: the tile's offset plus earlier warps
  for (int d = threadIdx.x; d < kDigits; d += kSortThreads) {
    uint32_t run = offsets[(int64_t)d * nb + blockIdx.x];
    for (int q = 0; q < kSortWarps; ++q) {
      const uint32_t c = wpos[q][d];
      wpos[q][d] = run;
      run += c;
    }
  }
  __syncthreads();
  // 3) chunks in order; inside a chunk, equal digits keep lane order
  for (int c = 0; c < kSubTile; c += 32) {
    const int64_t i = s0 + c + lane;
    const bool act = i < n;
    const uint32_t k = act ? kin[i] : 0u;
    const uint32_t d = act ? (k >> shift) & mask : (uint32_t)kDigits;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (act) {
      const uint32_t pos = wpos[w][d] + __popc(peers & below);
      kout[pos] = k;
      vout[pos] = vin[i];
    }
    __syncwarp();
    if (act && (peers & below) == 0) wpos[w][d] += __popc(peers);
    __syncwarp();
  }
}

__global__ void iota_kernel(int32_t* __restrict__ p, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int32_t)i;
}

__global__ void gather_keys_kernel(const int32_t* __restrict__ key, const int32_t* __restrict__ perm,
                                   uint32_t* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint32_t)key[perm[i]];
}

// Equal neighbours in mode-0 order; records the first position found.
__global__ void duplicate_kernel(const int32_t* __restrict__ keys, int64_t n, int N,
                                 const int32_t* __restrict__ perm, unsigned long long* first) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q + 1 >= n) return;
  const int32_t x = perm[q], y = perm[q + 1];
  for (int k = 0; k < N; ++k)
    if (keys[(int64_t)k * n + x] != keys[(int64_t)k * n + y]) return;
  atomicMin(first, (unsigned long long)q);
}

// The working copy in `perm` order: {int32 idx[N]; float val; zero padding}, or
// the packed 16-byte form (index bit fields in words 0..2, value in word 3).
__global__ void fill_elems_kernel(const int32_t* __restrict__ keys, const float* __restrict__ vals,
                                  int64_t n, int N, const int32_t* __restrict__ perm,
                                  uint8_t* __restrict__ out, int es, PackInfo pk) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int32_t x = perm[q];
  if (pk.packed) {
    uint64_t lo = 0, hi = 0;
    for (int k = 0; k < N; ++k) {
      const uint64_t v = (uint32_t)keys[(int64_t)k * n + x];
      const int off = pk.off[k];
      if (off < 64) {
        lo |= v << off;
        if (off + pk.bits[k] > 64) hi |= v >> (64 - off);
      } else {
        hi |= v << (off - 64);
      }
    }
    *reinterpret_cast<uint4*>(out + q * es) =
        make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, __float_as_uint(vals[x]));
    return;
  }
  uint4* d = reinterpret_cast<uint4*>(out + q * es);
  for (int v = 0; v < es / 16; ++v) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * v + j;
      w[j] = k < N ? (uint32_t)keys[(int64_t)k * n + x]
                   : (k == N ? __float_as_uint(vals[x]) : 0u);
    }
    d[v] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Remap ids carried in the stored nonzeros: word 4 + m of the nonzero at mode-0
// position pos0[x] is x's position q in mode m's order (cur = that order).
__global__ void alpha_fill_kernel(const int32_t* __restrict__ cur, const int32_t* __restrict__ pos0,
                                  int64_t n, int m, uint8_t* __restrict__ elems, int es) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) reinterpret_cast<int32_t*>(elems + (int64_t)pos0[cur[q]] * es)[4 + m] = (int32_t)q;
}

__device__ __forceinline__ bool row_start_at(const int32_t* key, const int32_t* cur, int64_t q) {
  return q == 0 || key[cur[q]] != key[cur[q - 1]];
}

__global__ void row_flags_kernel(const int32_t* __restrict__ key, const int32_t* __restrict__ cur,
                                 int64_t n, uint32_t* __restrict__ flags) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) flags[q] = row_start_at(key, cur, q) ? 1u : 0u;
}

__global__ void row_compact_kernel(const int32_t* __restrict__ key, const int32_t* __restrict__ cur,
                                   const uint32_t* __restrict__ pos, int64_t n,
                                   int32_t* __restrict__ starts, int32_t* __restrict__ ids) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n && row_start_at(key, cur, q)) {
    starts[pos[q]] = (int32_t)q;
    ids[pos[q]] = key[cur[q]];
  }
}

__global__ void inverse_kernel(const int32_t* __restrict__ perm, int32_t* __restrict__ inv,
                               int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) inv[perm[q]] = (int32_t)q;
}

__global__ void compose_kernel(const int32_t* __restrict__ inv, const int32_t* __restrict__ cur,
                               int32_t* __restrict__ out, int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = inv[cur[q]];
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

int bits_for(int64_t dim) {
  int b = 1;
  while (b < 31 && (int64_t(1) << b) < dim) ++b;
  return b;
}

// Device scratch of one build; freed on every exit path.
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* q : ptrs) cudaFree(q);
  }
  template <typename T>
  int alloc(T** out, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation
                                     ? fail(SPM_ERR_OOM, "device plan build: out of memory")
                                     : cuda_fail(e, "cudaMalloc (device plan build)");
    ptrs.push_back(q);
    *out = static_cast<T*>(q);
    return SPM_OK;
  }
};

struct Sorter {
  int64_t n = 0;
  int nb = 0;
  uint32_t *k0 = nullptr, *k1 = nullptr, *counts = nullptr, *partial = nullptr;
  cudaStream_t s = nullptr;

  int scan(uint32_t* a, int64_t m) {
    const int np = (int)((m + kScanChunk - 1) / kScanChunk);
    scan_partials_kernel<<<np, kScanThreads, 0, s>>>(a, m, partial);
    scan_top_kernel<<<1, kScanThreads, 0, s>>>(partial, np);
    scan_apply_kernel<<<np, kScanThreads, 0, s>>>(a, a, m, partial);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPM_OK : cuda_fail(e, "scan kernels");
  }

  // Stable sort of the element ids in *perm by key[id] (values < dim); *spare
  // is a second array of n ids.  The result is in *perm.
  int sort_by(const int32_t* key, int64_t dim, int32_t** perm, int32_t** spare) {
    gather_keys_kernel<<<grid_for(n, 256), 256, 0, s>>>(key, *perm, k0, n);
    const int bits = bits_for(dim);
    uint32_t *ki = k0, *ko = k1;
    int32_t *vi = *perm, *vo = *spare;
    for (int shift = 0; shift < bits; shift += 8) {
      const int b = std::min(8, bits - shift);
      const uint32_t mask = (1u << b) - 1u;
      radix_hist_kernel<<<nb, kSortThreads, 0, s>>>(ki, n, shift, mask, counts, nb);
      int st = scan(counts, (int64_t)kDigits * nb);
      if (st) return st;
      radix_scatter_kernel<<<nb, kSortThreads, 0, s>>>(ki, vi, ko, vo, n, shift, mask, counts, nb);
      std::swap(ki, ko);
      std::swap(vi, vo);
    }
    *perm = vi;
    *spare = vo;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPM_OK : cuda_fail(e, "radix sort kernels");
  }
};

}  // namespace

int build_device_orders(spmttkrp_plan* p, const std::vector<std::vector<int32_t>>& key,
                        const float* vals, uint8_t* elems, int32_t* const* next_pos) {
  const int N = p->N;
  const int64_t n = p->nnz;
  cudaStream_t s = p->stream;
  if (n <= 0) return SPM_OK;
  if (n >= (int64_t)1 << 31) return fail(SPM_ERR_UNSUPPORTED, "device plan build: nnz >= 2^31");
  Scratch sc;
  int32_t *d_keys, *cur, *spare, *nxt, *inv, *pos0 = nullptr;
  float* d_vals;
  unsigned long long* d_dup;
  Sorter so;
  so.n = n;
  so.nb = (int)((n + kSortTile - 1) / kSortTile);
  so.s = s;
  int st;
  if ((st = sc.alloc(&d_keys, (size_t)N * n)) || (st = sc.alloc(&d_vals, (size_t)n)) ||
      (st = sc.alloc(&cur, (size_t)n)) || (st = sc.alloc(&spare, (size_t)n)) ||
      (st = sc.alloc(&nxt, (size_t)n)) || (st = sc.alloc(&inv, (size_t)n)) ||
      (st = sc.alloc(&so.k0, (size_t)n)) || (st = sc.alloc(&so.k1, (size_t)n)) ||
      (st = sc.alloc(&so.counts, (size_t)kDigits * so.nb)) ||
      (st = sc.alloc(&so.partial, (size_t)(std::max<int64_t>((int64_t)kDigits * so.nb, n) /
                                               kScanChunk + 2))) ||
      (st = sc.alloc(&d_dup, 1)) || (p->alpha && (st = sc.alloc(&pos0, (size_t)n))))
    return st;
  for (int k = 0; k < N; ++k)
    SPM_CUDA(cudaMemcpyAsync(d_keys + (int64_t)k * n, key[(size_t)k].data(), (size_t)n * 4,
                             cudaMemcpyHostToDevice, s));
  SPM_CUDA(cudaMemcpyAsync(d_vals, vals, (size_t)n * 4, cudaMemcpyHostToDevice, s));

  // mode-0 order: stable sorts by i_1, i_2, ..., i_{N-1}, then i_0 (primary)
  iota_kernel<<<grid_for(n, 256), 256, 0, s>>>(cur, n);
  for (int j = 1; j <= N; ++j) {
    const int k = j % N;
    if ((st = so.sort_by(d_keys + (int64_t)k * n, p->dims[(size_t)k], &cur, &spare))) return st;
  }
  const unsigned long long none = ~0ull;
  SPM_CUDA(cudaMemcpyAsync(d_dup, &none, sizeof(none), cudaMemcpyHostToDevice, s));
  duplicate_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_keys, n, N, cur, d_dup);
  unsigned long long dup = 0;
  SPM_CUDA(cudaMemcpyAsync(&dup, d_dup, sizeof(dup), cudaMemcpyDeviceToHost, s));
  SPM_CUDA(cudaStreamSynchronize(s));
  if (dup != none) return fail(SPM_ERR_DUPLICATE, "duplicate coordinate in the COO input");
  fill_elems_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_keys, d_vals, n, N, cur, elems, p->es,
                                                      p->pack);
  if (p->alpha) inverse_kernel<<<grid_for(n, 256), 256, 0, s>>>(cur, pos0, n);

  // per mode: row starts (to the host), the next order, next_pos (stays on the device)
  p->row_start.assign((size_t)2 * N, {});
  std::vector<int32_t> hs, hid;
  for (int m = 0; m < N; ++m) {
    if (p->alpha) alpha_fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(cur, pos0, n, m, elems, p->es);
    const int32_t* km = d_keys + (int64_t)m * n;
    uint32_t* pos = so.k0;  // scratch between sorts
    row_flags_kernel<<<grid_for(n, 256), 256, 0, s>>>(km, cur, n, pos);
    uint32_t last_flag = 0, last_pos = 0;
    SPM_CUDA(cudaMemcpyAsync(&last_flag, pos + n - 1, 4, cudaMemcpyDeviceToHost, s));
    if ((st = so.scan(pos, n))) return st;
    SPM_CUDA(cudaMemcpyAsync(&last_pos, pos + n - 1, 4, cudaMemcpyDeviceToHost, s));
    SPM_CUDA(cudaStreamSynchronize(s));
    const int64_t nu = (int64_t)last_pos + last_flag;
    int32_t* starts = reinterpret_cast<int32_t*>(so.k1);
    int32_t* ids = inv;  // scratch until the inverse below
    row_compact_kernel<<<grid_for(n, 256), 256, 0, s>>>(km, cur, pos, n, starts, ids);
    hs.resize((size_t)nu);
    hid.resize((size_t)nu);
    SPM_CUDA(cudaMemcpyAsync(hs.data(), starts, (size_t)nu * 4, cudaMemcpyDeviceToHost, s));
    SPM_CUDA(cudaMemcpyAsync(hid.data(), ids, (size_t)nu * 4, cudaMemcpyDeviceToHost, s));
    SPM_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t>& us = p->row_start[(size_t)m];
    std::vector<int64_t>& ur = p->row_start[(size_t)N + m];
    us.assign((size_t)nu + 1, n);
    ur.assign((size_t)nu, 0);
    for (int64_t u = 0; u < nu; ++u) {
      us[(size_t)u] = hs[(size_t)u];
      ur[(size_t)u] = hid[(size_t)u];
    }
    // next order: stable sort of K_m by i_{m+1}; next_pos_m = its inverse at cur
    const int mx = (m + 1) % N;
    SPM_CUDA(cudaMemcpyAsync(nxt, cur, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    if ((st = so.sort_by(d_keys + (int64_t)mx * n, p->dims[(size_t)mx], &nxt, &spare))) return st;
    inverse_kernel<<<grid_for(n, 256), 256, 0, s>>>(nxt, inv, n);
    compose_kernel<<<grid_for(n, 256), 256, 0, s>>>(inv, cur, next_pos[m], n);
    std::swap(cur, nxt);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "device plan build kernels");
  SPM_CUDA(cudaStreamSynchronize(s));
  return SPM_OK;
}

}  // namespace spm

// ---------------------------------------------------------------------------
// Write orders of the tile form.

namespace spm {
namespace {

// One CTA per tile of mode m's order: sort the tile's (next_pos, local index)
// pairs by next_pos (bitonic network in shared memory; next_pos values are
// distinct) and store, for slot j, the local index of the j-th smallest.
__global__ void __launch_bounds__(256) write_order_kernel(const int32_t* __restrict__ next_pos,
                                                          int64_t n,
                                                          uint16_t* __restrict__ worder) {
  constexpr int P = 1024;  // the network's size: kTileNnz rounded up to a power of two
  static_assert(kTileNnz <= P, "tile larger than the sorting network");
  __shared__ unsigned long long key[P];
  const int64_t base = (int64_t)blockIdx.x * kTileNnz;
  const int len = (int)min((int64_t)kTileNnz, n - base);
  for (int i = threadIdx.x; i < P; i += blockDim.x)
    key[i] = i < len ? (((unsigned long long)(uint32_t)next_pos[base + i] << 10) | (unsigned)i)
                     : ~0ull;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long x = key[i], y = key[ixj];
          const bool up = (i & k) == 0;
          if (up ? (x > y) : (x < y)) {
            key[i] = y;
            key[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < len; i += blockDim.x)
    worder[base + i] = (uint16_t)(key[i] & 1023u);
}

// Word 7 of each nonzero (copy in mode-0 order): the write orders of the slots
// it occupies in the three orders (its position p in mode 0, alpha_1, alpha_2).
__global__ void write_order_fill_kernel(uint8_t* __restrict__ elems, int64_t n,
                                        const uint16_t* __restrict__ w0,
                                        const uint16_t* __restrict__ w1,
                                        const uint16_t* __restrict__ w2) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  uint32_t* e = reinterpret_cast<uint32_t*>(elems + q * 32);
  const uint32_t a1 = e[5] & kAlphaMask, a2 = e[6] & kAlphaMask;
  e[kTileWordW] = (uint32_t)w0[q] | ((uint32_t)w1[a1] << 10) | ((uint32_t)w2[a2] << 20);
}

}  // namespace

int build_write_orders(spmttkrp_plan* p, uint8_t* elems) {
  if (!(p->N == 3 && p->es == 32 && p->alpha) || p->nnz <= 0) return SPM_OK;
  const int64_t n = p->nnz;
  cudaStream_t s = p->stream;
  Scratch sc;
  uint16_t* w;
  int st = sc.alloc(&w, (size_t)3 * n);
  if (st) return st;
  const unsigned tiles = (unsigned)((n + kTileNnz - 1) / kTileNnz);
  for (int m = 0; m < 3; ++m)
    write_order_kernel<<<tiles, 256, 0, s>>>(p->md[(size_t)m].next_pos, n, w + (size_t)m * n);
  write_order_fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(elems, n, w, w + n, w + 2 * n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "write-order kernels");
  SPM_CUDA(cudaStreamSynchronize(s));
  p->worders = 1;
  return SPM_OK;
}

}  // namespace spm

// ---------------------------------------------------------------------------
// Hot-row flags.
namespace spm {
namespace {

__global__ void hot_flag_kernel(uint8_t* __restrict__ elems, int64_t n,
                                const uint8_t* __restrict__ h0, const uint8_t* __restrict__ h1,
                                const uint8_t* __restrict__ h2) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  uint32_t* e = reinterpret_cast<uint32_t*>(elems + q * 32);
  const uint8_t* h[3] = {h0, h1, h2};
#pragma unroll
  for (int k = 0; k < 3; ++k)
    e[4 + k] = (e[4 + k] & kAlphaMask) | (h[k][e[k]] ? 0x80000000u : 0u);
}

}  // namespace

int build_hot_flags(spmttkrp_plan* p, uint8_t* elems) {
  if (!(p->N == 3 && p->es == 32 && p->alpha) || p->nnz <= 0) return SPM_OK;
  // rows per factor: the two gathered factors' hot rows together fill about 48 KB
  // of L1 (192 rows of 32 FP32 values)
  const int s = p->dtype == SPM_DTYPE_BF16 ? 2 : 4;
  const int H = std::max(16, 24576 / (p->R * s));
  Scratch sc;
  uint8_t* dh[3];
  for (int k = 0; k < 3; ++k) {
    const int64_t I = p->dims[(size_t)k];
    const std::vector<int64_t>& us = p->row_start[(size_t)k];
    const std::vector<int64_t>& ur = p->row_start[(size_t)3 + k];
    std::vector<std::pair<int64_t, int64_t>> deg(ur.size());  // (-degree, row)
    for (size_t u = 0; u < ur.size(); ++u) deg[u] = {-(us[u + 1] - us[u]), ur[u]};
    const size_t take = std::min<size_t>((size_t)H, deg.size());
    std::partial_sort(deg.begin(), deg.begin() + (std::ptrdiff_t)take, deg.end());
    std::vector<uint8_t> hot((size_t)I, 0);
    for (size_t u = 0; u < take; ++u) hot[(size_t)deg[u].second] = 1;
    int st = sc.alloc(&dh[k], (size_t)I);
    if (st) return st;
    SPM_CUDA(cudaMemcpyAsync(dh[k], hot.data(), (size_t)I, cudaMemcpyHostToDevice, p->stream));
  }
  hot_flag_kernel<<<grid_for(p->nnz, 256), 256, 0, p->stream>>>(elems, p->nnz, dh[0], dh[1], dh[2]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "hot_flag_kernel launch");
  SPM_CUDA(cudaStreamSynchronize(p->stream));
  p->hot_rows = H;
  return SPM_OK;
}

}  // namespace spm
