// mttkrp_kernel.cuh - the fused mode-n spMTTKRP + dynamic remap kernel,
// one warp per block of the split.
//
// Every warp owns one block [lo, hi) of the mode-n ordered working copy (the
// paper's thread block over a tensor partition, Algorithm 4, shrunk to a warp
// so that no CTA-wide synchronisation is ever needed).  The warp is cut into
// G groups of L lanes, each lane owning a 16-byte slice of a rank-R row, and
// the block into G equal contiguous runs, one per group.  Each group streams
// its run through the warp's shared-memory ring: its leader lane issues 1D
// bulk-async copies (cp.async.bulk) of the next K nonzeros and of their remap
// ids S-1 tiles ahead, completion is counted on per-warp mbarriers (one
// arrival per group), and every wait is bounded.  For every tile:
//   * remap (Algorithm 3): the group's lanes copy its nonzeros to their places
//     in the next mode's order, T_out[next_pos[p]] = x_p;
//   * elementwise computation (Algorithm 2): the group walks its segment U
//     nonzeros at a time, issues all gathers A_k[i_k, slice] (k != n, 16-byte
//     read-only loads; indices come from shared memory) into packed
//     registers, then accumulates val * Hadamard product in order while the
//     output row is unchanged; rows that start and end inside the run are
//     written straight to M_n, and the run state carries over to the next
//     tile.
// At the end of the block the first and last row of every run, left as
// partial sums in shared memory, are added by the warp in run order; a row
// that continues past the block is written as a partial to `part` and summed
// by the fix-up kernel in block order.  No atomics: results are bit-identical
// from run to run and every output row is written exactly once (empty rows are
// zero-filled by the writer of the next nonempty row, or of the last one).
#pragma once

#include "mttkrp_common.cuh"
#include "mttkrp_tile.cuh"  // the write-order tiles (kTileNnz, kTileWordW)

namespace spm {

constexpr int kMaxStages = 4;  // tiles per warp ring: stages - 1 in flight while one is used
constexpr int kWarps = kThreads / 32;

// Per-warp shared-memory layout (bytes, in order).
struct WarpLayout {
  size_t ebuf, npbuf, sacc, cacc, srow, sprev, mbar, total;
};

// Remap ids staged per group segment of k nonzeros: k + 3 ids at most (the
// copy starts at the 16-byte boundary at or below the segment) rounded up to a
// multiple of 4 ints, so that every bulk-copy destination stays 16-byte aligned.
__host__ __device__ inline int np_stage_ints(int tw) { return (tw + 8 + 3) & ~3; }

__host__ __device__ inline WarpLayout warp_layout(int es, int tw, int R, int G, int stages) {
  WarpLayout l;
  size_t o = 0;
  l.ebuf = o;
  o += (size_t)stages * tw * es;
  l.npbuf = o;
  o += (size_t)stages * G * np_stage_ints(tw / G) * 4;
  l.sacc = o;
  o += (size_t)2 * G * R * 4;
  l.cacc = o;
  o += (size_t)R * 4;
  l.srow = o;
  o += (size_t)2 * G * 4;
  l.sprev = o;
  o += (size_t)2 * G * 4;
  o = (o + 7) & ~(size_t)7;
  l.mbar = o;
  o += (size_t)(stages + 1) * 8;  // the ring, plus one barrier only the stall test waits on
  l.total = (o + 127) & ~(size_t)127;
  return l;
}


// Registers a gathered factor-row slice lands in before it is used: one
// 16-byte vector (4 FP32 or 8 packed BF16) on the vector path, RC scalars on
// the scalar path.  Keeping BF16 packed until use halves the registers that
// loads in flight occupy.
template <typename T, int VW, int RC>
struct Landing {
  using type = uint4;
  __device__ __forceinline__ static void load(const void* base, int64_t row, int R, int sub,
                                              int L, uint64_t pol, type& out) {
    if (sub * VW < R)
      out = ld_nc_hint_v4(reinterpret_cast<const uint4*>(static_cast<const T*>(base) + row * R) +
                              sub,
                          pol);
    else
      out = make_uint4(0u, 0u, 0u, 0u);
  }
  __device__ __forceinline__ static void unpack(const type& v, float* x) {
    if constexpr (VW == 4) {
      x[0] = __uint_as_float(v.x);
      x[1] = __uint_as_float(v.y);
      x[2] = __uint_as_float(v.z);
      x[3] = __uint_as_float(v.w);
    } else {
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[2 * j] = __uint_as_float(w[j] << 16);
        x[2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
      }
    }
  }
};

// BF16 rows in 8-byte lane slices (4 values per lane)
template <>
struct Landing<__nv_bfloat16, 4, 1> {
  using type = uint2;
  __device__ __forceinline__ static void load(const void* base, int64_t row, int R, int sub,
                                              int L, uint64_t pol, type& out) {
    if (sub * 4 < R)
      out = ld_nc_hint_v2(
          reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(base) + row * R) + sub,
          pol);
    else
      out = make_uint2(0u, 0u);
  }
  __device__ __forceinline__ static void unpack(const type& v, float* x) {
    x[0] = __uint_as_float(v.x << 16);
    x[1] = __uint_as_float(v.x & 0xffff0000u);
    x[2] = __uint_as_float(v.y << 16);
    x[3] = __uint_as_float(v.y & 0xffff0000u);
  }
};

// One lane's slice of a factor row at ptr (16 or 8 bytes); with `flagged`, the L1
// choice of a hot-row flag (keep: evict_last; else evict_first).
template <typename LT>
__device__ __forceinline__ LT load_lane(const uint8_t* ptr, uint64_t pol, bool flagged, bool keep);
template <>
__device__ __forceinline__ uint4 load_lane<uint4>(const uint8_t* ptr, uint64_t pol, bool flagged,
                                                  bool keep) {
  return flagged ? ld_nc_l1_v4(ptr, pol, keep) : ld_nc_hint_v4(ptr, pol);
}
template <>
__device__ __forceinline__ uint2 load_lane<uint2>(const uint8_t* ptr, uint64_t pol, bool flagged,
                                                  bool keep) {
  return flagged ? ld_nc_l1_v2(ptr, pol, keep) : ld_nc_hint_v2(ptr, pol);
}

template <typename T, int RC>
struct Landing<T, 1, RC> {
  struct type {
    float v[RC];
  };
  __device__ __forceinline__ static void load(const void* base, int64_t row, int R, int sub,
                                              int L, uint64_t, type& out) {
#pragma unroll
    for (int j = 0; j < RC; ++j) {
      const int r = sub + L * j;
      out.v[j] = r < R ? load_scalar<T>(base, row * R + r) : 0.f;
    }
  }
  __device__ __forceinline__ static void unpack(const type& v, float* x) {
#pragma unroll
    for (int j = 0; j < RC; ++j) x[j] = v.v[j];
  }
};

// NT: modes at compile time (0 = runtime); T: factor type; VW: values per lane
// per 16-byte load (1 = scalar path); RC: rank chunks per lane (scalar path);
// U: nonzeros in flight per lane group; MODE: output mode at compile time (3
// modes only; -1 = runtime); ESB: element bytes when fixed (0 = the smallest
// multiple of 16 that holds N indices and the value).
// LOSS (3 modes, 16- or 32-byte nonzeros): the fused first pass of the CP loss.  Each
// nonzero's own factor row A_n[i_n] is gathered as well; the model value
// m_e = sum_r prod_k A_k[i_k, r] and the residual e = m_e - x_e replace the
// value in the pass (so `out` receives the mode-n gradient of L = 1/2 sum e^2),
// the remapped copy written is the residual copy (the value word holds e), and
// every block leaves its FP64 partial of sum e^2 in loss_part.
// Sums four per-lane partials m[0..3] over the L >= 4 lanes of a lane group
// (lane `sub` of the group; gmask: the group's lanes) and leaves the four totals
// in every lane.  A butterfly per value takes 4 log2(L) shuffles; here the lanes
// first split the values over the two highest lane bits (each keeps the half the
// partner passes), add over the remaining bits, and gather the totals back:
// log2(L) + 4 shuffles.  Every total adds the same pairs in the same order as
// the butterfly (xor L/2 first, then L/4, ...), so the results are bit-identical.
__device__ __forceinline__ void group_sum4(float (&m)[4], int sub, int L, unsigned gmask) {
  const int h = L >> 1, q = L >> 2;
  const bool bh = (sub & h) != 0, bq = (sub & q) != 0;
  // bit h: lanes with it clear keep values 0 and 1, the others 2 and 3
  const float k0 = (bh ? m[2] : m[0]) + __shfl_xor_sync(gmask, bh ? m[0] : m[2], h);
  const float k1 = (bh ? m[3] : m[1]) + __shfl_xor_sync(gmask, bh ? m[1] : m[3], h);
  // bit q: keep one of the two (value 2 bh + bq)
  float t = (bq ? k1 : k0) + __shfl_xor_sync(gmask, bq ? k0 : k1, q);
  for (int off = q >> 1; off > 0; off >>= 1) t += __shfl_xor_sync(gmask, t, off);
  // gather: the partner across bit q holds value 2 bh + !bq, across bit h 2 !bh + ..
  const float t2 = __shfl_xor_sync(gmask, t, q);
  const float lo = bq ? t2 : t, hi = bq ? t : t2;
  const float lo2 = __shfl_xor_sync(gmask, lo, h), hi2 = __shfl_xor_sync(gmask, hi, h);
  m[0] = bh ? lo2 : lo;
  m[1] = bh ? hi2 : hi;
  m[2] = bh ? lo : lo2;
  m[3] = bh ? hi : hi2;
}

// RWARP (3 modes, 32-byte nonzeros carrying remap ids and write orders; form 3):
// the CTA's last warp does the remap of the CTA's blocks, the other warps only
// compute.  The remap warp takes the 960-nonzero write-order tiles that start in
// the CTA's range of the mode order; it stages each with one bulk copy into its
// shared-memory region (`region`: an mbarrier, then the tile at +128) and stores
// the tile's nonzeros in the order of their destinations, so stores that land
// side by side leave together.  The two roles share nothing but the input.
constexpr int kRemapRegion = 128 + kTileNnz * 32;  // bytes of the remap warp's region
__device__ __forceinline__ void remap_warp_tiles(const MttkrpArgs& a, int mode, int cw,
                                                 uint8_t* region, unsigned long long wait_ns) {
  const int lane = threadIdx.x & 31;
  const int b0 = blockIdx.x * cw, b1 = min(b0 + cw, a.nblk) - 1;
  if (b0 > b1) return;
  // a tile belongs to the block holding its first nonzero; the tiles are taken
  // in the compute warps' wavefront order: the k-th tile of each block in turn
  int64_t ft[kWarps], et[kWarps];
  int64_t kmax = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    ft[w] = et[w] = 0;
    if (w < cw && b0 + w <= b1) {
      const int4 bw = a.blkinfo[b0 + w];
      ft[w] = ((int64_t)bw.x + kTileNnz - 1) / kTileNnz;
      et[w] = ((int64_t)bw.y + kTileNnz - 1) / kTileNnz;
      kmax = max(kmax, et[w] - ft[w]);
    }
  }
  int64_t kk = 0;
  int ww = -1;
  auto next_tile = [&]() -> int64_t {  // advances (kk, ww); -1 when done
    for (;;) {
      if (++ww == cw) {
        ww = 0;
        ++kk;
      }
      if (kk >= kmax) return -1;
      int64_t t = -1;
#pragma unroll
      for (int w = 0; w < kWarps; ++w)
        if (w == ww && ft[w] + kk < et[w]) t = ft[w] + kk;
      if (t >= 0) return t;
    }
  };
  int64_t t = next_tile();
  if (t < 0) return;
  uint64_t* bar = reinterpret_cast<uint64_t*>(region);
  uint8_t* buf = region + 128;
  const int nx = (mode + 1) % 3;
  const uint64_t pol = make_policy(1);
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  auto issue = [&](int64_t t) {  // lane 0: stage tile t
    const int64_t base = t * kTileNnz;
    const uint32_t bytes = (uint32_t)min((int64_t)kTileNnz, a.nnz - base) * 32u;
    fence_proxy_async_smem();
    mbar_expect_tx(bar, bytes);
    bulk_g2s_hint(buf, a.elems_in + base * 32, bytes, bar, make_policy(0));
  };
  if (lane == 0) issue(t);
  for (uint32_t it = 0; t >= 0; ++it) {
    const uint32_t parity = it & 1u;
    const bool ok = mbar_wait_bounded(bar, parity, wait_ns);
    if (!__all_sync(0xffffffffu, ok)) {
      // the copy did not complete in time: record it, wait (bounded) for it, leave
      if (lane == 0) {
        if (a.err) atomicOr(a.err, 1);
        (void)mbar_wait_bounded(bar, parity);
      }
      return;
    }
    const int len = (int)min((int64_t)kTileNnz, a.nnz - t * kTileNnz);
    for (int j = lane; j < len; j += 32) {
      const uint32_t wo = reinterpret_cast<const uint32_t*>(buf + (size_t)j * 32)[kTileWordW];
      const int k = (int)((wo >> (10 * mode)) & 1023u);
      if (k >= len) {  // damaged write order: skip and report
        if (a.err) atomicOr(a.err, 2);
        continue;
      }
      const uint4* sp = reinterpret_cast<const uint4*>(buf + (size_t)k * 32);
      const uint4 lo4 = sp[0], hi4 = sp[1];
      const uint32_t dst = (nx == 0 ? hi4.x : (nx == 1 ? hi4.y : hi4.z)) & kAlphaMask;
      if ((int64_t)dst >= a.nnz) {
        if (a.err) atomicOr(a.err, 2);
        continue;
      }
      st_hint_v8(a.elems_out + (int64_t)dst * 32, lo4, hi4, pol);
    }
    __syncwarp();  // every lane has read the tile before the next copy lands on it
    t = next_tile();
    if (lane == 0 && t >= 0) issue(t);
  }
}

// A lane group's change of output row on the vector path (VW values a lane, VW
// >= 4): the row that ends (cur, partial sums acc) goes to the group's head slot
// if it is the run's first row, else straight to M_n after the empty rows before
// it (and, for the mode's last row, the empty rows after it).  Returns the run's
// previous row and head flag.  Kept out of line: the batch code, unrolled over its
// nonzeros, carries one call per nonzero instead of a copy of this.
template <int VW>
struct RowAcc {
  float v[VW];
};
template <int VW>
__device__ __noinline__ int2 close_row(RowAcc<VW> acc, int cur, int prev_in_run, int head,
                                       float* __restrict__ out, int R, int sub, float sc,
                                       int last_row, int64_t out_rows, int no_fill, int slot,
                                       int* __restrict__ srow, int* __restrict__ sprev,
                                       float* __restrict__ sacc) {
  const bool live = sub * VW < R;
  if (head) {
    if (cur >= 0) {
      if (sub == 0) {
        srow[slot] = cur;
        sprev[slot] = -2;
      }
#pragma unroll
      for (int j = 0; j < VW; ++j)
        if (sub * VW + j < R) sacc[(size_t)slot * R + sub * VW + j] = acc.v[j];
      head = 0;
    }
  } else {
    if (!no_fill && live)
      for (int64_t z = (int64_t)prev_in_run + 1; z < cur; ++z) {
        float4* d = reinterpret_cast<float4*>(out + z * R + sub * VW);
#pragma unroll
        for (int q = 0; q < VW / 4; ++q) d[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    if (live) {
      float4* d = reinterpret_cast<float4*>(out + (int64_t)cur * R + sub * VW);
#pragma unroll
      for (int q = 0; q < VW / 4; ++q)
        d[q] = make_float4(acc.v[4 * q] * sc, acc.v[4 * q + 1] * sc, acc.v[4 * q + 2] * sc,
                           acc.v[4 * q + 3] * sc);
    }
    if (cur == last_row && !no_fill && live)
      for (int64_t z = (int64_t)cur + 1; z < out_rows; ++z) {
        float4* d = reinterpret_cast<float4*>(out + z * R + sub * VW);
#pragma unroll
        for (int q = 0; q < VW / 4; ++q) d[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
  }
  if (cur >= 0) prev_in_run = cur;
  return make_int2(prev_in_run, head);
}

template <int NT, typename T, int VW, int RC, int U, int MODE, int ESB = 0, bool LOSS = false,
          bool RWARP = false>
__global__ void __launch_bounds__(kThreads, ((U <= 4 && VW > 1 && NT <= 3 && !LOSS) ? 3 : 2))
    mttkrp_warp_kernel(const MttkrpArgs a, const int L) {
  static_assert(!LOSS || (NT == 3 && MODE >= 0 && VW > 1 && (ESB == 32 || ESB == 16)),
                "the fused CP-loss pass is built for 3 modes and 16- or 32-byte nonzeros");
  static_assert(!RWARP || (NT == 3 && MODE >= 0 && VW > 1 && ESB == 32 && !LOSS),
                "the remap warp is built for 3 modes and 32-byte nonzeros");
  constexpr int CW = RWARP ? kWarps - 1 : kWarps;  // warps that compute
  constexpr int NV = VW * RC;
  const int N = NT > 0 ? NT : a.nmodes;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = 32 / L, sub = lane % L, gw = lane / L;
  // element stride: a compile-time constant when the number of modes is
  // (packed nonzeros of 4 or more modes are 16 bytes: the plan's stride)
  constexpr int ES_C = ESB > 0 ? ESB : (NT > 0 ? (((4 * NT + 4) + 15) & ~15) : 0);
  const int es = (NT > 0 && !a.pk.packed) ? ES_C : a.es;
  const int R = a.R, mode = MODE >= 0 ? MODE : a.mode;
  const int TW = a.tile, K = TW / G, NPK = np_stage_ints(K);
  if constexpr (RWARP) {
    if (warp == kWarps - 1) {
      extern __shared__ __align__(128) uint8_t smem_r[];
      const WarpLayout lr = warp_layout(es, TW, R, G, a.stages);
      if (a.elems_out)
        remap_warp_tiles(a, MODE, CW, smem_r + (size_t)CW * lr.total,
                         a.wait_ns ? a.wait_ns : kWaitLimitNs);
      return;
    }
  }
  const int wb = blockIdx.x * CW + warp;
  if (wb >= a.nblk) return;
  const int4 bi = a.blkinfo[wb];
  const int lo = bi.x, hi = bi.y;
  if (lo >= hi) {
    if (LOSS && lane == 0) a.loss_part[wb] = 0.0;
    return;
  }

  extern __shared__ __align__(128) uint8_t smem[];
  const int S = a.stages;
  const WarpLayout lay = warp_layout(es, TW, R, G, S);
  uint8_t* wbase = smem + (size_t)warp * lay.total;
  uint8_t* ebuf = wbase + lay.ebuf;
  int32_t* npbuf = reinterpret_cast<int32_t*>(wbase + lay.npbuf);
  float* sacc = reinterpret_cast<float*>(wbase + lay.sacc);
  float* cacc = reinterpret_cast<float*>(wbase + lay.cacc);  // carry row partial (lanes over R)
  int* srow = reinterpret_cast<int*>(wbase + lay.srow);
  int* sprev = reinterpret_cast<int*>(wbase + lay.sprev);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(wbase + lay.mbar);

  // this group's run [ga, gb) of the block
  const int64_t len = hi - lo;
  const int ga = lo + (int)(len * gw / G), gb = lo + (int)(len * (gw + 1) / G);
  const int maxrun = (int)((len + G - 1) / G);
  const int ntiles = (maxrun + K - 1) / K;
  const bool remap = a.elems_out != nullptr && !RWARP;  // RWARP: the remap warp's work
  const bool leader = (sub == 0);
  const float sc = a.scale ? __ldg(a.scale) : 1.0f;
  const int64_t out_rows = a.out_rows;
  float* __restrict__ out = a.out;
  // L2 policies: the element stream, remap ids and remapped copy are touched
  // once per mode (evict first); factor rows are reused (evict last)
  const uint64_t pol_stream = make_policy((a.hints & 1) ? 1 : 0);
  const uint64_t pol_factor = make_policy((a.hints & 2) ? 2 : 0);
  // static 3-mode vector path: this lane's slice (VW values) of the two input
  // factors' rows (lanes past R read slice 0; their values are never stored)
  const uint32_t rowb = (uint32_t)R * (uint32_t)sizeof(T);
  constexpr int LB = VW * (int)sizeof(T);  // bytes of a lane's slice (16, or 8 for BF16 VW 4)
  const uint8_t* lane_base[2];
  {
    const int lsub = (sub * VW < R) ? sub : 0;
    const int k1 = (MODE >= 0 ? MODE : 0) + 1, k2 = (MODE >= 0 ? MODE : 0) + 2;
    lane_base[0] = static_cast<const uint8_t*>(a.factors[k1 % 3 < N ? k1 % 3 : 0]) + lsub * LB;
    lane_base[1] = static_cast<const uint8_t*>(a.factors[k2 % 3 < N ? k2 % 3 : 0]) + lsub * LB;
  }
  // fused CP loss: this lane's slice of the output mode's own factor, and the
  // lane's running sum of squared residuals (FP32 per batch, FP64 across)
  const uint8_t* own_base = nullptr;
  const bool lane_live = sub * VW < R;
  double lsum = 0.0;
  if constexpr (LOSS)
    own_base = static_cast<const uint8_t*>(a.factors[MODE]) + (lane_live ? sub : 0) * LB;

  // the group's leader stages the group's segment of tile t (one mbarrier
  // arrival per group and tile, with the segment's byte count)
  auto issue = [&](int t) {
    const int st = t % S;
    const int seg = ga + t * K;
    const int n = max(0, min(K, gb - seg));
    uint32_t ebytes = (uint32_t)n * es, npbytes = 0;
    int np0 = 0;
    if (remap && !a.alpha_word && n > 0) {  // remap ids from the next_pos array
      np0 = seg & ~3;
      npbytes = ((uint32_t)(seg + n - np0) * 4u + 15u) & ~15u;
    }
    fence_proxy_async_smem();
    mbar_expect_tx(&mbar[st], ebytes + npbytes);
    if (n > 0) {
      bulk_g2s_hint(ebuf + ((size_t)st * TW + (size_t)gw * K) * es, a.elems_in + (size_t)seg * es,
                    ebytes, &mbar[st], pol_stream);
      if (npbytes)
        bulk_g2s_hint(npbuf + (st * G + gw) * NPK, a.next_pos + np0, npbytes, &mbar[st],
                      pol_stream);
    }
  };

  if (lane == 0) {
    for (int b = 0; b <= S; ++b) mbar_init(&mbar[b], G);  // mbar[S]: never completed
    fence_mbar_init();
  }
  __syncwarp();
  if (leader)
    for (int q = 0; q < S - 1 && q < ntiles; ++q) issue(q);
  const unsigned long long wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;

  auto rank_of = [&](int j) -> int {
    if constexpr (VW > 1) return sub * VW + j;
    return sub + L * j;
  };
  auto zero_rows_group = [&](int64_t from, int64_t to) {
    if (a.no_fill) return;  // Algorithm 1 blocks: empty rows are zeroed from a list
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
  auto store_slot = [&](int s, int row, int prev, const float* acc) {
    if (sub == 0) {
      srow[s] = row;
      sprev[s] = prev;
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      const int r = rank_of(j);
      if (r < R) sacc[(size_t)s * R + r] = acc[j];
    }
  };

  // run state of this group, carried from tile to tile
  float acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.f;
  int cur = -1;
  bool head = true;
  int prev_in_run = -1;
  const uint8_t* eb = nullptr;  // this group's segment of the current tile

  constexpr int NI = (NT > 0 ? NT : 2) - 1;
  auto batch = [&](int e, int nb) {
    // 1) element fields from shared memory, 2) every gather of the batch
    // issued into packed registers, 3) products consumed in order
    int rows[U];
    float vals[U];
    int ixs[U][NI];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (u < nb) {
        const uint8_t* ep = eb + (size_t)(e + u) * es;
        if constexpr (NT == 3 && MODE >= 0) {
          const int4 v = *reinterpret_cast<const int4*>(ep);
          const int f[3] = {v.x, v.y, v.z};
          rows[u] = f[MODE];
          ixs[u][0] = f[(MODE + 1) % 3];
          ixs[u][1] = f[(MODE + 2) % 3];
          vals[u] = __int_as_float(v.w);
        } else if (a.pk.packed) {  // 4-6 modes in 16 bytes (bit fields)
          const uint4 w4 = *reinterpret_cast<const uint4*>(ep);
          const uint32_t w[3] = {w4.x, w4.y, w4.z};
          rows[u] = (int)pk_field(w, a.pk.off[mode], a.pk.bits[mode]);
          vals[u] = __uint_as_float(w4.w);
          int k = mode;
#pragma unroll
          for (int j = 0; j < NI; ++j) {
            if (j < N - 1) {
              k = (k + 1 == N) ? 0 : k + 1;
              ixs[u][j] = (int)pk_field(w, a.pk.off[k], a.pk.bits[k]);
            }
          }
        } else {
          const int* el = reinterpret_cast<const int*>(ep);
          rows[u] = el[mode];
          vals[u] = __int_as_float(el[N]);
          int k = mode;
#pragma unroll
          for (int j = 0; j < NI; ++j) {
            if (j < N - 1) {
              k = (k + 1 == N) ? 0 : k + 1;
              ixs[u][j] = el[k];
            }
          }
        }
      }
    }
    typename Landing<T, VW, RC>::type raw[U][NI];
    typename Landing<T, VW, RC>::type rown[LOSS ? U : 1];  // A_n[i_n] slices (fused loss)
    float hh[LOSS ? U : 1][NV];  // fused loss: the product of the two gathered slices
    if constexpr (LOSS) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (u < nb)
          rown[u] = load_lane<typename Landing<T, VW, RC>::type>(
              own_base + (uint64_t)(uint32_t)rows[u] * rowb, pol_factor, false, false);
    }
    if constexpr (NT == 3 && MODE >= 0 && VW > 1) {
      // static modes: one 32 x 32 -> 64-bit multiply per row address
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (u < nb) {
            using LT = typename Landing<T, VW, RC>::type;
            raw[u][j] = load_lane<LT>(lane_base[j] + (uint64_t)(uint32_t)ixs[u][j] * rowb,
                                      pol_factor, false, false);
          }
    } else {
#pragma unroll
      for (int j = 0; j < NI; ++j) {
        if (j < N - 1) {
          const int kj = (NT == 3 && MODE >= 0) ? (MODE + 1 + j) % 3 : (mode + 1 + j) % N;
          const void* Ak = a.factors[kj];
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (u < nb) Landing<T, VW, RC>::load(Ak, ixs[u][j], R, sub, L, pol_factor, raw[u][j]);
        }
      }
    }
    if constexpr (LOSS) {
      // the residual of each nonzero: m_e = sum over the lanes of the group of
      // sum_q A_k1 A_k2 A_n, then e = m_e - x_e replaces the value
      float m[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        m[u] = 0.f;
        if (u < nb) {
          float p[NV], x[NV], y[NV];
          Landing<T, VW, RC>::unpack(raw[u][0], p);
          Landing<T, VW, RC>::unpack(raw[u][1], x);
          Landing<T, VW, RC>::unpack(rown[u], y);
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            hh[u][q] = p[q] * x[q];  // kept: the gradient's product below
            m[u] = fmaf(hh[u][q], y[q], m[u]);
          }
          if (!lane_live) m[u] = 0.f;
        }
      }
      // the group's lanes run together (their segment lengths agree), other
      // groups may be on another batch size: shuffle within the group only
      const unsigned gmask = L >= 32 ? 0xffffffffu : (((1u << L) - 1u) << (gw * L));
      if constexpr (U == 4) {
        if (L >= 4) {
          group_sum4(m, sub, L, gmask);
        } else {
#pragma unroll
          for (int u = 0; u < U; ++u)
            for (int off = L / 2; off > 0; off >>= 1) m[u] += __shfl_xor_sync(gmask, m[u], off);
        }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
          for (int off = L / 2; off > 0; off >>= 1) m[u] += __shfl_xor_sync(gmask, m[u], off);
      }
      float sq = 0.f;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u < nb) {
          const float r = m[u] - vals[u];
          vals[u] = r;
          sq = fmaf(r, r, sq);
          if (sub == 0)  // the residual copy: the staged nonzero's value becomes e
            reinterpret_cast<float*>(const_cast<uint8_t*>(eb) + (size_t)(e + u) * es)[3] = r;
        }
      }
      if (sub == 0) lsum += (double)sq;
    }
    // rows are sorted within a run: if the batch's last nonzero is still in the
    // current row, every nonzero of the batch is, and no per-nonzero check is needed
    bool same_row = true;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (u == nb - 1) same_row = (rows[u] == cur);
    if (same_row) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u < nb) {
          float prod[NV], x[NV];
          if constexpr (LOSS) {
#pragma unroll
            for (int q = 0; q < NV; ++q) prod[q] = hh[u][q];
          } else {
            Landing<T, VW, RC>::unpack(raw[u][0], prod);
          }
          if constexpr (NV % 2 == 0) {  // paired FP32: half the instructions
            float2* p2 = reinterpret_cast<float2*>(prod);
            if constexpr (!LOSS) {
#pragma unroll
              for (int j = 1; j < NI; ++j) {
                if (j < N - 1) {
                  Landing<T, VW, RC>::unpack(raw[u][j], x);
                  const float2* x2 = reinterpret_cast<const float2*>(x);
#pragma unroll
                  for (int q = 0; q < NV / 2; ++q) p2[q] = mul2(p2[q], x2[q]);
                }
              }
            }
            float2* a2 = reinterpret_cast<float2*>(acc);
            const float2 vv = make_float2(vals[u], vals[u]);
#pragma unroll
            for (int q = 0; q < NV / 2; ++q) a2[q] = fma2(p2[q], vv, a2[q]);
          } else {
            if constexpr (!LOSS) {
#pragma unroll
              for (int j = 1; j < NI; ++j) {
                if (j < N - 1) {
                  Landing<T, VW, RC>::unpack(raw[u][j], x);
#pragma unroll
                  for (int q = 0; q < NV; ++q) prod[q] *= x[q];
                }
              }
            }
#pragma unroll
            for (int q = 0; q < NV; ++q) acc[q] = fmaf(prod[q], vals[u], acc[q]);
          }
        }
      }
      return;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (u < nb) {
        float prod[NV], x[NV];
        if constexpr (LOSS) {
#pragma unroll
          for (int q = 0; q < NV; ++q) prod[q] = hh[u][q];
        } else {
          Landing<T, VW, RC>::unpack(raw[u][0], prod);
#pragma unroll
          for (int j = 1; j < NI; ++j) {
            if (j < N - 1) {
              Landing<T, VW, RC>::unpack(raw[u][j], x);
#pragma unroll
              for (int q = 0; q < NV; ++q) prod[q] *= x[q];
            }
          }
        }
        if (rows[u] != cur) {
          if constexpr (VW > 1 && RC == 1 && NT >= 3 && NT <= 5) {  // (6 modes: more spills)
            RowAcc<NV> ra;
#pragma unroll
            for (int q = 0; q < NV; ++q) ra.v[q] = acc[q];
            const int2 st2 = close_row<NV>(ra, cur, prev_in_run, head ? 1 : 0, out, R, sub, sc,
                                           a.last_row, out_rows, a.no_fill, 2 * gw, srow, sprev,
                                           sacc);
            prev_in_run = st2.x;
            head = st2.y != 0;
          } else {
            if (head) {
              if (cur >= 0) {
                store_slot(2 * gw, cur, -2, acc);
                head = false;
              }
            } else {
              write_row_group(cur, acc, prev_in_run);
            }
            if (cur >= 0) prev_in_run = cur;
          }
          cur = rows[u];
#pragma unroll
          for (int q = 0; q < NV; ++q) acc[q] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] = fmaf(prod[q], vals[u], acc[q]);
      }
    }
  };
  // runtime number of modes: multiply each gathered slice in as it lands
  auto batch_generic = [&](int e, int nb) {
    float prod[U][NV];
    float vals[U];
    int rows[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (u < nb) {
        const uint8_t* ep = eb + (size_t)(e + u) * es;
        rows[u] = elem_index(ep, mode, a.pk);
        vals[u] = elem_value(ep, N, a.pk);
#pragma unroll
        for (int q = 0; q < NV; ++q) prod[u][q] = vals[u];
      }
    }
    for (int k = 0; k < N; ++k) {
      if (k == mode) continue;
      const void* Ak = a.factors[k];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u < nb) {
          typename Landing<T, VW, RC>::type raw;
          float x[NV];
          Landing<T, VW, RC>::load(Ak, elem_index(eb + (size_t)(e + u) * es, k, a.pk), R, sub, L,
                                   pol_factor, raw);
          Landing<T, VW, RC>::unpack(raw, x);
#pragma unroll
          for (int q = 0; q < NV; ++q) prod[u][q] *= x[q];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (u < nb) {
        if (rows[u] != cur) {
          if (head) {
            if (cur >= 0) {
              store_slot(2 * gw, cur, -2, acc);
              head = false;
            }
          } else {
            write_row_group(cur, acc, prev_in_run);
          }
          if (cur >= 0) prev_in_run = cur;
          cur = rows[u];
#pragma unroll
          for (int q = 0; q < NV; ++q) acc[q] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += prod[u][q];
      }
    }
  };

  int issued = min(ntiles, S - 1);
  for (int t = 0; t < ntiles; ++t) {
    const int st = t % S;
    // the stall test waits first on mbar[S], which no copy and no thread completes
    const bool stall = a.stall_test && t == 0;
    const bool ok = mbar_wait_bounded(stall ? &mbar[S] : &mbar[st],
                                      stall ? 0u : (uint32_t)((t / S) & 1), wait_ns);
    if (!__all_sync(0xffffffffu, ok)) {
      // a bulk copy did not complete in time: record it, wait (bounded) for
      // the copies still in flight, and leave without writing anything else
      if (lane == 0) {
        atomicOr(a.err, 1);
        for (int q = t; q < issued; ++q)
          (void)mbar_wait_bounded(&mbar[q % S], (uint32_t)((q / S) & 1));
      }
      return;
    }
    // the stage of tile t+S-1 held tile t-1, whose readers passed the last __syncwarp
    if (leader && t + S - 1 < ntiles) issue(t + S - 1);
    issued = min(ntiles, t + S);
    const int seg = ga + t * K;
    const int n = max(0, min(K, gb - seg));
    eb = ebuf + ((size_t)st * TW + (size_t)gw * K) * es;

    auto do_remap = [&]() {  // Algorithm 3: every element to its place in the next mode's order
      const int32_t* np = npbuf + (st * G + gw) * NPK + (seg & 3);
      if (es % 32 == 0) {  // whole 32-byte sectors per store (no read of the old sector)
        const int nv = es >= 32 ? es / 32 : 1;
        const int aw = a.alpha_word;  // remap id carried in the staged nonzero (Section 3.5)
        for (int i = sub; i < n * nv; i += L) {
          const int e = (nv == 1) ? i : i / nv, c = (nv == 1) ? 0 : i - e * nv;
          const uint4* src = reinterpret_cast<const uint4*>(eb + (size_t)e * es) + 2 * c;
          const uint4 lo = src[0], hi = src[1];
          // with the ids in the nonzero (32-byte stride, one sector: c == 0) the id is
          // word aw of the sector, i.e. component aw - 4 of its upper half
          // (bit 31 of the id words is a hot-row flag, not part of the id)
          const int dst = aw ? (int)((aw == 4 ? hi.x : (aw == 5 ? hi.y : hi.z)) & 0x7fffffffu)
                             : np[e];
          st_hint_v8(a.elems_out + (size_t)dst * es + 32 * c, lo, hi, pol_stream);
        }
      } else {
        const int nv = es / 16;  // 16-byte vectors per element (constant when NT > 0)
        for (int i = sub; i < n * nv; i += L) {
          const int e = (nv == 1) ? i : i / nv, c = (nv == 1) ? 0 : i - e * nv;
          const uint4 v = reinterpret_cast<const uint4*>(eb + (size_t)e * es)[c];
          st_hint_v4(reinterpret_cast<uint4*>(a.elems_out + (size_t)np[e] * es) + c, v,
                     pol_stream);
        }
      }
    };
    if (remap && !LOSS) do_remap();

    // Algorithm 2 over this group's segment [0, n) of the tile
    int e = 0;
    if constexpr (NT > 0) {
      for (; e + U <= n; e += U) batch(e, U);
      for (; e < n; ++e) batch(e, 1);
    } else {
      for (; e + U <= n; e += U) batch_generic(e, U);
      for (; e < n; ++e) batch_generic(e, 1);
    }
    if constexpr (LOSS) {  // the residual nonzeros, now in shared memory, to the next order
      __syncwarp();
      if (remap) do_remap();
    }
    __syncwarp();
  }

  // the run's first row (head) and last row (tail) as partial sums
  if (cur < 0) {  // empty run
    if (sub == 0) {
      srow[2 * gw] = -1;
      srow[2 * gw + 1] = -1;
    }
  } else if (head) {
    store_slot(2 * gw, cur, -2, acc);
    if (sub == 0) srow[2 * gw + 1] = -1;
  } else {
    store_slot(2 * gw + 1, cur, prev_in_run, acc);
  }
  __syncwarp();

  // warp combine: run-boundary rows in run order, then the block's last row
  int crow = -1, cprev = bi.z, emitted = 0;
  auto emit = [&](int row, int prev, bool first, bool last) {
    const bool split = (first && (bi.w & BLK_HEAD_SPLIT)) || (last && (bi.w & BLK_TAIL_SPLIT));
    if (split) {
      float* d = a.part + ((size_t)wb * 2 + (first ? 0 : 1)) * R;
      for (int r = lane; r < R; r += 32) d[r] = cacc[r];
      return;
    }
    for (int64_t z = a.no_fill ? (int64_t)row : (int64_t)prev + 1; z < row; ++z)
      for (int r = lane; r < R; r += 32) out[z * R + r] = 0.f;
    for (int r = lane; r < R; r += 32) out[(int64_t)row * R + r] = cacc[r] * sc;
    if (!a.no_fill && row == a.last_row)
      for (int64_t z = (int64_t)row + 1; z < out_rows; ++z)
        for (int r = lane; r < R; r += 32) out[z * R + r] = 0.f;
  };
  for (int s = 0; s < 2 * G; ++s) {
    const int row = srow[s];
    if (row < 0) continue;
    const float* sa = sacc + (size_t)s * R;
    if (row == crow) {
      for (int r = lane; r < R; r += 32) cacc[r] += sa[r];
    } else {
      if (crow >= 0) {
        emit(crow, cprev, emitted == 0, false);
        emitted = 1;
      }
      const int pv = sprev[s];
      cprev = (pv != -2) ? pv : (crow >= 0 ? crow : cprev);
      crow = row;
      for (int r = lane; r < R; r += 32) cacc[r] = sa[r];
    }
    __syncwarp();
  }
  if (crow >= 0) emit(crow, cprev, emitted == 0, true);
  if constexpr (LOSS) {  // fixed-order warp sum of the lanes' partials
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
    if (lane == 0) a.loss_part[wb] = lsum;
  }
}

// Nonzeros per warp tile for a requested size: G runs of an odd length K, so
// that the groups' elements fall on distinct shared-memory banks.
__host__ __device__ inline int warp_tile_for(int tile, int G) {
  int K = tile / G;
  if (K < 1) K = 1;
  if (!(K & 1)) K += 1;
  return G * K;
}

template <int NT, typename T, int VW, int RC, int U, int MODE = -1, int ESB = 0, bool LOSS = false,
          bool RWARP = false>
int launch_warp_kernel(const MttkrpArgs& a0, int L, cudaStream_t s) {
  const int G = 32 / L;
  MttkrpArgs a = a0;
  a.tile = warp_tile_for(a0.tile, G);
  // form 3: seven compute warps' slots, then the remap warp's region
  const size_t smem = RWARP ? (size_t)(kWarps - 1) * warp_layout(a.es, a.tile, a.R, G, a.stages).total +
                                  kRemapRegion
                            : (size_t)kWarps * warp_layout(a.es, a.tile, a.R, G, a.stages).total;
  auto kfn = mttkrp_warp_kernel<NT, T, VW, RC, U, MODE, ESB, LOSS, RWARP>;
  int st = ensure_dyn_smem((const void*)kfn, smem, "cudaFuncSetAttribute(mttkrp_warp)");
  if (st) return st;
  constexpr int CW = RWARP ? kWarps - 1 : kWarps;  // blocks per CTA
  const int grid = (a.nblk + CW - 1) / CW;
  kfn<<<grid, kThreads, smem, s>>>(a, L);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mttkrp_warp_kernel launch");
  return SPM_OK;
}

}  // namespace spm
