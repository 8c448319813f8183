// mttkrp_tile.cuh - the fused mode-n spMTTKRP + dynamic remap kernel over
// contiguous CTA tiles (form 2: 3-mode tensors whose 32-byte nonzeros carry
// their remap ids and write orders).
//
// Persistent CTAs (one per SM) take blocks of the mode's order (the contiguous
// split of Section 3.4 with heavy-row splitting) from a device counter, so SMs
// that finish early take more blocks, and walk each block in tiles of kTileNnz
// consecutive positions.  Warp roles:
//   * the control warp stages each tile into a shared-memory ring with one 1D
//     bulk-async copy (cp.async.bulk, completion on the stage's mbarrier), and,
//     once the compute warps are done with a tile, adds the tile's row partials
//     in position order and writes every finished row once;
//   * kTileComputeWarps compute warps first copy the tile's nonzeros to their
//     places in the next mode's order (Algorithm 3), then run the elementwise
//     computation (Algorithm 2) on their slice of the tile.
// Remap stores go out in destination order: the plan stores, in each nonzero,
// the tile-local index of the nonzero whose destination is the j-th smallest
// of the tile (for the slot j that nonzero occupies).  Nonzeros with the same
// next-mode index land on consecutive slots (the remap is a stable partition,
// Observation 1), so consecutive lanes store consecutive 32-byte sectors and
// the stores fill whole 128-byte lines wherever such runs exist.
// Gathers: each lane group (8 lanes, lanes over the rank) keeps U nonzeros in
// flight in a ring of registers; the next nonzero's two factor-row slices are
// requested as soon as a slot is consumed, across tile boundaries.  Rows that
// start and end inside a group's slice are written by the group; the first and
// last row of each slice become partial sums that the warp combines, and the
// first and last row of each warp's slice are combined by the control warp,
// all in position order (no atomics; results identical run to run).  A row
// that continues past its block goes to the split-row partials, summed by the
// fix-up kernels in block order.  Every wait is bounded; a wait that runs out
// sets an abort flag that every warp of the CTA polls, and the control warp
// waits for its copies in flight before the CTA exits.
#pragma once

#include "mttkrp_common.cuh"

namespace spm {

// Compute warps per CTA and nonzeros per lane group and tile (compile-time
// configuration).  15 compute warps and the control warp make 4 warps per SM
// sub-partition, so each thread may hold 128 registers (a 17th warp would cut
// that to 96).
#ifndef SPM_TILE_COMPUTE_WARPS
#define SPM_TILE_COMPUTE_WARPS 15
#endif
#ifndef SPM_TILE_SLICE
#define SPM_TILE_SLICE 16
#endif
#ifndef SPM_TILE_U
#define SPM_TILE_U 8
#endif
constexpr int kTileComputeWarps = SPM_TILE_COMPUTE_WARPS;
constexpr int kTileThreads = (kTileComputeWarps + 1) * 32;
constexpr int kTileGroups = 4;        // lane groups of 8 lanes per warp
constexpr int kTileSlice = SPM_TILE_SLICE;  // nonzeros per group per tile
constexpr int kTileU = SPM_TILE_U;          // nonzeros in flight per group (R <= 32)
constexpr int kTileNnz = kTileComputeWarps * kTileGroups * kTileSlice;  // 960 per tile
static_assert(kTileNnz <= 1024, "write-order fields are 10 bits");
constexpr int kTileStages = 4;        // tiles in the ring
constexpr int kTilePartRing = kTileStages + 1;  // tiles whose warp partials are kept
constexpr int kTileWordW = 7;         // word of a stored nonzero holding its write orders
constexpr int kStageBytes = kTileNnz * 32;
__host__ __device__ __forceinline__ int tile_offset(int li) { return li * 32; }
constexpr uint32_t kAlphaMask = 0x7fffffffu;

struct TileMeta {  // one per stage; written by the control warp before its copy
  int base;        // first position of the tile
  int len;         // nonzeros in the tile
  int l0, l1;      // the block's share of the tile, tile-local [l0, l1)
  int blk;         // block id
  int flags;       // TM_* bits
  int prev;        // row before the block (-1: none)
  int split;       // the block's split flags (BLK_HEAD_SPLIT / BLK_TAIL_SPLIT)
};
// TM_END marks a stage with no tile: the CTA's stream of tiles has ended
enum { TM_REMAP = 1, TM_FIRST = 2, TM_LAST = 4, TM_END = 8 };

struct TileLayout {
  size_t ebuf, meta, wpart, wrow, bars, total;
};

__host__ __device__ inline TileLayout tile_layout(int R) {
  TileLayout l;
  size_t o = 0;
  l.ebuf = o;
  o += (size_t)kTileStages * kStageBytes;
  l.meta = o;
  o += (size_t)kTileStages * sizeof(TileMeta);
  l.wpart = o;  // per ring slot, per compute warp: head and tail partial sums
  o += (size_t)kTilePartRing * kTileComputeWarps * 2 * R * 4;
  l.wrow = o;  // per ring slot, per compute warp, head and tail: {row, prev}
  o += (size_t)kTilePartRing * kTileComputeWarps * 2 * 2 * 4;
  o = (o + 15) & ~(size_t)15;
  l.bars = o;  // full[S], computed[S], stall, abort word (+pad)
  o += (size_t)(2 * kTileStages + 2) * 8;
  l.total = (o + 127) & ~(size_t)127;
  return l;
}

// A lane's slice of a factor row: LW 32-bit words (NV values of type T).
template <int LW>
struct RowSlice {
  uint32_t w[LW];
};

// keep: the row is hot (L1 evict_last); otherwise L1 evict_first
template <int LW>
__device__ __forceinline__ void load_slice(RowSlice<LW>& d, const uint8_t* p, uint64_t pol,
                                           bool keep) {
  if constexpr (LW == 1) {
    if (keep)
      asm volatile("ld.global.nc.L1::evict_last.L2::cache_hint.b32 %0, [%1], %2;"
                   : "=r"(d.w[0]) : "l"(p), "l"(pol));
    else
      asm volatile("ld.global.nc.L1::evict_first.L2::cache_hint.b32 %0, [%1], %2;"
                   : "=r"(d.w[0]) : "l"(p), "l"(pol));
  } else if constexpr (LW == 2) {
    if (keep)
      asm volatile("ld.global.nc.L1::evict_last.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;"
                   : "=r"(d.w[0]), "=r"(d.w[1]) : "l"(p), "l"(pol));
    else
      asm volatile("ld.global.nc.L1::evict_first.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;"
                   : "=r"(d.w[0]), "=r"(d.w[1]) : "l"(p), "l"(pol));
  } else {
#pragma unroll
    for (int q = 0; q < LW / 4; ++q) {
      const uint4 v = ld_nc_l1_v4(p + 16 * q, pol, keep);
      d.w[4 * q] = v.x;
      d.w[4 * q + 1] = v.y;
      d.w[4 * q + 2] = v.z;
      d.w[4 * q + 3] = v.w;
    }
  }
}

template <typename T, int NV, int LW>
__device__ __forceinline__ void unpack_slice(const RowSlice<LW>& s, float* x) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < NV; ++i) x[i] = __uint_as_float(s.w[i]);
  } else {
#pragma unroll
    for (int i = 0; i < NV / 2; ++i) {
      x[2 * i] = __uint_as_float(s.w[i] << 16);
      x[2 * i + 1] = __uint_as_float(s.w[i] & 0xffff0000u);
    }
  }
}

// Bounded wait that also gives up once another warp of the CTA has aborted.
// On running out it records the timeout and raises the CTA's abort flag.
__device__ __forceinline__ bool tile_wait(uint64_t* bar, uint32_t parity,
                                          unsigned long long limit_ns, volatile int* abort_flag,
                                          int* err) {
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
    if (*abort_flag) return false;
    if (global_ns() - t0 > limit_ns) {
      *abort_flag = 1;
      if (err) atomicOr(err, 1);
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// T: factor type; NV: rank values per lane (R = 8 NV); MODE: output mode; U:
// nonzeros in flight per lane group.
template <typename T, int NV, int MODE, int U>
__global__ void __launch_bounds__(kTileThreads, 1) mttkrp_tile_kernel(const MttkrpArgs a) {
  constexpr int R = 8 * NV;
  constexpr int LB = NV * (int)sizeof(T);  // bytes of a lane's row slice
  constexpr int LW = LB / 4;
  constexpr int RND = kTileSlice / U;      // rounds of U nonzeros per slice
  static_assert(kTileSlice % U == 0, "slice must be a multiple of U");
  constexpr int K1 = (MODE + 1) % 3, K2 = (MODE + 2) % 3;  // gathered factors
  constexpr int S = kTileStages;
  constexpr int PR = kTilePartRing;

  extern __shared__ __align__(128) uint8_t smem[];
  const TileLayout lay = tile_layout(R);
  uint8_t* ebuf = smem + lay.ebuf;
  TileMeta* meta = reinterpret_cast<TileMeta*>(smem + lay.meta);
  float* wpart = reinterpret_cast<float*>(smem + lay.wpart);
  int* wrow = reinterpret_cast<int*>(smem + lay.wrow);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);
  uint64_t* computed = full + S;
  uint64_t* stallbar = full + 2 * S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(full + 2 * S + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;
  const float sc = a.scale ? __ldg(a.scale) : 1.0f;
  const int64_t out_rows = a.out_rows;
  float* __restrict__ out = a.out;
  const uint64_t pol_stream = make_policy((a.hints & 1) ? 1 : 0);
  const uint64_t pol_factor = make_policy((a.hints & 2) ? 2 : 0);

  if (threadIdx.x == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&computed[q], kTileComputeWarps);
    }
    mbar_init(stallbar, 1);  // nothing ever arrives here
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  // ------------------------------------------------------------ control warp
  if (warp == kTileComputeWarps) {
    // lane 0's position in the stream: block blk, its tiles t..tlast
    int blk = -1, t = 0, tlast = -1;
    int4 bi = make_int4(0, 0, -1, 0);
    auto next_tile = [&]() -> bool {  // lane 0
      if (blk >= 0 && t < tlast) {
        ++t;
        return true;
      }
      while (true) {
        blk = atomicAdd(a.sched, 1);
        if (blk >= a.nblk) return false;
        bi = a.blkinfo[blk];
        if (bi.x < bi.y) break;
      }
      t = bi.x / kTileNnz;
      tlast = (bi.y - 1) / kTileNnz;
      return true;
    };
    // lane 0: fills stage j % S with the next tile, or with the end mark
    auto issue = [&](int j) -> bool {
      const int st = j % S;
      TileMeta m;
      if (!next_tile()) {
        m.flags = TM_END;
        meta[st] = m;
        mbar_arrive(&full[st]);  // completes the phase without a copy
        return false;
      }
      m.base = t * kTileNnz;
      m.len = (int)min((int64_t)kTileNnz, a.nnz - (int64_t)m.base);
      m.l0 = max(bi.x, m.base) - m.base;
      m.l1 = min(bi.y, m.base + kTileNnz) - m.base;
      m.blk = blk;
      m.flags = ((a.elems_out != nullptr && bi.x <= m.base) ? TM_REMAP : 0) |
                (t == bi.x / kTileNnz ? TM_FIRST : 0) | (t == tlast ? TM_LAST : 0);
      m.prev = bi.z;
      m.split = bi.w;
      meta[st] = m;
      fence_proxy_async_smem();
      mbar_expect_tx(&full[st], (uint32_t)m.len * 32u);
      bulk_g2s_hint(ebuf + (size_t)st * kStageBytes, a.elems_in + (size_t)m.base * 32,
                    (uint32_t)m.len * 32u, &full[st], pol_stream);
      return true;
    };
    // stages 0..S-1; `end` = the stream index holding the end mark (INT_MAX: not yet)
    int end = 0x7fffffff, issued = 0;
    for (; issued < S; ++issued) {
      int ok = 0;
      if (lane == 0) ok = issue(issued) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        end = issued++;
        break;
      }
    }

    // carry of the current block: the open row and its partial sum (lanes over R)
    int crow = -1, cprev = -1, emitted = 0;
    float cacc[2] = {0.f, 0.f};
    auto emit = [&](const TileMeta& m, int row, int prev, bool first, bool last) {
      const bool split = (first && (m.split & BLK_HEAD_SPLIT)) || (last && (m.split & BLK_TAIL_SPLIT));
      if (split) {
        float* d = a.part + ((size_t)m.blk * 2 + (first ? 0 : 1)) * R;
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (lane + 32 * h < R) d[lane + 32 * h] = cacc[h];
        return;
      }
      for (int64_t z = (int64_t)prev + 1; z < row; ++z)
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (lane + 32 * h < R) out[z * R + lane + 32 * h] = 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (lane + 32 * h < R) out[(int64_t)row * R + lane + 32 * h] = cacc[h] * sc;
      if (row == a.last_row)
        for (int64_t z = (int64_t)row + 1; z < out_rows; ++z)
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (lane + 32 * h < R) out[z * R + lane + 32 * h] = 0.f;
    };
    for (int j = 0; j < end; ++j) {
      const int st = j % S;
      if (!tile_wait(&computed[st], (uint32_t)((j / S) & 1), wait_ns, abort_flag, a.err)) {
        // give up: wait (default limit) for the copies still in flight, then leave
        if (lane == 0)
          for (int q = j; q < issued; ++q)
            (void)mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1));
        return;
      }
      const TileMeta m = meta[st];
      __syncwarp();
      // the stage's nonzeros are consumed: stage the next tile first (its warp
      // partials go to another ring slot, so the combine below is unaffected)
      if (end == 0x7fffffff) {
        int ok = 0;
        if (lane == 0) ok = issue(issued) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) end = issued;
        ++issued;
      }
      if (m.flags & TM_FIRST) {
        crow = -1;
        cprev = m.prev;
        emitted = 0;
      }
      const int ps = j % PR;
      const float* wp = wpart + (size_t)ps * kTileComputeWarps * 2 * R;
      const int* wr = wrow + (size_t)ps * kTileComputeWarps * 2 * 2;
      for (int s = 0; s < 2 * kTileComputeWarps; ++s) {
        const int row = wr[2 * s];
        if (row < 0) continue;
        const float* sa = wp + (size_t)s * R;
        if (row == crow) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (lane + 32 * h < R) cacc[h] += sa[lane + 32 * h];
        } else {
          if (crow >= 0) {
            emit(m, crow, cprev, emitted == 0, false);
            emitted = 1;
          }
          const int pv = wr[2 * s + 1];
          cprev = (pv != -2) ? pv : (crow >= 0 ? crow : cprev);
          crow = row;
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (lane + 32 * h < R) cacc[h] = sa[lane + 32 * h];
        }
      }
      if ((m.flags & TM_LAST) && crow >= 0) {
        emit(m, crow, cprev, emitted == 0, true);
        crow = -1;
      }
      __syncwarp();
    }
    return;
  }

  // ------------------------------------------------------------ compute warps
  // Warp cw streams the sub-tile [cw*W, (cw+1)*W) of every tile (W = 4 x slice):
  // its four lane groups take consecutive nonzeros (group g the g-th of every
  // four), so the warp walks the sub-tile in position order, four nonzeros per
  // step.  The open row (cur) is the same in all lanes; each group keeps its
  // own partial of it, and the four partials are added by shuffles when the
  // row ends.  The sub-tile's first row (head) and last row (tail) go to the
  // control warp as partial sums; rows between them are written here.
  constexpr int W = kTileGroups * kTileSlice;  // nonzeros per warp and tile
  const int cw = warp, g = lane >> 3, sub = lane & 7;
  const uint8_t* fb1 = static_cast<const uint8_t*>(a.factors[K1]) + sub * LB;
  const uint8_t* fb2 = static_cast<const uint8_t*>(a.factors[K2]) + sub * LB;
  constexpr uint32_t rowb = (uint32_t)R * sizeof(T);
  const int w0 = cw * W + g;  // tile-local index of this group's first nonzero

  RowSlice<LW> raw[U][2];
  int srow[U];
  float sval[U];

  // slot u <- the nonzero at tile-local index li of stage buffer eb
  auto issue_slot = [&](int u, const uint8_t* eb, int li, bool valid) {
    if (valid) {
      const int4 e = *reinterpret_cast<const int4*>(eb + tile_offset(li));
      const int4 h = *reinterpret_cast<const int4*>(eb + tile_offset(li) + 16);
      const int f[3] = {e.x, e.y, e.z};
      const int hf[3] = {h.x, h.y, h.z};  // bit 31: hot-row flag of each index
      srow[u] = f[MODE];
      sval[u] = __int_as_float(e.w);
      load_slice<LW>(raw[u][0], fb1 + (uint64_t)(uint32_t)f[K1] * rowb, pol_factor,
                     a.hot_flags && hf[K1] < 0);
      load_slice<LW>(raw[u][1], fb2 + (uint64_t)(uint32_t)f[K2] * rowb, pol_factor,
                     a.hot_flags && hf[K2] < 0);
    } else {
      srow[u] = -1;
    }
  };

  // run state of the warp's sub-tile (cur, head and prev are the same in all lanes)
  float acc[NV];
  int cur = -1, prev = -1;
  bool head = true;
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.f;

  auto zero_rows = [&](int64_t from, int64_t to) {  // lanes of group 0
    for (int64_t z = from; z < to; ++z) {
      float* d = out + z * R + sub * NV;
#pragma unroll
      for (int q = 0; q < NV; q += 2) *reinterpret_cast<float2*>(d + q) = make_float2(0.f, 0.f);
    }
  };
  auto accumulate = [&](int u) {
    float p[NV], x[NV];
    unpack_slice<T, NV, LW>(raw[u][0], p);
    unpack_slice<T, NV, LW>(raw[u][1], x);
    float2* a2 = reinterpret_cast<float2*>(acc);
    const float2* p2 = reinterpret_cast<const float2*>(p);
    const float2* x2 = reinterpret_cast<const float2*>(x);
    const float2 vv = make_float2(sval[u], sval[u]);
#pragma unroll
    for (int q = 0; q < NV / 2; ++q) a2[q] = fma2(mul2(p2[q], x2[q]), vv, a2[q]);
  };
  // the open row's total over the four groups (in group order), then acc = 0
  auto row_total = [&](float* tot) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const float v1 = __shfl_down_sync(0xffffffffu, acc[q], 8);
      const float v2 = __shfl_down_sync(0xffffffffu, acc[q], 16);
      const float v3 = __shfl_down_sync(0xffffffffu, acc[q], 24);
      tot[q] = ((acc[q] + v1) + v2) + v3;  // valid in group 0's lanes
      acc[q] = 0.f;
    }
  };
  // the open row ends: head partial to the control warp, or the row written
  auto close_row = [&](int ps) {
    float tot[NV];
    row_total(tot);
    if (head) {
      if (g == 0) {
        float* wp = wpart + ((size_t)ps * kTileComputeWarps + cw) * 2 * R;
#pragma unroll
        for (int q = 0; q < NV; ++q) wp[sub * NV + q] = tot[q];
      }
      if (lane == 0) {
        int* wr = wrow + ((size_t)ps * kTileComputeWarps + cw) * 2 * 2;
        wr[0] = cur;
        wr[1] = -2;
      }
      head = false;
    } else if (g == 0) {
      zero_rows((int64_t)prev + 1, cur);
      float* d = out + (int64_t)cur * R + sub * NV;
#pragma unroll
      for (int q = 0; q < NV; q += 2)
        *reinterpret_cast<float2*>(d + q) = make_float2(tot[q] * sc, tot[q + 1] * sc);
      if (cur == a.last_row) zero_rows((int64_t)cur + 1, out_rows);
    }
    prev = cur;
  };
  // step u: the four nonzeros held in slot u of the four groups, in order
  auto step = [&](int u, int ps) {
    if (__all_sync(0xffffffffu, srow[u] == cur) && cur >= 0) {
      accumulate(u);
      return;
    }
#pragma unroll
    for (int q = 0; q < kTileGroups; ++q) {
      const int rq = __shfl_sync(0xffffffffu, srow[u], q * 8);
      if (rq < 0) continue;
      if (rq != cur) {
        if (cur >= 0) close_row(ps);
        cur = rq;
      }
      if (g == q) accumulate(u);
    }
  };

  // the first tile: wait for it (or, in the stall test, for a barrier nothing completes)
  {
    const bool ok = a.stall_test
                        ? tile_wait(stallbar, 0u, wait_ns, abort_flag, a.err)
                        : tile_wait(&full[0], 0u, wait_ns, abort_flag, a.err);
    if (!ok) return;
    const TileMeta m = meta[0];
    if (m.flags & TM_END) return;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int li = w0 + 4 * u;
      issue_slot(u, ebuf, li, li >= m.l0 && li < m.l1);
    }
  }

  for (int j = 0;; ++j) {
    const int st = j % S;
    const int ps = j % PR;
    const uint8_t* eb = ebuf + (size_t)st * kStageBytes;
    const TileMeta m = meta[st];

    // Algorithm 3: this warp's share of the tile's remap, in destination order
    if (m.flags & TM_REMAP) {
#pragma unroll
      for (int q = 0; q < (kTileNnz + kTileComputeWarps * 32 - 1) / (kTileComputeWarps * 32); ++q) {
        const int slot = (q * kTileComputeWarps + cw) * 32 + lane;
        if (slot < m.len) {
          const uint32_t wo = *reinterpret_cast<const uint32_t*>(eb + tile_offset(slot) +
                                                                 4 * kTileWordW);
          const int src = (int)((wo >> (10 * MODE)) & 1023u);
          const uint4* sp = reinterpret_cast<const uint4*>(eb + tile_offset(min(src, kTileNnz - 1)));
          const uint4 lo = sp[0], hi = sp[1];
          const uint32_t dst = (K1 == 0 ? hi.x : (K1 == 1 ? hi.y : hi.z)) & kAlphaMask;
          if (src < m.len && (int64_t)dst < a.nnz)
            st_hint_v8(a.elems_out + (size_t)dst * 32, lo, hi, pol_stream);
          else if (a.err)
            atomicOr(a.err, 2);  // inconsistent write order or remap id: store skipped
        }
      }
    }

    // Algorithm 2 over the sub-tile, U nonzeros in flight per group
    bool next_end = false;
    for (int r = 0; r < RND; ++r) {
      const bool last_round = (r == RND - 1);
      const uint8_t* nb = eb;
      int nl0 = m.l0, nl1 = m.l1, noff = (r + 1) * U;
      if (last_round) {
        const int sn = (j + 1) % S;
        if (!tile_wait(&full[sn], (uint32_t)(((j + 1) / S) & 1), wait_ns, abort_flag, a.err))
          return;
        const TileMeta mn = meta[sn];
        next_end = (mn.flags & TM_END) != 0;
        nb = ebuf + (size_t)sn * kStageBytes;
        nl0 = next_end ? 0 : mn.l0;
        nl1 = next_end ? 0 : mn.l1;
        noff = 0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        step(u, ps);
        const int li = w0 + 4 * (noff + u);
        issue_slot(u, nb, li, li >= nl0 && li < nl1);
      }
    }

    // the sub-tile's last row: the tail partial (or the head, if it is the only row)
    {
      int* wr = wrow + ((size_t)ps * kTileComputeWarps + cw) * 2 * 2;
      float* wp = wpart + ((size_t)ps * kTileComputeWarps + cw) * 2 * R;
      if (cur >= 0) {
        float tot[NV];
        row_total(tot);
        const int h = head ? 0 : 1;
        if (g == 0) {
#pragma unroll
          for (int q = 0; q < NV; ++q) wp[(size_t)h * R + sub * NV + q] = tot[q];
        }
        if (lane == 0) {
          wr[2 * h] = cur;
          wr[2 * h + 1] = head ? -2 : prev;
          if (head) wr[2] = -1;
        }
      } else if (lane == 0) {  // no nonzero of the block in this sub-tile
        wr[0] = -1;
        wr[2] = -1;
      }
      cur = -1;
      prev = -1;
      head = true;
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q] = 0.f;
      __syncwarp();
      if (lane == 0) mbar_arrive(&computed[st]);
    }
    if (next_end) return;
  }
}

template <typename T, int NV, int MODE, int U>
int launch_tile_kernel(const MttkrpArgs& a, cudaStream_t s) {
  const size_t smem = tile_layout(8 * NV).total;
  auto kfn = mttkrp_tile_kernel<T, NV, MODE, U>;
  int st = ensure_dyn_smem((const void*)kfn, smem, "cudaFuncSetAttribute(mttkrp_tile)");
  if (st) return st;
  if (!a.sched) return fail(SPM_ERR_INVALID_ARG, "tile form needs a block counter");
  SPM_CUDA(cudaMemsetAsync(a.sched, 0, sizeof(int), s));  // blocks are taken from 0 up
  const int grid = std::max(1, std::min(a.nblk, a.grid_ctas > 0 ? a.grid_ctas : a.nblk));
  kfn<<<grid, kTileThreads, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mttkrp_tile_kernel launch");
  return SPM_OK;
}

}  // namespace spm
