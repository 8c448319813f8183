// mttkrp_tile.cuh - the fused mode-n spMTTKRP + dynamic remap kernel over
// contiguous CTA tiles (form 2: 3-mode tensors whose 32-byte nonzeros carry
// their remap ids and write orders).
//
// A persistent CTA walks its blocks of the mode's order (the contiguous split of
// Section 3.4 with heavy-row splitting) in tiles of kTileNnz consecutive
// positions.  Warp roles:
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

// 15 compute warps and the control warp: 4 warps per SM sub-partition, so each
// thread may hold 128 registers (a 17th warp would cut that to 96)
constexpr int kTileComputeWarps = 15;
constexpr int kTileThreads = (kTileComputeWarps + 1) * 32;
constexpr int kTileGroups = 4;        // lane groups of 8 lanes per warp
constexpr int kTileSlice = 16;        // nonzeros per group per tile
constexpr int kTileNnz = kTileComputeWarps * kTileGroups * kTileSlice;  // 960 per tile
static_assert(kTileNnz <= 1024, "write-order fields are 10 bits");
constexpr int kTileStages = 3;        // tiles in the ring
constexpr int kTileWordW = 7;         // word of a stored nonzero holding its write orders
constexpr uint32_t kAlphaMask = 0x7fffffffu;

struct TileMeta {  // one per stage; written by the control warp before its copy
  int base;        // first position of the tile
  int len;         // nonzeros in the tile
  int l0, l1;      // the block's share of the tile, tile-local [l0, l1)
  int blk;         // block id
  int flags;       // bit0: remap this tile; bit1: first tile of the block; bit2: last
  int pad0, pad1;
};
enum { TM_REMAP = 1, TM_FIRST = 2, TM_LAST = 4 };

struct TileLayout {
  size_t ebuf, meta, wpart, wrow, gslot, grow, bars, total;
};

__host__ __device__ inline TileLayout tile_layout(int R) {
  TileLayout l;
  size_t o = 0;
  l.ebuf = o;
  o += (size_t)kTileStages * kTileNnz * 32;
  l.meta = o;
  o += (size_t)kTileStages * sizeof(TileMeta);
  l.wpart = o;  // per stage, per compute warp: head and tail partial sums
  o += (size_t)kTileStages * kTileComputeWarps * 2 * R * 4;
  l.wrow = o;  // per stage, per compute warp, head and tail: {row, prev}
  o += (size_t)kTileStages * kTileComputeWarps * 2 * 2 * 4;
  l.gslot = o;  // per compute warp: the 2 slots of each of its 4 groups
  o += (size_t)kTileComputeWarps * 2 * kTileGroups * R * 4;
  l.grow = o;  // per compute warp, per group slot: {row, prev}
  o += (size_t)kTileComputeWarps * 2 * kTileGroups * 2 * 4;
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

template <int LW>
__device__ __forceinline__ void load_slice(RowSlice<LW>& d, const uint8_t* p, uint64_t pol) {
  if constexpr (LW == 1) {
    asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;"
                 : "=r"(d.w[0])
                 : "l"(p), "l"(pol));
  } else if constexpr (LW == 2) {
    asm volatile("ld.global.nc.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;"
                 : "=r"(d.w[0]), "=r"(d.w[1])
                 : "l"(p), "l"(pol));
  } else {
#pragma unroll
    for (int q = 0; q < LW / 4; ++q)
      asm volatile("ld.global.nc.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;"
                   : "=r"(d.w[4 * q]), "=r"(d.w[4 * q + 1]), "=r"(d.w[4 * q + 2]),
                     "=r"(d.w[4 * q + 3])
                   : "l"(p + 16 * q), "l"(pol));
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

  extern __shared__ __align__(128) uint8_t smem[];
  const TileLayout lay = tile_layout(R);
  uint8_t* ebuf = smem + lay.ebuf;
  TileMeta* meta = reinterpret_cast<TileMeta*>(smem + lay.meta);
  float* wpart = reinterpret_cast<float*>(smem + lay.wpart);
  int* wrow = reinterpret_cast<int*>(smem + lay.wrow);
  float* gslot = reinterpret_cast<float*>(smem + lay.gslot);
  int* grow = reinterpret_cast<int*>(smem + lay.grow);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);
  uint64_t* computed = full + S;
  uint64_t* stallbar = full + 2 * S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(full + 2 * S + 1);
  __shared__ int s_total;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;
  const float sc = a.scale ? __ldg(a.scale) : 1.0f;
  const int64_t out_rows = a.out_rows;
  float* __restrict__ out = a.out;
  const uint64_t pol_stream = make_policy((a.hints & 1) ? 1 : 0);
  const uint64_t pol_factor = make_policy((a.hints & 2) ? 2 : 0);

  if (threadIdx.x == 0) {
    int total = 0;
    for (int b = blockIdx.x; b < a.nblk; b += gridDim.x) {
      const int4 bi = a.blkinfo[b];
      if (bi.x < bi.y) total += (bi.y - 1) / kTileNnz - bi.x / kTileNnz + 1;
    }
    s_total = total;
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&computed[q], kTileComputeWarps);
    }
    mbar_init(stallbar, 1);  // nothing ever arrives here
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const int total = s_total;
  if (total == 0) return;

  // ------------------------------------------------------------ control warp
  if (warp == kTileComputeWarps) {
    // stream position of this CTA: block blk (its tiles t..tlast)
    int blk = blockIdx.x, t = 0, tlast = -1;
    int4 bi = make_int4(0, 0, -1, 0);
    auto advance = [&]() {  // to the next (block, tile) of this CTA
      if (t < tlast) {
        ++t;
        return;
      }
      if (tlast >= 0) blk += gridDim.x;
      while (blk < a.nblk) {
        bi = a.blkinfo[blk];
        if (bi.x < bi.y) break;
        blk += gridDim.x;
      }
      t = bi.x / kTileNnz;
      tlast = (bi.y - 1) / kTileNnz;
    };
    auto issue = [&](int j) {  // lane 0: stage tile j of the stream
      const int st = j % S;
      TileMeta m;
      m.base = t * kTileNnz;
      m.len = (int)min((int64_t)kTileNnz, (int64_t)a.nnz - m.base);
      m.l0 = max(bi.x, m.base) - m.base;
      m.l1 = min(bi.y, m.base + kTileNnz) - m.base;
      m.blk = blk;
      m.flags = ((a.elems_out != nullptr && bi.x <= m.base) ? TM_REMAP : 0) |
                (t == bi.x / kTileNnz ? TM_FIRST : 0) | (t == tlast ? TM_LAST : 0);
      m.pad0 = bi.z;  // row before the block
      m.pad1 = bi.w;  // split flags of the block
      meta[st] = m;
      fence_proxy_async_smem();
      mbar_expect_tx(&full[st], (uint32_t)m.len * 32u);
      bulk_g2s_hint(ebuf + (size_t)st * kTileNnz * 32, a.elems_in + (size_t)m.base * 32,
                    (uint32_t)m.len * 32u, &full[st], pol_stream);
    };
    int issued = 0;
    if (lane == 0) {
      for (; issued < S && issued < total; ++issued) {
        advance();
        issue(issued);
      }
    }
    issued = __shfl_sync(0xffffffffu, issued, 0);

    // carry of the current block: the open row and its partial sum (lanes over R)
    int crow = -1, cprev = -1, emitted = 0;
    float cacc[2] = {0.f, 0.f};
    auto emit = [&](const TileMeta& m, int row, int prev, bool first, bool last) {
      const bool split = (first && (m.pad1 & BLK_HEAD_SPLIT)) || (last && (m.pad1 & BLK_TAIL_SPLIT));
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
    for (int j = 0; j < total; ++j) {
      const int st = j % S;
      if (!tile_wait(&computed[st], (uint32_t)((j / S) & 1), wait_ns, abort_flag, a.err)) {
        // give up: wait (default limit) for the copies still in flight, then leave
        if (lane == 0)
          for (int q = j; q < issued; ++q)
            (void)mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1));
        return;
      }
      const TileMeta m = meta[st];
      if (m.flags & TM_FIRST) {
        crow = -1;
        cprev = m.pad0;
        emitted = 0;
      }
      const float* wp = wpart + (size_t)st * kTileComputeWarps * 2 * R;
      const int* wr = wrow + (size_t)st * kTileComputeWarps * 2 * 2;
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
      // the stage is free: stage tile j + S into it
      if (issued < total) {
        if (lane == 0) {
          advance();
          issue(issued);
        }
        ++issued;
      }
    }
    return;
  }

  // ------------------------------------------------------------ compute warps
  const int cw = warp, g = lane >> 3, sub = lane & 7;
  const uint8_t* fb1 = static_cast<const uint8_t*>(a.factors[K1]) + sub * LB;
  const uint8_t* fb2 = static_cast<const uint8_t*>(a.factors[K2]) + sub * LB;
  constexpr uint32_t rowb = (uint32_t)R * sizeof(T);
  const int slice0 = cw * (kTileGroups * kTileSlice) + g * kTileSlice;  // tile-local
  float* gs = gslot + (size_t)cw * 2 * kTileGroups * R;
  int* gr = grow + (size_t)cw * 2 * kTileGroups * 2;

  RowSlice<LW> raw[U][2];
  int srow[U];
  float sval[U];

  // slot u <- the nonzero at tile-local index li of stage buffer eb
  auto issue_slot = [&](int u, const uint8_t* eb, int li, bool valid) {
    if (valid) {
      const int4 e = *reinterpret_cast<const int4*>(eb + (size_t)li * 32);
      const int f[3] = {e.x, e.y, e.z};
      srow[u] = f[MODE];
      sval[u] = __int_as_float(e.w);
      load_slice<LW>(raw[u][0], fb1 + (uint64_t)(uint32_t)f[K1] * rowb, pol_factor);
      load_slice<LW>(raw[u][1], fb2 + (uint64_t)(uint32_t)f[K2] * rowb, pol_factor);
    } else {
      srow[u] = -1;
    }
  };

  // run state of this group's slice of the current tile
  float acc[NV];
  int cur = -1, prev_in_run = -1;
  bool head = true;
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.f;

  auto zero_rows = [&](int64_t from, int64_t to) {
    for (int64_t z = from; z < to; ++z) {
      float* d = out + z * R + sub * NV;
#pragma unroll
      for (int q = 0; q < NV; q += 2) *reinterpret_cast<float2*>(d + q) = make_float2(0.f, 0.f);
    }
  };
  auto write_row = [&](int row, const float* v, int prev) {
    zero_rows((int64_t)prev + 1, row);
    float* d = out + (int64_t)row * R + sub * NV;
#pragma unroll
    for (int q = 0; q < NV; q += 2)
      *reinterpret_cast<float2*>(d + q) = make_float2(v[q] * sc, v[q + 1] * sc);
    if (row == a.last_row) zero_rows((int64_t)row + 1, out_rows);
  };
  auto store_gslot = [&](int s, int row, int prev, const float* v) {
    if (sub == 0) {
      gr[2 * s] = row;
      gr[2 * s + 1] = prev;
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) gs[(size_t)s * R + sub * NV + q] = v[q];
  };
  auto consume = [&](int u) {
    if (srow[u] < 0) return;
    float p[NV], x[NV];
    unpack_slice<T, NV, LW>(raw[u][0], p);
    unpack_slice<T, NV, LW>(raw[u][1], x);
    if (srow[u] != cur) {
      if (cur >= 0) {
        if (head) {
          store_gslot(2 * g, cur, -2, acc);
          head = false;
        } else {
          write_row(cur, acc, prev_in_run);
        }
        prev_in_run = cur;
      }
      cur = srow[u];
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q] = 0.f;
    }
    float2* a2 = reinterpret_cast<float2*>(acc);
    const float2* p2 = reinterpret_cast<const float2*>(p);
    const float2* x2 = reinterpret_cast<const float2*>(x);
    const float2 vv = make_float2(sval[u], sval[u]);
#pragma unroll
    for (int q = 0; q < NV / 2; ++q) a2[q] = fma2(mul2(p2[q], x2[q]), vv, a2[q]);
  };

  // the first tile: wait for it (or, in the stall test, for a barrier nothing completes)
  {
    const bool ok = a.stall_test
                        ? tile_wait(stallbar, 0u, wait_ns, abort_flag, a.err)
                        : tile_wait(&full[0], 0u, wait_ns, abort_flag, a.err);
    if (!ok) return;
    const TileMeta m = meta[0];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int li = slice0 + u;
      issue_slot(u, ebuf, li, li >= m.l0 && li < m.l1);
    }
  }

  for (int j = 0; j < total; ++j) {
    const int st = j % S;
    const uint8_t* eb = ebuf + (size_t)st * kTileNnz * 32;
    const TileMeta m = meta[st];

    // Algorithm 3: this warp's share of the tile's remap, in destination order
    if (m.flags & TM_REMAP) {
#pragma unroll
      for (int q = 0; q < (kTileNnz + kTileComputeWarps * 32 - 1) / (kTileComputeWarps * 32); ++q) {
        const int slot = (q * kTileComputeWarps + cw) * 32 + lane;
        if (slot < m.len) {
          const uint32_t wo = *reinterpret_cast<const uint32_t*>(eb + (size_t)slot * 32 +
                                                                 4 * kTileWordW);
          const int src = (int)((wo >> (10 * MODE)) & 1023u);
          const uint4* sp = reinterpret_cast<const uint4*>(eb + (size_t)min(src, kTileNnz - 1) * 32);
          const uint4 lo = sp[0], hi = sp[1];
          const uint32_t dst = (K1 == 0 ? hi.x : (K1 == 1 ? hi.y : hi.z)) & kAlphaMask;
          if (src < m.len && (int64_t)dst < a.nnz)
            st_hint_v8(a.elems_out + (size_t)dst * 32, lo, hi, pol_stream);
          else if (a.err)
            atomicOr(a.err, 2);  // inconsistent write order or remap id: store skipped
        }
      }
    }

    // Algorithm 2 over the slice, U nonzeros in flight
    const bool has_next = j + 1 < total;
    for (int r = 0; r < RND; ++r) {
      const bool last_round = (r == RND - 1);
      const uint8_t* nb = eb;
      int nl0 = m.l0, nl1 = m.l1, noff = (r + 1) * U;
      if (last_round) {
        if (has_next) {
          const int sn = (j + 1) % S;
          if (!tile_wait(&full[sn], (uint32_t)(((j + 1) / S) & 1), wait_ns, abort_flag, a.err))
            return;
          nb = ebuf + (size_t)sn * kTileNnz * 32;
          const TileMeta mn = meta[sn];
          nl0 = mn.l0;
          nl1 = mn.l1;
        } else {
          nl0 = nl1 = 0;  // nothing left to issue
        }
        noff = 0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        consume(u);
        const int li = slice0 + noff + u;
        issue_slot(u, nb, li, li >= nl0 && li < nl1);
      }
    }

    // the slice's first (head) and last (tail) rows as partial sums
    if (cur < 0) {
      if (sub == 0) {
        gr[2 * (2 * g)] = -1;
        gr[2 * (2 * g + 1)] = -1;
      }
    } else if (head) {
      store_gslot(2 * g, cur, -2, acc);
      if (sub == 0) gr[2 * (2 * g + 1)] = -1;
    } else {
      store_gslot(2 * g + 1, cur, prev_in_run, acc);
    }
    cur = -1;
    prev_in_run = -1;
    head = true;
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.f;
    __syncwarp();

    // warp combine of the 8 group slots (lanes over R): the warp's first row
    // and last row go to the control warp, rows between them are finished here
    {
      float* wp = wpart + ((size_t)st * kTileComputeWarps + cw) * 2 * R;
      int* wr = wrow + ((size_t)st * kTileComputeWarps + cw) * 2 * 2;
      int crow = -1, cprev = -1, nrows = 0;
      float cv[2] = {0.f, 0.f};
      auto put = [&](int h, int row, int prev) {  // warp slot h (0 head, 1 tail)
        if (lane == 0) {
          wr[2 * h] = row;
          wr[2 * h + 1] = prev;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
          if (lane + 32 * q < R) wp[(size_t)h * R + lane + 32 * q] = cv[q];
      };
      for (int s = 0; s < 2 * kTileGroups; ++s) {
        const int row = gr[2 * s];
        if (row < 0) continue;
        const float* sa = gs + (size_t)s * R;
        if (row == crow) {
#pragma unroll
          for (int q = 0; q < 2; ++q)
            if (lane + 32 * q < R) cv[q] += sa[lane + 32 * q];
        } else {
          if (crow >= 0) {
            if (nrows == 0) {
              put(0, crow, -2);
            } else {  // a row strictly inside the warp's slice: finished here
              for (int64_t z = (int64_t)cprev + 1; z < crow; ++z)
#pragma unroll
                for (int q = 0; q < 2; ++q)
                  if (lane + 32 * q < R) out[z * R + lane + 32 * q] = 0.f;
#pragma unroll
              for (int q = 0; q < 2; ++q)
                if (lane + 32 * q < R) out[(int64_t)crow * R + lane + 32 * q] = cv[q] * sc;
              if (crow == a.last_row)
                for (int64_t z = (int64_t)crow + 1; z < out_rows; ++z)
#pragma unroll
                  for (int q = 0; q < 2; ++q)
                    if (lane + 32 * q < R) out[z * R + lane + 32 * q] = 0.f;
            }
            ++nrows;
          }
          const int pv = gr[2 * s + 1];
          cprev = (pv != -2) ? pv : (crow >= 0 ? crow : cprev);
          crow = row;
#pragma unroll
          for (int q = 0; q < 2; ++q)
            if (lane + 32 * q < R) cv[q] = sa[lane + 32 * q];
        }
      }
      if (crow < 0) {
        if (lane == 0) {
          wr[0] = -1;
          wr[2] = -1;
        }
      } else if (nrows == 0) {
        put(0, crow, -2);
        if (lane == 0) wr[2] = -1;
      } else {
        put(1, crow, cprev);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&computed[st]);
    }
  }
}

template <typename T, int NV, int MODE, int U>
int launch_tile_kernel(const MttkrpArgs& a, cudaStream_t s) {
  const size_t smem = tile_layout(8 * NV).total;
  auto kfn = mttkrp_tile_kernel<T, NV, MODE, U>;
  int st = ensure_dyn_smem((const void*)kfn, smem, "cudaFuncSetAttribute(mttkrp_tile)");
  if (st) return st;
  const int grid = std::max(1, std::min(a.nblk, a.grid_ctas > 0 ? a.grid_ctas : a.nblk));
  kfn<<<grid, kTileThreads, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mttkrp_tile_kernel launch");
  return SPM_OK;
}

}  // namespace spm
