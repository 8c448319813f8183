// mttkrp_kernel.cuh - the fused mode-n spMTTKRP + dynamic remap kernel,
// one warp per block of the split.
//
// Every warp owns one block [lo, hi) of the mode-n ordered working copy (the
// paper's thread block over a tensor partition, Algorithm 4, shrunk to a warp
// so that no CTA-wide synchronisation is ever needed).  The warp streams its
// block through its own shared-memory ring: lane 0 issues 1D bulk-async
// copies (cp.async.bulk) of the nonzeros and of their remap ids two tiles
// ahead, completion is signalled on per-warp mbarriers, and every wait is
// bounded.  For every tile:
//   * remap (Algorithm 3): the 32 lanes copy the tile's nonzeros to their
//     places in the next mode's order, T_out[next_pos[p]] = x_p;
//   * elementwise computation (Algorithm 2): the warp is cut into groups of L
//     lanes, each lane owning a 16-byte slice of a rank-R row; a group walks
//     a contiguous run of the tile U nonzeros at a time, issues the factor-row
//     gathers A_k[i_k, slice] (k != n, 16-byte read-only loads; the indices
//     come from shared memory, so all U x (N-1) gathers leave at once), and
//     accumulates val * Hadamard product in registers while the output row
//     is unchanged; rows that start and end inside the run are written
//     straight to M_n;
//   * the first and last row of every run leave partial sums in shared-memory
//     slots, which the warp adds in run order, carrying the row that
//     continues into the next tile in registers.
// A row that continues past the block is written as a partial to `part` and
// summed by the fix-up kernel in block order.  No atomics: results are
// bit-identical from run to run and every output row is written exactly once
// (empty rows are zero-filled by the writer of the next nonempty row, or of
// the last one).
#pragma once

#include "mttkrp_common.cuh"

namespace spm {

constexpr int kStages = 2;  // tiles per warp ring (one in flight while one is used)
constexpr int kWarps = kThreads / 32;

// Per-warp shared-memory layout (bytes, in order).
struct WarpLayout {
  size_t ebuf, npbuf, sacc, cacc, srow, sprev, mbar, total;
};

// Remap ids staged per tile: tw + 3 ids at most (the copy starts at the
// 16-byte boundary at or below the tile) rounded up to a multiple of 4 ints,
// so that every stage's bulk-copy destination stays 16-byte aligned.
__host__ __device__ inline int np_stage_ints(int tw) { return (tw + 8 + 3) & ~3; }

__host__ __device__ inline WarpLayout warp_layout(int es, int tw, int R, int G) {
  WarpLayout l;
  size_t o = 0;
  l.ebuf = o;
  o += (size_t)kStages * tw * es;
  l.npbuf = o;
  o += (size_t)kStages * np_stage_ints(tw) * 4;
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
  o += (size_t)kStages * 8;
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
// modes only; -1 = runtime).
template <int NT, typename T, int VW, int RC, int U, int MODE>
__global__ void __launch_bounds__(kThreads, ((U <= 4 && VW > 1 && NT <= 3) ? 3 : 2))
    mttkrp_warp_kernel(const MttkrpArgs a, const int L) {
  constexpr int NV = VW * RC;
  const int N = NT > 0 ? NT : a.nmodes;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = 32 / L, sub = lane % L, gw = lane / L;
  const int es = a.es, R = a.R, mode = MODE >= 0 ? MODE : a.mode;
  const int TW = a.tile, K = TW / G;
  const int wb = blockIdx.x * kWarps + warp;
  if (wb >= a.nblk) return;
  const int4 bi = a.blkinfo[wb];
  const int lo = bi.x, hi = bi.y;
  if (lo >= hi) return;

  extern __shared__ __align__(128) uint8_t smem[];
  const WarpLayout lay = warp_layout(es, TW, R, G);
  uint8_t* wbase = smem + (size_t)warp * lay.total;
  uint8_t* ebuf = wbase + lay.ebuf;
  int32_t* npbuf = reinterpret_cast<int32_t*>(wbase + lay.npbuf);
  float* sacc = reinterpret_cast<float*>(wbase + lay.sacc);
  float* cacc = reinterpret_cast<float*>(wbase + lay.cacc);  // carry row partial (lanes over R)
  int* srow = reinterpret_cast<int*>(wbase + lay.srow);
  int* sprev = reinterpret_cast<int*>(wbase + lay.sprev);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(wbase + lay.mbar);

  const int ntiles = (hi - lo + TW - 1) / TW;
  const bool remap = a.elems_out != nullptr;
  const float sc = a.scale ? __ldg(a.scale) : 1.0f;
  const int64_t out_rows = a.out_rows;
  float* __restrict__ out = a.out;
  // L2 policies: the element stream, remap ids and remapped copy are touched
  // once per mode (evict first); factor rows are reused (evict last)
  const uint64_t pol_stream = make_policy((a.hints & 1) ? 1 : 0);
  const uint64_t pol_factor = make_policy((a.hints & 2) ? 2 : 0);
  // static 3-mode vector path: this lane's 16-byte slice of the two input
  // factors' rows (lanes past R read slice 0; their values are never stored)
  const uint32_t rowb = (uint32_t)R * (uint32_t)sizeof(T);
  const uint8_t* lane_base[2];
  {
    const int lsub = (sub * VW < R) ? sub : 0;
    const int k1 = (MODE >= 0 ? MODE : 0) + 1, k2 = (MODE >= 0 ? MODE : 0) + 2;
    lane_base[0] = static_cast<const uint8_t*>(a.factors[k1 % 3 < N ? k1 % 3 : 0]) + lsub * 16;
    lane_base[1] = static_cast<const uint8_t*>(a.factors[k2 % 3 < N ? k2 % 3 : 0]) + lsub * 16;
  }

  auto issue = [&](int t) {  // lane 0 only
    const int st = t % kStages;
    const int tlo = lo + t * TW;
    const int n = min(TW, hi - tlo);
    const uint32_t ebytes = (uint32_t)n * es;
    uint32_t npbytes = 0;
    int np0 = 0;
    if (remap) {
      np0 = tlo & ~3;
      npbytes = ((uint32_t)(tlo + n - np0) * 4u + 15u) & ~15u;
    }
    fence_proxy_async_smem();
    mbar_expect_tx(&mbar[st], ebytes + npbytes);
    bulk_g2s_hint(ebuf + (size_t)st * TW * es, a.elems_in + (size_t)tlo * es, ebytes, &mbar[st],
                  pol_stream);
    if (remap)
      bulk_g2s_hint(npbuf + st * np_stage_ints(TW), a.next_pos + np0, npbytes, &mbar[st],
                    pol_stream);
  };

  if (lane == 0) {
    for (int b = 0; b < kStages; ++b) mbar_init(&mbar[b], 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (lane == 0)
    for (int q = 0; q < kStages - 1 && q < ntiles; ++q) issue(q);

  auto rank_of = [&](int j) -> int {
    if constexpr (VW > 1) return sub * VW + j;
    return sub + L * j;
  };
  auto zero_rows_group = [&](int64_t from, int64_t to) {
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

  // carry of the warp combine: the row continuing into the next tile; its
  // partial sum lives in shared memory (lanes over R) to keep registers for
  // the gathers in flight
  int crow = -1, cprev = bi.z, emitted = 0;
  auto emit = [&](int row, int prev, bool first, bool last) {
    const bool split = (first && (bi.w & BLK_HEAD_SPLIT)) || (last && (bi.w & BLK_TAIL_SPLIT));
    if (split) {
      float* d = a.part + ((size_t)wb * 2 + (first ? 0 : 1)) * R;
      for (int r = lane; r < R; r += 32) d[r] = cacc[r];
      return;
    }
    for (int64_t z = (int64_t)prev + 1; z < row; ++z)
      for (int r = lane; r < R; r += 32) out[z * R + r] = 0.f;
    for (int r = lane; r < R; r += 32) out[(int64_t)row * R + r] = cacc[r] * sc;
    if (row == a.last_row)
      for (int64_t z = (int64_t)row + 1; z < out_rows; ++z)
        for (int r = lane; r < R; r += 32) out[z * R + r] = 0.f;
  };

  int issued = min(ntiles, kStages - 1);
  for (int t = 0; t < ntiles; ++t) {
    const int st = t % kStages;
    const bool ok = mbar_wait_bounded(&mbar[st], (uint32_t)((t / kStages) & 1));
    if (!__all_sync(0xffffffffu, ok)) {
      // a bulk copy did not complete in time: record it, wait (bounded) for
      // the copies still in flight, and leave without writing anything else
      if (lane == 0) {
        atomicOr(a.err, 1);
        for (int q = t; q < issued; ++q)
          (void)mbar_wait_bounded(&mbar[q % kStages], (uint32_t)((q / kStages) & 1));
      }
      return;
    }
    // the stage of tile t+kStages-1 held tile t-1, whose readers passed the last __syncwarp
    if (lane == 0 && t + kStages - 1 < ntiles) {
      issue(t + kStages - 1);
      issued = t + kStages;
    }
    const int tlo = lo + t * TW;
    const int n = min(TW, hi - tlo);
    const uint8_t* eb = ebuf + (size_t)st * TW * es;

    if (remap) {  // Algorithm 3: every element to its place in the next mode's order
      const int32_t* np = npbuf + st * np_stage_ints(TW) + (tlo & 3);
      const int nv = es / 16;
      for (int i = lane; i < n * nv; i += 32) {
        const int e = i / nv, c = i - e * nv;
        const uint4 v = reinterpret_cast<const uint4*>(eb + (size_t)e * es)[c];
        st_hint_v4(reinterpret_cast<uint4*>(a.elems_out + (size_t)np[e] * es) + c, v, pol_stream);
      }
    }

    // Algorithm 2 over this group's run [a0, b0) of the tile
    const int a0 = gw * K, b0 = min(a0 + K, n);
    if (a0 >= b0) {
      if (sub == 0) {
        srow[2 * gw] = -1;
        srow[2 * gw + 1] = -1;
      }
    } else {
      float acc[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) acc[j] = 0.f;
      int cur = reinterpret_cast<const int*>(eb + (size_t)a0 * es)[mode];
      bool head = true;
      int prev_in_run = -1;
      // input modes of this pass: km[j] = (mode + 1 + j) mod N, j < N - 1
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
        if constexpr (NT == 3 && MODE >= 0 && VW > 1) {
          // static modes: one 32 x 32 -> 64-bit multiply per row address
#pragma unroll
          for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int u = 0; u < U; ++u)
              if (u < nb)
                raw[u][j] = ld_nc_hint_v4(lane_base[j] + (uint64_t)(uint32_t)ixs[u][j] * rowb,
                                          pol_factor);
        } else {
#pragma unroll
          for (int j = 0; j < NI; ++j) {
            if (j < N - 1) {
              const int kj = (NT == 3 && MODE >= 0) ? (MODE + 1 + j) % 3 : (mode + 1 + j) % N;
              const void* Ak = a.factors[kj];
#pragma unroll
              for (int u = 0; u < U; ++u)
                if (u < nb)
                  Landing<T, VW, RC>::load(Ak, ixs[u][j], R, sub, L, pol_factor, raw[u][j]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (u < nb) {
            float prod[NV], x[NV];
            Landing<T, VW, RC>::unpack(raw[u][0], prod);
#pragma unroll
            for (int j = 1; j < NI; ++j) {
              if (j < N - 1) {
                Landing<T, VW, RC>::unpack(raw[u][j], x);
#pragma unroll
                for (int q = 0; q < NV; ++q) prod[q] *= x[q];
              }
            }
            if (rows[u] != cur) {
              if (head) {
                store_slot(2 * gw, cur, -2, acc);
                head = false;
              } else {
                write_row_group(cur, acc, prev_in_run);
              }
              prev_in_run = cur;
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
            const int* el = reinterpret_cast<const int*>(eb + (size_t)(e + u) * es);
            rows[u] = el[mode];
            vals[u] = __int_as_float(el[N]);
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
              Landing<T, VW, RC>::load(Ak, reinterpret_cast<const int*>(eb + (size_t)(e + u) * es)[k],
                                       R, sub, L, pol_factor, raw);
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
                store_slot(2 * gw, cur, -2, acc);
                head = false;
              } else {
                write_row_group(cur, acc, prev_in_run);
              }
              prev_in_run = cur;
              cur = rows[u];
#pragma unroll
              for (int q = 0; q < NV; ++q) acc[q] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < NV; ++q) acc[q] += prod[u][q];
          }
        }
      };
      int e = a0;
      if constexpr (NT > 0) {
        for (; e + U <= b0; e += U) batch(e, U);
        for (; e < b0; ++e) batch(e, 1);
      } else {
        for (; e + U <= b0; e += U) batch_generic(e, U);
        for (; e < b0; ++e) batch_generic(e, 1);
      }
      if (head) {
        store_slot(2 * gw, cur, -2, acc);
        if (sub == 0) srow[2 * gw + 1] = -1;
      } else {
        store_slot(2 * gw + 1, cur, prev_in_run, acc);
      }
    }
    __syncwarp();

    // warp combine: run-boundary rows of this tile in run order
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
    }
    __syncwarp();
  }
  if (crow >= 0) emit(crow, cprev, emitted == 0, true);
}

// Nonzeros per warp tile for a requested size: G runs of an odd length K, so
// that the groups' elements fall on distinct shared-memory banks.
__host__ __device__ inline int warp_tile_for(int tile, int G) {
  int K = tile / G;
  if (K < 1) K = 1;
  if (!(K & 1)) K += 1;
  return G * K;
}

template <int NT, typename T, int VW, int RC, int U, int MODE = -1>
int launch_warp_kernel(const MttkrpArgs& a0, int L, cudaStream_t s) {
  const int G = 32 / L;
  MttkrpArgs a = a0;
  a.tile = warp_tile_for(a0.tile, G);
  const size_t smem = (size_t)kWarps * warp_layout(a.es, a.tile, a.R, G).total;
  auto kfn = mttkrp_warp_kernel<NT, T, VW, RC, U, MODE>;
  static size_t configured = 0;  // per instantiation: raise the dynamic smem limit once
  if (configured < smem) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max<size_t>(smem, 48 * 1024));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(mttkrp_warp)");
    configured = std::max<size_t>(smem, 48 * 1024);
  }
  const int grid = (a.nblk + kWarps - 1) / kWarps;
  kfn<<<grid, kThreads, smem, s>>>(a, L);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mttkrp_warp_kernel launch");
  return SPM_OK;
}

}  // namespace spm
