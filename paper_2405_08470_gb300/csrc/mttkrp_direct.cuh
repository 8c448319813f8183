// mttkrp_direct.cuh - barrier-free variant of the fused mode-n spMTTKRP +
// dynamic remap kernel.
//
// One CTA owns one block [lo, hi) of the mode-n ordered working copy (the
// paper's thread block over a tensor partition, Algorithm 4).  The block is
// cut into NG equal contiguous runs, one per group of L lanes; a group walks
// its run without any CTA-wide synchronisation: U nonzeros at a time it loads
// the elements (16-byte read-only loads; consecutive elements share L1
// lines), scatters them to their place in the next mode's order (Algorithm
// 3), gathers the factor-row slices of the other modes (Algorithm 2), and
// accumulates val * Hadamard product in registers while the output row is
// unchanged.  Rows that start and end inside a run are written straight to
// M_n.  The first and last row of every run leave partial sums in shared
// memory; after one barrier a single warp adds them in run order and writes
// those rows (or, for a row that continues past the block, a partial summed
// later by the fix-up kernel in block order).  No atomics: results are
// bit-identical from run to run and every output row is written once.
#pragma once

#include "mttkrp_kernel.cuh"

namespace spm {

__host__ __device__ inline size_t direct_smem_bytes(int R, int NG) {
  return (size_t)2 * NG * R * 4 + (size_t)2 * NG * 4 * 2;
}

// Loads the N indices and the value of element e into registers.
template <int NT>
struct ElemLoad {
  __device__ __forceinline__ static void load(const uint8_t* base, int64_t e, int es, int N,
                                              int* idx, float& val) {
    const int* el = reinterpret_cast<const int*>(base + e * es);
    for (int k = 0; k < N; ++k) idx[k] = __ldg(el + k);
    val = __int_as_float(__ldg(el + N));
  }
};
template <>
struct ElemLoad<3> {
  __device__ __forceinline__ static void load(const uint8_t* base, int64_t e, int, int, int* idx,
                                              float& val) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(base + e * 16));
    idx[0] = v.x;
    idx[1] = v.y;
    idx[2] = v.z;
    val = __int_as_float(v.w);
  }
};

template <int NT, typename T, int VW, int RC, int U>
__global__ void __launch_bounds__(kThreads, 3) mttkrp_direct_kernel(const MttkrpArgs a, const int L) {
  constexpr int NV = VW * RC;
  constexpr int NI = NT > 0 ? NT : kMaxModes;
  const int N = NT > 0 ? NT : a.nmodes;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = 32 / L, NG = (kThreads / 32) * G;
  const int es = a.es, R = a.R, mode = a.mode;
  const int sub = lane % L, gw = lane / L, gi = warp * G + gw;

  extern __shared__ __align__(128) uint8_t smem[];
  float* sacc = reinterpret_cast<float*>(smem);
  int* srow = reinterpret_cast<int*>(smem + (size_t)2 * NG * R * 4);
  int* sprev = srow + 2 * NG;

  const int4 bi = a.blkinfo[blockIdx.x];
  const int lo = bi.x, hi = bi.y;
  if (lo >= hi) return;
  const bool remap = a.elems_out != nullptr;
  const float sc = a.scale ? __ldg(a.scale) : 1.0f;
  const int64_t out_rows = a.out_rows;
  float* __restrict__ out = a.out;
  const int64_t len = hi - lo;
  const int a0 = lo + (int)(len * gi / NG), b0 = lo + (int)(len * (gi + 1) / NG);

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

  if (a0 >= b0) {
    if (sub == 0) {
      srow[2 * gi] = -1;
      srow[2 * gi + 1] = -1;
    }
  } else {
    float acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = 0.f;
    int cur = __ldg(reinterpret_cast<const int*>(a.elems_in + (int64_t)a0 * es) + mode);
    bool head = true;
    int prev_in_run = -1;
    for (int e = a0; e < b0; e += U) {
      float prod[U][NV];
      int rows[U];
      int idx[U][NI];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (e + u < b0) {
          float v;
          ElemLoad<NT>::load(a.elems_in, e + u, es, N, idx[u], v);
          if constexpr (NT > 0) {  // static indexing keeps idx in registers
            rows[u] = idx[u][0];
#pragma unroll
            for (int k = 1; k < NT; ++k)
              if (k == mode) rows[u] = idx[u][k];
          } else {
            rows[u] = idx[u][mode];
          }
#pragma unroll
          for (int j = 0; j < NV; ++j) prod[u][j] = v;
          if (remap && sub == 0) {  // Algorithm 3: T_out[next_pos[p]] = x_p
            const int64_t dst = __ldg(a.next_pos + e + u);
            const uint4* src = reinterpret_cast<const uint4*>(a.elems_in + (int64_t)(e + u) * es);
            uint4* d = reinterpret_cast<uint4*>(a.elems_out + dst * es);
            for (int c = 0; c < es / 16; ++c) d[c] = __ldg(src + c);
          }
        }
      }
      for (int k = 0; k < N; ++k) {
        if (k == mode) continue;
        const void* Ak = a.factors[k];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (e + u < b0) {
            const int64_t ix = idx[u][k];
            float x[NV];
            if constexpr (VW > 1) {
              if (sub * VW < R) {
                Slice<T, VW>::load(Ak, ix, R, sub, x);
              } else {
#pragma unroll
                for (int j = 0; j < NV; ++j) x[j] = 0.f;
              }
            } else {
#pragma unroll
              for (int j = 0; j < NV; ++j) {
                const int r = rank_of(j);
                x[j] = (r < R) ? load_scalar<T>(Ak, ix * R + r) : 0.f;
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
              store_slot(2 * gi, cur, -2, acc);
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
      store_slot(2 * gi, cur, -2, acc);
      if (sub == 0) srow[2 * gi + 1] = -1;
    } else {
      store_slot(2 * gi + 1, cur, prev_in_run, acc);
    }
  }
  __syncthreads();
  if (warp != 0) return;

  // ---- one warp: run-boundary rows in run order, then the block's last row
  constexpr int CC = (kMaxRank + 31) / 32;
  const int ncc = (R + 31) / 32;
  int crow = -1, cprev = bi.z, emitted = 0;
  float ca[CC];
#pragma unroll
  for (int c = 0; c < CC; ++c) ca[c] = 0.f;
  auto emit = [&](int row, int prev, bool first, bool last) {
    const bool split = (first && (bi.w & BLK_HEAD_SPLIT)) || (last && (bi.w & BLK_TAIL_SPLIT));
    if (split) {
      float* d = a.part + ((size_t)blockIdx.x * 2 + (first ? 0 : 1)) * R;
#pragma unroll
      for (int c = 0; c < CC; ++c)
        if (c < ncc && lane + 32 * c < R) d[lane + 32 * c] = ca[c];
      return;
    }
    for (int64_t z = a.no_fill ? (int64_t)row : (int64_t)prev + 1; z < row; ++z)
#pragma unroll
      for (int c = 0; c < CC; ++c)
        if (c < ncc && lane + 32 * c < R) out[z * R + lane + 32 * c] = 0.f;
#pragma unroll
    for (int c = 0; c < CC; ++c)
      if (c < ncc && lane + 32 * c < R) out[(int64_t)row * R + lane + 32 * c] = ca[c] * sc;
    if (!a.no_fill && row == a.last_row)
      for (int64_t z = (int64_t)row + 1; z < out_rows; ++z)
#pragma unroll
        for (int c = 0; c < CC; ++c)
          if (c < ncc && lane + 32 * c < R) out[z * R + lane + 32 * c] = 0.f;
  };
  for (int s = 0; s < 2 * NG; ++s) {
    const int row = srow[s];
    if (row < 0) continue;
    const float* sa = sacc + (size_t)s * R;
    if (row == crow) {
#pragma unroll
      for (int c = 0; c < CC; ++c)
        if (c < ncc && lane + 32 * c < R) ca[c] += sa[lane + 32 * c];
    } else {
      if (crow >= 0) {
        emit(crow, cprev, emitted == 0, false);
        emitted = 1;
      }
      const int pv = sprev[s];
      cprev = (pv != -2) ? pv : (crow >= 0 ? crow : cprev);
      crow = row;
#pragma unroll
      for (int c = 0; c < CC; ++c)
        if (c < ncc && lane + 32 * c < R) ca[c] = sa[lane + 32 * c];
    }
  }
  if (crow >= 0) emit(crow, cprev, emitted == 0, true);
}

template <int NT, typename T, int VW, int RC, int U>
int launch_direct(const MttkrpArgs& a, int L, cudaStream_t s) {
  const int NG = (kThreads / 32) * (32 / L);
  const size_t smem = direct_smem_bytes(a.R, NG);
  auto kfn = mttkrp_direct_kernel<NT, T, VW, RC, U>;
  int st = ensure_dyn_smem((const void*)kfn, smem, "cudaFuncSetAttribute(direct)");
  if (st) return st;
  kfn<<<a.nblk, kThreads, smem, s>>>(a, L);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mttkrp_direct_kernel launch");
  return SPM_OK;
}

}  // namespace spm
