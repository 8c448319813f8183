// kernels_als.cu - the CP-ALS update around the fused spMTTKRP (Section 2.1.4;
// the update itself is Kolda-Bader's CP-ALS, which the paper cites):
//   G_k = A_k^T A_k            FP32 per-chunk partials, FP64 fixed-order sum
//   V   = Hadamard_{k!=n} G_k  FP64, Cholesky V = L L^T and V^-1 in FP64
//   U   = M_n V^-1             FP32 (V^-1 stored as FP32), column norms^2
//                              (R <= 64: U stays on chip; the scale pass
//                              forms it again from M_n)
//   lambda = sqrt(sum_i U^2)   FP64 fixed-order sum
//   A_n = U / lambda           stored as the factor type (FP32 or BF16)
//   fit from |X|^2, lambda, the G_k and <X, Y> (last mode).
// Every reduction runs in a fixed order over a fixed grid, so the results are
// bit-identical from run to run.  A failed Cholesky sets a device status word
// that makes the remaining update kernels of the iteration return at once.
#include <cuda_bf16.h>

#include "engine.h"
#include "als.h"
#include "mttkrp_common.cuh"  // paired FP32 arithmetic (fma2)

namespace spm {

template <typename T>
__device__ __forceinline__ float to_f(T x);
template <>
__device__ __forceinline__ float to_f<float>(float x) {
  return x;
}
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}
template <typename T>
__device__ __forceinline__ T from_f(float x);
template <>
__device__ __forceinline__ float from_f<float>(float x) {
  return x;
}
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}

// ---- Gram partials: block (chunk, rt, st) computes G[rt*32.., st*32..] over its rows
template <typename T>
__global__ void __launch_bounds__(256) gram_partial_kernel(const T* __restrict__ A, int64_t I,
                                                           int R, int64_t rows_per_chunk,
                                                           double* __restrict__ part) {
  __shared__ float Ar[64][33];
  __shared__ float As[64][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int chunk = blockIdx.x, r0 = blockIdx.y * 32, s0 = blockIdx.z * 32;
  const int64_t lo = (int64_t)chunk * rows_per_chunk;
  const int64_t hi = min(I, lo + rows_per_chunk);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const bool diag = blockIdx.y == blockIdx.z;  // the two column tiles are the same
  float(*Bs)[33] = diag ? Ar : As;
  for (int64_t base = lo; base < hi; base += 64) {
    for (int q = threadIdx.x; q < 64 * 32; q += 256) {
      const int rr = q >> 5, cc = q & 31;
      const int64_t row = base + rr;
      const bool ok = row < hi;
      Ar[rr][cc] = (ok && r0 + cc < R) ? to_f<T>(A[row * R + r0 + cc]) : 0.f;
      if (!diag) As[rr][cc] = (ok && s0 + cc < R) ? to_f<T>(A[row * R + s0 + cc]) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < 64; ++q) {
      const float a = Ar[q][tx];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] += a * Bs[q][ty + 8 * j];
    }
    __syncthreads();
  }
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + tx, s = s0 + ty + 8 * j;
    if (r < R && s < R) part[((size_t)chunk * R + r) * R + s] = (double)acc[j];
  }
}

// gram_reduce: one warp per entry; lane l sums chunks l, l+32, ... in order,
// then a fixed tree over the lanes (deterministic for a given chunk count).
__global__ void gram_reduce_kernel(const double* __restrict__ part, int nchunk, int R,
                                   double* __restrict__ G) {
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= R * R) return;
  double s = 0.0;
  for (int c = lane; c < nchunk; c += 32) s += part[(size_t)c * R * R + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) G[q] = s;
}

// R <= 64 (RP = 16, 32 or 64 columns, zero-padded): the chunk's rows are staged
// in shared memory 64 at a time (the next tile's loads are issued into registers
// before the current tile is used).  G is symmetric, so only its 4 x 4 blocks on
// and above the diagonal are formed: thread q of group g adds the outer-product
// block (r0.., c0..), r0 <= c0, of rows g, g + NG, ... of each tile; the NG
// groups' sums are added in group order and mirrored below the diagonal.  FP32
// within a chunk.
template <typename T, int RP>
__global__ void __launch_bounds__(256) gram_tile_kernel(const T* __restrict__ A, int64_t I, int R,
                                                        int64_t rows_per_chunk,
                                                        double* __restrict__ part) {
  constexpr int RT = 64, LD = RP + 4;        // tile rows; row stride keeps float4 alignment
  constexpr int CB = RP / 4;                 // 4-column blocks per side
  constexpr int NB = CB * (CB + 1) / 2;      // blocks on and above the diagonal
  constexpr int NG = 256 / NB;               // thread groups (25, 7 or 1)
  constexpr int PT = RT * RP / 256;          // tile values each thread loads
  constexpr int TILE = RT * LD, RED = NG * RP * RP;
  __shared__ __align__(16) float sm[TILE > RED ? TILE : RED];
  const int tid = threadIdx.x, g = tid / NB;
  int bi = 0, t = tid % NB;
  while (t >= CB - bi) {
    t -= CB - bi;
    ++bi;
  }
  const int r0 = 4 * bi, c0 = 4 * (bi + t);
  const bool active = g < NG;
  const int64_t lo = (int64_t)blockIdx.x * rows_per_chunk;
  const int64_t hi = min(I, lo + rows_per_chunk);
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  float pre[PT];
  auto fetch = [&](int64_t base) {
#pragma unroll
    for (int p = 0; p < PT; ++p) {
      const int e = tid + 256 * p, rr = e / RP, cc = e % RP;
      const int64_t row = base + rr;
      pre[p] = (row < hi && cc < R) ? to_f<T>(A[row * R + cc]) : 0.f;
    }
  };
  if (lo < hi) fetch(lo);
  for (int64_t base = lo; base < hi; base += RT) {
    __syncthreads();  // the previous tile's reads are done
#pragma unroll
    for (int p = 0; p < PT; ++p) {
      const int e = tid + 256 * p;
      sm[(e / RP) * LD + e % RP] = pre[p];
    }
    __syncthreads();
    if (base + RT < hi) fetch(base + RT);
    if (active) {
      for (int rr = g; rr < RT; rr += NG) {
        const float4 x = *reinterpret_cast<const float4*>(&sm[rr * LD + r0]);
        const float4 y = *reinterpret_cast<const float4*>(&sm[rr * LD + c0]);
        const float xv[4] = {x.x, x.y, x.z, x.w};
        const float2 y01 = make_float2(y.x, y.y), y23 = make_float2(y.z, y.w);
#pragma unroll
        for (int a = 0; a < 4; ++a) {  // paired FMAs: the same result as four fmaf
          float2* a2 = reinterpret_cast<float2*>(acc[a]);
          const float2 xa = make_float2(xv[a], xv[a]);
          a2[0] = fma2(xa, y01, a2[0]);
          a2[1] = fma2(xa, y23, a2[1]);
        }
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) sm[(g * RP + r0 + a) * RP + c0 + b] = acc[a][b];
  }
  __syncthreads();
  for (int e = tid; e < R * R; e += 256) {
    const int r = e / R, c = e % R;
    const int u = min(r, c), w = max(r, c);  // the entry's place on or above the diagonal
    float v = 0.f;
    for (int k = 0; k < NG; ++k) v += sm[(k * RP + u) * RP + w];
    part[(size_t)blockIdx.x * R * R + e] = (double)v;
  }
}

// ---- V = Hadamard of the other Grams, Cholesky, V^-1 (one block, FP64)
// Every step is spread over the block, so no thread runs a long dependent chain:
//   Cholesky, right-looking: column j is scaled by 1 / sqrt(V_jj), then the
//     trailing lower triangle takes the rank-1 update -L_ij L_kj;
//   X = L^-1 by forward substitution on the identity, row i at step i (scaled
//     by 1 / L_ii), the rows below updated in parallel;
//   V^-1 = X^T X.
// V (holding L) and X live in dynamic shared memory when it holds them
// (in_smem; R <= 64), else in the global work buffer.
__global__ void __launch_bounds__(256) als_prep_kernel(const double* __restrict__ grams, int N,
                                                       int n, int R, double* __restrict__ work,
                                                       float* __restrict__ vinv,
                                                       int* __restrict__ status, int in_smem) {
  extern __shared__ double prep_smem[];
  double* V = in_smem ? prep_smem : work;
  double* X = V + (size_t)R * R;
  __shared__ int bad;
  __shared__ double rdiag[256];  // 1 / L[j][j] (R <= 256): FP64 divides are slow
  const int tid = threadIdx.x;
  if (tid == 0) bad = *status;
  __syncthreads();
  if (bad) return;
  for (int q = tid; q < R * R; q += blockDim.x) {
    double v = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != n) v *= grams[(size_t)k * R * R + q];
    V[q] = v;
    X[q] = (q / R == q % R) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < R; ++j) {
    if (tid == 0) {
      const double d = V[(size_t)j * R + j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
      } else {
        const double l = sqrt(d);
        V[(size_t)j * R + j] = l;
        rdiag[j] = 1.0 / l;
      }
    }
    __syncthreads();
    if (bad) break;
    const double rj = rdiag[j];
    for (int i = j + 1 + tid; i < R; i += blockDim.x) V[(size_t)i * R + j] *= rj;
    __syncthreads();
    const int m = R - j - 1;  // trailing block: rows and columns j+1 .. R-1
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) V[(size_t)i * R + k] -= V[(size_t)i * R + j] * V[(size_t)k * R + j];
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) *status = SPM_ERR_NOT_SPD;
    return;
  }
  for (int i = 0; i < R; ++i) {
    const double ri = rdiag[i];
    for (int c = tid; c <= i; c += blockDim.x) X[(size_t)i * R + c] *= ri;
    __syncthreads();
    const int rows = R - i - 1, cols = i + 1;
    for (int e = tid; e < rows * cols; e += blockDim.x) {
      const int k = i + 1 + e / cols, c = e % cols;
      X[(size_t)k * R + c] -= V[(size_t)k * R + i] * X[(size_t)i * R + c];
    }
    __syncthreads();
  }
  // V^-1 = X^T X (X lower triangular)
  for (int q = tid; q < R * R; q += blockDim.x) {
    const int i = q / R, j = q % R;
    double s = 0.0;
    for (int k = max(i, j); k < R; ++k) s += X[(size_t)k * R + i] * X[(size_t)k * R + j];
    vinv[q] = (float)s;
  }
}

// ---- U = M V^-1 (warp per row), per-block column sums of U^2
template <int CC>
__global__ void __launch_bounds__(256) als_solve_kernel(const float* __restrict__ M,
                                                        float* __restrict__ U,
                                                        const float* __restrict__ vinv, int64_t I,
                                                        int R, double* __restrict__ colsq_part,
                                                        const int* __restrict__ status) {
  extern __shared__ float vs[];  // R x R when R <= 128, else unused
  __shared__ float wsum[8][CC * 32];
  if (*status) return;
  const bool in_smem = R <= 128;
  if (in_smem)
    for (int q = threadIdx.x; q < R * R; q += 256) vs[q] = vinv[q];
  __syncthreads();
  const float* V = in_smem ? vs : vinv;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float csq[CC];
#pragma unroll
  for (int c = 0; c < CC; ++c) csq[c] = 0.f;
  // RW rows per warp and step: their loads are in flight together
  constexpr int RW = 4;
  const int64_t stride = (int64_t)gridDim.x * 8;
  for (int64_t i0 = (int64_t)blockIdx.x * 8 + w; i0 < I; i0 += stride * RW) {
    float m[RW][CC], u[RW][CC];
#pragma unroll
    for (int t = 0; t < RW; ++t) {
      const int64_t i = i0 + t * stride;
#pragma unroll
      for (int c = 0; c < CC; ++c) {
        const int r = lane + 32 * c;
        m[t][c] = (i < I && r < R) ? M[i * R + r] : 0.f;
        u[t][c] = 0.f;
      }
    }
#pragma unroll
    for (int cj = 0; cj < CC; ++cj) {
      for (int jj = 0; jj < 32; ++jj) {
        const int j = cj * 32 + jj;
        if (j < R) {
          float vj[CC];
#pragma unroll
          for (int c = 0; c < CC; ++c) {
            const int r = lane + 32 * c;
            vj[c] = r < R ? V[(size_t)j * R + r] : 0.f;
          }
#pragma unroll
          for (int t = 0; t < RW; ++t) {
            const float mj = __shfl_sync(0xffffffffu, m[t][cj], jj);
#pragma unroll
            for (int c = 0; c < CC; ++c) u[t][c] = fmaf(mj, vj[c], u[t][c]);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < RW; ++t) {
      const int64_t i = i0 + t * stride;
      if (i < I) {
#pragma unroll
        for (int c = 0; c < CC; ++c) {
          const int r = lane + 32 * c;
          if (r < R) {
            U[i * R + r] = u[t][c];
            csq[c] = fmaf(u[t][c], u[t][c], csq[c]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CC; ++c) wsum[w][lane + 32 * c] = csq[c];
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += 256) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += (double)wsum[q][r];
    colsq_part[(size_t)blockIdx.x * R + r] = s;
  }
}

// R <= 64 (RP = 16, 32 or 64 columns, zero-padded): U = M V^-1 on row tiles
// staged in shared memory.  Thread (rs, cb) holds the 4 x 4 block of rows rs +
// RS k and columns 4 cb..; every entry adds m_ij V^-1_jr over j in ascending
// order with fmaf, as the warp-per-row kernel does.
//   SCALE = false: per-block column sums of U^2 (for lambda); U is not stored.
//   SCALE = true:  U is formed again from M (the same arithmetic, so the same
//                  values), A = U / lambda is stored as T, and per-block column
//                  sums of M * A (for <X, Y>) are left in part.
template <typename T, int RP, bool SCALE>
__global__ void __launch_bounds__(256) als_rows_kernel(const float* __restrict__ M,
                                                       const float* __restrict__ vinv,
                                                       T* __restrict__ A,
                                                       const double* __restrict__ lam64,
                                                       int64_t I, int R,
                                                       double* __restrict__ part,
                                                       const int* __restrict__ status) {
  constexpr int CB = RP / 4, RS = 256 / CB, RT = 4 * RS, LD = RP + 1;
  __shared__ float Ms[RT * LD];
  __shared__ __align__(16) float Vs[RP * RP];
  __shared__ float red[RS][RP];
  if (*status) return;
  const int tid = threadIdx.x, cb = tid % CB, rs = tid / CB, c0 = 4 * cb;
  for (int e = tid; e < RP * RP; e += 256) {
    const int j = e / RP, c = e % RP;
    Vs[e] = (j < R && c < R) ? vinv[j * R + c] : 0.f;
  }
  float inv[4], sum[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    inv[b] = (SCALE && c0 + b < R) ? (float)(1.0 / lam64[c0 + b]) : 0.f;
    sum[b] = 0.f;
  }
  const int64_t ntiles = (I + RT - 1) / RT;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i0 = t * RT;
    __syncthreads();  // the previous tile's reads of Ms are done
    for (int e = tid; e < RT * RP; e += 256) {
      const int rr = e / RP, cc = e % RP;
      const int64_t i = i0 + rr;
      Ms[rr * LD + cc] = (i < I && cc < R) ? M[i * R + cc] : 0.f;
    }
    __syncthreads();
    float u[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int b = 0; b < 4; ++b) u[k][b] = 0.f;
#pragma unroll 8
    for (int j = 0; j < RP; ++j) {
      const float4 v = *reinterpret_cast<const float4*>(&Vs[j * RP + c0]);
      const float2 v01 = make_float2(v.x, v.y), v23 = make_float2(v.z, v.w);
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // paired FMAs: the same result as four fmaf
        const float m = Ms[(rs + RS * k) * LD + j];
        const float2 mm = make_float2(m, m);
        float2* u2 = reinterpret_cast<float2*>(u[k]);
        u2[0] = fma2(mm, v01, u2[0]);
        u2[1] = fma2(mm, v23, u2[1]);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + rs + RS * k;
      if (i >= I) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + b;
        if (c >= R) continue;
        if constexpr (SCALE) {
          const T a = from_f<T>(u[k][b] * inv[b]);
          A[i * R + c] = a;
          sum[b] = fmaf(Ms[(rs + RS * k) * LD + c], to_f<T>(a), sum[b]);
        } else {
          sum[b] = fmaf(u[k][b], u[k][b], sum[b]);
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) red[rs][c0 + b] = sum[b];
  __syncthreads();
  for (int c = tid; c < R; c += 256) {
    double acc = 0.0;
    for (int q = 0; q < RS; ++q) acc += (double)red[q][c];
    part[(size_t)blockIdx.x * R + c] = acc;
  }
}

// Sum over nb per-block partials of column r: lane l takes blocks l, l+32, ...
// in order, then a fixed tree over the lanes (deterministic).
__device__ __forceinline__ double warp_column_sum(const double* __restrict__ part, int nb, int R,
                                                  int r) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
#pragma unroll 8
  for (int b = lane; b < nb; b += 32) s += part[(size_t)b * R + r];  // loads run ahead
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  return __shfl_sync(0xffffffffu, s, 0);
}

__global__ void als_lambda_kernel(const double* __restrict__ colsq_part, int nb, int R,
                                  double* __restrict__ lam64, float* __restrict__ lam_out,
                                  const int* __restrict__ status) {
  if (*status) return;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);  // one warp per column
  if (r >= R) return;
  const double l = sqrt(warp_column_sum(colsq_part, nb, R, r));
  if ((threadIdx.x & 31) == 0) {
    lam64[r] = l;
    lam_out[r] = (float)l;
  }
}

// ---- Column-scale folding (cp_als_run).  The mode-n update followed by the
// 2-norm normalisation does not depend on the column scales of the other
// factors: scaling column r of A_k (k != n) by c scales column r of M_n by c and
// row and column r of V by c, so M_n V^-1 changes by 1/c in column r, which the
// normalisation removes.  The loop therefore stores U_n = M_n V^-1 as it is,
// with its Gram taken from the stored factor, and normalises once after the
// last iteration: A_k = U_k / |U_k[:, r]| with the norms read off the diagonals
// of the Grams, lambda_r = prod_k |U_k[:, r]|, the weight of rank-one term r of
// the same model.
__global__ void fill_f64_kernel(double* __restrict__ p, int n, double v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void als_fold_lambda_kernel(const double* __restrict__ grams, int N, int R,
                                       double* __restrict__ lam64, float* __restrict__ lam_out,
                                       const int* __restrict__ status) {
  if (*status) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double l = 1.0;
  for (int k = 0; k < N; ++k) l *= sqrt(grams[(size_t)k * R * R + (size_t)r * R + r]);
  lam64[r] = l;
  lam_out[r] = (float)l;
}

template <typename T>
__global__ void __launch_bounds__(256) als_normalize_kernel(T* __restrict__ A, int64_t I, int R,
                                                            const double* __restrict__ gram,
                                                            const int* __restrict__ status) {
  __shared__ float inv[256];
  if (*status) return;
  for (int r = threadIdx.x; r < R; r += 256)
    inv[r] = (float)(1.0 / sqrt(gram[(size_t)r * R + r]));
  __syncthreads();
  const int64_t n = I * R;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256)
    A[e] = from_f<T>(to_f<T>(A[e]) * inv[(int)(e % R)]);
}

// ---- A_n = U / lambda (stored as T); per-block sums of M * A_n (for <X, Y>)
template <typename T, int CC>
__global__ void __launch_bounds__(256) als_scale_kernel(const float* __restrict__ U,
                                                        const float* __restrict__ M,
                                                        T* __restrict__ A,
                                                        const double* __restrict__ lam64,
                                                        int64_t I, int R,
                                                        double* __restrict__ mdot_part,
                                                        const int* __restrict__ status) {
  __shared__ float wsum[8][CC * 32];
  if (*status) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float inv[CC], md[CC];
#pragma unroll
  for (int c = 0; c < CC; ++c) {
    const int r = lane + 32 * c;
    inv[c] = r < R ? (float)(1.0 / lam64[r]) : 0.f;
    md[c] = 0.f;
  }
  constexpr int RW = 4;  // rows per warp and step (loads in flight together)
  const int64_t stride = (int64_t)gridDim.x * 8;
  for (int64_t i0 = (int64_t)blockIdx.x * 8 + w; i0 < I; i0 += stride * RW) {
    float uu[RW][CC], mm[RW][CC];
#pragma unroll
    for (int t = 0; t < RW; ++t) {
      const int64_t i = i0 + t * stride;
#pragma unroll
      for (int c = 0; c < CC; ++c) {
        const int r = lane + 32 * c;
        const bool ok = i < I && r < R;
        uu[t][c] = ok ? U[i * R + r] : 0.f;
        mm[t][c] = ok ? M[i * R + r] : 0.f;
      }
    }
#pragma unroll
    for (int t = 0; t < RW; ++t) {
      const int64_t i = i0 + t * stride;
      if (i < I) {
#pragma unroll
        for (int c = 0; c < CC; ++c) {
          const int r = lane + 32 * c;
          if (r < R) {
            const T a = from_f<T>(uu[t][c] * inv[c]);
            A[i * R + r] = a;
            md[c] = fmaf(mm[t][c], to_f<T>(a), md[c]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CC; ++c) wsum[w][lane + 32 * c] = md[c];
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += 256) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += (double)wsum[q][r];
    mdot_part[(size_t)blockIdx.x * R + r] = s;
  }
}

// ---- fit = 1 - sqrt(|X|^2 + |Y|^2 - 2 <X,Y>) / |X|
// One block of kFitThreads: a warp per column of <M, A> (the column sums of the
// per-block partials), then a fixed-order tree over the threads' parts.
constexpr int kFitThreads = 1024;
__global__ void __launch_bounds__(kFitThreads) als_fit_kernel(const double* __restrict__ grams,
                                                              int N, int R,
                                                              const double* __restrict__ lam64,
                                                              const double* __restrict__ mdot_part,
                                                              int nb, double normx2,
                                                              double* __restrict__ fit_out,
                                                              const int* __restrict__ status) {
  __shared__ double red[kFitThreads];
  __shared__ double red2[kFitThreads];
  const int tid = threadIdx.x;
  double y2 = 0.0, xy = 0.0;
  for (int q = tid; q < R * R; q += kFitThreads) {
    const int r = q / R, s = q % R;
    double h = 1.0;
    for (int k = 0; k < N; ++k) h *= grams[(size_t)k * R * R + q];
    y2 += lam64[r] * lam64[s] * h;
  }
  for (int r = tid >> 5; r < R; r += kFitThreads / 32) {  // one warp per column
    const double m = warp_column_sum(mdot_part, nb, R, r);
    if ((tid & 31) == 0) xy += lam64[r] * m;
  }
  red[tid] = y2;
  red2[tid] = xy;
  __syncthreads();
  for (int w = kFitThreads / 2; w > 0; w >>= 1) {
    if (tid < w) {
      red[tid] += red[tid + w];
      red2[tid] += red2[tid + w];
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double res2 = fmax(normx2 + red[0] - 2.0 * red2[0], 0.0);
    fit_out[0] = *status ? nan("") : 1.0 - sqrt(res2) / sqrt(normx2);
  }
}

// ------------------------------------------------------------ launchers

int launch_gram(const void* A, int dtype, int64_t I, int R, double* part, int max_chunks,
                double* G, cudaStream_t s) {
  int64_t rpc = std::max<int64_t>(512, (I + max_chunks - 1) / max_chunks);
  int nchunk = (int)std::max<int64_t>(1, (I + rpc - 1) / rpc);
  const int nt = (R + 31) / 32;
  dim3 grid(nchunk, nt, nt);
  if (R <= 64) {
    const bool bf = dtype == SPM_DTYPE_BF16;
    const auto* Ab = static_cast<const __nv_bfloat16*>(A);
    const auto* Af = static_cast<const float*>(A);
    if (R <= 16) {
      if (bf) gram_tile_kernel<__nv_bfloat16, 16><<<nchunk, 256, 0, s>>>(Ab, I, R, rpc, part);
      else gram_tile_kernel<float, 16><<<nchunk, 256, 0, s>>>(Af, I, R, rpc, part);
    } else if (R <= 32) {
      if (bf) gram_tile_kernel<__nv_bfloat16, 32><<<nchunk, 256, 0, s>>>(Ab, I, R, rpc, part);
      else gram_tile_kernel<float, 32><<<nchunk, 256, 0, s>>>(Af, I, R, rpc, part);
    } else {
      if (bf) gram_tile_kernel<__nv_bfloat16, 64><<<nchunk, 256, 0, s>>>(Ab, I, R, rpc, part);
      else gram_tile_kernel<float, 64><<<nchunk, 256, 0, s>>>(Af, I, R, rpc, part);
    }
  } else if (dtype == SPM_DTYPE_BF16) {
    gram_partial_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(
        static_cast<const __nv_bfloat16*>(A), I, R, rpc, part);
  } else {
    gram_partial_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(A), I, R, rpc,
                                                    part);
  }
  gram_reduce_kernel<<<(R * R + 7) / 8, 256, 0, s>>>(part, nchunk, R, G);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "gram kernels");
}

int launch_als_prep(const double* grams, int N, int n, int R, double* work, float* vinv,
                    int* status, cudaStream_t s) {
  const size_t smem = (size_t)2 * R * R * sizeof(double);
  const int in_smem = R <= 64;
  if (in_smem) {
    int st = ensure_dyn_smem((const void*)als_prep_kernel, 2 * 64 * 64 * sizeof(double),
                             "cudaFuncSetAttribute(als_prep)");
    if (st) return st;
  }
  als_prep_kernel<<<1, 256, in_smem ? smem : 0, s>>>(grams, N, n, R, work, vinv, status, in_smem);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "als_prep_kernel");
}

template <int CC>
static int solve_cc(const float* M, float* U, const float* vinv, int64_t I, int R,
                    double* colsq, const int* status, int nb, cudaStream_t s) {
  const size_t smem = R <= 128 ? (size_t)R * R * 4 : 0;
  int st = ensure_dyn_smem((const void*)als_solve_kernel<CC>, 128 * 128 * 4,
                           "cudaFuncSetAttribute(als_solve)");
  if (st) return st;
  als_solve_kernel<CC><<<nb, 256, smem, s>>>(M, U, vinv, I, R, colsq, status);
  return SPM_OK;
}

int launch_als_solve(const float* M, float* U, const float* vinv, int64_t I, int R,
                     double* colsq, const int* status, int nb, cudaStream_t s) {
  const int cc = (R + 31) / 32;
  if (R <= 16)  // column norms only: the scale pass forms U again
    als_rows_kernel<float, 16, false><<<nb, 256, 0, s>>>(M, vinv, nullptr, nullptr, I, R, colsq,
                                                          status);
  else if (R <= 32)
    als_rows_kernel<float, 32, false><<<nb, 256, 0, s>>>(M, vinv, nullptr, nullptr, I, R, colsq,
                                                          status);
  else if (R <= 64)
    als_rows_kernel<float, 64, false><<<nb, 256, 0, s>>>(M, vinv, nullptr, nullptr, I, R, colsq,
                                                          status);
  else if (cc <= 1) solve_cc<1>(M, U, vinv, I, R, colsq, status, nb, s);
  else if (cc <= 2) solve_cc<2>(M, U, vinv, I, R, colsq, status, nb, s);
  else if (cc <= 4) solve_cc<4>(M, U, vinv, I, R, colsq, status, nb, s);
  else solve_cc<8>(M, U, vinv, I, R, colsq, status, nb, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "als_solve_kernel");
}

int launch_als_lambda(const double* colsq, int nb, int R, double* lam64, float* lam_out,
                      const int* status, cudaStream_t s) {
  als_lambda_kernel<<<(R + 7) / 8, 256, 0, s>>>(colsq, nb, R, lam64, lam_out, status);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "als_lambda_kernel");
}

template <typename T, int CC>
static void scale_cc(const float* U, const float* M, void* A, const double* lam64, int64_t I,
                     int R, double* mdot, const int* status, int nb, cudaStream_t s) {
  als_scale_kernel<T, CC><<<nb, 256, 0, s>>>(U, M, static_cast<T*>(A), lam64, I, R, mdot,
                                             status);
}

template <typename T>
static void rows_scale(const float* M, const float* vinv, void* A, const double* lam64, int64_t I,
                       int R, double* mdot, const int* status, int nb, cudaStream_t s) {
  T* At = static_cast<T*>(A);
  if (R <= 16)
    als_rows_kernel<T, 16, true><<<nb, 256, 0, s>>>(M, vinv, At, lam64, I, R, mdot, status);
  else if (R <= 32)
    als_rows_kernel<T, 32, true><<<nb, 256, 0, s>>>(M, vinv, At, lam64, I, R, mdot, status);
  else
    als_rows_kernel<T, 64, true><<<nb, 256, 0, s>>>(M, vinv, At, lam64, I, R, mdot, status);
}

int launch_als_scale(const float* U, const float* M, const float* vinv, void* A, int dtype,
                     const double* lam64, int64_t I, int R, double* mdot, const int* status,
                     int nb, cudaStream_t s) {
  const int cc = (R + 31) / 32;
  if (R <= 64) {
    if (dtype == SPM_DTYPE_BF16)
      rows_scale<__nv_bfloat16>(M, vinv, A, lam64, I, R, mdot, status, nb, s);
    else
      rows_scale<float>(M, vinv, A, lam64, I, R, mdot, status, nb, s);
  } else if (dtype == SPM_DTYPE_BF16) {
    if (cc <= 1) scale_cc<__nv_bfloat16, 1>(U, M, A, lam64, I, R, mdot, status, nb, s);
    else if (cc <= 2) scale_cc<__nv_bfloat16, 2>(U, M, A, lam64, I, R, mdot, status, nb, s);
    else if (cc <= 4) scale_cc<__nv_bfloat16, 4>(U, M, A, lam64, I, R, mdot, status, nb, s);
    else scale_cc<__nv_bfloat16, 8>(U, M, A, lam64, I, R, mdot, status, nb, s);
  } else {
    if (cc <= 1) scale_cc<float, 1>(U, M, A, lam64, I, R, mdot, status, nb, s);
    else if (cc <= 2) scale_cc<float, 2>(U, M, A, lam64, I, R, mdot, status, nb, s);
    else if (cc <= 4) scale_cc<float, 4>(U, M, A, lam64, I, R, mdot, status, nb, s);
    else scale_cc<float, 8>(U, M, A, lam64, I, R, mdot, status, nb, s);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "als_scale_kernel");
}

int launch_fill_f64(double* p, int n, double v, cudaStream_t s) {
  fill_f64_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, n, v);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "fill_f64_kernel");
}

int launch_als_fold_finish(void* const* factors, int dtype, const int64_t* dims, int N, int R,
                           const double* grams, double* lam64, float* lam_out, const int* status,
                           int nb, cudaStream_t s) {
  if (R > 256) return fail(SPM_ERR_UNSUPPORTED, "rank above 256");
  als_fold_lambda_kernel<<<(R + 127) / 128, 128, 0, s>>>(grams, N, R, lam64, lam_out, status);
  for (int k = 0; k < N; ++k) {
    const double* G = grams + (size_t)k * R * R;
    if (dtype == SPM_DTYPE_BF16)
      als_normalize_kernel<__nv_bfloat16><<<nb, 256, 0, s>>>(
          static_cast<__nv_bfloat16*>(factors[k]), dims[k], R, G, status);
    else
      als_normalize_kernel<float><<<nb, 256, 0, s>>>(static_cast<float*>(factors[k]), dims[k], R,
                                                     G, status);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "ALS normalisation kernels");
}

int launch_als_fit(const double* grams, int N, int R, const double* lam64, const double* mdot,
                   int nb, double normx2, double* fit_out, const int* status, cudaStream_t s) {
  als_fit_kernel<<<1, kFitThreads, 0, s>>>(grams, N, R, lam64, mdot, nb, normx2, fit_out,
                                           status);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "als_fit_kernel");
}

}  // namespace spm

namespace spm {

// Convergence check of iteration t inside a CP-ALS graph: records the fit,
// counts the iteration, and lets the next iteration's conditional node run only
// while the fit still moves by tol or more (and no mode failed).
__global__ void als_converge_kernel(const double* __restrict__ fit, const int* __restrict__ status,
                                    double* __restrict__ fits, int* __restrict__ iters, int t,
                                    double tol, cudaGraphConditionalHandle next, int has_next) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double f = fit[0];
  fits[t] = f;
  iters[0] = t + 1;
  const bool stop = status[0] != 0 || (t > 0 && fabs(f - fits[t - 1]) < tol);
  if (has_next) cudaGraphSetConditional(next, stop ? 0u : 1u);
}

int launch_als_converge(const double* fit, const int* status, double* fits, int* iters, int t,
                        double tol, cudaGraphConditionalHandle next, int has_next,
                        cudaStream_t s) {
  als_converge_kernel<<<1, 32, 0, s>>>(fit, status, fits, iters, t, tol, next, has_next);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPM_OK : cuda_fail(e, "als_converge_kernel");
}

}  // namespace spm
