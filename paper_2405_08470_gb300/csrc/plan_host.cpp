// plan_host.cpp - host-side planning of the all-mode sparse MTTKRP engine.
//
// This is the preprocessing step of the paper (Section 3.4-3.5; the
// evaluation's preprocessing is also done on the CPU): it sorts the nonzeros
// into every mode's canonical order, computes the remap ids that the dynamic
// remap (Section 3.1, Algorithm 3) scatters by, and cuts every mode into
// blocks that own disjoint output rows (Observation 2).
//
// Canonical order of mode n: lexicographic by K_n = (i_n, i_{n-1}, ..., i_0,
// i_{N-1}, ..., i_{n+1}).  A stable sort of the mode-n order by i_{n+1} is the
// mode-(n+1) order, so every order follows from the previous one by one
// stable counting pass, and next_pos_n is exactly the destination of that
// pass.  All sorts here are stable LSD radix passes (16-bit digits at most),
// parallelised over contiguous slices with per-slice histograms, so the
// result does not depend on the thread count.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <queue>
#include <thread>
#include <utility>
#include <vector>

#include "engine.h"

namespace spm {

static int pick_threads(int64_t work) {
  unsigned hw = std::thread::hardware_concurrency();
  int t = hw ? (int)hw : 4;
  if (t > 32) t = 32;
  if (work < (1 << 16)) t = 1;
  return t;
}

// Runs f(slice_index, begin, end) over T contiguous slices of [0, n).
static void parallel_slices(int T, int64_t n, const std::function<void(int, int64_t, int64_t)>& f) {
  if (T <= 1) {
    f(0, 0, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(T);
  for (int t = 0; t < T; ++t) {
    int64_t b = n * t / T, e = n * (t + 1) / T;
    th.emplace_back([&f, t, b, e] { f(t, b, e); });
  }
  for (auto& x : th) x.join();
}

static int bits_for(int64_t dim) {
  int b = 1;
  while (b < 31 && (int64_t(1) << b) < dim) ++b;
  return b;
}

// One stable counting pass: out = in ordered by digit ((key[in[p]] >> shift) & mask).
static void radix_pass(const int32_t* key, const int32_t* in, int32_t* out, int64_t n, int shift,
                       int bits, int T) {
  const int D = 1 << bits;
  const uint32_t mask = (uint32_t)D - 1;
  std::vector<int64_t> hist((size_t)T * D, 0);
  parallel_slices(T, n, [&](int t, int64_t b, int64_t e) {
    int64_t* h = &hist[(size_t)t * D];
    for (int64_t p = b; p < e; ++p) h[((uint32_t)key[in[p]] >> shift) & mask]++;
  });
  int64_t run = 0;
  for (int d = 0; d < D; ++d)
    for (int t = 0; t < T; ++t) {
      int64_t c = hist[(size_t)t * D + d];
      hist[(size_t)t * D + d] = run;
      run += c;
    }
  parallel_slices(T, n, [&](int t, int64_t b, int64_t e) {
    int64_t* h = &hist[(size_t)t * D];
    for (int64_t p = b; p < e; ++p) {
      int32_t v = in[p];
      out[h[((uint32_t)key[v] >> shift) & mask]++] = v;
    }
  });
}

// Stable sort of perm (element ids) by key[] in [0, dim): LSD passes low digit first.
static void stable_sort_by(const int32_t* key, int64_t dim, std::vector<int32_t>& perm,
                           std::vector<int32_t>& tmp, int T) {
  int bits = bits_for(dim);
  int passes = (bits + 15) / 16;
  int per = (bits + passes - 1) / passes;
  int shift = 0;
  for (int ps = 0; ps < passes; ++ps) {
    int b = std::min(per, bits - shift);
    radix_pass(key, perm.data(), tmp.data(), (int64_t)perm.size(), shift, b, T);
    perm.swap(tmp);
    shift += b;
  }
}

int default_nblk(int64_t nnz, int num_sms, int variant) {
  if (nnz <= 0) return 1;
  int64_t nb;
  if (variant == 0 || variant == 3) {
    // warp blocks (forms 0 and 3): about 16 waves of 24 warps per SM, each block >= 256
    // nonzeros, and never more than 4K nonzeros per block (measured: blocks of
    // 1.7-4K nonzeros sweep fastest on 60M-200M nonzero tensors)
    nb = std::max<int64_t>(std::min<int64_t>((int64_t)num_sms * 24 * 16, (nnz + 255) / 256),
                           (nnz + 4095) / 4096);
  } else if (variant == 2) {
    // tile form: about 16 blocks per SM, taken dynamically by the persistent
    // CTAs, each at least four 960-nonzero tiles long
    nb = std::min<int64_t>((int64_t)num_sms * 16, (nnz + 3839) / 3840);
  } else {
    // CTA blocks: about 32K nonzeros each, at least 4 per SM while each keeps
    // >= 256 nonzeros
    nb = std::max<int64_t>((nnz + 32767) / 32768,
                           std::min<int64_t>((int64_t)num_sms * 4, (nnz + 255) / 256));
  }
  return (int)std::max<int64_t>(1, std::min<int64_t>(nb, 1 << 22));
}

// Nonzeros per warp tile (the plan halves it while two 8-warp CTAs per SM would
// not fit in shared memory: a 3-stage ring of 128 32-byte nonzeros per warp
// would leave room for one, a 2-stage ring for two).
int default_tile(int) { return 128; }

// Position -> index of the nonempty row holding it (ustart ascending, size nu+1).
static inline int64_t row_index_of(const std::vector<int64_t>& ustart, int64_t pos) {
  return (int64_t)(std::upper_bound(ustart.begin(), ustart.end(), pos) - ustart.begin()) - 1;
}

// Algorithm 1 (Section 3.4): the mode's vertices (output rows) in descending
// degree, equal degrees in ascending index, each to the block holding the fewest
// hyperedges so far, ties to the lowest block.  blk[v] = block of row v.
static void lpt_assign(const std::vector<int64_t>& deg, int kappa, std::vector<int32_t>& blk,
                       std::vector<int64_t>& load) {
  const int64_t V = (int64_t)deg.size();
  std::vector<int32_t> order((size_t)V);
  for (int64_t v = 0; v < V; ++v) order[(size_t)v] = (int32_t)v;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return deg[(size_t)a] > deg[(size_t)b]; });
  using Fill = std::pair<int64_t, int32_t>;  // (hyperedges in the block, block id)
  std::priority_queue<Fill, std::vector<Fill>, std::greater<Fill>> least;
  for (int b = 0; b < kappa; ++b) least.push({0, b});
  blk.assign((size_t)V, 0);
  load.assign((size_t)kappa, 0);
  for (int32_t v : order) {
    const int32_t b = least.top().second;
    least.pop();
    blk[(size_t)v] = b;
    load[(size_t)b] += deg[(size_t)v];
    least.push({load[(size_t)b], b});
  }
}

// Blocks of Algorithm 1: block b is the range of the mode order (block, K_n)
// holding its rows; no row is split, so no block has a split head or tail and
// no kernel fills gaps between rows (the mode's empty rows are listed).
static int partition_mode_lpt(const spmttkrp_plan* p, int n, int nblk, ModeHost* out) {
  if (nblk != p->lpt_kappa)
    return fail(SPM_ERR_UNSUPPORTED, "partition 1 fixes the block count when the plan is built");
  const std::vector<int64_t>& load = p->lpt_load[(size_t)n];
  ModeHost m;
  m.nblk = nblk;
  m.bounds.assign((size_t)nblk + 1, 0);
  for (int b = 0; b < nblk; ++b) m.bounds[(size_t)b + 1] = m.bounds[(size_t)b] + load[(size_t)b];
  m.blkinfo.assign((size_t)nblk * 4, 0);
  for (int b = 0; b < nblk; ++b) {
    int32_t* bi = &m.blkinfo[(size_t)b * 4];
    bi[0] = (int32_t)m.bounds[(size_t)b];
    bi[1] = (int32_t)m.bounds[(size_t)b + 1];
    bi[2] = -1;
    bi[3] = 0;
  }
  m.last_row = -1;
  m.lpt_load = load;
  m.empty_rows = p->lpt_empty[(size_t)n];
  *out = std::move(m);
  return SPM_OK;
}

// Contiguous split of one mode with heavy-row splitting (the engine's reading
// of Section 3.4 for rows heavier than a block):
//   T = ceil(nnz / nblk); for j = 1..nblk-1, t = min(j*T, nnz), r = the row
//   holding t.  t == start(r): boundary t.  deg(r) <= T: snap to start(r) or
//   end(r), whichever is nearer (ties to start).  Else: boundary t, r is split.
int partition_mode(const spmttkrp_plan* p, int n, int nblk, ModeHost* out) {
  if (nblk < 1) return fail(SPM_ERR_INVALID_ARG, "nblk must be >= 1");
  if (p->partition == 1) return partition_mode_lpt(p, n, nblk, out);
  const int64_t nnz = p->nnz;
  const std::vector<int64_t>& us = p->row_start[n];   // nonempty-row starts (+nnz)
  const std::vector<int64_t>& ur = p->row_start[p->N + n];  // nonempty-row ids
  ModeHost m;
  m.nblk = nblk;
  m.bounds.assign((size_t)nblk + 1, 0);
  m.bounds[nblk] = nnz;
  if (nnz > 0) {
    const int64_t T = (nnz + nblk - 1) / nblk;
    for (int j = 1; j < nblk; ++j) {
      int64_t t = std::min<int64_t>((int64_t)j * T, nnz);
      if (t >= nnz) {
        m.bounds[j] = nnz;
        continue;
      }
      int64_t u = row_index_of(us, t);
      int64_t s = us[u], e = us[u + 1];
      if (t == s)
        m.bounds[j] = t;
      else if (e - s <= T)
        m.bounds[j] = (t - s <= e - t) ? s : e;
      else
        m.bounds[j] = t;
    }
    m.last_row = (int)ur.back();
  }
  // per-block descriptors
  m.blkinfo.assign((size_t)nblk * 4, 0);
  for (int b = 0; b < nblk; ++b) {
    int64_t lo = m.bounds[b], hi = m.bounds[b + 1];
    int32_t* bi = &m.blkinfo[(size_t)b * 4];
    bi[0] = (int32_t)lo;
    bi[1] = (int32_t)hi;
    bi[2] = -1;
    bi[3] = 0;
    if (lo < hi) {
      int64_t ulo = row_index_of(us, lo);
      if (lo > 0) {
        int64_t uprev = row_index_of(us, lo - 1);
        bi[2] = (int32_t)ur[uprev];
        if (uprev == ulo) bi[3] |= BLK_HEAD_SPLIT;
      }
      if (hi < nnz) {
        if (row_index_of(us, hi) == row_index_of(us, hi - 1)) bi[3] |= BLK_TAIL_SPLIT;
      }
    }
  }
  // split rows: a boundary strictly inside a row
  int64_t last_u = -1;
  for (int j = 1; j < nblk; ++j) {
    int64_t t = m.bounds[j];
    if (t <= 0 || t >= nnz) continue;
    int64_t u = row_index_of(us, t);
    if (us[u] < t && t < us[u + 1] && u != last_u) {
      SplitRow sr;
      int64_t s = us[u], e = us[u + 1];
      sr.row = (int)ur[u];
      sr.first_blk =
          (int)(std::upper_bound(m.bounds.begin(), m.bounds.end(), s) - m.bounds.begin()) - 1;
      sr.last_blk =
          (int)(std::upper_bound(m.bounds.begin(), m.bounds.end(), e - 1) - m.bounds.begin()) - 1;
      sr.first_slot = (m.bounds[sr.first_blk] == s) ? 0 : 1;
      sr.prev_row = u > 0 ? (int)ur[u - 1] : -1;
      sr.is_last = (e == nnz) ? 1 : 0;
      sr.chunk0 = m.nchunk;
      sr.pad1 = 0;
      m.nchunk += (sr.last_blk - sr.first_blk + kFixChunk) / kFixChunk;
      m.splits.push_back(sr);
      last_u = u;
    }
  }
  *out = std::move(m);
  return SPM_OK;
}

// Key columns (int32, input order) with range validation, and |X|^2.
int plan_keys(spmttkrp_plan* p, const int64_t* coo, const float* vals,
              std::vector<std::vector<int32_t>>& key) {
  const int N = p->N;
  const int64_t nnz = p->nnz;
  const int T = pick_threads(nnz);
  key.assign((size_t)N, {});
  for (int k = 0; k < N; ++k) key[k].resize((size_t)nnz);
  std::atomic<int64_t> bad{-1};
  parallel_slices(T, nnz, [&](int, int64_t b, int64_t e) {
    for (int64_t q = b; q < e; ++q)
      for (int k = 0; k < N; ++k) {
        int64_t v = coo[q * N + k];
        if (v < 0 || v >= p->dims[k]) {
          int64_t expect = -1;
          bad.compare_exchange_strong(expect, q);
          return;
        }
        key[k][q] = (int32_t)v;
      }
  });
  if (bad.load() >= 0)
    return fail(SPM_ERR_INDEX_RANGE,
                "coordinate out of range at nonzero " + std::to_string(bad.load()));

  // sum of squared values, fixed 1M chunks added in order (deterministic)
  {
    const int64_t C = 1 << 20;
    int64_t nchunk = (nnz + C - 1) / C;
    std::vector<double> part((size_t)std::max<int64_t>(nchunk, 1), 0.0);
    parallel_slices(std::min<int64_t>(T, std::max<int64_t>(nchunk, 1)), nchunk,
                    [&](int, int64_t b, int64_t e) {
                      for (int64_t c = b; c < e; ++c) {
                        double s = 0.0;
                        for (int64_t q = c * C; q < std::min(nnz, (c + 1) * C); ++q)
                          s += (double)vals[q] * (double)vals[q];
                        part[(size_t)c] = s;
                      }
                    });
    double s = 0.0;
    for (int64_t c = 0; c < nchunk; ++c) s += part[(size_t)c];
    p->normx2 = s;
  }
  return SPM_OK;
}

// Block tables of every mode from the row starts (partition 0) or Algorithm 1's
// loads (partition 1).
int plan_partitions(spmttkrp_plan* p, int nblk_opt) {
  p->mh.assign((size_t)p->N, ModeHost());
  for (int n = 0; n < p->N; ++n) {
    int nb = p->partition == 1
                 ? p->lpt_kappa
                 : (nblk_opt > 0 ? nblk_opt : default_nblk(p->nnz, p->num_sms, p->variant));
    int st = partition_mode(p, n, nb, &p->mh[(size_t)n]);
    if (st != SPM_OK) return st;
  }
  return SPM_OK;
}

int build_host_plan(spmttkrp_plan* p, const int64_t* coo, const float* vals, int nblk_opt) {
  const int N = p->N;
  const int64_t nnz = p->nnz;
  const int T = pick_threads(nnz);
  std::vector<std::vector<int32_t>> key;
  int kst = plan_keys(p, coo, vals, key);
  if (kst) return kst;

  // mode-0 order: LSD over keys i_1, i_2, ..., i_{N-1}, then i_0 (primary)
  std::vector<int32_t> perm0((size_t)nnz), tmp((size_t)nnz);
  for (int64_t q = 0; q < nnz; ++q) perm0[(size_t)q] = (int32_t)q;
  for (int j = 1; j <= N; ++j) {
    int k = j % N;
    stable_sort_by(key[k].data(), p->dims[k], perm0, tmp, T);
  }

  // duplicates: equal neighbours in mode-0 order
  std::atomic<int64_t> dup{-1};
  parallel_slices(T, std::max<int64_t>(nnz - 1, 0), [&](int, int64_t b, int64_t e) {
    for (int64_t q = b; q < e; ++q) {
      int32_t x = perm0[(size_t)q], y = perm0[(size_t)q + 1];
      bool same = true;
      for (int k = 0; k < N && same; ++k) same = key[k][x] == key[k][y];
      if (same) {
        int64_t expect = -1;
        dup.compare_exchange_strong(expect, q);
        return;
      }
    }
  });
  if (dup.load() >= 0) return fail(SPM_ERR_DUPLICATE, "duplicate coordinate in the COO input");

  // The working copy's order for mode n: K_n (partition 0), or with Algorithm 1
  // (partition 1) the nonzeros grouped by the block of their i_n, in K_n order
  // inside a block (Section 3.4: hyperedges follow their mode-n vertex).
  std::vector<std::vector<int32_t>> blk;
  if (p->partition == 1) {
    const int kappa = nblk_opt > 0 ? nblk_opt : default_nblk(nnz, p->num_sms, p->variant);
    p->lpt_kappa = kappa;
    p->lpt_load.assign((size_t)N, {});
    p->lpt_empty.assign((size_t)N, {});
    blk.assign((size_t)N, {});
    for (int n = 0; n < N; ++n) {
      std::vector<int64_t> deg((size_t)p->dims[n], 0);
      for (int64_t q = 0; q < nnz; ++q) ++deg[(size_t)key[n][(size_t)q]];
      lpt_assign(deg, kappa, blk[(size_t)n], p->lpt_load[(size_t)n]);
      for (int64_t r = 0; r < p->dims[n]; ++r)
        if (deg[(size_t)r] == 0) p->lpt_empty[(size_t)n].push_back((int32_t)r);
    }
  }
  std::vector<int32_t> bkey;
  auto order_of = [&](int n, const std::vector<int32_t>& kord) {
    std::vector<int32_t> o = kord;
    if (p->partition != 1) return o;
    bkey.resize((size_t)nnz);
    parallel_slices(T, nnz, [&](int, int64_t b, int64_t e) {
      for (int64_t q = b; q < e; ++q)
        bkey[(size_t)q] = blk[(size_t)n][(size_t)key[n][(size_t)q]];
    });
    stable_sort_by(bkey.data(), p->lpt_kappa, o, tmp, T);
    return o;
  };

  // working copy in mode-0 order: {int32 idx[N]; float val; zero padding}
  std::vector<int32_t> kcur = perm0;         // K_n order
  std::vector<int32_t> cur = order_of(0, kcur);  // order of the working copy for mode n
  const int es = p->es;
  p->h_elems.assign((size_t)nnz * es, 0);
  parallel_slices(T, nnz, [&](int, int64_t b, int64_t e) {
    for (int64_t q = b; q < e; ++q) {
      int32_t x = cur[(size_t)q];
      int32_t* d = reinterpret_cast<int32_t*>(&p->h_elems[(size_t)q * es]);
      if (p->pack.packed) {  // Section 3.5 bit fields, value in word 3
        int32_t idx[kMaxModes];
        for (int k = 0; k < N; ++k) idx[k] = key[k][x];
        pack_nonzero(p->pack, N, idx, vals[x], reinterpret_cast<uint32_t*>(d));
      } else {
        for (int k = 0; k < N; ++k) d[k] = key[k][x];
        std::memcpy(&d[N], &vals[x], 4);
      }
    }
  });

  // with p->alpha every stored nonzero also carries its remap ids: word 4 + m holds
  // its position in mode m's order (pos0 = position in the mode-0 copy)
  std::vector<int32_t> pos0;
  if (p->alpha) {
    pos0.resize((size_t)nnz);
    parallel_slices(T, nnz, [&](int, int64_t b, int64_t e) {
      for (int64_t q = b; q < e; ++q) pos0[(size_t)cur[(size_t)q]] = (int32_t)q;
    });
  }

  // per mode: nonempty rows and their starts, and next_pos_n
  p->row_start.assign((size_t)2 * N, {});
  p->h_next_pos.assign((size_t)N, {});
  std::vector<int32_t> inv((size_t)nnz);
  for (int n = 0; n < N; ++n) {
    if (p->alpha)
      parallel_slices(T, nnz, [&](int, int64_t b, int64_t e) {
        for (int64_t q = b; q < e; ++q) {
          int32_t* d = reinterpret_cast<int32_t*>(&p->h_elems[(size_t)pos0[(size_t)cur[(size_t)q]] * es]);
          d[4 + n] = (int32_t)q;
        }
      });
    // nonempty rows of mode n in the mode-n order `cur` (each row is contiguous)
    const int32_t* kn = key[n].data();
    std::vector<int64_t> cnt((size_t)T + 1, 0);
    parallel_slices(T, nnz, [&](int t, int64_t b, int64_t e) {
      int64_t c = 0;
      for (int64_t q = b; q < e; ++q)
        if (q == 0 || kn[cur[(size_t)q]] != kn[cur[(size_t)q - 1]]) ++c;
      cnt[(size_t)t + 1] = c;
    });
    for (int t = 0; t < T; ++t) cnt[(size_t)t + 1] += cnt[(size_t)t];
    int64_t nu = cnt[(size_t)T];
    std::vector<int64_t>& us = p->row_start[(size_t)n];
    std::vector<int64_t>& ur = p->row_start[(size_t)N + n];
    us.assign((size_t)nu + 1, nnz);
    ur.assign((size_t)nu, 0);
    parallel_slices(T, nnz, [&](int t, int64_t b, int64_t e) {
      int64_t c = cnt[(size_t)t];
      for (int64_t q = b; q < e; ++q)
        if (q == 0 || kn[cur[(size_t)q]] != kn[cur[(size_t)q - 1]]) {
          us[(size_t)c] = q;
          ur[(size_t)c] = kn[cur[(size_t)q]];
          ++c;
        }
    });
    // next K order: stable sort of K_n by i_{n+1}; the next working-copy order from it
    const int nx = (n + 1) % N;
    std::vector<int32_t> knext = kcur;
    stable_sort_by(key[nx].data(), p->dims[nx], knext, tmp, T);
    std::vector<int32_t> nxt = order_of(nx, knext);
    parallel_slices(T, nnz, [&](int, int64_t b, int64_t e) {
      for (int64_t q = b; q < e; ++q) inv[(size_t)nxt[(size_t)q]] = (int32_t)q;
    });
    std::vector<int32_t>& np = p->h_next_pos[(size_t)n];
    np.resize((size_t)nnz);
    parallel_slices(T, nnz, [&](int, int64_t b, int64_t e) {
      for (int64_t q = b; q < e; ++q) np[(size_t)q] = inv[(size_t)cur[(size_t)q]];
    });
    kcur.swap(knext);
    cur.swap(nxt);
  }

  return plan_partitions(p, nblk_opt);
}

}  // namespace spm
