// api.cu - the C ABI of the engine: plan lifetime, remap, per-mode compute and
// the all-mode sweep (Algorithm 5), plus plan queries and error reporting.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>

#include "als.h"
#include "engine.h"
#include "mttkrp_kernel.cuh"

namespace spm {

static thread_local std::string g_last_error;

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return SPM_ERR_CUDA;
}

int ensure_dyn_smem(const void* kernel, size_t bytes, const char* what) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;  // (kernel, device) -> limit set
  int dev = 0;
  SPM_CUDA(cudaGetDevice(&dev));
  const size_t want = std::max<size_t>(bytes, 48 * 1024);
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[std::make_pair(kernel, dev)];
  if (have >= want) return SPM_OK;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)want);
  if (e != cudaSuccess) return cuda_fail(e, what);
  have = want;
  return SPM_OK;
}

int plan_dalloc(spmttkrp_plan* p, void** ptr, size_t bytes) {
  bytes = std::max<size_t>(bytes, 16);
  if (p->max_bytes && p->dev_bytes + bytes > p->max_bytes)
    return fail(SPM_ERR_OOM, "plan device memory cap (max_bytes) exceeded");
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(SPM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  p->dev_bytes += bytes;
  return SPM_OK;
}

static void dfree(void* ptr) {
  if (ptr) cudaFree(ptr);
}

// Uploads one mode's block descriptors and split table (after (re)partitioning).
int upload_mode_tables(spmttkrp_plan* p, int n) {
  ModeHost& h = p->mh[(size_t)n];
  ModeDev& d = p->md[(size_t)n];
  if (d.blkinfo) {
    cudaFree(d.blkinfo);
    p->dev_bytes -= std::max<size_t>((size_t)d.nblk * sizeof(int4), 16);
    d.blkinfo = nullptr;
  }
  if (d.splits) {
    cudaFree(d.splits);
    p->dev_bytes -= std::max<size_t>((size_t)d.nsplit * sizeof(SplitRow), 16);
    d.splits = nullptr;
  }
  if (d.empty_rows) {
    cudaFree(d.empty_rows);
    p->dev_bytes -= std::max<size_t>((size_t)d.nempty * sizeof(int32_t), 16);
    d.empty_rows = nullptr;
  }
  d.nblk = h.nblk;
  d.nsplit = (int)h.splits.size();
  d.nchunk = h.nchunk;
  d.last_row = h.last_row;
  int st = plan_dalloc(p, (void**)&d.blkinfo, (size_t)d.nblk * sizeof(int4));
  if (st) return st;
  st = plan_dalloc(p, (void**)&d.splits, (size_t)d.nsplit * sizeof(SplitRow));
  if (st) return st;
  SPM_CUDA(cudaMemcpyAsync(d.blkinfo, h.blkinfo.data(), (size_t)d.nblk * sizeof(int4),
                           cudaMemcpyHostToDevice, p->stream));
  if (d.nsplit)
    SPM_CUDA(cudaMemcpyAsync(d.splits, h.splits.data(), (size_t)d.nsplit * sizeof(SplitRow),
                             cudaMemcpyHostToDevice, p->stream));
  d.nempty = (int)h.empty_rows.size();
  if (d.nempty) {
    st = plan_dalloc(p, (void**)&d.empty_rows, (size_t)d.nempty * sizeof(int32_t));
    if (st) return st;
    SPM_CUDA(cudaMemcpyAsync(d.empty_rows, h.empty_rows.data(), (size_t)d.nempty * sizeof(int32_t),
                             cudaMemcpyHostToDevice, p->stream));
  }
  // fix-up scratch: one R-float sum per chunk of a split row's blocks
  const size_t fneed = (size_t)std::max(d.nchunk, 1) * p->R;
  if (fneed > p->fixsum_cap) {
    if (p->d_fixsum) {
      cudaFree(p->d_fixsum);
      p->dev_bytes -= std::max<size_t>(p->fixsum_cap * 4, 16);
      p->d_fixsum = nullptr;
    }
    st = plan_dalloc(p, (void**)&p->d_fixsum, fneed * 4);
    if (st) return st;
    p->fixsum_cap = fneed;
  }
  // partial-sum buffer: 2 slots of R floats per block
  size_t need = (size_t)d.nblk * 2 * p->R;
  if (need > p->part_cap) {
    if (p->d_part) {
      cudaFree(p->d_part);
      p->dev_bytes -= std::max<size_t>(p->part_cap * 4, 16);
      p->d_part = nullptr;
    }
    st = plan_dalloc(p, (void**)&p->d_part, need * 4);
    if (st) return st;
    p->part_cap = need;
  }
  SPM_CUDA(cudaStreamSynchronize(p->stream));  // host vectors may change after return
  return SPM_OK;
}

// Index k of a packed nonzero from its words 0..2 (host side of pk_field).
uint32_t host_field(const uint32_t* w, int off, int b) {
  uint64_t x;
  if (off < 32)
    x = (((uint64_t)w[1] << 32) | w[0]) >> off;
  else if (off < 64)
    x = (((uint64_t)w[2] << 32) | w[1]) >> (off - 32);
  else
    x = (uint64_t)(w[2] >> (off - 64));
  return (uint32_t)x & ((1u << b) - 1u);
}

// Packs the N indices of one nonzero into words 0..2 (bit fields of the plan's
// widths) and the value into word 3.
void pack_nonzero(const PackInfo& pk, int N, const int32_t* idx, float v, uint32_t* w) {
  uint64_t lo = 0, hi = 0;  // bits 0..63 and 64..127 of the field
  for (int k = 0; k < N; ++k) {
    const uint64_t x = (uint32_t)idx[k];
    const int off = pk.off[k];
    if (off < 64) {
      lo |= x << off;
      if (off + pk.bits[k] > 64) hi |= x >> (64 - off);
    } else {
      hi |= x << (off - 64);
    }
  }
  w[0] = (uint32_t)lo;
  w[1] = (uint32_t)(lo >> 32);
  w[2] = (uint32_t)hi;
  std::memcpy(&w[3], &v, 4);
}

static int check_plan(spmttkrp_plan* p, bool need_device = true) {
  if (!p || p->destroyed) return fail(SPM_ERR_INVALID_ARG, "null or destroyed plan");
  if (need_device && p->host_only) return fail(SPM_ERR_STATE, "plan was built host-only");
  return SPM_OK;
}

static int check_factors(const spmttkrp_plan* p, const void* const* f, int skip) {
  if (!f) return fail(SPM_ERR_INVALID_ARG, "factors array is null");
  for (int k = 0; k < p->N; ++k)
    if (k != skip && !f[k]) return fail(SPM_ERR_INVALID_ARG, "null factor pointer");
  return SPM_OK;
}

// One remap-only pass of the working copy: mode cur_mode -> cur_mode + 1.
// With keep_base, mode N-1 -> 0 needs no pass: the mode-0 copy is resident.
static int remap_step(spmttkrp_plan* p) {
  const int m = p->cur_mode;
  if (p->keep_base && m == p->N - 1) {
    p->cur_mode = 0;
    return SPM_OK;
  }
  const int dst = next_buf(p);
  int st = p->worders
               ? launch_remap_ordered(cur_elems(p), p->d_elem[dst], p->nnz, m, p->d_err, p->stream)
               : launch_remap_only(cur_elems(p), p->d_elem[dst], p->md[(size_t)m].next_pos,
                                   p->nnz, p->es, p->stream);
  if (st) return st;
  p->cur_buf = dst;
  p->cur_mode = (m + 1) % p->N;
  return SPM_OK;
}

static int check_device_word(spmttkrp_plan* p) {
  SPM_CUDA(cudaStreamSynchronize(p->stream));
  int h = 0;
  SPM_CUDA(cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    SPM_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
    if (h & 2)
      return fail(SPM_ERR_STATE,
                  "a stored nonzero's write order or remap id was out of range (store skipped)");
    return fail(SPM_ERR_TIMEOUT, "a bounded device wait gave up (bulk copy did not complete)");
  }
  return SPM_OK;
}

// Mode-n fused compute + remap on an explicit element copy pair.
int run_mode(spmttkrp_plan* p, int mode, const void* const* factors, float* out,
             const uint8_t* ein, uint8_t* eout, const float* scale, double* loss_part) {
  if (p->nnz == 0) return launch_zero_rows(out, p->dims[(size_t)mode], p->R, p->stream);
  const ModeDev& d = p->md[(size_t)mode];
  MttkrpArgs a;
  std::memset(&a, 0, sizeof(a));
  a.elems_in = ein;
  a.elems_out = eout;
  a.next_pos = d.next_pos;
  a.blkinfo = d.blkinfo;
  a.nblk = d.nblk;
  for (int k = 0; k < p->N; ++k) a.factors[k] = factors[k];
  a.out = out;
  a.out_rows = p->dims[(size_t)mode];
  a.R = p->R;
  a.mode = mode;
  a.nmodes = p->N;
  a.es = p->es;
  a.tile = p->tile;
  a.part = p->d_part;
  a.last_row = d.last_row;
  a.err = p->d_err;
  a.scale = scale;
  a.dtype = p->dtype;
  a.variant = p->variant;
  a.hints = p->hints;
  a.unroll = p->unroll;
  a.stages = p->stages;
  a.no_fill = p->partition == 1;
  a.wait_ns = p->wait_ns;
  a.stall_test = p->stall_test;
  a.nnz = p->nnz;
  a.grid_ctas = p->num_sms;
  a.sched = p->d_err + 1;
  a.pk = p->pack;
  if (p->pack.packed && a.variant == 1) a.variant = 0;  // form 1 reads plain indices only
  a.hot_flags = p->hot_rows > 0 && (p->hints & 4);  // read by the tile form only
  a.loss_part = loss_part;  // the fused CP-loss pass (always the warp-block form)
  if (loss_part) a.variant = 0;
  if ((a.variant == 2 || a.variant == 3) && !p->worders) a.variant = 0;  // no write orders
  // the pass's elements carry their remap ids: word 4 + (next mode)
  a.alpha_word = p->alpha ? 4 + (mode + 1) % p->N : 0;
  int st = launch_mttkrp(a, p->stream);
  if (st) return st;
  st = launch_fixup(p->d_part, d.splits, d.nsplit, d.nchunk, p->d_fixsum, out, a.out_rows, p->R,
                    scale, p->stream);
  if (st) return st;
  return launch_zero_listed_rows(out, d.empty_rows, d.nempty, p->R, p->stream);
}

const char* nvtx_mode_name(int n) {
  static const char* names[] = {
      "spmttkrp mode 0",  "spmttkrp mode 1",  "spmttkrp mode 2",  "spmttkrp mode 3",
      "spmttkrp mode 4",  "spmttkrp mode 5",  "spmttkrp mode 6",  "spmttkrp mode 7",
      "spmttkrp mode 8",  "spmttkrp mode 9",  "spmttkrp mode 10", "spmttkrp mode 11",
      "spmttkrp mode 12", "spmttkrp mode 13", "spmttkrp mode 14", "spmttkrp mode 15"};
  return (n >= 0 && n < 16) ? names[n] : "spmttkrp mode";
}

int compute_mode(spmttkrp_plan* p, int mode, const void* const* factors, float* out,
                 bool keep_order) {
  NvtxRange range(nvtx_mode_name(mode));
  while (p->cur_mode != mode) {
    int st = remap_step(p);
    if (st) return st;
  }
  if (keep_order)  // no remap: the working copy stays in mode order
    return run_mode(p, mode, factors, out, cur_elems(p), nullptr, nullptr);
  // with keep_base the last mode's pass writes no remap (mode-0 copy resident)
  const bool last = p->keep_base && mode == p->N - 1;
  const int dst = next_buf(p);
  int st = run_mode(p, mode, factors, out, cur_elems(p), last ? nullptr : p->d_elem[dst],
                    nullptr);
  if (st) return st;
  if (p->nnz > 0 && !last) p->cur_buf = dst;
  p->cur_mode = (mode + 1) % p->N;
  return SPM_OK;
}

static int sweep_eager(spmttkrp_plan* p, const void* const* factors, float* const* outs) {
  const int start = p->cur_mode;
  for (int i = 0; i < p->N; ++i) {
    const int n = (start + i) % p->N;
    int st = compute_mode(p, n, factors, outs[n], false);
    if (st) return st;
  }
  return SPM_OK;
}

}  // namespace spm

using namespace spm;

extern "C" {

int spmttkrp_version(void) { return 100; }

const char* spmttkrp_last_error(void) { return g_last_error.c_str(); }

int spmttkrp_opts_init(spmttkrp_opts_t* o) {
  if (!o) return fail(SPM_ERR_INVALID_ARG, "opts is null");
  std::memset(o, 0, sizeof(*o));
  return SPM_OK;
}

int spmttkrp_plan_create(spmttkrp_plan_t* out, const int64_t* coo, const float* vals,
                         int64_t nnz, const int64_t* dims, int nmodes, int rank,
                         const spmttkrp_opts_t* opts) {
  if (!out) return fail(SPM_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  NvtxRange range("spmttkrp plan build");
  if (nmodes < 2) return fail(SPM_ERR_INVALID_ARG, "nmodes must be >= 2");
  if (nmodes > kMaxModes) return fail(SPM_ERR_UNSUPPORTED, "nmodes > 16");
  if (rank < 1) return fail(SPM_ERR_INVALID_ARG, "rank must be >= 1");
  if (rank > kMaxRank) return fail(SPM_ERR_UNSUPPORTED, "rank > 256");
  if (nnz < 0) return fail(SPM_ERR_INVALID_ARG, "nnz < 0");
  if (nnz >= (int64_t(1) << 31) - 4) return fail(SPM_ERR_UNSUPPORTED, "nnz >= 2^31");
  if (!dims) return fail(SPM_ERR_INVALID_ARG, "dims is null");
  if (nnz > 0 && (!coo || !vals)) return fail(SPM_ERR_INVALID_ARG, "coo or vals is null");
  for (int k = 0; k < nmodes; ++k) {
    if (dims[k] < 1) return fail(SPM_ERR_INVALID_ARG, "dims[k] must be >= 1");
    if (dims[k] > 2147483647LL) return fail(SPM_ERR_UNSUPPORTED, "dims[k] > 2^31-1");
  }
  spmttkrp_opts_t o;
  spmttkrp_opts_init(&o);
  if (opts) o = *opts;
  if (o.factor_dtype != SPM_DTYPE_F32 && o.factor_dtype != SPM_DTYPE_BF16)
    return fail(SPM_ERR_INVALID_ARG, "factor_dtype must be F32 or BF16");
  if (o.partition != 0 && o.partition != 1)
    return fail(SPM_ERR_INVALID_ARG, "partition must be 0 (contiguous split) or 1 (Algorithm 1)");
  if (o.tile != 0 && o.tile != 32 && o.tile != 64 && o.tile != 128 && o.tile != 256)
    return fail(SPM_ERR_INVALID_ARG, "tile must be 0, 32, 64, 128 or 256");
  if (o.nblk < 0) return fail(SPM_ERR_INVALID_ARG, "nblk must be >= 0");
  if (o.variant < 0 || o.variant > 3)
    return fail(SPM_ERR_INVALID_ARG, "variant must be 0, 1, 2 or 3");
  if (o.unroll != 0 && o.unroll != 4 && o.unroll != 8)
    return fail(SPM_ERR_INVALID_ARG, "unroll must be 0, 4 or 8");
  if (o.stages != 0 && (o.stages < 2 || o.stages > 4))
    return fail(SPM_ERR_INVALID_ARG, "stages must be 0 or in [2, 4]");
  if (o.cache_hints < -1 || o.cache_hints > 7)
    return fail(SPM_ERR_INVALID_ARG, "cache_hints must be in [-1, 7]");
  if (o.keep_base != 0 && o.keep_base != 1)
    return fail(SPM_ERR_INVALID_ARG, "keep_base must be 0 or 1");
  if (o.wait_limit_ns < 0) return fail(SPM_ERR_INVALID_ARG, "wait_limit_ns must be >= 0");
  if (o.inject_wait_stall != 0 && o.inject_wait_stall != 1)
    return fail(SPM_ERR_INVALID_ARG, "inject_wait_stall must be 0 or 1");

  spmttkrp_plan* p = new (std::nothrow) spmttkrp_plan();
  if (!p) return fail(SPM_ERR_OOM, "host allocation failed");
  p->N = nmodes;
  p->R = rank;
  p->nnz = nnz;
  p->dtype = o.factor_dtype;
  p->variant = o.variant;
  p->unroll = o.unroll ? o.unroll : 8;
  p->stages = o.stages;
  p->hints = o.cache_hints == 0 ? 3 : (o.cache_hints < 0 ? 0 : o.cache_hints);
  p->checks = o.checks;
  p->keep_base = o.keep_base;
  p->partition = o.partition;
  p->wait_ns = (unsigned long long)o.wait_limit_ns;
  p->stall_test = o.inject_wait_stall;
  p->host_only = o.host_only;
  p->max_bytes = o.max_bytes;
  p->stream = (cudaStream_t)o.stream;
  p->dims.assign(dims, dims + nmodes);
  // a nonzero is N int32 indices and an FP32 value; by default it is stored in a
  // whole 32-byte sector when it fits one, so that remap stores never write part
  // of a sector (which costs DRAM a read of the old sector first)
  const int es_min = ((4 * nmodes + 4) + 15) & ~15;
  p->es = es_min <= 32 ? 32 : es_min;
  if (o.element_bytes != 0) {
    // 16 bytes with 4 or more modes: the indices packed into bit fields (Section
    // 3.5) of their exact widths, when they fit 96 bits
    int packed_bits = 0;
    for (int k = 0; k < nmodes; ++k) {
      int b = 1;
      while (b < 31 && (int64_t(1) << b) < dims[k]) ++b;
      p->pack.off[k] = (uint8_t)std::min(packed_bits, 255);
      p->pack.bits[k] = (uint8_t)b;
      packed_bits += b;
    }
    const bool pack = o.element_bytes == 16 && nmodes >= 4 && packed_bits <= 96;
    if ((o.element_bytes != 16 && o.element_bytes != 32) ||
        (o.element_bytes < es_min && !pack)) {
      delete p;
      return fail(SPM_ERR_INVALID_ARG,
                  "element_bytes must be 0, 16 (up to 3 modes, or packed indices of at most "
                  "96 bits) or 32 (up to 7 modes)");
    }
    p->es = o.element_bytes;
    p->pack.packed = pack ? 1 : 0;
  }
  p->pack.vword = p->pack.packed ? 3 : nmodes;
  // 3-mode nonzeros in 32-byte sectors carry their remap ids in the padding (the
  // element tuple of Section 3.5), so the fused pass reads no next_pos array
  p->alpha = (nmodes == 3 && p->es == 32) ? 1 : 0;
  // ring depth: 2 stages for 32-byte and wider nonzeros (a tile of 128 of
  // them is 4 KB, so two in flight keep the copies ahead), 3 for 16-byte ones
  if (!p->stages) p->stages = p->es >= 32 ? 2 : 3;
  p->tile = o.tile ? o.tile : default_tile(p->es);
  // a default tile keeps two CTAs per SM (<= 110 KB each); a requested one is
  // only cut down to what one CTA can hold
  const size_t smem_cap = (o.tile ? 200 : 110) * 1024;
  while (p->tile > 32 && mttkrp_smem_bytes(p->es, p->tile, p->R, p->dtype, p->stages) > smem_cap)
    p->tile /= 2;
  if (!p->host_only) {
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "cudaGetDevice");
    }
  }
  // The orders (sorts, remap ids, working copy) are built on the device for a
  // device plan with the contiguous split, unless the host is asked for; the
  // partition itself always runs on the host.
  const bool device_orders =
      !p->host_only && p->nnz > 0 && p->partition == 0 && !o.plan_on_host;
  std::vector<std::vector<int32_t>> keys;
  int st;
  try {
    st = device_orders ? plan_keys(p, coo, vals, keys) : build_host_plan(p, coo, vals, o.nblk);
  } catch (const std::bad_alloc&) {
    st = fail(SPM_ERR_OOM, "host allocation failed while planning");
  }
  if (st) {
    delete p;
    return st;
  }
  if (!p->host_only) {
    const int N = p->N;
    p->md.assign((size_t)N, ModeDev());
    const size_t eb = (size_t)p->nnz * p->es;
    st = plan_dalloc(p, (void**)&p->d_elem[0], eb);
    if (!st) st = plan_dalloc(p, (void**)&p->d_elem[1], eb);
    if (!st && p->keep_base) st = plan_dalloc(p, (void**)&p->d_base, eb);
    // d_err[0]: device error word; d_err[1]: the tile form's block counter
    if (!st) st = plan_dalloc(p, (void**)&p->d_err, 4 * sizeof(int));
    if (!st) {
      cudaError_t e = cudaMemsetAsync(p->d_err, 0, 4 * sizeof(int), p->stream);
      if (e == cudaSuccess && eb && !device_orders)
        e = cudaMemcpyAsync(p->keep_base ? p->d_base : p->d_elem[0], p->h_elems.data(), eb,
                            cudaMemcpyHostToDevice, p->stream);
      if (e != cudaSuccess) st = cuda_fail(e, "upload of the working copy");
    }
    for (int n = 0; n < N && !st; ++n) {
      ModeDev& d = p->md[(size_t)n];
      st = plan_dalloc(p, (void**)&d.next_pos, ((size_t)p->nnz + 4) * sizeof(int32_t));
      if (!st) {
        cudaError_t e = cudaMemsetAsync(d.next_pos, 0, ((size_t)p->nnz + 4) * 4, p->stream);
        if (e == cudaSuccess && p->nnz && !device_orders)
          e = cudaMemcpyAsync(d.next_pos, p->h_next_pos[(size_t)n].data(),
                              (size_t)p->nnz * sizeof(int32_t), cudaMemcpyHostToDevice, p->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "upload of next_pos");
      }
    }
    if (!st && device_orders) {
      NvtxRange orders("spmttkrp plan orders on the device");
      std::vector<int32_t*> np((size_t)N);
      for (int n = 0; n < N; ++n) np[(size_t)n] = p->md[(size_t)n].next_pos;
      try {
        st = build_device_orders(p, keys, vals, p->keep_base ? p->d_base : p->d_elem[0],
                                 np.data());
        std::vector<std::vector<int32_t>>().swap(keys);
        if (!st) st = plan_partitions(p, o.nblk);
      } catch (const std::bad_alloc&) {
        st = fail(SPM_ERR_OOM, "host allocation failed while planning");
      }
    }
    // the tile form's write orders (3 modes, nonzeros carrying remap ids)
    if (!st && p->alpha)
      st = build_write_orders(p, p->keep_base ? p->d_base : p->d_elem[0]);
    if (!st && p->alpha) st = build_hot_flags(p, p->keep_base ? p->d_base : p->d_elem[0]);
    for (int n = 0; n < N && !st; ++n) st = upload_mode_tables(p, n);
    if (!st) {
      cudaError_t e = cudaStreamSynchronize(p->stream);
      if (e != cudaSuccess) st = cuda_fail(e, "plan upload");
    }
    if (st) {
      spmttkrp_plan_destroy(p);
      return st;
    }
    // the device holds the data now
    std::vector<uint8_t>().swap(p->h_elems);
    std::vector<std::vector<int32_t>>().swap(p->h_next_pos);
  }
  *out = p;
  return SPM_OK;
}

int spmttkrp_plan_destroy(spmttkrp_plan_t p) {
  if (!p || p->destroyed) return fail(SPM_ERR_INVALID_ARG, "null or destroyed plan");
  if (!p->host_only) cudaStreamSynchronize(p->stream);
  for (auto& g : p->sweep_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& g : p->als_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& g : p->als_run_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (int i = 0; i < 3; ++i) dfree(p->d_elem[i]);
  dfree(p->d_base);
  for (auto& d : p->md) {
    dfree(d.next_pos);
    dfree(d.blkinfo);
    dfree(d.splits);
    dfree(d.empty_rows);
  }
  dfree(p->d_part);
  dfree(p->d_fixsum);
  dfree(p->d_err);
  dfree(p->d_M);
  dfree(p->d_U);
  dfree(p->d_gram);
  dfree(p->d_gpart);
  dfree(p->d_red);
  dfree(p->d_chol);
  dfree(p->d_scal);
  dfree(p->d_vinv);
  dfree(p->d_lossgrad);
  dfree(p->d_fits);
  dfree(p->d_lpart);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->als_side) cudaStreamDestroy(p->als_side);
  if (p->als_fork) cudaEventDestroy(p->als_fork);
  if (p->als_join) cudaEventDestroy(p->als_join);
  p->destroyed = true;
  delete p;
  return SPM_OK;
}

int spmttkrp_set_stream(spmttkrp_plan_t p, void* stream) {
  int st = check_plan(p, false);
  if (st) return st;
  p->stream = (cudaStream_t)stream;
  return SPM_OK;
}

int spmttkrp_remap(spmttkrp_plan_t p, int mode) {
  int st = check_plan(p);
  if (st) return st;
  if (mode < 0 || mode >= p->N) return fail(SPM_ERR_INVALID_ARG, "mode out of range");
  while (p->cur_mode != mode) {
    st = remap_step(p);
    if (st) return st;
  }
  return SPM_OK;
}

int spmttkrp_compute_ex(spmttkrp_plan_t p, int mode, const void* const* factors, float* out,
                        int flags) {
  int st = check_plan(p);
  if (st) return st;
  if (mode < 0 || mode >= p->N) return fail(SPM_ERR_INVALID_ARG, "mode out of range");
  if (flags & ~SPM_COMPUTE_KEEP_ORDER) return fail(SPM_ERR_INVALID_ARG, "unknown compute flag");
  st = check_factors(p, factors, mode);
  if (st) return st;
  if (!out) return fail(SPM_ERR_INVALID_ARG, "out is null");
  st = compute_mode(p, mode, factors, out, (flags & SPM_COMPUTE_KEEP_ORDER) != 0);
  if (st) return st;
  if (p->checks) return check_device_word(p);
  return SPM_OK;
}

int spmttkrp_compute(spmttkrp_plan_t p, int mode, const void* const* factors, float* out) {
  return spmttkrp_compute_ex(p, mode, factors, out, 0);
}

int spmttkrp_sweep(spmttkrp_plan_t p, const void* const* factors, float* const* outs,
                   int flags) {
  NvtxRange range("spmttkrp sweep");
  int st = check_plan(p);
  if (st) return st;
  st = check_factors(p, factors, -1);
  if (st) return st;
  if (!outs) return fail(SPM_ERR_INVALID_ARG, "outs is null");
  for (int k = 0; k < p->N; ++k)
    if (!outs[k]) return fail(SPM_ERR_INVALID_ARG, "null output pointer");
  if (!(flags & SPM_SWEEP_GRAPH)) {
    st = sweep_eager(p, factors, outs);
    if (st) return st;
    return p->checks ? check_device_word(p) : SPM_OK;
  }
  // graph replay: one captured graph per (pointers, buffer parity, start mode)
  std::vector<const void*> key;
  for (int k = 0; k < p->N; ++k) key.push_back(factors[k]);
  for (int k = 0; k < p->N; ++k) key.push_back(outs[k]);
  key.push_back((const void*)(intptr_t)(p->cur_buf * 64 + p->cur_mode));
  GraphCache* hit = nullptr;
  for (auto& g : p->sweep_graphs)
    if (g.key == key) hit = &g;
  const int buf0 = p->cur_buf, mode0 = p->cur_mode;
  if (!hit) {
    // first run eagerly: configures every kernel outside of stream capture
    st = sweep_eager(p, factors, outs);
    if (st) return st;
    const int buf1 = p->cur_buf, mode1 = p->cur_mode;
    p->cur_buf = buf0;
    p->cur_mode = mode0;
    cudaGraph_t g = nullptr;
    // capture on an internal stream (the legacy default stream cannot capture)
    if (!p->cap_stream) SPM_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = p->stream;
    p->stream = p->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      p->stream = user;
      return cuda_fail(e, "cudaStreamBeginCapture(sweep)");
    }
    st = sweep_eager(p, factors, outs);
    e = cudaStreamEndCapture(p->stream, &g);
    p->stream = user;
    p->cur_buf = buf1;
    p->cur_mode = mode1;
    if (st) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(sweep)");
    GraphCache gc;
    gc.key = key;
    gc.end_buf = buf1;
    gc.end_mode = mode1;
    e = cudaGraphInstantiate(&gc.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(sweep)");
    if (p->sweep_graphs.size() >= 8) {
      cudaGraphExecDestroy(p->sweep_graphs.front().exec);
      p->sweep_graphs.erase(p->sweep_graphs.begin());
    }
    p->sweep_graphs.push_back(gc);
    return p->checks ? check_device_word(p) : SPM_OK;
  }
  SPM_CUDA(cudaGraphLaunch(hit->exec, p->stream));
  p->cur_buf = hit->end_buf;
  p->cur_mode = hit->end_mode;
  return p->checks ? check_device_word(p) : SPM_OK;
}

int spmttkrp_plan_query(spmttkrp_plan_t p, int what, int mode, void* dst, size_t bytes) {
  int st = check_plan(p, false);
  if (st) return st;
  if (!dst) return fail(SPM_ERR_INVALID_ARG, "dst is null");
  const int N = p->N;
  const int64_t nnz = p->nnz;
  auto need = [&](size_t b) -> int {
    return bytes < b ? fail(SPM_ERR_INVALID_ARG, "destination too small") : SPM_OK;
  };
  if (what != SPM_Q_INFO && what != SPM_Q_ELEMS && what != SPM_Q_VALS && what != SPM_Q_RAW &&
      (mode < 0 || mode >= N))
    return fail(SPM_ERR_INVALID_ARG, "mode out of range");
  switch (what) {
    case SPM_Q_INFO: {
      if ((st = need(16 * sizeof(int64_t)))) return st;
      int m = (mode >= 0 && mode < N) ? mode : 0;
      int64_t* o = (int64_t*)dst;
      std::memset(o, 0, 16 * sizeof(int64_t));
      o[0] = nnz;
      o[1] = N;
      o[2] = p->R;
      o[3] = p->es;
      o[4] = p->cur_mode;
      o[5] = p->dtype;
      o[6] = p->tile;
      o[7] = p->mh[(size_t)m].nblk;
      o[8] = (int64_t)p->mh[(size_t)m].splits.size();
      int64_t launches = 0;
      for (int n = 0; n < N; ++n)
        launches += 1 + (p->mh[(size_t)n].splits.empty() ? 0 : 2) +
                    (p->mh[(size_t)n].empty_rows.empty() ? 0 : 1);
      o[9] = nnz > 0 ? launches : N;
      o[10] = (int64_t)p->dev_bytes;
      o[11] = p->cur_buf;
      o[12] = p->host_only;
      o[13] = p->num_sms;
      std::memcpy(&o[14], &p->normx2, 8);
      o[15] = lane_config(p->R, p->dtype, true).L;
      o[12] = (int64_t)p->host_only | ((int64_t)(p->variant & 1) << 1) |
              ((int64_t)p->keep_base << 2) | ((int64_t)p->stages << 3) |
              ((int64_t)p->partition << 6) | ((int64_t)p->alpha << 7) |
              ((int64_t)p->variant << 8) | ((int64_t)p->worders << 10) |
              ((int64_t)p->hot_rows << 11);
      return SPM_OK;
    }
    case SPM_Q_NEXT_POS: {
      if ((st = need((size_t)nnz * 4))) return st;
      if (nnz == 0) return SPM_OK;
      if (p->host_only) {
        std::memcpy(dst, p->h_next_pos[(size_t)mode].data(), (size_t)nnz * 4);
        return SPM_OK;
      }
      SPM_CUDA(cudaStreamSynchronize(p->stream));
      SPM_CUDA(cudaMemcpy(dst, p->md[(size_t)mode].next_pos, (size_t)nnz * 4,
                          cudaMemcpyDeviceToHost));
      return SPM_OK;
    }
    case SPM_Q_BOUNDS: {
      const ModeHost& h = p->mh[(size_t)mode];
      if ((st = need(h.bounds.size() * 8))) return st;
      std::memcpy(dst, h.bounds.data(), h.bounds.size() * 8);
      return SPM_OK;
    }
    case SPM_Q_SPLITS: {
      const ModeHost& h = p->mh[(size_t)mode];
      if ((st = need(h.splits.size() * 24))) return st;
      int64_t* o = (int64_t*)dst;
      for (size_t i = 0; i < h.splits.size(); ++i) {
        o[3 * i] = h.splits[i].row;
        o[3 * i + 1] = h.splits[i].first_blk;
        o[3 * i + 2] = h.splits[i].last_blk;
      }
      return SPM_OK;
    }
    case SPM_Q_ELEMS:
    case SPM_Q_VALS: {
      const size_t per = (what == SPM_Q_ELEMS) ? (size_t)N * 4 : 4;
      if ((st = need((size_t)nnz * per))) return st;
      if (nnz == 0) return SPM_OK;
      std::vector<uint8_t> tmp;
      const uint8_t* src;
      if (p->host_only) {
        src = p->h_elems.data();
      } else {
        tmp.resize((size_t)nnz * p->es);
        SPM_CUDA(cudaStreamSynchronize(p->stream));
        SPM_CUDA(cudaMemcpy(tmp.data(), cur_elems(p), tmp.size(), cudaMemcpyDeviceToHost));
        src = tmp.data();
      }
      uint8_t* o = (uint8_t*)dst;
      for (int64_t q = 0; q < nnz; ++q) {
        const uint8_t* e = src + (size_t)q * p->es;
        if (what == SPM_Q_ELEMS) {
          if (p->pack.packed) {  // bit fields of words 0..2
            uint32_t w[3];
            std::memcpy(w, e, 12);
            int32_t* oi = reinterpret_cast<int32_t*>(o + (size_t)q * N * 4);
            for (int k = 0; k < N; ++k) oi[k] = (int32_t)host_field(w, p->pack.off[k],
                                                                    p->pack.bits[k]);
          } else {
            std::memcpy(o + (size_t)q * N * 4, e, (size_t)N * 4);
          }
        } else {
          std::memcpy(o + (size_t)q * 4, e + (size_t)p->pack.vword * 4, 4);
        }
      }
      return SPM_OK;
    }
    case SPM_Q_RAW: {
      const size_t bytes = (size_t)nnz * p->es;
      if ((st = need(bytes))) return st;
      if (nnz == 0) return SPM_OK;
      if (p->host_only) {
        std::memcpy(dst, p->h_elems.data(), bytes);
        return SPM_OK;
      }
      SPM_CUDA(cudaStreamSynchronize(p->stream));
      SPM_CUDA(cudaMemcpy(dst, cur_elems(p), bytes, cudaMemcpyDeviceToHost));
      return SPM_OK;
    }
    default:
      return fail(SPM_ERR_INVALID_ARG, "unknown query");
  }
}

int spmttkrp_device_status(spmttkrp_plan_t p) {
  int st = check_plan(p);
  if (st) return st;
  return check_device_word(p);
}

}  // extern "C"
