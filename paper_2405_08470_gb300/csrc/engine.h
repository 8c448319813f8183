// engine.h - internal declarations shared by the host plan builder, the
// kernels and the C ABI of the all-mode sparse MTTKRP engine.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/spmttkrp.h"

namespace spm {

constexpr int kMaxModes = 16;
constexpr int kMaxRank = 256;
constexpr int kThreads = 256;  // threads per CTA of the fused kernel

// Stored layout of a nonzero's indices: plain (N int32 words, the value in word
// N) or packed (Section 3.5: index k in bits [off[k], off[k] + bits[k]) of the
// 96-bit little-endian field in words 0..2, the value in word 3; 16 bytes for
// up to 6 modes whose index widths sum to at most 96 bits).
struct PackInfo {
  int packed = 0;
  int vword = 0;  // word of the FP32 value
  uint8_t off[kMaxModes] = {};
  uint8_t bits[kMaxModes] = {};
};

// Per-block descriptor of one mode's contiguous split (int4 on the device):
//   x = first position, y = one past the last position,
//   z = row of position x-1 (the row before the block; -1 for none),
//   w = flags: bit0 = the block's first row started in an earlier block,
//              bit1 = the block's last row continues into a later block.
enum { BLK_HEAD_SPLIT = 1, BLK_TAIL_SPLIT = 2 };

// Split-row descriptor (int4 pairs on the device):
//   a = {row, first_blk, last_blk, slot of first_blk (0 or 1)}
//   b = {row before this row (-1 for none), 1 if it is the last nonempty row, 0, 0}
struct SplitRow {
  int row, first_blk, last_blk, first_slot;
  int prev_row, is_last;
  int chunk0;  // the row's first chunk (of kFixChunk blocks) in the fix-up's scratch
  int pad1;
};
constexpr int kFixChunk = 256;  // blocks summed by one CTA of the fix-up's first pass

// Host-side result of planning one mode.
struct ModeHost {
  int nblk = 0;
  std::vector<int64_t> bounds;     // nblk + 1
  std::vector<int32_t> blkinfo;    // 4 * nblk
  std::vector<SplitRow> splits;    // ascending rows
  int nchunk = 0;                  // fix-up chunks over all split rows
  int last_row = -1;               // row of position nnz-1
  // partition 1 (Algorithm 1): nonzeros per block and the rows with none
  std::vector<int64_t> lpt_load;
  std::vector<int32_t> empty_rows;
};

// Device tables of one mode.
struct ModeDev {
  int nblk = 0;
  int nsplit = 0;
  int last_row = -1;
  int4* blkinfo = nullptr;
  SplitRow* splits = nullptr;
  int32_t* empty_rows = nullptr;  // partition 1: rows of this mode with no nonzero
  int nempty = 0;
  int nchunk = 0;                  // fix-up chunks of this mode's split rows
  int32_t* next_pos = nullptr;  // nnz (+4 padding ints)
};

struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;
  int end_buf = 0, end_mode = 0;  // working-copy state after one replay
};

}  // namespace spm

struct spmttkrp_plan {
  int N = 0, R = 0, dtype = 0, tile = 512, checks = 0, host_only = 0;
  int variant = 0;  // fused-kernel form (see MttkrpArgs::variant)
  int hints = 3;    // L2 cache policy bits of the fused kernel (see MttkrpArgs)
  int unroll = 0;   // nonzeros in flight per lane group of the warp-block form
  int stages = 3;   // tiles per warp ring of the warp-block form
  unsigned long long wait_ns = 0;  // first-wait limit of the fused kernels (0 = 2 s)
  int stall_test = 0;              // test only: the fused kernels' first wait never completes
  int64_t nnz = 0;
  int es = 16;  // element stride in bytes: {int32 idx[N]; float val}, rounded up to 16
  std::vector<int64_t> dims;
  size_t max_bytes = 0, dev_bytes = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // internal stream used only for graph capture
  // CP-ALS: a side stream that forms each updated factor's Gram and the next
  // mode's Cholesky beside that mode's spMTTKRP, and its fork / join events
  cudaStream_t als_side = nullptr;
  cudaEvent_t als_fork = nullptr, als_join = nullptr;
  int device = 0;
  int num_sms = 148;

  // host copies kept for re-partitioning and queries: row_start[n] = starts of
  // the nonempty rows of mode n (+ nnz), row_start[N + n] = their row ids
  std::vector<std::vector<int64_t>> row_start;
  std::vector<std::vector<int32_t>> h_next_pos;  // host-only plans keep these
  std::vector<spm::ModeHost> mh;                 // per mode
  std::vector<uint8_t> h_elems;                  // host-only plans: mode-0 working copy
  double normx2 = 0.0;                           // sum of squared values (FP64)

  // device state
  uint8_t* d_elem[3] = {nullptr, nullptr, nullptr};  // working copy ping/pong + residual copy
  int cur_buf = 0;   // which of d_elem[0..1] holds the working copy
  int cur_mode = 0;  // canonical order the working copy is in
  float* d_fixsum = nullptr;     // fix-up scratch: one R-float sum per chunk
  size_t fixsum_cap = 0;         // floats
  int keep_base = 0;             // the mode-0 copy stays resident in d_base
  int partition = 0;             // 0 = contiguous split, 1 = Algorithm 1 (LPT)
  int alpha = 0;  // stored nonzeros carry their remap ids: words 4..6 = position in
                  // the mode-0/1/2 order (3 modes in 32-byte sectors)
  int worders = 0;  // word 7 holds the write orders of the tile form (form 2)
  int hot_rows = 0;   // rows per factor marked hot (bit 31 of words 4..6); 0 = none
  spm::PackInfo pack;  // index layout of the stored nonzeros (packed: 16 bytes, 4-6 modes)
  int lpt_kappa = 0;                               // partition 1: blocks per mode
  std::vector<std::vector<int64_t>> lpt_load;      // partition 1: nonzeros per block
  std::vector<std::vector<int32_t>> lpt_empty;     // partition 1: rows with no nonzero
  uint8_t* d_base = nullptr;     // read-only mode-0 copy (keep_base only)
  std::vector<spm::ModeDev> md;
  float* d_part = nullptr;   // split-row partials: max nblk x 2 x R
  size_t part_cap = 0;       // floats
  int* d_err = nullptr;      // device error word [0] and the tile form's block counter [1]
  // ALS / CP-loss scratch (allocated on first use)
  float* d_M = nullptr;       // max_n dims[n] x R: spMTTKRP output of the ALS mode
  float* d_U = nullptr;       // max_n dims[n] x R: M V^-1 before normalisation (R > 64)
  double* d_gram = nullptr;   // N x R x R Gram matrices
  double* d_gpart = nullptr;  // kGramChunks x R x R Gram partials
  double* d_red = nullptr;    // 2 x red_nb x R reduction partials
  int red_nb = 0;             // blocks of the row-wise ALS kernels (fixed per plan)
  double* d_chol = nullptr;   // 2 x R x R FP64 Cholesky work (R > 64)
  double* d_scal = nullptr;   // [0] status (as int), [1] fit, [2] loss, [8..8+R) lambda
  float* d_vinv = nullptr;    // R x R
  int res_valid = 0;          // residual copy d_elem[2] is current (after cp_loss_fwd)
  int res_mode = 0;           // order the residual copy is in
  int res_grad = -1;          // >= 0: the fused forward left that mode's gradient in d_lossgrad
  float* d_lossgrad = nullptr;  // max_n dims[n] x R: gradient of the fused forward's mode
  double* d_lpart = nullptr;    // per-block partials of sum e^2 (fused forward)
  size_t lpart_cap = 0;
  std::vector<spm::GraphCache> sweep_graphs;  // by parity
  std::vector<spm::GraphCache> als_graphs;
  std::vector<spm::GraphCache> als_run_graphs;  // whole ALS loops (cp_als_run)
  double* d_fits = nullptr;    // cp_als_run: fit of every iteration, then the count
  int fits_cap = 0;
  bool destroyed = false;
};

namespace spm {

// Named NVTX range over a host-side scope (plan build, a mode's pass, a sweep,
// an ALS iteration ...), so a profiler timeline shows the engine's phases.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
// "spmttkrp mode <n>" for n < kMaxModes
const char* nvtx_mode_name(int n);

// ---- error reporting (thread-local last error) ----
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
#define SPM_CUDA(call)                                   \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return spm::cuda_fail(_e, #call); \
  } while (0)

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device (once per kernel and device; thread-safe).
int ensure_dyn_smem(const void* kernel, size_t bytes, const char* what);

// packed nonzeros (PackInfo) on the host
uint32_t host_field(const uint32_t* w, int off, int b);
void pack_nonzero(const PackInfo& pk, int N, const int32_t* idx, float v, uint32_t* w);

// ---- host planning (plan_host.cpp) ----
int build_host_plan(spmttkrp_plan* p, const int64_t* coo, const float* vals, int nblk_opt);
int plan_keys(spmttkrp_plan* p, const int64_t* coo, const float* vals,
              std::vector<std::vector<int32_t>>& key);
int plan_partitions(spmttkrp_plan* p, int nblk_opt);
// ---- device planning (plan_device.cu) ----
int build_device_orders(spmttkrp_plan* p, const std::vector<std::vector<int32_t>>& key,
                        const float* vals, uint8_t* elems, int32_t* const* next_pos);
// Write orders of the tile form (3 modes, 32-byte nonzeros carrying remap ids):
// for every mode m and every tile of kTileNnz positions of its order, the
// tile-local indices sorted by destination (next_pos_m), stored 10 bits per mode
// in word 7 of the nonzero occupying each slot.  `elems` is the copy in mode-0
// order.
int build_write_orders(spmttkrp_plan* p, uint8_t* elems);
// Hot-row flags (3 modes, 32-byte nonzeros carrying remap ids): for every mode k,
// the hot_rows rows of largest degree (ties to the lower row id); bit 31 of word
// 4 + k of each nonzero (copy in mode-0 order) is set when its i_k is one of them.
int build_hot_flags(spmttkrp_plan* p, uint8_t* elems);
int default_tile(int es);
int partition_mode(const spmttkrp_plan* p, int n, int nblk, ModeHost* out);
int default_nblk(int64_t nnz, int num_sms, int variant);

// ---- kernel launchers (kernels_*.cu) ----
struct MttkrpArgs {
  const uint8_t* elems_in;
  uint8_t* elems_out;      // null: no remap
  const int32_t* next_pos;
  const int4* blkinfo;
  int nblk;
  const void* factors[kMaxModes];
  float* out;
  int64_t out_rows;
  int R, mode, nmodes, es, tile;
  float* part;
  int last_row;
  int* err;
  const float* scale;      // device scalar multiplier or null
  int dtype;
  int variant;             // 0 = warp blocks, staged tiles; 1 = CTA blocks, direct runs
  int hints;               // bit0: streams evict_first in L2; bit1: factor rows evict_last;
                           // bit2: L1 choice by the hot-row flags (hot rows evict_last,
                           // others evict_first)
  int unroll;              // nonzeros in flight per lane group (4 or 8; 0 = default)
  int stages;              // tiles per warp ring of the staged form (2..4)
  int no_fill;             // 1: blocks own non-contiguous row sets (Algorithm 1), so
                           // no kernel writes the empty rows between its rows
  int alpha_word;          // > 0: int32 word of a stored nonzero holding its position in
                           // the next mode's order (the remap id carried in the
                           // element); 0: the next_pos array
  unsigned long long wait_ns;  // limit of the first bounded wait that gives up
                               // (0 = the default 2 s); draining copies in flight
                               // after a give-up always uses the default
  int stall_test;          // test only: each warp's first wait is on a barrier that
                           // nothing completes, so it gives up after wait_ns
  int64_t nnz;             // nonzeros of the working copy (form 2 stages whole tiles)
  int grid_ctas;           // form 2: persistent CTAs (0 = one per block)
  int* sched;              // form 2: device block counter (zeroed by the launcher)
  PackInfo pk;             // index layout of the stored nonzeros
  double* loss_part;       // fused CP-loss pass: one FP64 partial of sum e^2 per block
                           // (non-null selects the fused pass: see mttkrp_warp_kernel)
  int hot_flags;           // bit 31 of word 4 + k of a stored nonzero marks i_k as one
                           // of the hot rows of factor k (3 modes, 32-byte nonzeros)
};
int launch_mttkrp(const MttkrpArgs& a, cudaStream_t s);
// the tile form (form 2) covers 3 modes, 32-byte nonzeros carrying remap ids, R 16/32/64
bool tile_form_supported(int nmodes, int es, int alpha_word, int R);
int launch_fixup(const float* part, const SplitRow* splits, int nsplit, int nchunk,
                 float* chunk_sums, float* out, int64_t out_rows, int R, const float* scale,
                 cudaStream_t s);
int launch_zero_rows(float* out, int64_t rows, int R, cudaStream_t s);
int launch_zero_listed_rows(float* out, const int32_t* rows, int nrows, int R, cudaStream_t s);
int launch_remap_only(const uint8_t* in, uint8_t* out, const int32_t* next_pos, int64_t nnz,
                      int es, cudaStream_t s);
int launch_scale_copy(const float* src, float* dst, int64_t n, const float* scale,
                      cudaStream_t s);
int launch_loss_reduce(const double* part, int64_t n, float* loss, double* loss64,
                       cudaStream_t s);
// remap-only pass in destination order (plans with write orders): mode -> mode+1
int launch_remap_ordered(const uint8_t* in, uint8_t* out, int64_t nnz, int mode, int* err,
                         cudaStream_t s);
size_t mttkrp_smem_bytes(int es, int tile, int R, int dtype, int stages);

// The copy of the nonzeros in the working order (the resident mode-0 copy
// when keep_base is on and the order is mode 0).
inline uint8_t* cur_elems(const spmttkrp_plan* p) {
  return (p->keep_base && p->cur_mode == 0) ? p->d_base : p->d_elem[p->cur_buf];
}
// Buffer of the pair that the next remap of the working copy writes.
inline int next_buf(const spmttkrp_plan* p) {
  return (p->keep_base && p->cur_mode == 0) ? 0 : 1 - p->cur_buf;
}

}  // namespace spm
