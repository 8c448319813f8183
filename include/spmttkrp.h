/*
 * spmttkrp.h - C ABI of the GB300 all-mode sparse MTTKRP engine.
 *
 * Method: Wijeratne, Kannan, Prasanna, "Sparse MTTKRP Acceleration for Tensor
 * Decomposition on GPU" (CF '24).  A COO tensor X with N modes is kept on the
 * device as ONE working copy of its nonzeros.  Computing the mode-n MTTKRP
 *     M_n = X_(n) (Khatri-Rao product of the A_k, k != n)          (Eq. 1)
 * streams that copy, gathers the factor rows A_k[i_k, :], and at the same
 * time scatters every nonzero to its place in the next mode's order (the
 * dynamic tensor remap, Section 3.1, Algorithm 3), so that mode n+1 again
 * reads a copy sorted by its own output index (Algorithm 5).  The nonzeros of
 * one mode are cut into blocks that own disjoint output rows, so no global
 * atomics are used (Observation 2); rows heavier than a block are split and
 * summed afterwards in block order.  Every output row is written once.
 *
 * Conventions (all entry points):
 *   - Every call returns an int status (SPM_OK or a negative SPM_ERR_*) and
 *     never aborts; spmttkrp_last_error() gives a thread-local message.
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device, owned by the caller, unless stated otherwise.  "host" pointers
 *     are ordinary CPU memory owned by the caller.
 *   - Work is queued asynchronously on the plan's stream (opts.stream, or
 *     spmttkrp_set_stream); only calls documented as synchronizing wait.
 *   - Indices are 0-based; every dims[k] must be in [1, 2^31-1]; nnz < 2^31;
 *     2 <= nmodes <= 16; 1 <= rank <= 256.
 *   - Factor matrices are dense, row-major I_k x R, with row stride R
 *     elements; FP32, or BF16 when the plan was made with SPM_DTYPE_BF16.
 *     Outputs and gradients are FP32, row-major I_n x R.
 */
#ifndef SPMTTKRP_H
#define SPMTTKRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spmttkrp_plan* spmttkrp_plan_t;

enum spm_status {
  SPM_OK = 0,
  SPM_ERR_INVALID_ARG = -1, /* null pointer, bad mode, bad size or option        */
  SPM_ERR_INDEX_RANGE = -2, /* a coordinate outside [0, dims[k])                   */
  SPM_ERR_DUPLICATE = -3,   /* two nonzeros share a coordinate                      */
  SPM_ERR_OOM = -4,         /* host or device allocation failed, or max_bytes hit  */
  SPM_ERR_CUDA = -5,        /* a CUDA runtime call failed                           */
  SPM_ERR_UNSUPPORTED = -6, /* sizes beyond the limits above                        */
  SPM_ERR_NOT_SPD = -7,     /* ALS: the Hadamard of Gram matrices is not SPD        */
  SPM_ERR_STATE = -8,       /* call not valid for this plan (host-only, destroyed) */
  SPM_ERR_TIMEOUT = -9      /* a bounded device wait gave up (no hang, no trap)     */
};

enum spm_dtype { SPM_DTYPE_F32 = 0, SPM_DTYPE_BF16 = 1 };

typedef struct {
  int factor_dtype; /* SPM_DTYPE_F32 or SPM_DTYPE_BF16 (factor storage only)     */
  int partition;    /* 0 = contiguous split of each mode's order with heavy-row
                       splitting and an ordered fix-up of split rows (default);
                       1 = Algorithm 1 (Section 3.4): each mode's rows go, in
                       descending degree, to the block with the fewest nonzeros
                       so far (ties to the lowest block); the working copy of
                       mode n is ordered by (block of i_n, K_n); no row is split
                       (a heavy row stays in one block); rows without nonzeros
                       are zeroed from a per-mode list; nblk (the block count
                       kappa) is fixed when the plan is built                    */
  int nblk;         /* blocks per mode (warp blocks for variant 0, CTA blocks for
                       variant 1); 0 = size-based default                         */
  int tile;         /* nonzeros per staged warp tile: 0 (= 128, halved while two
                       CTAs per SM would not fit), 32, 64, 128 or 256             */
  size_t max_bytes; /* cap on the plan's device memory; 0 = no cap               */
  int checks;       /* 1 = synchronize and read the device error word after every
                       compute call (slow; for debugging)                         */
  int host_only;    /* 1 = build the plan on the host only (no device memory);
                       only spmttkrp_plan_query and destroy are then valid        */
  int variant;      /* fused kernel form: 0 = one warp per block, tiles staged in
                       shared memory by bulk async copies (default); 1 = one CTA
                       per block, each lane group streams one contiguous run;
                       2 = tile form (3 modes, 32-byte nonzeros, R = 16, 32 or 64,
                       16-byte aligned factors and outputs; otherwise form 0 runs):
                       persistent CTAs stage tiles of 960 consecutive nonzeros,
                       issue the remap stores in destination order, and keep
                       several gathers in flight per lane group;
                       3 = form 0 with one remap warp per CTA (3 modes, 32-byte
                       nonzeros carrying their ids and write orders, partition
                       0; otherwise form 0 runs): 7 warps per CTA compute and
                       the 8th stores the CTA's 960-nonzero write-order tiles
                       in destination order                                     */
  int unroll;       /* nonzeros in flight per lane group in form 0: 0 (= 8), 4, 8 */
  int stages;       /* tiles per warp ring in form 0: 0 (= 2 for 32-byte and wider
                       nonzeros, 3 for 16-byte ones), 2, 3 or 4                   */
  int element_bytes;/* stride of a stored nonzero (N int32 indices + FP32 value):
                       0 = default, 32 when that fits (up to 7 modes: remap stores
                       then write whole 32-byte sectors, and DRAM never reads an
                       old sector to merge half of it), else the smallest multiple
                       of 16; 16 = unpadded (up to 3 modes, half the memory);
                       32 = padded (up to 7 modes).  A 3-mode nonzero in 32 bytes
                       carries its remap ids in the padding (Section 3.5): its
                       positions in the three modes' orders                       */
  int cache_hints;  /* fused-kernel cache policy: -1 = none, 0 = default (= 3);
                       bit0: the nonzero stream, remap ids and remapped copy evict
                       first in L2; bit1: factor rows evict last in L2; bit2 (tile
                       form only): L1 by the hot-row flags of 3-mode 32-byte
                       nonzeros (the rows of each factor holding the most
                       nonzeros evict last, the others first)                     */
  void* stream;     /* cudaStream_t for all work; NULL = default stream           */
  int keep_base;    /* 1 = keep the mode-0 copy resident and read-only next to the
                       two working copies (one more copy of the nonzeros): mode 0
                       reads it, and the pass of mode N-1 writes no remap, since
                       the mode-0 order it would produce is already resident.  A
                       sweep then does N-1 remap scatters instead of N.  0 = two
                       copies, every pass remaps (Algorithm 3 as written).       */
  int plan_on_host; /* 0 = a device plan with partition 0 builds its orders on the
                       device (stable LSD radix sorts of K_n, duplicate check,
                       working copy, next_pos; temporary device memory of about
                       5 int32 per nonzero plus the key columns, not counted in
                       max_bytes); 1 = on the host (parallel C++ radix passes).
                       Both give the same plan bit for bit.  Host-only plans and
                       partition 1 always build on the host.                    */
  int64_t wait_limit_ns; /* limit of the fused kernels' bounded waits on their
                       bulk-copy barriers before they give up and record
                       SPM_ERR_TIMEOUT (read by spmttkrp_device_status);
                       0 = 2 s.  Copies already in flight are still awaited
                       (with the 2 s limit) before a giving-up warp returns.    */
  int inject_wait_stall; /* failure-injection test switch: 1 = the first wait of
                       every warp of the fused kernel is on a barrier that nothing
                       completes, so it runs out after wait_limit_ns and the
                       pass reports SPM_ERR_TIMEOUT without writing its outputs;
                       the device context stays usable.  0 = off (always, except
                       in tests of the give-up path).                          */
} spmttkrp_opts_t;

/* Fills *opts with the defaults (FP32, contiguous split, automatic sizes). */
int spmttkrp_opts_init(spmttkrp_opts_t* opts);

/*
 * Builds a plan (the paper's preprocessing, Section 3.4 / 3.5 and the
 * evaluation's preprocessing step): validates the COO, sorts the nonzeros
 * into every mode's canonical order K_n = (i_n, i_{n-1}, ..., i_{n+1})
 * (lexicographic), computes the remap ids next_pos_n (position in the
 * mode-(n+1) order of the nonzero at position p of the mode-n order), the
 * block boundaries of every mode and the split-row tables, and uploads the
 * working copy (mode-0 order) and these tables to the device.
 *   out    host, receives the plan handle (owned by the caller; destroy it).
 *   coo    host, int64 [nnz][nmodes] row-major coordinates, any order.
 *   vals   host, float [nnz] values.
 *   nnz    number of nonzeros (0 allowed: every output is then all zeros).
 *   dims   host, int64 [nmodes].
 *   rank   R of the factor matrices the plan will be used with.
 *   opts   host, nullable (defaults).
 * Errors: INVALID_ARG, INDEX_RANGE, DUPLICATE, UNSUPPORTED, OOM, CUDA.
 * Synchronizes the plan's stream before returning.
 */
int spmttkrp_plan_create(spmttkrp_plan_t* out, const int64_t* coo, const float* vals,
                         int64_t nnz, const int64_t* dims, int nmodes, int rank,
                         const spmttkrp_opts_t* opts);

/* Frees the plan and every device buffer it owns (synchronizes its stream). */
int spmttkrp_plan_destroy(spmttkrp_plan_t plan);

/* Sets the stream (cudaStream_t) later calls queue their work on. */
int spmttkrp_set_stream(spmttkrp_plan_t plan, void* stream);

/*
 * Dynamic tensor remap only (Section 3.1, Algorithm 3): brings the working
 * copy into the given mode's canonical order by pure remap passes (no-op when
 * it is already there).  Errors: INVALID_ARG (mode), STATE.
 */
int spmttkrp_remap(spmttkrp_plan_t plan, int mode);

/*
 * Mode-n spMTTKRP (Eq. 1; Algorithms 2, 4) fused with the remap of the
 * working copy into mode (n+1) mod N order (Algorithm 3).  Remaps first if the
 * copy is not in mode-n order.  With opts.keep_base the pass of mode N-1 skips
 * the remap (the resident mode-0 copy becomes the working copy).
 *   factors  host array of nmodes device pointers (the mode-n one is not read).
 *   out      device, float [dims[mode]][rank], fully overwritten (rows with no
 *            nonzero are written as zeros); must not alias a factor.
 * Errors: INVALID_ARG, STATE, CUDA, TIMEOUT (with opts.checks).
 */
int spmttkrp_compute(spmttkrp_plan_t plan, int mode, const void* const* factors, float* out);

/* flags for spmttkrp_compute_ex */
enum { SPM_COMPUTE_KEEP_ORDER = 1 /* write no remap: the copy stays in mode order */ };

/*
 * spmttkrp_compute with flags.  SPM_COMPUTE_KEEP_ORDER: the pass computes M_n
 * (Eq. 1) from the copy in mode-n order and writes no remap (Algorithm 3 is
 * skipped), so the working copy stays in mode-n order and the call can be
 * repeated (e.g. the same mode with new factors, or timing the elementwise
 * computation without the dynamic remap, the split of Section 5.2).  Other
 * arguments and errors as spmttkrp_compute.
 */
int spmttkrp_compute_ex(spmttkrp_plan_t plan, int mode, const void* const* factors, float* out,
                        int flags);

/* flags for spmttkrp_sweep */
enum { SPM_SWEEP_GRAPH = 1 /* replay the sweep as one captured CUDA graph */ };

/*
 * All-mode spMTTKRP (Algorithm 5): M_n for every mode n with the same input
 * factors, one fused compute+remap pass per mode, starting from the mode the
 * working copy is in; afterwards the copy is back in that mode's order.
 *   factors  host array of nmodes device pointers.
 *   outs     host array of nmodes device pointers, float [dims[n]][rank].
 *   flags    0 or SPM_SWEEP_GRAPH.
 */
int spmttkrp_sweep(spmttkrp_plan_t plan, const void* const* factors, float* const* outs,
                   int flags);

/*
 * One CP-ALS iteration over modes 0..N-1 (Section 2.1.4; Kolda-Bader update):
 * per mode M_n = spMTTKRP, V = Hadamard of the Gram matrices A_k^T A_k (k != n)
 * in FP64, Cholesky of V in FP64, A_n = M_n V^-1, lambda = column 2-norms of
 * A_n, A_n /= lambda.  Replayed from a captured CUDA graph after the first
 * call with the same pointers.
 *   factors  host array of nmodes device pointers, read and overwritten.
 *   lambda   device, float [rank], written.
 *   fit      host, receives 1 - |X - Y|_F / |X|_F; this call synchronizes.
 * Errors: NOT_SPD (factors unchanged from the failing mode on), INVALID_ARG,
 * STATE, CUDA.
 */
int cp_als_iter(spmttkrp_plan_t plan, void* const* factors, float* lambda, double* fit);

/*
 * Up to max_iters CP-ALS iterations run as ONE graph launch, stopping on the
 * device once the fit changes by less than tol between two iterations (the
 * convergence check of the ALS loop, Section 2.1.4): a chain of conditional
 * graph nodes, each holding one iteration and its check, which decides whether
 * the next node runs.  Column scales are folded: inside the loop each
 * U_n = M_n V^-1 is stored unnormalised (the mode update followed by the
 * normalisation does not depend on the other factors' column scales), the fit is
 * that of the stored factors' model, and after the last iteration every factor
 * is divided by its column 2-norms and lambda_r = prod_k |U_k[:, r]|.  The
 * results are cp_als_iter's up to rounding.  No host synchronisation happens
 * between iterations; the call synchronizes once at the end.  The graph is built
 * on the first call and replayed by later calls with the same pointers,
 * max_iters, tol and working-copy buffer.
 *   factors   host array of nmodes device pointers, read and overwritten.
 *   lambda    device, float [rank], written.
 *   max_iters 1..256.   tol  >= 0 (0: always max_iters iterations).
 *   fits      host, double [max_iters]: fit after each iteration that ran.
 *   iters     host, receives the number of iterations that ran.
 * Errors: NOT_SPD (the loop stops at the failing iteration), INVALID_ARG,
 * STATE, CUDA.
 */
int cp_als_run(spmttkrp_plan_t plan, void* const* factors, float* lambda, int max_iters,
               double tol, double* fits, int* iters);

/*
 * CP loss on the observed entries: L = 1/2 sum_e (m_e - x_e)^2 with
 * m_e = sum_r prod_k A_k[i_k(e), r]; keeps the residuals m_e - x_e in the plan.
 *   factors  host array of nmodes device pointers.
 *   loss     device, float scalar, written.
 */
int cp_loss_fwd(spmttkrp_plan_t plan, const void* const* factors, float* loss);

/* flags for cp_loss_fwd_ex */
enum { SPM_LOSS_FORWARD_ONLY = 1 /* no gradient will follow: the plain forward pass */ };

/*
 * cp_loss_fwd with flags.  By default (flags 0) a plan whose nonzeros are
 * 3-mode, 16 or 32 bytes (and whose factors are 16-byte aligned, R a multiple
 * of 4), split contiguously, runs one fused pass in the working copy's current mode n: it computes
 * the residuals, the loss, the gradient dL/dA_n (kept in the plan until the
 * next cp_loss_bwd scales it by grad_out), and writes the residual copy
 * directly in the mode-(n+1) order, so the backward needs N-1 passes instead
 * of N.  SPM_LOSS_FORWARD_ONLY runs the plain forward (residual copy in mode n
 * order, no gradient), the cheaper choice when no backward follows.  Other
 * plans always run the plain forward.  Arguments and errors as cp_loss_fwd.
 */
int cp_loss_fwd_ex(spmttkrp_plan_t plan, const void* const* factors, float* loss, int flags);

/*
 * Gradient of the CP loss: grads[n] = grad_out * spMTTKRP_n(residual tensor)
 * for every mode, one all-mode sweep on a remapped copy of the residuals (after
 * the fused forward: the forward's mode is a scaled copy of the gradient it left,
 * and the sweep covers the other N-1 modes).  Needs a previous cp_loss_fwd with
 * the same factors; it consumes that forward's residuals.
 *   grad_out device, float scalar (dL_total/dL).
 *   grads    host array of nmodes device pointers, float [dims[n]][rank].
 */
int cp_loss_bwd(spmttkrp_plan_t plan, const void* const* factors, const float* grad_out,
                float* const* grads);

/*
 * Chooses blocks per mode (2 to 32 waves of 24 warps per SM, and the size-based
 * default), tile size, ring depth and kernel form by timing all-mode sweeps
 * with CUDA events on the plan's own data, and applies the winner
 * (deterministic argmin of the median of 3, ties to the first candidate).  With
 * partition 1 the block count stays as built.  Results are cached in the text
 * file named by $SPMTTKRP_TUNE_CACHE when set (one line per key: "<shape key>
 * <blocks per SM, -1 = default> <tile> <kernel form> <ring depth>"); the key
 * holds modes, rank, dtype, nonzero stride, partition, log2 nnz, the heaviest
 * row's share and the SM count.
 *   factors  host array of nmodes device pointers used for the trial sweeps.
 *   scratch  host array of nmodes device output buffers for the trial sweeps.
 *   flags    bit 0: ignore the cache.
 */
int spmttkrp_autotune(spmttkrp_plan_t plan, const void* const* factors, float* const* scratch,
                      int flags);

/* what for spmttkrp_plan_query */
enum {
  SPM_Q_INFO = 0,     /* int64[16]: nnz, nmodes, rank, elem_bytes, cur_mode, dtype,
                         tile, nblk(mode), nsplit(mode), launches per sweep,
                         device bytes, working buffer, flags (bit0 host_only, bit1
                         variant & 1, bit2 keep_base, bits 3-5 ring stages, bit6
                         partition, bit7 nonzeros carry their remap ids, bits 8-9
                         variant, bit10 nonzeros carry write orders, bits 11-31
                         hot rows per factor, 0 = no hot-row flags), SMs,
                         |X|^2 (double), lanes                                      */
  SPM_Q_NEXT_POS = 1, /* int32[nnz]: next_pos of `mode`                            */
  SPM_Q_BOUNDS = 2,   /* int64[nblk+1]: block boundaries of `mode`                 */
  SPM_Q_SPLITS = 3,   /* int64[nsplit][3]: (row, first_blk, last_blk) of `mode`   */
  SPM_Q_ELEMS = 4,    /* int32[nnz][nmodes] indices of the working copy, in its
                         current order                                             */
  SPM_Q_VALS = 5,     /* float[nnz] values of the working copy, same order         */
  SPM_Q_RAW = 6       /* uint8[nnz][elem_bytes]: the stored nonzeros of the working
                         copy in its current order, padding words included (for a
                         3-mode plan in 32-byte sectors: words 4..6 = the nonzero's
                         positions in the three orders, word 7 = the write orders
                         of the tile form, 10 bits per mode)                       */
};

/* Copies plan data into host memory (synchronizes).  bytes must be >= the
 * size stated above for `what`.  Errors: INVALID_ARG, STATE, CUDA. */
int spmttkrp_plan_query(spmttkrp_plan_t plan, int what, int mode, void* host_dst,
                        size_t bytes);

/*
 * Mode-n spMTTKRP (and, optionally, the remap into mode n+1 order) for callers
 * that cannot allocate device memory: code running where cudaMalloc is not
 * allowed or not possible (an allocator-free region of a host framework, a
 * process whose device memory is owned by another pool).  Such callers cannot
 * create a plan, so everything is passed in; the call allocates nothing.  The
 * paper has no counterpart: this is an engineering entry point.
 *   elems      device, nnz nonzeros in mode-`mode` canonical order, each
 *              {int32 idx[nmodes]; float val} padded with zeros to a stride of
 *              (4*nmodes+4) rounded up to 16 bytes (the plan's layout).
 *   dims       host, int64 [nmodes];  factors: host array of device pointers.
 *   out        device, float [dims[mode]][rank], fully overwritten.
 *   elems_out, next_pos  both NULL (no remap) or both device: element p is
 *              written to elems_out[next_pos[p]] (int32 [nnz]).
 *   nblk       blocks of the even split (0 = automatic), at most 4096.
 *   stream     cudaStream_t (NULL = default stream); the call is asynchronous.
 * Scratch (block descriptors, split-row table, split-row partial sums) lives in
 * one static device array of 8.25 MiB that every device using the library
 * keeps until the process exits: at most 4096 blocks and rank <= 256; larger
 * requests return SPM_ERR_UNSUPPORTED.  The first call on a device looks up
 * that array's device address; make that first call before any stream
 * capture.  All calls share the array, so calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Every scratch entry a call reads is written earlier in the same call.
 */
int spmttkrp_compute_noalloc(const void* elems, int64_t nnz, int nmodes, int mode,
                             const int64_t* dims, int rank, int factor_dtype,
                             const void* const* factors, float* out, void* elems_out,
                             const int32_t* next_pos, int nblk, void* stream);

/* Synchronizes, returns SPM_OK or the first recorded device-side error
 * (e.g. SPM_ERR_TIMEOUT) and clears it. */
int spmttkrp_device_status(spmttkrp_plan_t plan);

/* Consistency check of a working copy on the device (Section 3.5: one pass's
 * remap scatters every nonzero to exactly one place of the next order).  It
 * reads only; nothing traps.  Checks, in this order of reported status:
 *   - every index of every nonzero lies in [0, dims[k])     -> SPM_ERR_INDEX_RANGE
 *   - next_pos (if given) holds ids in [0, nnz), each hit
 *     exactly once (a permutation)                           -> SPM_ERR_STATE
 *   - word alpha_word of every nonzero (if > 0) equals its
 *     next_pos entry (remap ids carried in the padding)      -> SPM_ERR_STATE
 * The last-error text gives the count of violations and the first position.
 *   elems       device, nnz nonzeros of elem_bytes each: int32 idx[nmodes],
 *               float value, then padding (elem_bytes a multiple of 16).
 *   dims        host, int64 [nmodes].
 *   next_pos    device int32 [nnz] or NULL (no remap checks).
 *   alpha_word  0, or the 32-bit word index (> nmodes, inside elem_bytes) of
 *               the remap id carried in each nonzero.
 *   stream      cudaStream_t (NULL = default); the call synchronizes it.
 * Allocates nnz * 4 bytes of device scratch for the hit counters (freed before
 * return; not counted against a plan's max_bytes).  Errors: INVALID_ARG, CUDA,
 * and the statuses above. */
int spmttkrp_check_elements(const void* elems, int64_t nnz, int nmodes, const int64_t* dims,
                            int elem_bytes, const int32_t* next_pos, int alpha_word,
                            void* stream);

/* The same check on a plan's own working copy in its current mode's order,
 * with that mode's next_pos and, for plans that carry remap ids in their
 * nonzeros, the id word of the next mode.  Errors: INVALID_ARG, STATE
 * (host-only plan, or a failed check), INDEX_RANGE, CUDA. */
int spmttkrp_plan_check(spmttkrp_plan_t plan);

/*
 * Memory-system probe (a measurement utility; the paper has no counterpart):
 * one kernel over n records of 32 bytes that the caller times, for the access
 * patterns of the dynamic remap.
 *   kind 0  copy: dst[i] = src[i]
 *   kind 1  scatter: dst[pi(i)] = src[i]
 *   kind 2  gather: dst[i] = src[pi(i)]
 * pi keeps runs of `run` consecutive records together (run 4 = one 128-byte
 * line) and sends run q to run (A q + 12345) mod (n / run), A a fixed prime not
 * dividing n / run (a permutation of the runs).
 *   src, dst  device, n * 32 bytes each, 32-byte aligned, not overlapping.
 *   run       >= 1 and dividing n.
 *   stream    cudaStream_t (NULL = default); asynchronous.
 * Errors: INVALID_ARG, CUDA.
 */
int spmttkrp_memprobe(int kind, const void* src, void* dst, int64_t n, int run, void* stream);

/* Thread-local text for the last non-OK status of this thread. */
const char* spmttkrp_last_error(void);

/* ABI version (major * 100 + minor). */
int spmttkrp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPMTTKRP_H */
