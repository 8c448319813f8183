// api_ext.cu - CP-ALS iteration (captured as a CUDA graph), CP loss forward /
// backward, and the autotuner, on top of the fused spMTTKRP + remap path.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "als.h"
#include "engine.h"
#include "mttkrp_kernel.cuh"

namespace spm {

constexpr int kMaxAlsRun = 256;  // iterations one cp_als_run graph may hold

// Row chunks of a Gram matrix (FP32 within a chunk, FP64 across chunks in a fixed
// order): enough chunks to fill the GPU, at most 32 MB of partials.
static int gram_chunks(int R) { return R <= 64 ? 1024 : (R <= 128 ? 256 : 64); }

static int ensure(spmttkrp_plan* p, void** ptr, size_t bytes) {
  if (*ptr) return SPM_OK;
  return plan_dalloc(p, ptr, bytes);
}

static int64_t max_dim(const spmttkrp_plan* p) {
  int64_t m = 0;
  for (int64_t d : p->dims) m = std::max(m, d);
  return m;
}

static int ensure_als(spmttkrp_plan* p) {
  const size_t R = (size_t)p->R, N = (size_t)p->N, I = (size_t)max_dim(p);
  if (!p->red_nb) p->red_nb = std::max(1, p->num_sms * 8);
  int st;
  if ((st = ensure(p, (void**)&p->d_M, I * R * 4))) return st;
  if (R > 64 && (st = ensure(p, (void**)&p->d_U, I * R * 4))) return st;  // M V^-1 (R > 64)
  if ((st = ensure(p, (void**)&p->d_gram, N * R * R * 8))) return st;
  if ((st = ensure(p, (void**)&p->d_gpart, (size_t)gram_chunks((int)R) * R * R * 8))) return st;
  if ((st = ensure(p, (void**)&p->d_red, (size_t)2 * p->red_nb * R * 8))) return st;
  if ((st = ensure(p, (void**)&p->d_chol, 2 * R * R * 8))) return st;
  if ((st = ensure(p, (void**)&p->d_vinv, R * R * 4))) return st;
  if (!p->d_scal) {  // [8, 8 + R): lambda; [8 + R, 8 + 2R): ones (the folded loop's lambda)
    if ((st = plan_dalloc(p, (void**)&p->d_scal, (8 + 2 * R) * 8))) return st;
    if ((st = launch_fill_f64(p->d_scal + 8 + R, (int)R, 1.0, p->stream))) return st;
  }
  if (!p->als_side) SPM_CUDA(cudaStreamCreateWithFlags(&p->als_side, cudaStreamNonBlocking));
  if (!p->als_fork) SPM_CUDA(cudaEventCreateWithFlags(&p->als_fork, cudaEventDisableTiming));
  if (!p->als_join) SPM_CUDA(cudaEventCreateWithFlags(&p->als_join, cudaEventDisableTiming));
  return SPM_OK;
}

// Queues one CP-ALS iteration (modes 0..N-1) on p->stream.  The working copy
// must be in mode-0 order; afterwards it is again.  Mode n's spMTTKRP needs the
// factors but not their Grams, so the Gram of the factor just updated and the
// next mode's Cholesky run on a side stream beside it (forked from and joined
// into p->stream; under stream capture they become a parallel branch).
// grams_current: the plan's Grams already belong to these factors (the previous
// iteration of the same loop formed them), so none is formed first.
// fold: column-scale folding (cp_als_run): each U_n = M_n V^-1 is stored as it
// is, with no column norms, lambda or normalisation; the fit is that of the model
// of the stored factors (lambda = 1), the same model; the loop normalises at its
// end (launch_als_fold_finish).
static int als_enqueue(spmttkrp_plan* p, void* const* factors, float* lambda,
                       bool grams_current = false, bool fold = false) {
  const int N = p->N, R = p->R;
  int* status = reinterpret_cast<int*>(p->d_scal);
  double* fit = p->d_scal + 1;
  double* lam64 = p->d_scal + 8;
  const double* lam_one = p->d_scal + 8 + R;
  double* colsq = p->d_red;
  double* mdot = p->d_red + (size_t)p->red_nb * R;
  cudaStream_t s = p->stream, side = p->als_side;
  SPM_CUDA(cudaMemsetAsync(p->d_scal, 0, 8, s));
  int st;
  for (int k = 0; k < N && !grams_current; ++k)
    if ((st = launch_gram(factors[k], p->dtype, p->dims[(size_t)k], R, p->d_gpart, gram_chunks(R),
                          p->d_gram + (size_t)k * R * R, s)))
      return st;
  // side: mode 0's Cholesky
  SPM_CUDA(cudaEventRecord(p->als_fork, s));
  SPM_CUDA(cudaStreamWaitEvent(side, p->als_fork, 0));
  if ((st = launch_als_prep(p->d_gram, N, 0, R, p->d_chol, p->d_vinv, status, side))) return st;
  SPM_CUDA(cudaEventRecord(p->als_join, side));
  std::vector<const void*> cf(factors, factors + N);
  for (int n = 0; n < N; ++n) {
    const int64_t I = p->dims[(size_t)n];
    if ((st = compute_mode(p, n, cf.data(), p->d_M, false))) return st;
    SPM_CUDA(cudaStreamWaitEvent(s, p->als_join, 0));  // V^-1 of mode n is ready
    if (!fold || R > 64) {  // the column norms (R > 64: U itself, for the scale pass)
      if ((st = launch_als_solve(p->d_M, p->d_U, p->d_vinv, I, R, colsq, status, p->red_nb, s)))
        return st;
    }
    if (!fold && (st = launch_als_lambda(colsq, p->red_nb, R, lam64, lambda, status, s)))
      return st;
    // A_n = U / lambda, or with folding U / 1 = U itself; and <M, A_n>
    if ((st = launch_als_scale(p->d_U, p->d_M, p->d_vinv, factors[n], p->dtype,
                               fold ? lam_one : lam64, I, R, mdot, status, p->red_nb, s)))
      return st;
    // side: the updated factor's Gram, then the next mode's Cholesky
    SPM_CUDA(cudaEventRecord(p->als_fork, s));
    SPM_CUDA(cudaStreamWaitEvent(side, p->als_fork, 0));
    if ((st = launch_gram(factors[n], p->dtype, I, R, p->d_gpart, gram_chunks(R),
                          p->d_gram + (size_t)n * R * R, side)))
      return st;
    if (n + 1 < N &&
        (st = launch_als_prep(p->d_gram, N, n + 1, R, p->d_chol, p->d_vinv, status, side)))
      return st;
    SPM_CUDA(cudaEventRecord(p->als_join, side));
  }
  SPM_CUDA(cudaStreamWaitEvent(s, p->als_join, 0));
  return launch_als_fit(p->d_gram, N, R, fold ? lam_one : lam64, mdot, p->red_nb, p->normx2, fit,
                        status, s);
}

static void drop_graphs(std::vector<GraphCache>& v) {
  for (auto& g : v)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  v.clear();
}

// Re-cuts every mode into nblk blocks and switches the kernel form / tile / ring.
static int apply_config(spmttkrp_plan* p, int nblk, int tile, int variant, int stages) {
  for (int n = 0; n < p->N; ++n) {
    int st = partition_mode(p, n, nblk, &p->mh[(size_t)n]);
    if (st) return st;
    st = upload_mode_tables(p, n);
    if (st) return st;
  }
  p->tile = tile;
  p->variant = variant;
  p->stages = stages;
  drop_graphs(p->sweep_graphs);
  drop_graphs(p->als_graphs);
  return SPM_OK;
}

// ---- autotune cache: one line per key, "key nblk_per_sm tile variant stages"
static std::string tune_key(const spmttkrp_plan* p) {
  int64_t maxdeg = 0;
  for (int n = 0; n < p->N; ++n) {
    const auto& us = p->row_start[(size_t)n];
    for (size_t u = 0; u + 1 < us.size(); ++u) maxdeg = std::max(maxdeg, us[u + 1] - us[u]);
  }
  const int zbucket = p->nnz > 0 ? (int)std::floor(std::log2((double)p->nnz)) : 0;
  const int skew = p->nnz > 0 ? (int)std::floor(20.0 * (double)maxdeg / (double)p->nnz) : 0;
  std::ostringstream o;
  o << "N" << p->N << "_R" << p->R << "_d" << p->dtype << "_e" << p->es << "_p" << p->partition
    << "_z" << zbucket << "_s" << skew << "_m" << p->num_sms;
  return o.str();
}

static bool cache_lookup(const std::string& key, int* nps, int* tile, int* variant,
                         int* stages) {
  const char* path = std::getenv("SPMTTKRP_TUNE_CACHE");
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string k;
    int a, b, c, d;
    if (is >> k >> a >> b >> c >> d && k == key) {
      *nps = a;
      *tile = b;
      *variant = c;
      *stages = d;
      return true;
    }
  }
  return false;
}

static void cache_store(const std::string& key, int nps, int tile, int variant, int stages) {
  const char* path = std::getenv("SPMTTKRP_TUNE_CACHE");
  if (!path) return;
  std::vector<std::string> keep;
  {
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
      std::istringstream is(line);
      std::string k;
      if (is >> k && k != key) keep.push_back(line);
    }
  }
  std::ofstream f(path, std::ios::trunc);
  for (auto& l : keep) f << l << "\n";
  f << key << " " << nps << " " << tile << " " << variant << " " << stages << "\n";
}

}  // namespace spm

using namespace spm;

extern "C" {

int cp_als_iter(spmttkrp_plan_t p, void* const* factors, float* lambda, double* fit) {
  NvtxRange range("cp_als_iter");
  if (!p || p->destroyed) return fail(SPM_ERR_INVALID_ARG, "null or destroyed plan");
  if (p->host_only) return fail(SPM_ERR_STATE, "plan was built host-only");
  if (!factors || !lambda || !fit) return fail(SPM_ERR_INVALID_ARG, "null argument");
  for (int k = 0; k < p->N; ++k)
    if (!factors[k]) return fail(SPM_ERR_INVALID_ARG, "null factor pointer");
  if (p->nnz == 0) return fail(SPM_ERR_INVALID_ARG, "CP-ALS needs at least one nonzero");
  int st = ensure_als(p);
  if (st) return st;
  st = spmttkrp_remap(p, 0);
  if (st) return st;
  std::vector<const void*> key(factors, factors + p->N);
  key.push_back(lambda);
  key.push_back((const void*)(intptr_t)p->cur_buf);
  GraphCache* hit = nullptr;
  for (auto& g : p->als_graphs)
    if (g.key == key) hit = &g;
  if (hit) {
    SPM_CUDA(cudaGraphLaunch(hit->exec, p->stream));
    p->cur_buf = hit->end_buf;
  } else {
    const int buf0 = p->cur_buf;
    st = als_enqueue(p, factors, lambda);  // eager first run
    if (st) return st;
    const int buf1 = p->cur_buf;
    // capture the same sequence for later calls with these pointers
    if (!p->cap_stream) SPM_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = p->stream;
    p->stream = p->cap_stream;
    p->cur_buf = buf0;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      st = als_enqueue(p, factors, lambda);
      e = cudaStreamEndCapture(p->stream, &g);
    }
    p->stream = user;
    p->cur_buf = buf1;
    p->cur_mode = 0;
    if (st) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "ALS graph capture");
    GraphCache gc;
    gc.key = key;
    gc.end_buf = buf1;
    e = cudaGraphInstantiate(&gc.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(ALS)");
    if (p->als_graphs.size() >= 4) {
      cudaGraphExecDestroy(p->als_graphs.front().exec);
      p->als_graphs.erase(p->als_graphs.begin());
    }
    p->als_graphs.push_back(gc);
  }
  p->cur_mode = 0;
  double host[2] = {0.0, 0.0};
  SPM_CUDA(cudaMemcpyAsync(host, p->d_scal, 16, cudaMemcpyDeviceToHost, p->stream));
  SPM_CUDA(cudaStreamSynchronize(p->stream));
  int status;
  std::memcpy(&status, host, sizeof(int));
  *fit = host[1];
  if (status) return fail(SPM_ERR_NOT_SPD, "Hadamard product of Gram matrices is not SPD");
  return SPM_OK;
}

// The fused CP-loss pass serves plans whose nonzeros are 3-mode, 16 or 32 bytes,
// and whose factors take the vector lanes (16-byte aligned, R a multiple of 4).
static bool loss_fusable(const spmttkrp_plan* p, const void* const* factors) {
  if (!(p->N == 3 && (p->es == 32 || p->es == 16) && p->partition == 0 && p->nnz > 0))
    return false;
  bool al = true;
  for (int k = 0; k < p->N; ++k) al = al && (((uintptr_t)factors[k] & 15u) == 0);
  return lane_config(p->R, p->dtype, al, true).vec;
}

int cp_als_run(spmttkrp_plan_t p, void* const* factors, float* lambda, int max_iters,
               double tol, double* fits, int* iters) {
  NvtxRange range("cp_als_run");
  if (!p || p->destroyed) return fail(SPM_ERR_INVALID_ARG, "null or destroyed plan");
  if (p->host_only) return fail(SPM_ERR_STATE, "plan was built host-only");
  if (!factors || !lambda || !fits || !iters) return fail(SPM_ERR_INVALID_ARG, "null argument");
  if (max_iters < 1 || max_iters > kMaxAlsRun)
    return fail(SPM_ERR_INVALID_ARG, "max_iters must be in [1, 256]");
  if (!(tol >= 0.0)) return fail(SPM_ERR_INVALID_ARG, "tol must be >= 0");
  for (int k = 0; k < p->N; ++k)
    if (!factors[k]) return fail(SPM_ERR_INVALID_ARG, "null factor pointer");
  if (p->nnz == 0) return fail(SPM_ERR_INVALID_ARG, "CP-ALS needs at least one nonzero");
  int st = ensure_als(p);
  if (st) return st;
  if (max_iters + 1 > p->fits_cap) {
    if (p->d_fits) {
      cudaFree(p->d_fits);
      p->dev_bytes -= std::max<size_t>((size_t)p->fits_cap * 8, 16);
      p->d_fits = nullptr;
    }
    if ((st = plan_dalloc(p, (void**)&p->d_fits, (size_t)(kMaxAlsRun + 1) * 8))) return st;
    p->fits_cap = kMaxAlsRun + 1;
  }
  st = spmttkrp_remap(p, 0);
  if (st) return st;
  int* d_iters = reinterpret_cast<int*>(p->d_fits + kMaxAlsRun);
  int* status = reinterpret_cast<int*>(p->d_scal);
  double tolbits;
  std::memcpy(&tolbits, &tol, 8);
  std::vector<const void*> key(factors, factors + p->N);
  key.push_back(lambda);
  key.push_back((const void*)(intptr_t)p->cur_buf);
  key.push_back((const void*)(intptr_t)max_iters);
  key.push_back(reinterpret_cast<const void*>(*reinterpret_cast<const intptr_t*>(&tolbits)));
  GraphCache* hit = nullptr;
  for (auto& g : p->als_run_graphs)
    if (g.key == key) hit = &g;
  const int buf0 = p->cur_buf;
  if (!hit) {
    // the loop as one graph: a chain of max_iters conditional nodes, node t
    // holding iteration t and its convergence check, which decides whether
    // node t+1 runs (an iteration of an odd number of modes moves the working
    // copy to the other buffer, so each iteration is captured with its own
    // buffer parity)
    cudaGraph_t g = nullptr;
    SPM_CUDA(cudaGraphCreate(&g, 0));
    std::vector<cudaGraphConditionalHandle> h((size_t)max_iters);
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < max_iters && e == cudaSuccess; ++t)
      e = cudaGraphConditionalHandleCreate(&h[(size_t)t], g, t == 0 ? 1u : 0u,
                                           cudaGraphCondAssignDefault);
    if (!p->cap_stream && e == cudaSuccess)
      e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    cudaGraphNode_t prev = nullptr;
    cudaStream_t user = p->stream;
    for (int t = 0; t < max_iters && e == cudaSuccess && !st; ++t) {
      alignas(cudaGraphNodeParams) unsigned char npb[sizeof(cudaGraphNodeParams)];
      std::memset(npb, 0, sizeof(npb));  // reserved fields must be zero
      cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npb);
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h[(size_t)t];
      np.conditional.type = cudaGraphCondTypeIf;
      np.conditional.size = 1;
      cudaGraphNode_t node = nullptr;
      e = cudaGraphAddNode(&node, g, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &np);
      if (e != cudaSuccess) break;
      cudaGraph_t body = np.conditional.phGraph_out[0];
      p->stream = p->cap_stream;
      e = cudaStreamBeginCaptureToGraph(p->stream, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        st = als_enqueue(p, factors, lambda, t > 0, true);  // iteration t-1 formed the Grams
        if (!st)
          st = launch_als_converge(p->d_scal + 1, status, p->d_fits, d_iters, t, tol,
                                   t + 1 < max_iters ? h[(size_t)t + 1] : h[(size_t)t],
                                   t + 1 < max_iters ? 1 : 0, p->stream);
        cudaGraph_t cap = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(p->stream, &cap);
        if (e == cudaSuccess) e = e2;
      }
      p->stream = user;
      prev = node;
    }
    // after the last iteration that ran: the folded column scales become lambda
    if (e == cudaSuccess && !st) {
      p->stream = p->cap_stream;
      e = cudaStreamBeginCaptureToGraph(p->stream, g, &prev, nullptr, 1,
                                        cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        st = launch_als_fold_finish(factors, p->dtype, p->dims.data(), p->N, p->R, p->d_gram,
                                    p->d_scal + 8, lambda, status, p->red_nb, p->stream);
        cudaGraph_t cap = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(p->stream, &cap);
        if (e == cudaSuccess) e = e2;
      }
      p->stream = user;
    }
    p->stream = user;
    p->cur_buf = buf0;
    p->cur_mode = 0;
    if (st || e != cudaSuccess) {
      cudaGraphDestroy(g);
      return st ? st : cuda_fail(e, "CP-ALS loop graph");
    }
    GraphCache gc;
    gc.key = key;
    e = cudaGraphInstantiate(&gc.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(CP-ALS loop)");
    if (p->als_run_graphs.size() >= 2) {
      cudaGraphExecDestroy(p->als_run_graphs.front().exec);
      p->als_run_graphs.erase(p->als_run_graphs.begin());
    }
    p->als_run_graphs.push_back(gc);
    hit = &p->als_run_graphs.back();
  }
  SPM_CUDA(cudaMemsetAsync(d_iters, 0, sizeof(int), p->stream));
  SPM_CUDA(cudaGraphLaunch(hit->exec, p->stream));
  int n = 0, stat = 0;
  SPM_CUDA(cudaMemcpyAsync(&n, d_iters, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  SPM_CUDA(cudaMemcpyAsync(&stat, status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  SPM_CUDA(cudaMemcpyAsync(fits, p->d_fits, (size_t)max_iters * 8, cudaMemcpyDeviceToHost,
                           p->stream));
  SPM_CUDA(cudaStreamSynchronize(p->stream));
  *iters = n;
  // each iteration of an odd number of modes flips the working-copy buffer
  if (!p->keep_base && (p->N & 1) && (n & 1)) p->cur_buf = 1 - buf0;
  p->cur_mode = 0;
  if (stat) return fail(SPM_ERR_NOT_SPD, "Hadamard product of Gram matrices is not SPD");
  return SPM_OK;
}

int cp_loss_fwd_ex(spmttkrp_plan_t p, const void* const* factors, float* loss, int flags) {
  NvtxRange range("cp_loss_fwd");
  if (!p || p->destroyed) return fail(SPM_ERR_INVALID_ARG, "null or destroyed plan");
  if (p->host_only) return fail(SPM_ERR_STATE, "plan was built host-only");
  if (!factors || !loss) return fail(SPM_ERR_INVALID_ARG, "null argument");
  if (flags & ~SPM_LOSS_FORWARD_ONLY) return fail(SPM_ERR_INVALID_ARG, "unknown cp_loss flag");
  for (int k = 0; k < p->N; ++k)
    if (!factors[k]) return fail(SPM_ERR_INVALID_ARG, "null factor pointer");
  int st = ensure_als(p);
  if (st) return st;
  if ((st = ensure(p, (void**)&p->d_elem[2], (size_t)p->nnz * p->es))) return st;
  p->res_valid = 0;
  p->res_grad = -1;
  const int n0 = p->cur_mode;
  if (!(flags & SPM_LOSS_FORWARD_ONLY) && loss_fusable(p, factors)) {
    // one pass: residuals, the mode-n0 gradient of L, the residual copy in the
    // next mode's order, and per-block partial sums of e^2
    if ((st = ensure(p, (void**)&p->d_lossgrad, (size_t)max_dim(p) * p->R * 4))) return st;
    const size_t need = (size_t)std::max(1, p->md[(size_t)n0].nblk);
    if (need > p->lpart_cap) {
      if (p->d_lpart) {
        cudaFree(p->d_lpart);
        p->dev_bytes -= std::max<size_t>(p->lpart_cap * 8, 16);
        p->d_lpart = nullptr;
      }
      if ((st = plan_dalloc(p, (void**)&p->d_lpart, need * 8))) return st;
      p->lpart_cap = need;
    }
    st = run_mode(p, n0, factors, p->d_lossgrad, cur_elems(p), p->d_elem[2], nullptr,
                  p->d_lpart);
    if (st) return st;
    st = launch_loss_reduce(p->d_lpart, p->md[(size_t)n0].nblk, loss, p->d_scal + 2, p->stream);
    if (st) return st;
    p->res_valid = 1;
    p->res_mode = (n0 + 1) % p->N;
    p->res_grad = n0;
    return p->checks ? spmttkrp_device_status(p) : SPM_OK;
  }
  FactorPtrs fp;
  for (int k = 0; k < p->N; ++k) fp.p[k] = factors[k];
  st = launch_cp_fwd(cur_elems(p), p->d_elem[2], p->nnz, p->es, p->N, fp, p->pack, p->R,
                     p->dtype, p->d_red, p->red_nb, loss, p->d_scal + 2, p->stream);
  if (st) return st;
  p->res_valid = 1;
  p->res_mode = p->cur_mode;
  return SPM_OK;
}

int cp_loss_fwd(spmttkrp_plan_t p, const void* const* factors, float* loss) {
  return cp_loss_fwd_ex(p, factors, loss, 0);
}

int cp_loss_bwd(spmttkrp_plan_t p, const void* const* factors, const float* grad_out,
                float* const* grads) {
  NvtxRange range("cp_loss_bwd");
  if (!p || p->destroyed) return fail(SPM_ERR_INVALID_ARG, "null or destroyed plan");
  if (p->host_only) return fail(SPM_ERR_STATE, "plan was built host-only");
  if (!factors || !grad_out || !grads) return fail(SPM_ERR_INVALID_ARG, "null argument");
  for (int k = 0; k < p->N; ++k)
    if (!factors[k] || !grads[k]) return fail(SPM_ERR_INVALID_ARG, "null factor or grad");
  if (!p->res_valid) return fail(SPM_ERR_STATE, "cp_loss_bwd needs a preceding cp_loss_fwd");
  // the residual copy ping-pongs between its own buffer and the free half of
  // the working-copy pair (both halves are free while the resident mode-0 copy
  // is the working copy); it is dropped afterwards, so the last pass writes no
  // remap
  uint8_t* bufs[2] = {p->d_elem[2], p->d_elem[1 - p->cur_buf]};
  int cur = 0, first = 0;
  if (p->res_grad >= 0) {  // the fused forward's mode: its gradient, scaled
    const int g = p->res_grad;
    int st = launch_scale_copy(p->d_lossgrad, grads[g], p->dims[(size_t)g] * p->R, grad_out,
                               p->stream);
    if (st) return st;
    first = 1;
  }
  for (int i = first; i < p->N; ++i) {
    const int n = (p->res_mode + i - first) % p->N;
    int st = run_mode(p, n, factors, grads[n], bufs[cur], i == p->N - 1 ? nullptr : bufs[1 - cur],
                      grad_out);
    if (st) return st;
    if (p->nnz > 0) cur ^= 1;
  }
  p->res_valid = 0;
  p->res_grad = -1;
  return p->checks ? spmttkrp_device_status(p) : SPM_OK;
}

int spmttkrp_autotune(spmttkrp_plan_t p, const void* const* factors, float* const* scratch,
                      int flags) {
  NvtxRange range("spmttkrp autotune");
  if (!p || p->destroyed) return fail(SPM_ERR_INVALID_ARG, "null or destroyed plan");
  if (p->host_only) return fail(SPM_ERR_STATE, "plan was built host-only");
  if (!factors || !scratch) return fail(SPM_ERR_INVALID_ARG, "null argument");
  if (p->nnz == 0) return SPM_OK;
  const std::string key = tune_key(p);
  int nps = 0, tile = 0, variant = 0, stages = 0;
  // Algorithm 1's blocks are fixed when the plan is built (the working copy is
  // ordered by them): only the tile, ring depth and form are tuned then
  const bool fixed_blocks = p->partition == 1;
  // n_per_sm < 0: the plan's size-based default block count
  const int nblk_default = default_nblk(p->nnz, p->num_sms, 0);
  auto nblk_for = [&](int n_per_sm) {
    if (fixed_blocks) return p->mh[0].nblk;
    return n_per_sm < 0 ? nblk_default : std::max(1, n_per_sm * p->num_sms);
  };
  if (!(flags & 1) && cache_lookup(key, &nps, &tile, &variant, &stages))
    return apply_config(p, nblk_for(nps), tile, variant, stages);

  struct Cand {
    int nps, tile, variant, stages;
  };
  // blocks per SM: warp blocks (form 0) from 48 to 768 (each block >= 256
  // nonzeros), tiles whose rings keep two CTAs per SM, 2- or 3-stage rings;
  // CTA blocks (form 1) in multiples of 4
  std::vector<Cand> cands;
  bool default_listed = false;
  for (int n : {48, 96, 192, 384, 768}) default_listed |= n * p->num_sms == nblk_default;
  for (int n : {-1, 48, 96, 192, 384, 768}) {
    if (n < 0 && (default_listed || fixed_blocks)) continue;
    if (n > 0 && (int64_t)n * p->num_sms * 256 > p->nnz && n > 48) continue;
    if (fixed_blocks && n > 48) continue;
    for (int t : {64, 128, 256})
      for (int sg : {2, 3})
        if (mttkrp_smem_bytes(p->es, t, p->R, p->dtype, sg) <= 110 * 1024)
          cands.push_back({n, t, 0, sg});
  }
  for (int n : {4, 8, 16, 32}) {
    if (p->pack.packed) break;  // form 1 reads plain indices only
    if ((int64_t)n * p->num_sms * 1024 > p->nnz && n > 4) continue;
    if (fixed_blocks && n > 4) continue;
    cands.push_back({n, p->tile, 1, p->stages});
  }
  cudaEvent_t e0, e1;
  SPM_CUDA(cudaEventCreate(&e0));
  SPM_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  Cand win = cands.front();
  int st = SPM_OK;
  for (const Cand& c : cands) {
    st = apply_config(p, nblk_for(c.nps), c.tile, c.variant, c.stages);
    if (st) break;
    st = spmttkrp_sweep(p, factors, scratch, 0);  // warm
    if (st) break;
    std::vector<float> ms;
    for (int rep = 0; rep < 3 && !st; ++rep) {
      cudaEventRecord(e0, p->stream);
      st = spmttkrp_sweep(p, factors, scratch, 0);
      cudaEventRecord(e1, p->stream);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      ms.push_back(t);
    }
    if (st) break;
    std::sort(ms.begin(), ms.end());
    if (ms[1] < best) {
      best = ms[1];
      win = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  st = apply_config(p, nblk_for(win.nps), win.tile, win.variant, win.stages);
  if (st) return st;
  cache_store(key, win.nps, win.tile, win.variant, win.stages);
  return SPM_OK;
}

}  // extern "C"
