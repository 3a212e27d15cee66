// Host runtime and C ABI of libkkm (declared in include/kkm.h).
//
// One kkm_ctx owns one run: the device state sized at kkm_init (see
// kkm_internal.cuh for the layout), the stream its work goes to, and a host
// mirror of the iteration counter. kkm_step queues the whole iteration as a
// fixed sequence of kernels on that stream. No step allocates, and nothing
// crosses to the host unless the caller asks for a host result.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <tuple>
#include <unordered_set>
#include <vector>

#include "kkm_internal.cuh"
#include "../../include/kkm.h"

#define KKM_API extern "C" __attribute__((visibility("default")))

using kkm::Dev;

// Steps of one kkm_steps_host chunk (one graph replay per chunk).
constexpr int HOST_CHUNK = 16;

struct kkm_ctx {
  Dev s{};
  cudaStream_t stream = nullptr;
  int32_t* h_status = nullptr;      // page-locked copy of the device status word (read after each sync)
  int device = 0;
  int64_t iteration = 1;
  int32_t max_iters = 0;
  int32_t wmax = 0;          // most rows a window can hold
  bool poisoned = false;
  bool use_tc = false;
  std::string err;
  std::vector<void*> allocs;
  int32_t* d_init_idx = nullptr;
  // kkm_step_host's staging area: page-locked, device-mapped memory, so the
  // step's kernels read the indices and write the results across the
  // CPU-GPU link with no copy-engine transfer. h_* are the host views.
  void* h_stage = nullptr;
  int32_t* h_hbatch = nullptr;
  int32_t* h_hassign = nullptr;
  double* h_hobj = nullptr;
  int32_t* d_hbatch = nullptr;
  int32_t* d_hassign = nullptr;
  double* d_hobj = nullptr;
  bool host_pending = false;         // a kkm_step_host call queued work it has not yet waited for
  // kkm_steps_host's staging: two slots of HOST_CHUNK steps each, page-locked
  // and device-mapped like h_stage. A slot holds, for step i of its chunk, the
  // indices at i * nb4 and the assignments at (HOST_CHUNK + i) * nb4, then the
  // chunk's f_B values. One graph per slot and index source replays a chunk.
  void* h_qstage = nullptr;
  char* h_qslot[2] = {nullptr, nullptr};
  char* d_qslot[2] = {nullptr, nullptr};
  size_t q_nb4 = 0;
  cudaEvent_t qdone[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec_q[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [slot][host indices]
  bool fin_pending = false;          // the last step's k_finalize is still to run (see flush)
  double* d_objpart = nullptr;
  double* d_obj2 = nullptr;   // kkm_fit: f_B before and after the update
  int32_t objpart_len = 0;
  bool timing = false;
  int32_t timing_reps = 1;          // distance-pass launches between one pair of events
  std::vector<cudaEvent_t> ev;
  std::vector<int32_t> ev_reps;     // launches between each recorded pair
  int64_t ev_used = 0;
  int64_t launches = 0;       // kernels launched (host count)
  alignas(64) unsigned char tmaps[512];   // TMA descriptors of the tensor-core passes (4 x 128 B)
  // CUDA graph of one step (kkm_graph_enable): captured on a private stream
  // per set of kkm_step pointer arguments and launched on `stream`
  bool graph_on = false;
  int64_t eager_steps = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t gexec_multi = nullptr;     // kkm_steps: STEPS_PER_GRAPH sampler steps per replay
  // table form of Algorithm 1 (kkm_config.algo = KKM_ALGO_TABLE)
  bool tab = false;
  kkm::TabBuf tb{};
  kkm::Dev g{};                              // Gram view: A = every row of X, B = the support buffer
  alignas(64) unsigned char gmaps[512];      // its TMA descriptors
  double* d_tabblk = nullptr;
  int32_t tabblk_n = 0;
  // workspace of kkm_objective_fwd / _bwd (grows with m, freed with the context)
  double* gws = nullptr;
  size_t gws_len = 0;
};

namespace {

thread_local std::string g_init_error;

kkm_status fail(kkm_ctx* c, kkm_status st, const std::string& msg) {
  if (c) c->err = msg; else g_init_error = msg;
  return st;
}

kkm_status cuda_fail(kkm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, KKM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
cudaError_t dalloc(kkm_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) { *p = nullptr; return e; }
  e = cudaMemset(q, 0, bytes);
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return e;
}

void free_all(kkm_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  for (int q = 0; q < 2; ++q) {
    for (int h = 0; h < 2; ++h) {
      if (c->gexec_q[q][h]) cudaGraphExecDestroy(c->gexec_q[q][h]);
      c->gexec_q[q][h] = nullptr;
    }
    if (c->qdone[q]) cudaEventDestroy(c->qdone[q]);
    c->qdone[q] = nullptr;
  }
  if (c->h_qstage) cudaFreeHost(c->h_qstage);
  c->h_qstage = nullptr;
  if (c->gexec_multi) cudaGraphExecDestroy(c->gexec_multi);
  c->gexec_multi = nullptr;
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->gws) cudaFree(c->gws);
  c->gws = nullptr;
  c->gws_len = 0;
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  if (c->h_status) cudaFreeHost(c->h_status);
  c->h_status = nullptr;
  if (c->h_stage) cudaFreeHost(c->h_stage);
  c->h_stage = nullptr;
}

kkm_status check_usable(kkm_ctx* c) {
  if (!c) return fail(nullptr, KKM_EINVAL, "null context");
  if (c->poisoned) return fail(c, KKM_ESTATE, "context poisoned by an earlier device-side fault");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, KKM_ECUDA, "cudaSetDevice failed");
  return KKM_OK;
}

// A step (windows form, kkm_step) ends with its window pass and leaves its
// weight update, k_finalize, to the start of the next step, where it runs
// beside the next batch's gather. Every call that reads or replaces the
// centers first runs it here (on the context's stream).
kkm_status flush(kkm_ctx* c) {
  if (!c->fin_pending) return KKM_OK;
  cudaError_t e = kkm::launch_finalize(c->s, c->stream, true);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->s.fin_pending, 0, sizeof(int32_t), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "pending weight update");
  c->fin_pending = false;
  c->launches += 1;
  return KKM_OK;
}

// check_usable, then the pending weight update.
kkm_status check_ready(kkm_ctx* c) {
  const kkm_status st = check_usable(c);
  return st != KKM_OK ? st : flush(c);
}

// Synchronises the stream and turns sticky device status bits into an error.
// The status word comes back with the stream's own work (an async copy into
// page-locked memory), so a call waits for the device once.
kkm_status sync_and_check(kkm_ctx* c) {
  cudaError_t e = cudaMemcpyAsync(c->h_status, c->s.status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "status read");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  const int32_t st = *c->h_status;
  if (st != 0) {
    c->poisoned = true;
    std::string m = "device status:";
    if (st & kkm::ST_BAD_BATCH_INDEX) m += " batch/data index out of range;";
    if (st & kkm::ST_BAD_ASSIGN) m += " forced assignment out of range;";
    if (st & kkm::ST_CAPACITY) m += " capacity exceeded;";
    if (st & kkm::ST_TIMEOUT) m += " bounded wait timed out;";
    return fail(c, (st & kkm::ST_TIMEOUT) ? KKM_ETIMEOUT : KKM_EINVAL, m);
  }
  return KKM_OK;
}

#define KKM_CU(expr, where)                                  \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return cuda_fail(c, _e, where);   \
  } while (0)

kkm_status launch_distance_pass(kkm_ctx* c, int rows) {
  if (c->use_tc) KKM_CU(kkm::launch_dist_tc(c->s, c->tmaps, rows, c->stream), "distance kernel (tcgen05)");
  else KKM_CU(kkm::launch_dist_simt(c->s, rows, c->stream), "distance kernel");
  return KKM_OK;
}

}  // namespace

KKM_API int32_t kkm_version(void) { return KKM_ABI_VERSION; }

KKM_API const char* kkm_last_error(const kkm_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

KKM_API kkm_status kkm_form_supported(int32_t precision, int32_t cc_major, int32_t cc_minor) {
  if (precision < KKM_PREC_FP32 || precision > KKM_PREC_TF32) return KKM_EINVAL;
  if (precision == KKM_PREC_FP32) return KKM_OK;       // CUDA-core kernels, any device the build runs on
  return (cc_major == 10 && cc_minor == 3) ? KKM_OK : KKM_ENOTSUP;   // tcgen05 passes built for sm_103a
}

KKM_API kkm_status kkm_kmeanspp(const float* X, int64_t n, int32_t d, int64_t ldx, int32_t k,
                                const kkm_kernel* kernel, uint64_t seed, int64_t* out_idx, void* stream) {
  if (!X || !kernel || !out_idx) return fail(nullptr, KKM_EINVAL, "X, kernel and out_idx are required");
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(nullptr, KKM_EINVAL, "n must be in [1, 2^31)");
  if (d < 1 || d > 4096) return fail(nullptr, KKM_EINVAL, "d must be in [1, 4096]");
  if (ldx < d) return fail(nullptr, KKM_EINVAL, "ldx must be >= d");
  if (k < 1 || k > n) return fail(nullptr, KKM_EINVAL, "k must be in [1, n]");
  if (kernel->kind < KKM_GAUSSIAN || kernel->kind > KKM_POLY)
    return fail(nullptr, KKM_EINVAL, "unknown kernel kind");
  if ((kernel->kind == KKM_GAUSSIAN || kernel->kind == KKM_LAPLACIAN) &&
      !(std::isfinite(kernel->param) && kernel->param > 0.0))
    return fail(nullptr, KKM_EINVAL, "kernel param (kappa or sigma) must be finite and > 0");
  if (kernel->kind == KKM_POLY &&
      (kernel->degree < 1 || kernel->degree > 8 || !std::isfinite(kernel->coef0)))
    return fail(nullptr, KKM_EINVAL, "polynomial degree must be in [1, 8] with a finite coef0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* d2 = nullptr;
  double* part = nullptr;
  int64_t* chosen = nullptr;
  const int64_t nblk = (n + 7) / 8;
  cudaError_t e = cudaMalloc(&d2, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&part, nblk * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&chosen, k * sizeof(int64_t));
  if (e == cudaSuccess)
    e = kkm::launch_kmeanspp(X, n, d, ldx, k, kernel->kind, kernel->param, kernel->coef0, kernel->degree, seed, d2,
                             part, chosen, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_idx, chosen, k * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d2);
  cudaFree(part);
  cudaFree(chosen);
  if (e != cudaSuccess) return fail(nullptr, KKM_ECUDA, std::string("k-means++: ") + cudaGetErrorString(e));
  return KKM_OK;
}

KKM_API kkm_status kkm_init(kkm_ctx** out, const float* X, int64_t n, int32_t d, int64_t ldx,
                            int32_t k, const kkm_kernel* kernel, int32_t b, const kkm_config* cfg,
                            const int64_t* init_idx, void* stream) {
  if (!out) return fail(nullptr, KKM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!X || !kernel || !cfg) return fail(nullptr, KKM_EINVAL, "X, kernel and cfg are required");
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(nullptr, KKM_EINVAL, "n must be in [1, 2^31)");
  if (d < 1 || d > 4096) return fail(nullptr, KKM_EINVAL, "d must be in [1, 4096]");
  if (ldx < d) return fail(nullptr, KKM_EINVAL, "ldx must be >= d");
  if (k < 1 || k > 1024 || k > n) return fail(nullptr, KKM_EINVAL, "k must be in [1, min(n, 1024)]");
  if (b < 1 || b > 8192) return fail(nullptr, KKM_EINVAL, "b must be in [1, 8192]");
  if (kernel->kind < KKM_GAUSSIAN || kernel->kind > KKM_POLY)
    return fail(nullptr, KKM_EINVAL, "unknown kernel kind");
  if ((kernel->kind == KKM_GAUSSIAN || kernel->kind == KKM_LAPLACIAN) &&
      !(std::isfinite(kernel->param) && kernel->param > 0.0))
    return fail(nullptr, KKM_EINVAL, "kernel param (kappa or sigma) must be finite and > 0");
  if (kernel->kind == KKM_POLY &&
      (kernel->degree < 1 || kernel->degree > 8 || !std::isfinite(kernel->coef0)))
    return fail(nullptr, KKM_EINVAL, "polynomial degree must be in [1, 8] with a finite coef0");
  if (cfg->lr != KKM_LR_BETA && cfg->lr != KKM_LR_CONST && cfg->lr != KKM_LR_SKLEARN)
    return fail(nullptr, KKM_EINVAL, "unknown learning rate");
  if (cfg->lr == KKM_LR_CONST && !(cfg->eta > 0.0 && cfg->eta <= 1.0))
    return fail(nullptr, KKM_EINVAL, "eta must be in (0, 1]");
  if (cfg->dist_tile != 0 && cfg->dist_tile != 64 && cfg->dist_tile != 128 && cfg->dist_tile != 256)
    return fail(nullptr, KKM_EINVAL, "dist_tile must be 0, 64, 128 or 256");
  if (cfg->algo != KKM_ALGO_WINDOWS && cfg->algo != KKM_ALGO_TABLE)
    return fail(nullptr, KKM_EINVAL, "unknown algo");
  const bool tab = cfg->algo == KKM_ALGO_TABLE;
  if (tab && cfg->tau > 0)
    return fail(nullptr, KKM_EINVAL, "the table form runs Algorithm 1: tau must be <= 0");
  if (tab && (int64_t)n * k >= (int64_t(1) << 40)) return fail(nullptr, KKM_EINVAL, "n*k too large for the table");
  if (cfg->precision < KKM_PREC_FP32 || cfg->precision > KKM_PREC_TF32)
    return fail(nullptr, KKM_EINVAL, "unknown precision");
  if (cfg->tau > 1000000) return fail(nullptr, KKM_EINVAL, "tau must be <= 1e6");
  if (cfg->tau <= 0 && cfg->max_iters < 1 && !tab)
    return fail(nullptr, KKM_EINVAL, "an untruncated run needs max_iters >= 1");
  if (init_idx)
    for (int j = 0; j < k; ++j)
      if (init_idx[j] < 0 || init_idx[j] >= n)
        return fail(nullptr, KKM_EINVAL, "init_idx entry out of [0, n)");

  // table form: the support store is one buffer of the center-sorted batch
  // (b rows in blocks of whole tiles, at most 256 rows each, plus slack),
  // sized as k regions
  const int64_t wmax = tab ? b : cfg->tau > 0 ? (int64_t)cfg->tau + b : 1 + (int64_t)cfg->max_iters * b;
  const int64_t cap = tab ? kkm::round_up((b + 256LL * k + 512 + k - 1) / k, 8)
                          : (cfg->tau > 0 ? kkm::round_up(2LL * cfg->tau + 4LL * b + 8, 8)
                                          : kkm::round_up(wmax, 8)) + kkm::REGION_PAD;
  const int64_t srows = (int64_t)k * cap + 256;
  if (srows >= (int64_t(1) << 31)) return fail(nullptr, KKM_EINVAL, "support store too large (k*cap)");

  kkm_ctx* c = new (std::nothrow) kkm_ctx();
  if (!c) return fail(nullptr, KKM_ENOMEM, "host allocation failed");
  auto bail = [&](kkm_status st) {
    g_init_error = c->err;
    free_all(c);
    delete c;
    return st;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    c->err = "no CUDA device";
    return bail(KKM_ECUDA);
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  c->stream = static_cast<cudaStream_t>(stream);
  c->max_iters = cfg->max_iters;
  c->wmax = (int32_t)wmax;

  Dev& s = c->s;
  s.n = n; s.d = d; s.k = k; s.b = b; s.ldx = ldx; s.X = X;
  s.tau = cfg->tau > 0 ? cfg->tau : 0;
  s.cap = (int32_t)cap;
  s.nbcap = tab ? 2 : cfg->tau > 0 ? cfg->tau + 2 : cfg->max_iters + 2;
  c->tab = tab;
  s.form = cfg->precision;
  s.kind = kernel->kind; s.degree = kernel->degree; s.lr = cfg->lr;
  s.param = kernel->param; s.coef0 = kernel->coef0; s.eta = cfg->eta;
  s.inv_b = 1.0 / (double)b;
  s.negc = (kernel->kind == KKM_GAUSSIAN || kernel->kind == KKM_LAPLACIAN)
               ? (float)(-1.4426950408889634 / kernel->param) : 0.0f;
  s.num_sms = sms > 0 ? sms : 148;
  s.seed = cfg->seed;
  s.pre_b = tab ? 0 : 1;
  if (s.form == kkm::FORM_FP32) { s.dp = 0; s.ld = (int32_t)kkm::round_up(d, 16); }
  else if (s.form == kkm::FORM_TF32) { s.dp = (int32_t)kkm::round_up(d, 32); s.ld = s.dp; }
  else { s.dp = (int32_t)kkm::round_up(d, 64); s.ld = 2 * s.dp; }
  s.bpad = (int32_t)kkm::round_up(b, 128);

  // the tensor-core forms run only on the tcgen05 passes built for sm_103a:
  // there is no CUDA-core stand-in for them
  c->use_tc = false;
  if (s.form != kkm::FORM_FP32) {
    int maj = 0, min = 0;
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, c->device);
    cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, c->device);
    if (kkm_form_supported(s.form, maj, min) != KKM_OK) {
      c->err = "the BF16, split-BF16 and TF32 forms need a compute capability 10.3 device (tcgen05)";
      return bail(KKM_ENOTSUP);
    }
    c->use_tc = true;
  }
  s.tn = c->use_tc ? (cfg->dist_tile == 0 ? (tab ? 64 : 256) : cfg->dist_tile) : 64;
  s.ppt = c->use_tc ? kkm::tc_parts_per_tile(s.tn) : 1;
  s.pair_rows = c->use_tc ? 128 : 64;
  s.pair_cols = c->use_tc ? kkm::WPASS_TNV : 64;
  s.walign = c->use_tc ? 4 : 1;
  const int64_t TR = s.pair_rows, TC = s.pair_cols;   // window-pass tile
  s.max_tiles = tab ? (int32_t)(k + (b + s.tn - 1) / s.tn + 1)
                    : (int32_t)((int64_t)k * ((wmax + s.tn - 1) / s.tn + 1));
  // window-pass tiles per step: per center, ceil((rows + a) / TR) x ceil((cols + a) / TC)
  // for the dropped rows against the window and the new block, and for the new
  // block against itself, with a < walign rows of alignment slack
  const int64_t smax = (int64_t)k * wmax, al = s.walign;
  const int64_t p1 = ((smax + al * k + TR - 1) / TR + k) * ((wmax + b + al + TC - 1) / TC + 1);
  const int64_t p2 = ((b + al * k + TR - 1) / TR + k) * ((b + al + TC - 1) / TC + 1);
  if (p1 + p2 >= (int64_t(1) << 31)) {
    c->err = "window pass would need too many tiles";
    return bail(KKM_EINVAL);
  }
  s.max_pairs = (int32_t)(p1 + p2);

  const int esz = kkm::f32_rows(s.form) ? 4 : 2;
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, count)                                        \
  do {                                                           \
    e = dalloc(c, &(ptr), (size_t)(count));                      \
    if (e != cudaSuccess) {                                      \
      c->err = std::string("device allocation: ") + cudaGetErrorString(e); \
      return bail(KKM_ENOMEM);                                   \
    }                                                            \
  } while (0)
  ALLOC(s.bidx, b);
  if (esz == 4) ALLOC(s.xb32, (size_t)s.bpad * s.ld);
  else ALLOC(s.xbh, (size_t)s.bpad * s.ld);
  ALLOC(s.xbn, s.bpad);
  ALLOC(s.xbi, s.bpad);
  if (esz == 4) ALLOC(s.y32, (size_t)srows * s.ld);
  else ALLOC(s.ybh, (size_t)srows * s.ld);
  ALLOC(s.yn, srows);
  ALLOC(s.yi, srows);
  ALLOC(s.w64, srows);
  ALLOC(s.w32, srows);
  ALLOC(s.head, k); ALLOC(s.tail, k); ALLOC(s.c1, k); ALLOC(s.wsum, k); ALLOC(s.cnorm, k);
  ALLOC(s.cnorm32, k); ALLOC(s.cmpart, (size_t)k * 32);
  ALLOC(s.blk_iter, (size_t)k * s.nbcap); ALLOC(s.blk_cnt, (size_t)k * s.nbcap);
  ALLOC(s.blk_first, k); ALLOC(s.blk_num, k);
  ALLOC(s.assign, s.bpad); ALLOC(s.mind, s.bpad); ALLOC(s.inner_a, s.bpad);
  ALLOC(s.counts, k); ALLOC(s.alpha, k); ALLOC(s.coff, k + 1); ALLOC(s.perm, s.bpad); ALLOC(s.mvdst, s.bpad);
  ALLOC(s.cmc, k); ALLOC(s.ncum, k); ALLOC(c->d_obj2, 2); ALLOC(s.plan, k); ALLOC(s.comp_off, k); ALLOC(s.comp_total, 1);
  ALLOC(s.tiles, s.max_tiles); ALLOC(s.ntiles, 1); ALLOC(s.tile_first, k); ALLOC(s.tile_cnt, k);
  ALLOC(s.part, (size_t)s.max_tiles * s.ppt * s.bpad);
  ALLOC(s.wpairs, s.max_pairs); ALLOC(s.nwpairs, 1); ALLOC(s.wpair_first, k); ALLOC(s.wpair_cnt, k);
  // window-pass partial slots (of four sums) per item: one per group of a team
  s.wslots = c->use_tc ? kkm::tc_parts_per_tile(kkm::WPASS_TNV) : 4;
  ALLOC(s.wpart, (size_t)s.max_pairs * s.wslots * 4);
  ALLOC(s.iter, 1); ALLOC(s.fin_pending, 1); ALLOC(s.status, 1); ALLOC(s.stats, 3); ALLOC(s.obj, 1);
  {
    // the finalise step's rate sqrt(n/b) and 1/n, by the host's correctly rounded
    // FP64 operations (the same values the device would compute)
    double* rt = nullptr;
    ALLOC(rt, 2 * ((int64_t)b + 1));
    std::vector<double> h(2 * ((size_t)b + 1), 0.0);
    for (int m = 1; m <= b; ++m) {
      h[m] = 1.0 / (double)m;
      h[b + 1 + m] = std::sqrt((double)m * s.inv_b);
    }
    e = cudaMemcpy(rt, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      c->err = std::string("rate table: ") + cudaGetErrorString(e);
      return bail(KKM_ECUDA);
    }
    s.rtab = rt;
  }
  e = cudaHostAlloc(reinterpret_cast<void**>(&c->h_status), sizeof(int32_t), cudaHostAllocDefault);
  if (e != cudaSuccess) {
    c->h_status = nullptr;
    c->err = std::string("host allocation: ") + cudaGetErrorString(e);
    return bail(KKM_ENOMEM);
  }
  ALLOC(c->d_init_idx, k);
  {
    // kkm_step_host's staging area: [b indices][b assignments][f_B], mapped into the device
    const size_t nb4 = ((size_t)b * sizeof(int32_t) + 15) & ~(size_t)15;
    e = cudaHostAlloc(&c->h_stage, 2 * nb4 + 16, cudaHostAllocMapped);
    void* dev = nullptr;
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&dev, c->h_stage, 0);
    if (e != cudaSuccess) {
      c->err = std::string("mapped host allocation: ") + cudaGetErrorString(e);
      return bail(KKM_ENOMEM);
    }
    std::memset(c->h_stage, 0, 2 * nb4 + 16);
    char* hb = static_cast<char*>(c->h_stage);
    char* db = static_cast<char*>(dev);
    c->h_hbatch = reinterpret_cast<int32_t*>(hb);
    c->h_hassign = reinterpret_cast<int32_t*>(hb + nb4);
    c->h_hobj = reinterpret_cast<double*>(hb + 2 * nb4);
    c->d_hbatch = reinterpret_cast<int32_t*>(db);
    c->d_hassign = reinterpret_cast<int32_t*>(db + nb4);
    c->d_hobj = reinterpret_cast<double*>(db + 2 * nb4);
    // kkm_steps_host's two chunk slots and their completion events
    const size_t slot = (2 * HOST_CHUNK * nb4 + 8 * HOST_CHUNK + 127) & ~(size_t)127;
    e = cudaHostAlloc(&c->h_qstage, 2 * slot, cudaHostAllocMapped);
    dev = nullptr;
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&dev, c->h_qstage, 0);
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = cudaEventCreateWithFlags(&c->qdone[q], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      c->err = std::string("mapped host allocation (chunk staging): ") + cudaGetErrorString(e);
      return bail(KKM_ENOMEM);
    }
    std::memset(c->h_qstage, 0, 2 * slot);
    c->q_nb4 = nb4;
    for (int q = 0; q < 2; ++q) {
      c->h_qslot[q] = static_cast<char*>(c->h_qstage) + q * slot;
      c->d_qslot[q] = static_cast<char*>(dev) + q * slot;
    }
  }
  c->objpart_len = 1024;
  ALLOC(c->d_objpart, c->objpart_len);
  if (tab) {
    // the Gram view: A = every row of X in the operand form
    const int64_t npad = kkm::round_up(n, 128);
    kkm::Dev& g = c->g;
    g = s;
    g.pre_b = 0;       // its B operand (the laid-out batch) is written by the kernel just before it
    g.xb32 = nullptr;
    g.xbh = nullptr;
    if (esz == 4) ALLOC(g.xb32, (size_t)npad * s.ld);
    else ALLOC(g.xbh, (size_t)npad * s.ld);
    ALLOC(g.xbn, npad);
    ALLOC(g.xbi, npad);
    g.bpad = (int32_t)npad;
    ALLOC(g.part, (size_t)s.max_tiles * s.ppt * npad);
    ALLOC(c->tb.T, (size_t)k * n);
    ALLOC(c->tb.bs_off, k + 1);
    c->tb.part = g.part;
    c->tb.npad = npad;
    c->tb.bs_rows = (int32_t)srows;
    c->tabblk_n = (int32_t)std::min<int64_t>(4 * s.num_sms, (n + 255) / 256);
    ALLOC(c->d_tabblk, c->tabblk_n);
  }
#undef ALLOC

  // initial centers: caller's indices, or k distinct ones from SplitMix64
  std::vector<int32_t> h_init(k);
  if (init_idx) {
    for (int j = 0; j < k; ++j) h_init[j] = (int32_t)init_idx[j];
  } else {
    std::unordered_set<int64_t> seen;
    uint64_t ctr = 0;
    for (int j = 0; j < k; ++j) {
      int64_t i;
      do { i = kkm::index_below(kkm::splitmix64(cfg->seed ^ 0x6a09e667f3bcc909ull, ctr++), n); }
      while (seen.count(i));
      seen.insert(i);
      h_init[j] = (int32_t)i;
    }
  }
  const int64_t one = 1;
  e = cudaMemcpyAsync(c->d_init_idx, h_init.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.iter, &one, sizeof(one), cudaMemcpyHostToDevice, c->stream);
  if (tab) {
    // T[j][x] = K(x, x_init_j): the Gram pass against the k initial rows, then T = S
    if (e == cudaSuccess) e = kkm::launch_tab_init(s, c->g, c->tb, c->d_init_idx, c->stream);
    if (e == cudaSuccess && c->use_tc) e = kkm::tc_prepare(c->g, c->gmaps);
    if (e == cudaSuccess)
      e = c->use_tc ? kkm::launch_dist_tc(c->g, c->gmaps, (int)n, c->stream)
                    : kkm::launch_dist_simt(c->g, (int)n, c->stream);
    if (e == cudaSuccess) e = kkm::launch_tab_update(s, c->tb, true, c->stream);
  } else {
    if (e == cudaSuccess) e = kkm::launch_init_centers(s, c->d_init_idx, c->stream);
    if (e == cudaSuccess && c->use_tc) e = kkm::tc_prepare(s, c->tmaps);
    if (e == cudaSuccess) e = kkm::launch_build_tiles(s, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->err = std::string("initialisation: ") + cudaGetErrorString(e);
    return bail(KKM_ECUDA);
  }
  int32_t st = 0;
  cudaMemcpy(&st, s.status, sizeof(st), cudaMemcpyDeviceToHost);
  if (st != 0) {
    c->err = "initialisation: invalid initial index";
    return bail(KKM_EINVAL);
  }
  *out = c;
  return KKM_OK;
}

// The kernel sequence of one step, queued on `st`.
// rotated (kkm_step, windows form): the previous step's k_finalize first (a
// no-op unless one is pending), the gather beside it, and this step's
// k_finalize left pending. Otherwise (run groups) finalize ends the step.
static kkm_status enqueue_step(kkm_ctx* c, cudaStream_t st, const int32_t* batch_idx,
                               const int32_t* forced_assign, int32_t* assign_out, float* dist_out,
                               double* batch_obj_out, bool timed, bool rotated) {
  const Dev& s = c->s;
  if (c->tab) {
    // table form (Appendix A): distances off the table, sort, lay out the batch,
    // the n x b Gram pass, the norm recurrence, the table update
    KKM_CU(kkm::launch_gather_batch(s, batch_idx, st), "batch gather");
    KKM_CU(kkm::launch_tab_batch_dist(s, c->tb, s.b, forced_assign, assign_out, nullptr, dist_out, true, st),
           "table distances");
    KKM_CU(kkm::launch_tab_plan(s, c->tb, batch_obj_out, st), "sort/layout");
    KKM_CU(kkm::launch_tab_fill(s, c->tb, st), "batch layout");
    if (timed) KKM_CU(cudaEventRecord(c->ev[2 * c->ev_used], st), "timing event");
    for (int r = 0; r < (timed ? c->timing_reps : 1); ++r) {   // the pass is idempotent
      if (c->use_tc) KKM_CU(kkm::launch_dist_tc(c->g, c->gmaps, (int)s.n, st), "Gram pass (tcgen05)");
      else KKM_CU(kkm::launch_dist_simt(c->g, (int)s.n, st), "Gram pass");
    }
    if (timed) {
      KKM_CU(cudaEventRecord(c->ev[2 * c->ev_used + 1], st), "timing event");
      c->ev_reps[c->ev_used++] = c->timing_reps;
    }
    KKM_CU(kkm::launch_tab_center(s, c->tb, st), "norm recurrence");
    KKM_CU(kkm::launch_tab_update(s, c->tb, false, st), "table update");
    return KKM_OK;
  }
  // with batch_idx NULL the gather draws the indices itself (SplitMix64)
  if (rotated) KKM_CU(kkm::launch_finalize(s, st, true), "pending weight update");
  KKM_CU(kkm::launch_gather_batch(s, batch_idx, st, rotated), "batch gather");
  if (timed) KKM_CU(cudaEventRecord(c->ev[2 * c->ev_used], st), "timing event");
  for (int r = 0; r < (timed ? c->timing_reps : 1); ++r) {   // the pass is idempotent
    if (c->use_tc) KKM_CU(kkm::launch_dist_tc(s, c->tmaps, s.b, st, true), "distance kernel (tcgen05)");
    else KKM_CU(kkm::launch_dist_simt(s, s.b, st), "distance kernel");
  }
  if (timed) {
    KKM_CU(cudaEventRecord(c->ev[2 * c->ev_used + 1], st), "timing event");
    c->ev_reps[c->ev_used++] = c->timing_reps;
  }
  KKM_CU(kkm::launch_argmin(s, s.b, forced_assign, assign_out, nullptr, dist_out, true, st), "argmin");
  KKM_CU(kkm::launch_sort_plan(s, batch_obj_out, st, rotated), "sort/plan");
  KKM_CU(kkm::launch_move(s, st), "row moves");
  if (c->use_tc) KKM_CU(kkm::launch_wgram_tc(s, c->tmaps, st), "window Gram (tcgen05)");
  else KKM_CU(kkm::launch_wgram(s, st), "window Gram");
  if (!rotated) KKM_CU(kkm::launch_finalize(s, st), "finalize");
  return KKM_OK;
}

KKM_API kkm_status kkm_step(kkm_ctx* c, const int32_t* batch_idx, const int32_t* forced_assign,
                            int32_t* assign_out, float* dist_out, double* batch_obj_out) {
  kkm_status st = check_usable(c);
  if (st != KKM_OK) return st;
  if (c->s.tau == 0 && !c->tab && c->iteration > c->max_iters)
    return fail(c, KKM_ESTATE, "untruncated run: max_iters iterations already done");
  const bool timed = c->timing && c->ev_used < (int64_t)c->ev.size() / 2;
  if (c->graph_on && !timed && c->eager_steps > 0) {
    const void* key[5] = {batch_idx, forced_assign, assign_out, dist_out, batch_obj_out};
    if (!c->gexec || std::memcmp(key, c->gkey, sizeof(key)) != 0) {
      if (!c->cap_stream)
        KKM_CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
      KKM_CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      st = enqueue_step(c, c->cap_stream, batch_idx, forced_assign, assign_out, dist_out, batch_obj_out, false, true);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
      if (st != KKM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
      cudaGraphExec_t ex = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) return cuda_fail(c, ei, "graph instantiate");
      if (c->gexec) cudaGraphExecDestroy(c->gexec);
      c->gexec = ex;
      std::memcpy(c->gkey, key, sizeof(key));
    }
    KKM_CU(cudaGraphLaunch(c->gexec, c->stream), "graph launch");
  } else {
    st = enqueue_step(c, c->stream, batch_idx, forced_assign, assign_out, dist_out, batch_obj_out, timed, true);
    if (st != KKM_OK) return st;
    ++c->eager_steps;
  }
  // (the previous step's finalize), gather, distance, argmin, sort/plan, moves,
  // window Gram (+ timing repeats)
  c->launches += 7 + (timed ? c->timing_reps - 1 : 0);
  c->fin_pending = !c->tab;
  ++c->iteration;
  return KKM_OK;
}

KKM_API kkm_status kkm_flush(kkm_ctx* c) { return check_ready(c); }

// Iterations the kkm_steps graph holds. Within it consecutive steps meet
// through programmatic dependent launch, as the kernels of one step do;
// between two graph launches they do not.
constexpr int STEPS_PER_GRAPH = 16;

KKM_API kkm_status kkm_steps(kkm_ctx* c, int64_t n) {
  kkm_status st = check_usable(c);
  if (st != KKM_OK) return st;
  if (n < 0) return fail(c, KKM_EINVAL, "n must be >= 0");
  if (c->s.tau == 0 && !c->tab && c->iteration - 1 + n > c->max_iters)
    return fail(c, KKM_ESTATE, "untruncated run: n steps would pass max_iters");
  const bool timed = c->timing && c->ev_used < (int64_t)c->ev.size() / 2;
  int64_t left = n;
  if (c->graph_on && !timed) {
    if (c->eager_steps == 0 && left > 0) {   // the first step runs eagerly, as kkm_step's does
      st = kkm_step(c, nullptr, nullptr, nullptr, nullptr, nullptr);
      if (st != KKM_OK) return st;
      --left;
    }
    if (left >= STEPS_PER_GRAPH && !c->gexec_multi) {
      if (!c->cap_stream)
        KKM_CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
      KKM_CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      for (int i = 0; i < STEPS_PER_GRAPH && st == KKM_OK; ++i)
        st = enqueue_step(c, c->cap_stream, nullptr, nullptr, nullptr, nullptr, nullptr, false, !c->tab);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
      if (st != KKM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
      const cudaError_t ei = cudaGraphInstantiate(&c->gexec_multi, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        c->gexec_multi = nullptr;
        return cuda_fail(c, ei, "graph instantiate");
      }
    }
    for (; left >= STEPS_PER_GRAPH; left -= STEPS_PER_GRAPH) {
      KKM_CU(cudaGraphLaunch(c->gexec_multi, c->stream), "graph launch");
      c->launches += 7 * STEPS_PER_GRAPH;
      c->iteration += STEPS_PER_GRAPH;
      c->fin_pending = !c->tab;
    }
  }
  for (; left > 0; --left) {
    st = kkm_step(c, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st != KKM_OK) return st;
  }
  return KKM_OK;
}

KKM_API kkm_status kkm_graph_enable(kkm_ctx* c, int32_t enable) {
  kkm_status st = check_usable(c);
  if (st != KKM_OK) return st;
  c->graph_on = enable != 0;
  return KKM_OK;
}

KKM_API kkm_status kkm_step_host(kkm_ctx* c, const int32_t* batch_idx, int32_t* assign_out,
                                 double* batch_obj_out) {
  kkm_status st = check_usable(c);
  if (st != KKM_OK) return st;
  const int b = c->s.b;
  if (c->host_pending) {            // an earlier call did not get to wait: its kernels may still read the area
    st = sync_and_check(c);
    if (st != KKM_OK) return st;
    c->host_pending = false;
  }
  // the kernels read the indices and write the results in the mapped area
  if (batch_idx) std::memcpy(c->h_hbatch, batch_idx, (size_t)b * sizeof(int32_t));
  c->host_pending = true;
  st = kkm_step(c, batch_idx ? c->d_hbatch : nullptr, nullptr, assign_out ? c->d_hassign : nullptr,
                nullptr, batch_obj_out ? c->d_hobj : nullptr);
  if (st != KKM_OK) return st;
  st = sync_and_check(c);
  if (st != KKM_OK) return st;
  c->host_pending = false;
  if (assign_out) std::memcpy(assign_out, c->h_hassign, (size_t)b * sizeof(int32_t));
  if (batch_obj_out) *batch_obj_out = *c->h_hobj;
  return KKM_OK;
}

// kkm_steps_host: chunks of HOST_CHUNK steps alternate between the two
// staging slots. While the device runs one chunk the host copies the next
// chunk's indices in and the results of the chunk before out, so the steps
// meet no host round trip. A slot is reused only after its event shows the
// chunk that used it done.
namespace {
int32_t* q_idx(char* slot, size_t nb4, int i) { return reinterpret_cast<int32_t*>(slot + (size_t)i * nb4); }
int32_t* q_asg(char* slot, size_t nb4, int i) {
  return reinterpret_cast<int32_t*>(slot + (size_t)(HOST_CHUNK + i) * nb4);
}
double* q_obj(char* slot, size_t nb4, int i) {
  return reinterpret_cast<double*>(slot + 2 * (size_t)HOST_CHUNK * nb4) + i;
}

// Queues m steps reading slot q (indices from it when host_idx, else the
// built-in sampler) and writing their results there.
kkm_status q_enqueue(kkm_ctx* c, int q, int m, bool host_idx) {
  const size_t nb4 = c->q_nb4;
  char* d = c->d_qslot[q];
  if (c->graph_on && m == HOST_CHUNK) {
    cudaGraphExec_t& ge = c->gexec_q[q][host_idx ? 1 : 0];
    if (!ge) {
      if (!c->cap_stream)
        KKM_CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
      KKM_CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      kkm_status st = KKM_OK;
      for (int i = 0; i < HOST_CHUNK && st == KKM_OK; ++i)
        st = enqueue_step(c, c->cap_stream, host_idx ? q_idx(d, nb4, i) : nullptr, nullptr, q_asg(d, nb4, i),
                          nullptr, q_obj(d, nb4, i), false, !c->tab);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
      if (st != KKM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
      const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        ge = nullptr;
        return cuda_fail(c, ei, "graph instantiate");
      }
    }
    KKM_CU(cudaGraphLaunch(ge, c->stream), "graph launch");
  } else {
    for (int i = 0; i < m; ++i) {
      const kkm_status st = enqueue_step(c, c->stream, host_idx ? q_idx(d, nb4, i) : nullptr, nullptr,
                                         q_asg(d, nb4, i), nullptr, q_obj(d, nb4, i), false, !c->tab);
      if (st != KKM_OK) return st;
      ++c->eager_steps;
    }
  }
  c->launches += 7 * m;
  c->iteration += m;
  c->fin_pending = !c->tab;
  return KKM_OK;
}
}  // namespace

KKM_API kkm_status kkm_steps_host(kkm_ctx* c, int64_t n, const int32_t* batch_idx, int32_t* assign_out,
                                  double* batch_obj_out) {
  kkm_status st = check_usable(c);
  if (st != KKM_OK) return st;
  if (n < 0) return fail(c, KKM_EINVAL, "n must be >= 0");
  if (c->s.tau == 0 && !c->tab && c->iteration - 1 + n > c->max_iters)
    return fail(c, KKM_ESTATE, "untruncated run: n steps would pass max_iters");
  const int b = c->s.b;
  const size_t row = (size_t)b * sizeof(int32_t);
  int64_t j = 0;
  // a context's first step, and every step while timing is on, go one at a
  // time through kkm_step_host (the first step runs eagerly, as kkm_step's does)
  while (j < n && (c->eager_steps == 0 || c->timing)) {
    st = kkm_step_host(c, batch_idx ? batch_idx + j * b : nullptr, assign_out ? assign_out + j * b : nullptr,
                       batch_obj_out ? batch_obj_out + j : nullptr);
    if (st != KKM_OK) return st;
    ++j;
  }
  if (c->host_pending) {
    st = sync_and_check(c);
    if (st != KKM_OK) return st;
    c->host_pending = false;
  }
  int64_t first[2] = {0, 0};
  int cnt[2] = {0, 0};
  // waits for the chunk in slot q and copies its results out
  auto drain = [&](int q) -> kkm_status {
    if (cnt[q] == 0) return KKM_OK;
    const cudaError_t e = cudaEventSynchronize(c->qdone[q]);
    if (e != cudaSuccess) return cuda_fail(c, e, "chunk wait");
    for (int i = 0; i < cnt[q]; ++i) {
      if (assign_out) std::memcpy(assign_out + (first[q] + i) * b, q_asg(c->h_qslot[q], c->q_nb4, i), row);
      if (batch_obj_out) batch_obj_out[first[q] + i] = *q_obj(c->h_qslot[q], c->q_nb4, i);
    }
    cnt[q] = 0;
    return KKM_OK;
  };
  // on a failure nothing may still read or write the slots once the call returns
  auto abort_with = [&](kkm_status s) {
    cudaStreamSynchronize(c->stream);
    return s;
  };
  int q = 0;
  while (j < n) {
    const int m = (int)std::min<int64_t>(HOST_CHUNK, n - j);
    st = drain(q);
    if (st != KKM_OK) return abort_with(st);
    if (batch_idx)
      for (int i = 0; i < m; ++i) std::memcpy(q_idx(c->h_qslot[q], c->q_nb4, i), batch_idx + (j + i) * b, row);
    st = q_enqueue(c, q, m, batch_idx != nullptr);
    if (st != KKM_OK) return abort_with(st);
    const cudaError_t e = cudaEventRecord(c->qdone[q], c->stream);
    if (e != cudaSuccess) return abort_with(cuda_fail(c, e, "chunk event"));
    first[q] = j;
    cnt[q] = m;
    j += m;
    q ^= 1;
  }
  // the device status first: results of a context that went bad are not reported
  st = sync_and_check(c);
  if (st != KKM_OK) return st;
  st = drain(q);   // the older of the two chunks in flight
  if (st == KKM_OK) st = drain(q ^ 1);
  return st;
}

// Runs the distance pass and argmin over query rows in chunks of b rows.
static kkm_status assign_chunks(kkm_ctx* c, const float* Q, int64_t m, int64_t ldq, int32_t* assign_out,
                                float* mind_out, float* dist_out, double* obj_sum) {
  const Dev& s = c->s;
  const bool is_x = (Q == s.X && ldq == s.ldx);
  std::vector<double> partials;
  int pending = 0;
  double total = 0.0;
  for (int64_t r0 = 0; r0 < m; r0 += s.b) {
    const int rows = (int)std::min<int64_t>(s.b, m - r0);
    KKM_CU(kkm::launch_gather_query(s, Q + r0 * ldq, ldq, rows, c->stream), "query gather");
    c->launches += 3 + (obj_sum ? 1 : 0);   // gather, distance, argmin (+ sum)
    if (is_x) {
      // query rows that are data points keep their index, so a point meeting
      // its own support copy gets ||x - y|| = 0 exactly
      std::vector<int32_t> ids(rows);
      for (int r = 0; r < rows; ++r) ids[r] = (int32_t)(r0 + r);
      KKM_CU(cudaMemcpyAsync(s.xbi, ids.data(), rows * sizeof(int32_t), cudaMemcpyHostToDevice,
                             c->stream), "query ids");
      KKM_CU(cudaStreamSynchronize(c->stream), "query ids sync");
    }
    kkm_status st = launch_distance_pass(c, rows);
    if (st != KKM_OK) return st;
    KKM_CU(kkm::launch_argmin(s, rows, nullptr, assign_out ? assign_out + r0 : nullptr,
                              obj_sum ? s.mind : (mind_out ? mind_out + r0 : nullptr),
                              dist_out ? dist_out + r0 * s.k : nullptr, false, c->stream),
           "query argmin");
    if (obj_sum) {
      if (mind_out)
        KKM_CU(cudaMemcpyAsync(mind_out + r0, s.mind, rows * sizeof(float), cudaMemcpyDeviceToDevice,
                               c->stream), "mind copy");
      KKM_CU(kkm::launch_mind_sum(s, rows, 1.0, c->d_objpart + pending, c->stream), "objective sum");
      if (++pending == c->objpart_len || r0 + s.b >= m) {
        partials.resize(pending);
        KKM_CU(cudaMemcpyAsync(partials.data(), c->d_objpart, pending * sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream), "objective download");
        KKM_CU(cudaStreamSynchronize(c->stream), "objective sync");
        for (double v : partials) total += v;
        pending = 0;
      }
    }
  }
  if (obj_sum) *obj_sum = total;
  return KKM_OK;
}

KKM_API kkm_status kkm_assign(kkm_ctx* c, const float* Q, int64_t m, int64_t ldq, int32_t* assign_out,
                              float* mind_out, float* dist_out) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  if (c->tab) return fail(c, KKM_ENOTSUP, "the table form scores only the rows of X (kkm_objective)");
  if (m < 0 || (m > 0 && (!Q || ldq < c->s.d))) return fail(c, KKM_EINVAL, "bad query matrix");
  return assign_chunks(c, Q, m, ldq, assign_out, mind_out, dist_out, nullptr);
}

KKM_API kkm_status kkm_objective(kkm_ctx* c, const float* Q, int64_t m, int64_t ldq, double* out) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  if (!out) return fail(c, KKM_EINVAL, "out is NULL");
  if (c->tab) {
    if (Q) return fail(c, KKM_ENOTSUP, "the table form scores only the rows of X (Q = NULL)");
    KKM_CU(kkm::launch_tab_objective(c->s, c->tb, c->g.xbn, c->d_tabblk, c->tabblk_n, c->stream), "objective");
    st = sync_and_check(c);
    if (st != KKM_OK) return st;
    std::vector<double> h(c->tabblk_n);
    KKM_CU(cudaMemcpy(h.data(), c->d_tabblk, h.size() * sizeof(double), cudaMemcpyDeviceToHost), "objective read");
    double total = 0.0;
    for (double v : h) total += v;
    *out = total / (double)c->s.n;
    return KKM_OK;
  }
  if (!Q) { Q = c->s.X; m = c->s.n; ldq = c->s.ldx; }
  if (m < 1 || ldq < c->s.d) return fail(c, KKM_EINVAL, "bad query matrix");
  double total = 0.0;
  st = assign_chunks(c, Q, m, ldq, nullptr, nullptr, nullptr, &total);
  if (st != KKM_OK) return st;
  st = sync_and_check(c);
  if (st != KKM_OK) return st;
  *out = total / (double)m;
  return KKM_OK;
}

namespace {

kkm_status objective_call(kkm_ctx* c, const float* Q, int64_t m, int64_t ldq, const int32_t* assign,
                          double log_sigma, double* loss, float* delta, const double* grad_loss, float* grad_q,
                          int64_t ldg, double* grad_s) {
  const kkm::Dev& s = c->s;
  if (c->tab) return fail(c, KKM_ENOTSUP, "the table form keeps no support rows");
  if (s.kind != kkm::K_GAUSS && s.kind != kkm::K_LAPLACE)
    return fail(c, KKM_ENOTSUP, "the bandwidth objective needs the Gaussian or Laplacian kernel");
  if (s.d > 1024) return fail(c, KKM_ENOTSUP, "the bandwidth objective supports d <= 1024");
  if (m < 1 || m >= ((int64_t)1 << 30) || !Q || ldq < s.d || !assign)
    return fail(c, KKM_EINVAL, "bad query rows or assignments (1 <= m < 2^30)");
  if (!std::isfinite(log_sigma)) return fail(c, KKM_EINVAL, "log_sigma must be finite");
  const size_t need = kkm::grad_workspace_doubles(s, m);
  if (need > c->gws_len) {
    if (c->gws) KKM_CU(cudaFree(c->gws), "workspace free");
    c->gws = nullptr;
    c->gws_len = 0;
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, need * sizeof(double));
    if (e != cudaSuccess) return fail(c, KKM_ENOMEM, std::string("workspace: ") + cudaGetErrorString(e));
    c->gws = static_cast<double*>(p);
    c->gws_len = need;
    KKM_CU(cudaMemsetAsync(p, 0, need * sizeof(double), c->stream), "workspace clear");   // the kernels' counter starts at 0
  }
  KKM_CU(kkm::launch_objective(s, log_sigma, Q, m, ldq, assign, loss, delta, grad_loss, grad_q, ldg, grad_s,
                               c->gws, c->stream), "objective kernels");
  c->launches += 2;
  return KKM_OK;
}

}  // namespace

KKM_API kkm_status kkm_objective_fwd(kkm_ctx* c, const float* Q, int64_t m, int64_t ldq, const int32_t* assign,
                                     double log_sigma, double* loss_out, float* delta_out) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  if (!loss_out) return fail(c, KKM_EINVAL, "loss_out is NULL");
  return objective_call(c, Q, m, ldq, assign, log_sigma, loss_out, delta_out, nullptr, nullptr, 0, nullptr);
}

KKM_API kkm_status kkm_objective_bwd(kkm_ctx* c, const float* Q, int64_t m, int64_t ldq, const int32_t* assign,
                                     double log_sigma, const double* grad_loss, float* grad_q, int64_t ldg,
                                     double* grad_log_sigma) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  if (!grad_loss || !grad_q || !grad_log_sigma || ldg < c->s.d)
    return fail(c, KKM_EINVAL, "grad_loss, grad_q (ldg >= d) and grad_log_sigma are required");
  return objective_call(c, Q, m, ldq, assign, log_sigma, nullptr, nullptr, grad_loss, grad_q, ldg, grad_log_sigma);
}

KKM_API kkm_status kkm_step_eval(kkm_ctx* c, const int32_t* batch_idx, double* obj_before_dev,
                                 double* obj_after_dev) {
  kkm_status st = check_usable(c);
  if (st != KKM_OK) return st;
  if (!obj_before_dev || !obj_after_dev) return fail(c, KKM_EINVAL, "obj_before_dev and obj_after_dev are required");
  st = kkm_step(c, batch_idx, nullptr, nullptr, nullptr, obj_before_dev);
  if (st != KKM_OK) return st;
  st = flush(c);                     // the step's weight update
  if (st != KKM_OK) return st;
  // f_{B_i}(C_{i+1}): the distance pass and argmin again on the same batch
  // rows, against the windows, weights and norms the step just wrote
  const Dev& s = c->s;
  if (c->tab) {
    KKM_CU(kkm::launch_tab_batch_dist(s, c->tb, s.b, nullptr, nullptr, s.mind, nullptr, false, c->stream),
           "table distances");
  } else {
    if (c->use_tc) KKM_CU(kkm::launch_dist_tc(s, c->tmaps, s.b, c->stream), "distance kernel (tcgen05)");
    else KKM_CU(kkm::launch_dist_simt(s, s.b, c->stream), "distance kernel");
    KKM_CU(kkm::launch_argmin(s, s.b, nullptr, nullptr, s.mind, nullptr, false, c->stream), "argmin");
  }
  KKM_CU(kkm::launch_mind_sum(s, s.b, s.inv_b, obj_after_dev, c->stream), "objective sum");
  c->launches += 3;
  return KKM_OK;
}

KKM_API kkm_status kkm_fit(kkm_ctx* c, int64_t max_iters, double eps, int64_t* iters_done,
                           double* last_improvement) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  if (max_iters < 0 || std::isnan(eps)) return fail(c, KKM_EINVAL, "max_iters >= 0 and a non-NaN eps required");
  int64_t done = 0;
  double imp = 0.0;
  for (; done < max_iters;) {
    st = kkm_step_eval(c, nullptr, c->d_obj2, c->d_obj2 + 1);
    if (st != KKM_OK) return st;
    ++done;
    st = sync_and_check(c);
    if (st != KKM_OK) return st;
    double h[2];
    KKM_CU(cudaMemcpy(h, c->d_obj2, sizeof(h), cudaMemcpyDeviceToHost), "objective read");
    imp = h[0] - h[1];   // the improvement on the batch (Sec. 5)
    if (imp < eps) break;
  }
  if (iters_done) *iters_done = done;
  if (last_improvement) *last_improvement = imp;
  return KKM_OK;
}

KKM_API kkm_status kkm_get_cum_counts(kkm_ctx* c, int64_t* counts) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  if (!counts) return fail(c, KKM_EINVAL, "counts is NULL");
  st = sync_and_check(c);
  if (st != KKM_OK) return st;
  std::vector<double> h(c->s.k);
  KKM_CU(cudaMemcpy(h.data(), c->s.ncum, h.size() * sizeof(double), cudaMemcpyDeviceToHost), "state read");
  for (int j = 0; j < c->s.k; ++j) counts[j] = (int64_t)h[j];
  return KKM_OK;
}

KKM_API kkm_status kkm_set_cum_counts(kkm_ctx* c, const int64_t* counts) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  if (!counts) return fail(c, KKM_EINVAL, "counts is NULL");
  std::vector<double> h(c->s.k);
  for (int j = 0; j < c->s.k; ++j) {
    if (counts[j] < 0 || counts[j] > (int64_t(1) << 53)) return fail(c, KKM_EINVAL, "counts out of range");
    h[j] = (double)counts[j];
  }
  st = sync_and_check(c);
  if (st != KKM_OK) return st;
  KKM_CU(cudaMemcpy(c->s.ncum, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice), "state write");
  return KKM_OK;
}

KKM_API kkm_status kkm_sync(kkm_ctx* c) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  return sync_and_check(c);
}

KKM_API kkm_status kkm_get_state_sizes(kkm_ctx* c, int64_t* total_rows, int64_t* total_blocks) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  if (c->tab) return fail(c, KKM_ENOTSUP, "the table form keeps no support rows");
  st = sync_and_check(c);
  if (st != KKM_OK) return st;
  const int k = c->s.k;
  std::vector<int32_t> head(k), tail(k), c1(k), nb(k);
  KKM_CU(cudaMemcpy(head.data(), c->s.head, k * 4, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(tail.data(), c->s.tail, k * 4, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(c1.data(), c->s.c1, k * 4, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(nb.data(), c->s.blk_num, k * 4, cudaMemcpyDeviceToHost), "state read");
  int64_t r = 0, bl = 0;
  for (int j = 0; j < k; ++j) { r += tail[j] - head[j]; bl += nb[j] + (c1[j] ? 1 : 0); }
  if (total_rows) *total_rows = r;
  if (total_blocks) *total_blocks = bl;
  return KKM_OK;
}

KKM_API kkm_status kkm_get_state(kkm_ctx* c, int64_t* iteration, int32_t* rows_per_center,
                                 int64_t* row_idx, double* row_w, int32_t* blocks_per_center,
                                 int64_t* block_iter, int32_t* block_count, uint8_t* c1_kept,
                                 double* cnorm) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  if (c->tab) return fail(c, KKM_ENOTSUP, "the table form keeps no support rows");
  st = sync_and_check(c);
  if (st != KKM_OK) return st;
  const Dev& s = c->s;
  const int k = s.k;
  std::vector<int32_t> head(k), tail(k), c1(k), bf(k), bn(k);
  std::vector<int32_t> bi((size_t)k * s.nbcap), bc((size_t)k * s.nbcap);
  std::vector<double> cn(k);
  int64_t it = 0;
  KKM_CU(cudaMemcpy(head.data(), s.head, k * 4, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(tail.data(), s.tail, k * 4, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(c1.data(), s.c1, k * 4, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(bf.data(), s.blk_first, k * 4, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(bn.data(), s.blk_num, k * 4, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(bi.data(), s.blk_iter, bi.size() * 4, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(bc.data(), s.blk_cnt, bc.size() * 4, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(cn.data(), s.cnorm, k * 8, cudaMemcpyDeviceToHost), "state read");
  KKM_CU(cudaMemcpy(&it, s.iter, 8, cudaMemcpyDeviceToHost), "state read");
  if (iteration) *iteration = it;
  int64_t ro = 0, bo = 0;
  for (int j = 0; j < k; ++j) {
    const int rows = tail[j] - head[j];
    if (rows_per_center) rows_per_center[j] = rows;
    if (rows > 0) {
      std::vector<int32_t> yi(rows);
      std::vector<double> w(rows);
      const int64_t g = (int64_t)j * s.cap + head[j];
      KKM_CU(cudaMemcpy(yi.data(), s.yi + g, rows * 4, cudaMemcpyDeviceToHost), "state read");
      KKM_CU(cudaMemcpy(w.data(), s.w64 + g, rows * 8, cudaMemcpyDeviceToHost), "state read");
      for (int r = 0; r < rows; ++r) {
        if (row_idx) row_idx[ro + r] = yi[r];
        if (row_w) row_w[ro + r] = w[r];
      }
    }
    ro += rows;
    const int nblk = bn[j] + (c1[j] ? 1 : 0);
    if (blocks_per_center) blocks_per_center[j] = nblk;
    int64_t q = bo;
    if (c1[j]) {
      if (block_iter) block_iter[q] = 0;
      if (block_count) block_count[q] = 1;
      ++q;
    }
    for (int t = 0; t < bn[j]; ++t, ++q) {
      const int slot = (bf[j] + t) % s.nbcap;
      if (block_iter) block_iter[q] = bi[(size_t)j * s.nbcap + slot];
      if (block_count) block_count[q] = bc[(size_t)j * s.nbcap + slot];
    }
    bo += nblk;
    if (c1_kept) c1_kept[j] = c1[j] ? 1 : 0;
    if (cnorm) cnorm[j] = cn[j];
  }
  return KKM_OK;
}

KKM_API kkm_status kkm_set_state(kkm_ctx* c, int64_t iteration, const int32_t* rows_per_center,
                                 const int64_t* row_idx, const double* row_w,
                                 const int32_t* blocks_per_center, const int64_t* block_iter,
                                 const int32_t* block_count, const uint8_t* c1_kept,
                                 const double* cnorm) {
  kkm_status st = check_ready(c);
  if (st != KKM_OK) return st;
  if (c->tab) return fail(c, KKM_ENOTSUP, "the table form keeps no support rows");
  const Dev& s = c->s;
  const int k = s.k;
  if (!rows_per_center || !row_idx || !row_w || !blocks_per_center || !block_iter || !block_count ||
      !c1_kept || !cnorm)
    return fail(c, KKM_EINVAL, "all state arrays are required");
  if (iteration < 1) return fail(c, KKM_EINVAL, "iteration must be >= 1");
  if (s.tau == 0 && iteration - 1 > c->max_iters)
    return fail(c, KKM_EINVAL, "iteration beyond max_iters of an untruncated run");
  // validate everything before touching the device
  int64_t ro = 0, bo = 0;
  for (int j = 0; j < k; ++j) {
    const int rows = rows_per_center[j], nblk = blocks_per_center[j];
    if (rows < 0 || rows > c->wmax) return fail(c, KKM_EINVAL, "rows_per_center out of range");
    if (nblk < 0) return fail(c, KKM_EINVAL, "blocks_per_center negative");
    int64_t sum = 0, prev_it = 0;
    int q0 = 0;
    if (c1_kept[j]) {
      if (nblk < 1 || block_iter[bo] != 0 || block_count[bo] != 1)
        return fail(c, KKM_EINVAL, "a kept C_1 must be the first block (iteration 0, count 1)");
      q0 = 1;
      sum = 1;
    }
    if (nblk - q0 > s.nbcap - 1) return fail(c, KKM_EINVAL, "too many blocks for the window ring");
    for (int q = q0; q < nblk; ++q) {
      const int64_t bi = block_iter[bo + q];
      if (bi <= prev_it || bi >= iteration) return fail(c, KKM_EINVAL, "block iterations must increase, below iteration");
      if (block_count[bo + q] < 1) return fail(c, KKM_EINVAL, "block counts must be >= 1");
      prev_it = bi;
      sum += block_count[bo + q];
    }
    if (sum != rows) return fail(c, KKM_EINVAL, "block counts do not add up to rows_per_center");
    if (!std::isfinite(cnorm[j])) return fail(c, KKM_EINVAL, "cnorm must be finite");
    for (int r = 0; r < rows; ++r) {
      if (row_idx[ro + r] < 0 || row_idx[ro + r] >= s.n) return fail(c, KKM_EINVAL, "row_idx out of range");
      if (!std::isfinite(row_w[ro + r])) return fail(c, KKM_EINVAL, "row weights must be finite");
    }
    ro += rows;
    bo += nblk;
  }
  KKM_CU(cudaStreamSynchronize(c->stream), "stream synchronize");
  // weights are 0 outside the windows
  KKM_CU(cudaMemset(s.w64, 0, ((size_t)k * s.cap + 256) * sizeof(double)), "state write");
  KKM_CU(cudaMemset(s.w32, 0, ((size_t)k * s.cap + 256) * sizeof(float)), "state write");
  std::vector<int32_t> head(k, 0), tail(k), c1(k), wsum(k), bf(k, 0), bn(k);
  std::vector<int32_t> bi((size_t)k * s.nbcap, 0), bc((size_t)k * s.nbcap, 0);
  ro = 0; bo = 0;
  for (int j = 0; j < k; ++j) {
    const int rows = rows_per_center[j], nblk = blocks_per_center[j];
    tail[j] = rows;
    c1[j] = c1_kept[j] ? 1 : 0;
    int q0 = c1[j];
    bn[j] = nblk - q0;
    int ws = 0;
    for (int q = q0; q < nblk; ++q) {
      bi[(size_t)j * s.nbcap + (q - q0)] = (int32_t)block_iter[bo + q];
      bc[(size_t)j * s.nbcap + (q - q0)] = block_count[bo + q];
      ws += block_count[bo + q];
    }
    wsum[j] = ws;
    if (rows > 0) {
      std::vector<int32_t> yi(rows);
      std::vector<float> w32(rows);
      for (int r = 0; r < rows; ++r) { yi[r] = (int32_t)row_idx[ro + r]; w32[r] = (float)row_w[ro + r]; }
      const int64_t g = (int64_t)j * s.cap;
      KKM_CU(cudaMemcpy(s.yi + g, yi.data(), rows * 4, cudaMemcpyHostToDevice), "state write");
      KKM_CU(cudaMemcpy(s.w64 + g, row_w + ro, rows * 8, cudaMemcpyHostToDevice), "state write");
      KKM_CU(cudaMemcpy(s.w32 + g, w32.data(), rows * 4, cudaMemcpyHostToDevice), "state write");
    }
    ro += rows;
    bo += nblk;
  }
  KKM_CU(cudaMemcpy(s.head, head.data(), k * 4, cudaMemcpyHostToDevice), "state write");
  KKM_CU(cudaMemcpy(s.tail, tail.data(), k * 4, cudaMemcpyHostToDevice), "state write");
  KKM_CU(cudaMemcpy(s.c1, c1.data(), k * 4, cudaMemcpyHostToDevice), "state write");
  KKM_CU(cudaMemcpy(s.wsum, wsum.data(), k * 4, cudaMemcpyHostToDevice), "state write");
  KKM_CU(cudaMemcpy(s.blk_first, bf.data(), k * 4, cudaMemcpyHostToDevice), "state write");
  KKM_CU(cudaMemcpy(s.blk_num, bn.data(), k * 4, cudaMemcpyHostToDevice), "state write");
  KKM_CU(cudaMemcpy(s.blk_iter, bi.data(), bi.size() * 4, cudaMemcpyHostToDevice), "state write");
  KKM_CU(cudaMemcpy(s.blk_cnt, bc.data(), bc.size() * 4, cudaMemcpyHostToDevice), "state write");
  KKM_CU(cudaMemcpy(s.cnorm, cnorm, k * 8, cudaMemcpyHostToDevice), "state write");
  KKM_CU(cudaMemcpy(s.iter, &iteration, 8, cudaMemcpyHostToDevice), "state write");
  KKM_CU(kkm::launch_load_rows(s, 0, c->stream), "support row gather");
  KKM_CU(kkm::launch_build_tiles(s, c->stream), "tile list");
  c->iteration = iteration;
  return sync_and_check(c);
}

KKM_API kkm_status kkm_stats(kkm_ctx* c, int64_t* steps, int64_t* support_rows, int64_t* gram_tiles,
                             int32_t reset) {
  kkm_status st = check_usable(c);
  if (st != KKM_OK) return st;
  st = sync_and_check(c);
  if (st != KKM_OK) return st;
  int64_t v[3] = {0, 0, 0};
  KKM_CU(cudaMemcpy(v, c->s.stats, sizeof(v), cudaMemcpyDeviceToHost), "stats read");
  if (steps) *steps = v[0];
  if (support_rows) *support_rows = v[1];
  if (gram_tiles) *gram_tiles = v[2];
  if (reset) KKM_CU(cudaMemset(c->s.stats, 0, sizeof(v)), "stats reset");
  return KKM_OK;
}

KKM_API kkm_status kkm_timing_enable(kkm_ctx* c, int32_t enable) {
  kkm_status st = check_usable(c);
  if (st != KKM_OK) return st;
  if (enable && c->ev.empty()) {
    c->ev.resize(2 * 4096);
    c->ev_reps.assign(4096, 1);
    for (auto& e : c->ev) KKM_CU(cudaEventCreate(&e), "event create");
  }
  if (enable < 0 || enable > 1000) return fail(c, KKM_EINVAL, "timing: enable must be in [0, 1000]");
  c->timing = enable != 0;
  c->timing_reps = enable > 1 ? enable : 1;
  return KKM_OK;
}

KKM_API kkm_status kkm_timing_read(kkm_ctx* c, int64_t* launches, double* total_ms, int32_t reset) {
  kkm_status st = check_usable(c);
  if (st != KKM_OK) return st;
  KKM_CU(cudaStreamSynchronize(c->stream), "stream synchronize");
  double tot = 0.0;
  for (int64_t i = 0; i < c->ev_used; ++i) {
    float ms = 0.0f;
    KKM_CU(cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]), "event elapsed");
    tot += (double)ms / c->ev_reps[i];
  }
  if (launches) *launches = c->ev_used;
  if (total_ms) *total_ms = tot;
  if (reset) c->ev_used = 0;
  return KKM_OK;
}

KKM_API kkm_status kkm_launches(kkm_ctx* c, int64_t* launches, int32_t reset) {
  if (!c) return fail(nullptr, KKM_EINVAL, "null context");
  if (launches) *launches = c->launches;
  if (reset) c->launches = 0;
  return KKM_OK;
}

// ------------------------------------------------------------ run groups
// Many independent runs stepped together. For runs of the windows form (the
// usual case) a group step is one launch per step phase over every run: the
// gather, the argmin, the sort/plan, the row moves and the weight update each
// cover all runs in one grid, and the two Gram passes take one launch per
// class of runs that share their kernel template (tensor-core or FP32 form,
// kernel kind, distance tile). Each block of such a launch plays one block of
// one run's own launch (kkm::GroupPhase), so every run computes what it
// would alone. The runs' Dev structs and TMA descriptors sit in device memory,
// written at creation. A group that holds table-form runs keeps the general
// path: a graph that forks into one branch per run, each branch that run's
// kernel sequence, and joins back. Either way the first group step runs
// eagerly and the second captures the step as a CUDA graph.
struct kkm_group {
  int device = 0;
  std::vector<kkm_ctx*> runs;
  cudaStream_t stream = nullptr;   // where the group's work is ordered
  bool own_stream = false;
  cudaStream_t root = nullptr;     // capture root
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> ev;     // [0] fork, [1 + i] join of run i
  cudaGraphExec_t gexec = nullptr;
  int64_t steps = 0;
  int64_t launches = 0;            // kernels launched by the group's steps (host count)
  std::string err;
  // the per-phase path
  bool batched = false;
  int32_t chains_req = 0;                // chains asked for (0: automatic)
  kkm::GroupRun* d_runs = nullptr;       // the runs, ordered by chain, then class
  int32_t* d_first = nullptr;            // every phase's first-block table
  struct Phase {
    kkm::GroupPhase g{};
    int blocks = 0;
  };
  struct Pass {                           // one class of runs: a Gram pass over all of them
    Phase ph;
    bool tc = false;
    int form = 0, kind = 0, tn = 0;
  };
  // A chain: a share of the runs stepped by one launch per phase, on a graph
  // branch of its own, so that one chain's short phases overlap another's
  // Gram passes; each chain's tensor-core passes take its share of the SMs.
  struct Chain {
    Phase gather, argmin, sort_plan, move, finalize;
    int sort_smem = 0;
    std::vector<Pass> dist, window;
  };
  std::vector<Chain> chains;
  int launches_per_step = 0;
};

namespace {

thread_local std::string g_group_error;

kkm_status gfail(kkm_group* g, kkm_status st, const std::string& msg) {
  if (g) g->err = msg; else g_group_error = msg;
  return st;
}

void group_free(kkm_group* g) {
  if (g->d_runs) cudaFree(g->d_runs);
  if (g->d_first) cudaFree(g->d_first);
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  for (cudaStream_t b : g->branch) cudaStreamDestroy(b);
  if (g->root) cudaStreamDestroy(g->root);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
}

// One step of the runs of one chain, one launch per phase (and per class for the Gram passes).
kkm_status chain_enqueue(kkm_group* g, const kkm_group::Chain& c, cudaStream_t st) {
  auto ok = [&](cudaError_t e, const char* what) {
    return e == cudaSuccess ? KKM_OK : gfail(g, KKM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  kkm_status r = ok(kkm::launch_group_gather(c.gather.g, c.gather.blocks, st), "group gather");
  for (const auto& p : c.dist) {
    if (r != KKM_OK) return r;
    r = ok(p.tc ? kkm::launch_group_tc(p.ph.g, 0, p.form, p.kind, p.tn, p.ph.blocks, st)
                : kkm::launch_group_simt(p.ph.g, 0, p.form, p.ph.blocks, st),
           "group distance pass");
  }
  if (r == KKM_OK) r = ok(kkm::launch_group_argmin(c.argmin.g, c.argmin.blocks, st), "group argmin");
  if (r == KKM_OK) r = ok(kkm::launch_group_sort_plan(c.sort_plan.g, c.sort_smem, st), "group sort/plan");
  if (r == KKM_OK) r = ok(kkm::launch_group_move(c.move.g, c.move.blocks, st), "group row moves");
  for (const auto& p : c.window) {
    if (r != KKM_OK) return r;
    r = ok(p.tc ? kkm::launch_group_tc(p.ph.g, 1, p.form, p.kind, p.tn, p.ph.blocks, st)
                : kkm::launch_group_simt(p.ph.g, 1, p.form, p.ph.blocks, st),
           "group window pass");
  }
  if (r == KKM_OK) r = ok(kkm::launch_group_finalize(c.finalize.g, c.finalize.blocks, st), "group finalize");
  return r;
}

// One step of every run: the chains on branches forked from `st` and joined back.
kkm_status group_enqueue_batched(kkm_group* g, cudaStream_t st) {
  if (g->chains.size() == 1) return chain_enqueue(g, g->chains[0], st);
  if (cudaEventRecord(g->ev[0], st) != cudaSuccess) return gfail(g, KKM_ECUDA, "fork event");
  for (size_t c = 0; c < g->chains.size(); ++c) {
    if (cudaStreamWaitEvent(g->branch[c], g->ev[0], 0) != cudaSuccess) return gfail(g, KKM_ECUDA, "fork wait");
    const kkm_status r = chain_enqueue(g, g->chains[c], g->branch[c]);
    if (r != KKM_OK) return r;
    if (cudaEventRecord(g->ev[1 + c], g->branch[c]) != cudaSuccess) return gfail(g, KKM_ECUDA, "join event");
    if (cudaStreamWaitEvent(st, g->ev[1 + c], 0) != cudaSuccess) return gfail(g, KKM_ECUDA, "join wait");
  }
  return KKM_OK;
}

// Fork from `from`, queue one step of every run on its branch, join back.
kkm_status group_enqueue(kkm_group* g, cudaStream_t from) {
  if (g->batched) return group_enqueue_batched(g, from);
  if (cudaEventRecord(g->ev[0], from) != cudaSuccess) return gfail(g, KKM_ECUDA, "fork event");
  for (size_t i = 0; i < g->runs.size(); ++i) {
    kkm_ctx* c = g->runs[i];
    if (cudaStreamWaitEvent(g->branch[i], g->ev[0], 0) != cudaSuccess) return gfail(g, KKM_ECUDA, "fork wait");
    const kkm_status st = enqueue_step(c, g->branch[i], nullptr, nullptr, nullptr, nullptr, nullptr, false, false);
    if (st != KKM_OK) return gfail(g, st, "run " + std::to_string(i) + ": " + c->err);
    if (cudaEventRecord(g->ev[1 + i], g->branch[i]) != cudaSuccess) return gfail(g, KKM_ECUDA, "join event");
    if (cudaStreamWaitEvent(from, g->ev[1 + i], 0) != cudaSuccess) return gfail(g, KKM_ECUDA, "join wait");
  }
  return KKM_OK;
}

// Estimated Gram-pass work of one run per step (support rows once the
// windows are full, times the batch, times the operand width): the weight by
// which runs are dealt to chains and chains get their share of the SMs.
double run_work(const kkm::Dev& s) {
  const double width = (double)std::max(s.d, 1) * (s.form == kkm::FORM_BF16X3 ? 3.0 : 1.0);
  const double tau = s.tau > 0 ? s.tau : (double)s.b;
  return (double)s.b * (s.k * tau + s.b) * (width + 64.0);   // + 64: the kernel values, whatever d is
}

// The per-phase layout of a group of windows-form runs: the runs dealt to
// `nchains` chains (longest work first, each to the least loaded chain),
// ordered by chain and class, every phase's first-block table, and the runs'
// Dev structs and descriptors copied to the device.
cudaError_t group_build_batched(kkm_group* g, int nchains) {
  const int n = (int)g->runs.size();
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
  if (sms < 1) sms = 148;
  if (g->d_runs) cudaFree(g->d_runs);
  if (g->d_first) cudaFree(g->d_first);
  g->d_runs = nullptr;
  g->d_first = nullptr;
  nchains = std::max(1, std::min(nchains, n));
  // distance-pass class (form, kind, tile); the window pass ignores the tile
  auto key = [](const kkm_ctx* c) {
    return std::make_tuple(c->use_tc ? 1 : 0, (int)c->s.form, (int)c->s.kind, (int)c->s.tn);
  };
  auto wkey = [](const kkm_ctx* c) { return std::make_tuple(c->use_tc ? 1 : 0, (int)c->s.form, (int)c->s.kind); };
  std::vector<double> work(n);
  for (int i = 0; i < n; ++i) work[i] = run_work(g->runs[i]->s);
  std::vector<int> by_work(n), chain_of(n);
  for (int i = 0; i < n; ++i) by_work[i] = i;
  std::stable_sort(by_work.begin(), by_work.end(), [&](int a, int b) { return work[a] > work[b]; });
  std::vector<double> load(nchains, 0.0);
  for (int i : by_work) {
    const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    chain_of[i] = c;
    load[c] += work[i];
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (chain_of[a] != chain_of[b]) return chain_of[a] < chain_of[b];
    return key(g->runs[a]) < key(g->runs[b]);
  });
  std::vector<kkm::GroupRun> hr(n);
  for (int i = 0; i < n; ++i) {
    const kkm_ctx* c = g->runs[order[i]];
    std::memcpy(hr[i].maps, c->tmaps, sizeof(hr[i].maps));
    hr[i].s = c->s;
    hr[i].s.pre_b = 0;   // the group passes read item counts after their grid-dependency wait
  }
  cudaError_t e = cudaMalloc(&g->d_runs, sizeof(kkm::GroupRun) * (size_t)n);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(g->d_runs, hr.data(), sizeof(kkm::GroupRun) * (size_t)n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;

  std::vector<int32_t> first;
  struct Pending { int chain, which; size_t off; int lo; int cnt; };
  std::vector<Pending> pend;
  // appends the first-block table of runs [lo, lo + blocks.size())
  auto table = [&](int chain, int which, int lo, const std::vector<int>& blocks) {
    const size_t off = first.size();
    int64_t acc = 0;
    for (int b : blocks) {
      first.push_back((int32_t)acc);
      acc += b;
    }
    first.push_back((int32_t)acc);
    pend.push_back({chain, which, off, lo, (int)blocks.size()});
    return (int)acc;
  };
  double total_load = 0.0;
  for (double l : load) total_load += l;
  g->chains.assign(nchains, kkm_group::Chain{});
  std::vector<std::vector<int>> dist_lo(nchains), win_lo(nchains);
  for (int c = 0, lo = 0; c < nchains; ++c) {
    int hi = lo;
    while (hi < n && chain_of[order[hi]] == c) ++hi;
    auto& ch = g->chains[c];
    std::vector<int> bg, ba, bs, bm, bf;
    for (int i = lo; i < hi; ++i) {
      const kkm::Dev& s = hr[i].s;
      bg.push_back((s.b * 32 + 255) / 256);
      ba.push_back((s.b + 31) / 32);
      bs.push_back(1);
      bm.push_back(std::max(1, (s.b + 7) / 8));
      bf.push_back(s.k);
      ch.sort_smem = std::max(ch.sort_smem, kkm::sort_plan_smem(s.k, s.b));
    }
    ch.gather.blocks = table(c, 0, lo, bg);
    ch.argmin.blocks = table(c, 1, lo, ba);
    ch.sort_plan.blocks = table(c, 2, lo, bs);
    ch.move.blocks = table(c, 3, lo, bm);
    ch.finalize.blocks = table(c, 4, lo, bf);
    // the Gram passes balance their runs on the device (a weighted item
    // space per class for the tensor-core passes, a flat one for the
    // CUDA-core passes) over the chain's share of the SMs
    const int share = std::max(1, (int)std::lround(sms * (total_load > 0 ? load[c] / total_load : 1.0)));
    for (int i = lo; i < hi;) {
      int j = i + 1;
      while (j < hi && key(g->runs[order[j]]) == key(g->runs[order[i]])) ++j;
      const kkm_ctx* c0 = g->runs[order[i]];
      kkm_group::Pass p;
      p.tc = c0->use_tc;
      p.form = c0->s.form;
      p.kind = c0->s.kind;
      p.tn = c0->s.tn;
      p.ph.blocks = p.tc ? share : 4 * share;
      p.ph.g.nruns = j - i;
      ch.dist.push_back(p);
      dist_lo[c].push_back(i);
      i = j;
    }
    for (int i = lo; i < hi;) {
      int j = i + 1;
      while (j < hi && wkey(g->runs[order[j]]) == wkey(g->runs[order[i]])) ++j;
      const kkm_ctx* c0 = g->runs[order[i]];
      kkm_group::Pass p;
      p.tc = c0->use_tc;
      p.form = c0->s.form;
      p.kind = c0->s.kind;
      p.tn = c0->s.tn;
      p.ph.blocks = p.tc ? share : 4 * share;
      p.ph.g.nruns = j - i;
      ch.window.push_back(p);
      win_lo[c].push_back(i);
      i = j;
    }
    lo = hi;
  }
  e = cudaMalloc(&g->d_first, sizeof(int32_t) * first.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(g->d_first, first.data(), sizeof(int32_t) * first.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  g->launches_per_step = 0;
  for (const auto& q : pend) {
    auto& ch = g->chains[q.chain];
    kkm_group::Phase* ph[5] = {&ch.gather, &ch.argmin, &ch.sort_plan, &ch.move, &ch.finalize};
    ph[q.which]->g = kkm::GroupPhase{g->d_runs + q.lo, g->d_first + q.off, q.cnt};
  }
  for (int c = 0; c < nchains; ++c) {
    auto& ch = g->chains[c];
    for (size_t i = 0; i < ch.dist.size(); ++i) {
      ch.dist[i].ph.g.runs = g->d_runs + dist_lo[c][i];
      ch.dist[i].ph.g.first = g->d_first;   // not read by the Gram passes
    }
    for (size_t i = 0; i < ch.window.size(); ++i) {
      ch.window[i].ph.g.runs = g->d_runs + win_lo[c][i];
      ch.window[i].ph.g.first = g->d_first;
    }
    g->launches_per_step += 5 + (int)ch.dist.size() + (int)ch.window.size();
  }
  g->batched = true;
  return cudaSuccess;
}

}  // namespace

KKM_API kkm_status kkm_group_create(kkm_group** out, kkm_ctx* const* runs, int32_t n, void* stream) {
  if (!out) return gfail(nullptr, KKM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !runs) return gfail(nullptr, KKM_EINVAL, "a group needs n >= 1 runs");
  if (n > 1024) return gfail(nullptr, KKM_EINVAL, "a group holds at most 1024 runs");
  for (int32_t i = 0; i < n; ++i) {
    if (!runs[i]) return gfail(nullptr, KKM_EINVAL, "null run");
    if (runs[i]->poisoned) return gfail(nullptr, KKM_ESTATE, "a run is poisoned");
    if (runs[i]->device != runs[0]->device) return gfail(nullptr, KKM_EINVAL, "runs on different devices");
    for (int32_t q = 0; q < i; ++q)
      if (runs[q] == runs[i]) return gfail(nullptr, KKM_EINVAL, "a run appears twice");
  }
  kkm_group* g = new (std::nothrow) kkm_group();
  if (!g) return gfail(nullptr, KKM_ENOMEM, "out of host memory");
  g->device = runs[0]->device;
  g->runs.assign(runs, runs + n);
  auto bail = [&](const char* what, cudaError_t e) {
    g_group_error = std::string(what) + ": " + cudaGetErrorString(e);
    group_free(g);
    delete g;
    return KKM_ECUDA;
  };
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return bail("cudaSetDevice", e);
  for (kkm_ctx* c : g->runs) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail("run stream synchronize", e);
  }
  if (stream) {
    g->stream = static_cast<cudaStream_t>(stream);
  } else {
    e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail("stream", e);
    g->own_stream = true;
  }
  e = cudaStreamCreateWithFlags(&g->root, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail("stream", e);
  g->branch.resize(n, nullptr);
  for (int32_t i = 0; i < n; ++i) {
    e = cudaStreamCreateWithFlags(&g->branch[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail("stream", e);
  }
  g->ev.resize(n + 1, nullptr);
  for (auto& ev : g->ev) {
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail("event", e);
  }
  bool all_windows = true;
  for (kkm_ctx* c : g->runs) all_windows = all_windows && !c->tab;
  if (all_windows) {
    e = group_build_batched(g, n >= 16 ? 2 : 1);
    if (e != cudaSuccess) return bail("group layout", e);
  } else {
    g->launches_per_step = 7 * n;   // seven kernels per run, on the run's branch
  }
  *out = g;
  return KKM_OK;
}

KKM_API kkm_status kkm_group_step(kkm_group* g) {
  if (!g) return gfail(nullptr, KKM_EINVAL, "null group");
  if (cudaSetDevice(g->device) != cudaSuccess) return gfail(g, KKM_ECUDA, "cudaSetDevice failed");
  for (kkm_ctx* c : g->runs) {
    if (c->poisoned) return gfail(g, KKM_ESTATE, "a run is poisoned");
    if (c->s.tau == 0 && !c->tab && c->iteration > c->max_iters)
      return gfail(g, KKM_ESTATE, "an untruncated run has done max_iters iterations");
    if (c->fin_pending) {               // a kkm_step on the run since the last group step
      if (flush(c) != KKM_OK || cudaStreamSynchronize(c->stream) != cudaSuccess)
        return gfail(g, KKM_ECUDA, "pending weight update of a run");
    }
  }
  if (g->steps == 0) {
    const kkm_status st = group_enqueue(g, g->stream);
    if (st != KKM_OK) return st;
  } else {
    if (!g->gexec) {
      if (cudaStreamBeginCapture(g->root, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return gfail(g, KKM_ECUDA, "begin capture");
      const kkm_status st = group_enqueue(g, g->root);
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(g->root, &graph);
      if (st != KKM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return gfail(g, KKM_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
      const cudaError_t ei = cudaGraphInstantiate(&g->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) return gfail(g, KKM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    }
    const cudaError_t e = cudaGraphLaunch(g->gexec, g->stream);
    if (e != cudaSuccess) return gfail(g, KKM_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  }
  for (kkm_ctx* c : g->runs) ++c->iteration;
  g->launches += g->launches_per_step;
  ++g->steps;
  return KKM_OK;
}

KKM_API kkm_status kkm_group_set_chains(kkm_group* g, int32_t chains) {
  if (!g) return gfail(nullptr, KKM_EINVAL, "null group");
  if (chains < 0 || chains > (int32_t)g->runs.size()) return gfail(g, KKM_EINVAL, "chains must be in [0, runs]");
  if (g->steps > 0) return gfail(g, KKM_ESTATE, "chains are set before the first group step");
  bool all_windows = true;
  for (kkm_ctx* c : g->runs) all_windows = all_windows && !c->tab;
  if (chains > 0 && !all_windows)
    return gfail(g, KKM_ENOTSUP, "a group with table-form runs steps each run on its own branch");
  if (cudaSetDevice(g->device) != cudaSuccess) return gfail(g, KKM_ECUDA, "cudaSetDevice failed");
  g->chains_req = chains;
  if (chains == 0) {             // one graph branch per run
    g->batched = false;
    g->chains.clear();
    g->launches_per_step = 7 * (int)g->runs.size();
    return KKM_OK;
  }
  const cudaError_t e = group_build_batched(g, chains);
  if (e != cudaSuccess) return gfail(g, KKM_ECUDA, std::string("group layout: ") + cudaGetErrorString(e));
  return KKM_OK;
}

KKM_API kkm_status kkm_group_launches(kkm_group* g, int64_t* launches, int32_t* per_step, int32_t reset) {
  if (!g) return gfail(nullptr, KKM_EINVAL, "null group");
  if (launches) *launches = g->launches;
  if (per_step) *per_step = g->launches_per_step;
  if (reset) g->launches = 0;
  return KKM_OK;
}

KKM_API kkm_status kkm_group_sync(kkm_group* g) {
  if (!g) return gfail(nullptr, KKM_EINVAL, "null group");
  if (cudaSetDevice(g->device) != cudaSuccess) return gfail(g, KKM_ECUDA, "cudaSetDevice failed");
  const cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return gfail(g, KKM_ECUDA, std::string("stream synchronize: ") + cudaGetErrorString(e));
  for (size_t i = 0; i < g->runs.size(); ++i) {
    const kkm_status st = sync_and_check(g->runs[i]);
    if (st != KKM_OK) return gfail(g, st, "run " + std::to_string(i) + ": " + g->runs[i]->err);
  }
  return KKM_OK;
}

KKM_API const char* kkm_group_last_error(kkm_group* g) {
  return g ? g->err.c_str() : g_group_error.c_str();
}

KKM_API kkm_status kkm_group_destroy(kkm_group* g) {
  if (!g) return KKM_OK;
  cudaSetDevice(g->device);
  cudaStreamSynchronize(g->stream);
  group_free(g);
  delete g;
  return KKM_OK;
}

KKM_API kkm_status kkm_destroy(kkm_ctx* c) {
  if (!c) return KKM_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  return KKM_OK;
}
