// Full-batch kernel k-means (kernel Lloyd): the baseline the paper's
// mini-batch algorithm is compared with in Sec. 6 (and whose per-iteration
// cost, O(n^2) kernel evaluations, motivates it in Sec. 1).
//
// One iteration, given the assignment a of every point:
//   1. counting sort of X by a (stable; ranks per chunk of rows, then offsets),
//   2. the center-sorted operand rows into the support buffer, weight 1/n_j,
//   3. the n x n Gram pass of X against that buffer, chunk by chunk of rows
//      of X, each chunk's tile partials summed into T[j][x] = <phi(x), C_j>,
//   4. ||C_j||^2 = (1/n_j) sum_{x in X_j} T[j][x],
//   5. the new assignment argmin_j K(x,x) - 2 T[j][x] + ||C_j||^2, f_X at the
//      new centers and the number of points whose assignment changed.
// Initialisation runs steps 3 and 5 against the k initial points (one
// support row each, weight 1, ||C_j||^2 = K(y_j, y_j) from the exact norm).
// A center that gets no points keeps its row of T and its norm, which is what
// C_j <- C_j means for the table. The Gram pass is the library's distance
// pass (tcgen05 for the BF16, split-BF16 and TF32 forms, CUDA cores for FP32)
// on a view of X's operand rows; nothing here runs on the host but sizing.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "kkm_internal.cuh"
#include "../../include/kkm.h"

#define KKM_API extern "C" __attribute__((visibility("default")))

struct kkm_lloyd {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool use_tc = false;
  bool poisoned = false;
  kkm::Dev g{};           // the Gram view: xb* = every row of X, y* = X sorted by center
  kkm::LloydBuf L{};
  int64_t npad = 0;       // rows of the operand buffer (multiple of 128)
  int64_t R = 0;          // rows of X per Gram-pass chunk (multiple of 128)
  int32_t nchunk = 0;
  unsigned char* maps = nullptr;   // 4 TMA descriptors (512 bytes, 64-byte aligned) per chunk
  std::vector<void*> allocs;
  int64_t iters = 0;      // center updates run
  int64_t launches = 0;   // kernels launched (host count)
  std::string err;
};

namespace {

thread_local std::string g_lloyd_init_error;

kkm_status lfail(kkm_lloyd* c, kkm_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_lloyd_init_error = msg;
  return st;
}

template <class T>
cudaError_t lalloc(kkm_lloyd* c, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  c->allocs.push_back(q);
  e = cudaMemset(q, 0, bytes);
  *p = static_cast<T*>(q);
  return e;
}

void lfree(kkm_lloyd* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  std::free(c->maps);
  c->maps = nullptr;
}

#define LL_CU(expr, where)                                                                   \
  do {                                                                                       \
    const cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess) {                                                                 \
      c->poisoned = true;                                                                    \
      return lfail(c, KKM_ECUDA, std::string(where) + ": " + cudaGetErrorString(_e));        \
    }                                                                                        \
  } while (0)

// The view of chunk q: its operand rows, norms and indices, and the shared
// partials buffer with the chunk's own row stride.
kkm::Dev chunk_view(const kkm_lloyd* c, int q) {
  kkm::Dev v = c->g;
  const int64_t r0 = (int64_t)q * c->R;
  if (v.xb32) v.xb32 += r0 * v.ld;
  if (v.xbh) v.xbh += r0 * v.ld;
  v.xbn += r0;
  v.xbi += r0;
  v.bpad = (int32_t)std::min<int64_t>(c->R, c->npad - r0);
  return v;
}

// Steps 3 (and the reduction of its partials) over every chunk of rows.
kkm_status gram_and_reduce(kkm_lloyd* c, bool all) {
  for (int q = 0; q < c->nchunk; ++q) {
    const kkm::Dev v = chunk_view(c, q);
    const int64_t r0 = (int64_t)q * c->R;
    const int rows = (int)std::min<int64_t>(c->R, c->g.n - r0);
    if (c->use_tc) LL_CU(kkm::launch_dist_tc(v, c->maps + 512 * (size_t)q, rows, c->stream), "Gram pass (tcgen05)");
    else LL_CU(kkm::launch_dist_simt(v, rows, c->stream), "Gram pass");
    LL_CU(kkm::launch_lloyd_reduce(v, c->L, r0, rows, all, c->stream), "Gram reduction");
    c->launches += 2;
  }
  return KKM_OK;
}

kkm_status check_status(kkm_lloyd* c) {
  int32_t st = 0;
  LL_CU(cudaMemcpyAsync(&st, c->g.status, sizeof(st), cudaMemcpyDeviceToHost, c->stream), "status read");
  LL_CU(cudaStreamSynchronize(c->stream), "synchronise");
  if (st == 0) return KKM_OK;
  c->poisoned = true;
  std::string m = "device status:";
  if (st & kkm::ST_BAD_BATCH_INDEX) m += " initial index out of range;";
  if (st & kkm::ST_CAPACITY) m += " internal capacity exceeded;";
  if (st & kkm::ST_TIMEOUT) m += " bounded wait timed out;";
  return lfail(c, (st & kkm::ST_TIMEOUT) ? KKM_ETIMEOUT : KKM_EINVAL, m);
}

}  // namespace

KKM_API const char* kkm_lloyd_last_error(const kkm_lloyd* c) {
  return c ? c->err.c_str() : g_lloyd_init_error.c_str();
}

KKM_API kkm_status kkm_lloyd_init(kkm_lloyd** out, const float* X, int64_t n, int32_t d, int64_t ldx, int32_t k,
                                  const kkm_kernel* kernel, int32_t precision, const int64_t* init_idx,
                                  int64_t chunk_rows, void* stream) {
  if (!out) return lfail(nullptr, KKM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!X || !kernel || !init_idx) return lfail(nullptr, KKM_EINVAL, "X, kernel and init_idx are required");
  if (n < 1 || n >= (int64_t(1) << 31) - 65536) return lfail(nullptr, KKM_EINVAL, "n must be in [1, 2^31 - 65536)");
  if (d < 1 || d > 4096) return lfail(nullptr, KKM_EINVAL, "d must be in [1, 4096]");
  if (ldx < d) return lfail(nullptr, KKM_EINVAL, "ldx must be >= d");
  if (k < 1 || k > 1024 || k > n) return lfail(nullptr, KKM_EINVAL, "k must be in [1, min(n, 1024)]");
  if (kernel->kind < KKM_GAUSSIAN || kernel->kind > KKM_POLY) return lfail(nullptr, KKM_EINVAL, "unknown kernel kind");
  if ((kernel->kind == KKM_GAUSSIAN || kernel->kind == KKM_LAPLACIAN) &&
      !(std::isfinite(kernel->param) && kernel->param > 0.0))
    return lfail(nullptr, KKM_EINVAL, "kernel param (kappa or sigma) must be finite and > 0");
  if (kernel->kind == KKM_POLY && (kernel->degree < 1 || kernel->degree > 8 || !std::isfinite(kernel->coef0)))
    return lfail(nullptr, KKM_EINVAL, "polynomial degree must be in [1, 8] with a finite coef0");
  if (precision < KKM_PREC_FP32 || precision > KKM_PREC_TF32) return lfail(nullptr, KKM_EINVAL, "unknown precision");
  if (chunk_rows < 0 || chunk_rows % 128 != 0)
    return lfail(nullptr, KKM_EINVAL, "chunk_rows must be 0 (automatic) or a positive multiple of 128");
  if ((int64_t)n * k >= (int64_t(1) << 40)) return lfail(nullptr, KKM_EINVAL, "n*k too large for the table");
  for (int j = 0; j < k; ++j)
    if (init_idx[j] < 0 || init_idx[j] >= n) return lfail(nullptr, KKM_EINVAL, "init_idx entry out of [0, n)");

  kkm_lloyd* c = new (std::nothrow) kkm_lloyd();
  if (!c) return lfail(nullptr, KKM_ENOMEM, "host allocation failed");
  auto bail = [&](kkm_status st) {
    g_lloyd_init_error = c->err;
    lfree(c);
    delete c;
    return st;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    c->err = "no CUDA device";
    return bail(KKM_ECUDA);
  }
  c->stream = static_cast<cudaStream_t>(stream);
  if (precision != KKM_PREC_FP32) {
    int maj = 0, min = 0;
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, c->device);
    cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, c->device);
    if (kkm_form_supported(precision, maj, min) != KKM_OK) {
      c->err = "the BF16, split-BF16 and TF32 forms need a compute capability 10.3 device (tcgen05)";
      return bail(KKM_ENOTSUP);
    }
    c->use_tc = true;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);

  kkm::Dev& g = c->g;
  g.n = n; g.d = d; g.k = k; g.b = 1; g.ldx = ldx; g.X = X;
  g.form = precision;
  g.kind = kernel->kind; g.degree = kernel->degree;
  g.param = kernel->param; g.coef0 = kernel->coef0;
  g.inv_b = 1.0;
  g.negc = (kernel->kind == KKM_GAUSSIAN || kernel->kind == KKM_LAPLACIAN)
               ? (float)(-1.4426950408889634 / kernel->param) : 0.0f;
  g.num_sms = sms > 0 ? sms : 148;
  g.pre_b = 0;   // the support buffer is written by the kernel just before each Gram pass
  if (g.form == kkm::FORM_FP32) { g.dp = 0; g.ld = (int32_t)kkm::round_up(d, 16); }
  else if (g.form == kkm::FORM_TF32) { g.dp = (int32_t)kkm::round_up(d, 32); g.ld = g.dp; }
  else { g.dp = (int32_t)kkm::round_up(d, 64); g.ld = 2 * g.dp; }
  // clusters hold thousands of rows: the widest tensor-core tile
  g.tn = c->use_tc ? 256 : 64;
  g.ppt = c->use_tc ? kkm::tc_parts_per_tile(g.tn) : 1;
  // every center in whole tiles: at most n / tn + k tiles, n + k tn rows
  g.max_tiles = (int32_t)((n + g.tn - 1) / g.tn + k + 1);
  g.cap = (int32_t)kkm::round_up((n + (int64_t)k * g.tn + k - 1) / k, 8);
  const int64_t srows = (int64_t)k * g.cap + 256;
  c->npad = kkm::round_up(n, 128);
  // chunk of rows of X per Gram pass: the partials of one chunk take at most 1 GiB
  const int64_t per_row = (int64_t)g.max_tiles * g.ppt * (int64_t)sizeof(float);
  int64_t R = chunk_rows > 0 ? chunk_rows : std::max<int64_t>(128, ((int64_t(1) << 30) / per_row) / 128 * 128);
  R = std::min<int64_t>(R, c->npad);
  c->R = R;
  c->nchunk = (int32_t)((n + R - 1) / R);
  g.bpad = (int32_t)R;

  const int esz = kkm::f32_rows(g.form) ? 4 : 2;
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, count)                                                  \
  do {                                                                     \
    e = lalloc(c, &(ptr), (size_t)(count));                                \
    if (e != cudaSuccess) {                                                \
      c->err = std::string("device allocation: ") + cudaGetErrorString(e); \
      return bail(KKM_ENOMEM);                                             \
    }                                                                      \
  } while (0)
  if (esz == 4) {
    ALLOC(g.xb32, (size_t)c->npad * g.ld);
    ALLOC(g.y32, (size_t)srows * g.ld);
  } else {
    ALLOC(g.xbh, (size_t)c->npad * g.ld);
    ALLOC(g.ybh, (size_t)srows * g.ld);
  }
  ALLOC(g.xbn, c->npad); ALLOC(g.xbi, c->npad);
  ALLOC(g.yn, srows); ALLOC(g.yi, srows); ALLOC(g.w64, srows); ALLOC(g.w32, srows);
  ALLOC(g.cnorm, k); ALLOC(g.cnorm32, k); ALLOC(g.counts, k); ALLOC(g.coff, k + 1);
  ALLOC(g.perm, n);
  ALLOC(g.tiles, g.max_tiles); ALLOC(g.ntiles, 1); ALLOC(g.tile_first, k); ALLOC(g.tile_cnt, k);
  ALLOC(g.part, (size_t)g.max_tiles * g.ppt * R);
  ALLOC(g.status, 1);
  kkm::LloydBuf& L = c->L;
  L.nrk = (int32_t)((n + kkm::LLOYD_RANK_ROWS - 1) / kkm::LLOYD_RANK_ROWS);
  L.nblk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(4LL * g.num_sms, (n + 255) / 256));
  ALLOC(L.T, (size_t)k * n);
  ALLOC(L.assign, n); ALLOC(L.mind, n); ALLOC(L.rank, n);
  ALLOC(L.ccnt, (size_t)L.nrk * k); ALLOC(L.cbase, (size_t)L.nrk * k);
  ALLOC(L.bs_off, k + 1);
  ALLOC(L.blk, L.nblk); ALLOC(L.blk_changed, L.nblk);
  ALLOC(L.obj, 1); ALLOC(L.changed, 1);
  int32_t* d_init = nullptr;
  ALLOC(d_init, k);
#undef ALLOC

  std::vector<int32_t> h_init(k);
  for (int j = 0; j < k; ++j) h_init[j] = (int32_t)init_idx[j];
  e = cudaMemcpyAsync(d_init, h_init.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
  if (c->use_tc && e == cudaSuccess) {
    c->maps = static_cast<unsigned char*>(std::aligned_alloc(64, 512 * (size_t)c->nchunk));
    if (!c->maps) {
      c->err = "host allocation failed";
      return bail(KKM_ENOMEM);
    }
    for (int q = 0; q < c->nchunk && e == cudaSuccess; ++q) {
      kkm::Dev v = chunk_view(c, q);
      e = kkm::tc_prepare(v, c->maps + 512 * (size_t)q);
    }
  }
  if (e != cudaSuccess) {
    c->err = std::string("initialisation: ") + cudaGetErrorString(e);
    return bail(KKM_ECUDA);
  }
  // operand rows of X, the initial centers as the support buffer, T against them
  const kkm::TabBuf none{};
  e = kkm::launch_tab_init(g, g, none, d_init, c->stream);
  c->launches += 2;
  if (e != cudaSuccess) {
    c->err = std::string("initialisation: ") + cudaGetErrorString(e);
    return bail(KKM_ECUDA);
  }
  kkm_status st = gram_and_reduce(c, true);
  if (st == KKM_OK) {
    e = kkm::launch_lloyd_assign(g, L, true, c->stream);
    c->launches += 2;
    if (e != cudaSuccess) st = lfail(c, KKM_ECUDA, std::string("assignment: ") + cudaGetErrorString(e));
  }
  if (st == KKM_OK) st = check_status(c);
  if (st != KKM_OK) return bail(st);
  *out = c;
  return KKM_OK;
}

KKM_API kkm_status kkm_lloyd_iterate(kkm_lloyd* c, int32_t iters) {
  if (!c) return lfail(nullptr, KKM_EINVAL, "handle is NULL");
  if (c->poisoned) return lfail(c, KKM_EINVAL, "an earlier failure left the run unusable");
  if (iters < 0) return lfail(c, KKM_EINVAL, "iters must be >= 0");
  for (int it = 0; it < iters; ++it) {
    LL_CU(kkm::launch_lloyd_sort(c->g, c->L, c->stream), "counting sort");
    LL_CU(kkm::launch_lloyd_scatter(c->g, c->L, c->stream), "support layout");
    c->launches += 3;
    const kkm_status st = gram_and_reduce(c, false);
    if (st != KKM_OK) return st;
    LL_CU(kkm::launch_lloyd_cnorm(c->g, c->L, c->stream), "center norms");
    LL_CU(kkm::launch_lloyd_assign(c->g, c->L, false, c->stream), "assignment");
    c->launches += 3;
    ++c->iters;
  }
  return KKM_OK;
}

KKM_API kkm_status kkm_lloyd_read(kkm_lloyd* c, double* obj, int64_t* changed, int64_t* iters_done) {
  if (!c) return lfail(nullptr, KKM_EINVAL, "handle is NULL");
  if (c->poisoned) return lfail(c, KKM_EINVAL, "an earlier failure left the run unusable");
  double o = 0.0;
  int64_t ch = 0;
  LL_CU(cudaMemcpyAsync(&o, c->L.obj, sizeof(o), cudaMemcpyDeviceToHost, c->stream), "objective read");
  LL_CU(cudaMemcpyAsync(&ch, c->L.changed, sizeof(ch), cudaMemcpyDeviceToHost, c->stream), "changed read");
  const kkm_status st = check_status(c);
  if (st != KKM_OK) return st;
  if (obj) *obj = o;
  if (changed) *changed = ch;
  if (iters_done) *iters_done = c->iters;
  return KKM_OK;
}

KKM_API kkm_status kkm_lloyd_assignments(kkm_lloyd* c, int32_t* assign_out, float* mind_out) {
  if (!c) return lfail(nullptr, KKM_EINVAL, "handle is NULL");
  if (c->poisoned) return lfail(c, KKM_EINVAL, "an earlier failure left the run unusable");
  const size_t n = (size_t)c->g.n;
  if (assign_out)
    LL_CU(cudaMemcpyAsync(assign_out, c->L.assign, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream),
          "assignment copy");
  if (mind_out)
    LL_CU(cudaMemcpyAsync(mind_out, c->L.mind, n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream),
          "distance copy");
  return KKM_OK;
}

KKM_API kkm_status kkm_lloyd_distances(kkm_lloyd* c, float* dist_out) {
  if (!c) return lfail(nullptr, KKM_EINVAL, "handle is NULL");
  if (c->poisoned) return lfail(c, KKM_EINVAL, "an earlier failure left the run unusable");
  if (!dist_out) return lfail(c, KKM_EINVAL, "dist_out is required");
  LL_CU(kkm::launch_lloyd_dist(c->g, c->L, dist_out, c->stream), "distances");
  ++c->launches;
  return KKM_OK;
}

KKM_API kkm_status kkm_lloyd_center_norms(kkm_lloyd* c, double* out) {
  if (!c) return lfail(nullptr, KKM_EINVAL, "handle is NULL");
  if (c->poisoned) return lfail(c, KKM_EINVAL, "an earlier failure left the run unusable");
  if (!out) return lfail(c, KKM_EINVAL, "out is required");
  LL_CU(cudaMemcpyAsync(out, c->g.cnorm, (size_t)c->g.k * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
        "center norm read");
  LL_CU(cudaStreamSynchronize(c->stream), "synchronise");
  return KKM_OK;
}

KKM_API kkm_status kkm_lloyd_info(const kkm_lloyd* c, int64_t* launches, int32_t* chunks, int64_t* chunk_rows) {
  if (!c) return lfail(nullptr, KKM_EINVAL, "handle is NULL");
  if (launches) *launches = c->launches;
  if (chunks) *chunks = c->nchunk;
  if (chunk_rows) *chunk_rows = c->R;
  return KKM_OK;
}

KKM_API kkm_status kkm_lloyd_destroy(kkm_lloyd* c) {
  if (!c) return KKM_OK;
  cudaStreamSynchronize(c->stream);
  lfree(c);
  delete c;
  return KKM_OK;
}
