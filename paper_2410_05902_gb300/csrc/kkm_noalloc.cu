// kkm_distances_noalloc: the FP32 distance pass without a context and without
// any allocation.
//
// Some callers cannot call cudaMalloc. Two kinds are common. One is a caller
// whose device memory is owned entirely by a framework's caching allocator or
// a pre-sized arena: a serving process that reserved the free memory at
// start-up, where a stray cudaMalloc fails or fragments that reservation. The
// other is a caller on a latency-critical loop, where cudaMalloc and cudaFree
// can synchronise the device and stall for milliseconds. This entry point lets
// such callers score query points against k centers that they hold
// themselves. They pass the inputs and the outputs. The only scratch is one
// file-scope __device__ array of fixed size (KKM_NOALLOC_SCRATCH_BYTES in
// kkm.h).
//
// CUDA loads modules lazily by default, so that array, and the code of this
// file's kernels, come onto a device when the first call on that device looks
// up the array's address and launches the kernels. The first call on each
// device therefore reserves the memory; a call with m = 0 does exactly that
// and nothing else. It must come before the caller reserves the rest of the
// device memory and before any stream capture. Later calls reserve nothing.
//
// Host code never dereferences the array's name: on the host that name is only
// a stand-in. Every call shares the one array, so two calls whose kernels
// overlap on the GPU (for example on two streams without ordering between
// them) race on it. Calls queued on one stream, one after another, are safe.
// Each call writes every scratch entry it later reads (tile list, norms,
// partial sums, the offsets' check), so nothing left over from an earlier call
// is ever used.
#include <algorithm>
#include <mutex>
#include <string>

#include "kkm_internal.cuh"
#include "../../include/kkm.h"

#define KKM_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr int NA_ROWS = KKM_NOALLOC_MAX_ROWS_PER_PASS;   // query rows per internal pass
constexpr int NA_TILE = 64;                               // support rows per tile
constexpr int NA_MAX_TILES = KKM_NOALLOC_MAX_TILES;
constexpr int NA_MAX_S = KKM_NOALLOC_MAX_SUPPORT;
constexpr int BK = 16, NT = 256;

struct Scratch {
  float part[NA_MAX_TILES * NA_ROWS];   // per-tile weighted kernel sums of each query row
  float yn[NA_MAX_S];                   // ||y||^2 of the support rows
  float qn[NA_ROWS];                    // ||q||^2 of the pass's query rows
  int4 tiles[NA_MAX_TILES];             // (center, first support row, rows, -)
  int32_t tile_first[1024];
  int32_t tile_cnt[1024];
  int32_t ntiles;                       // tiles written by this call's k_na_tiles
  int32_t bad;                          // the call's offsets were not non-decreasing within [0, S]
};
static_assert(sizeof(Scratch) <= KKM_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds its declared size");

static __device__ __align__(256) unsigned char kkm_noalloc_scratch[KKM_NOALLOC_SCRATCH_BYTES];

std::mutex g_na_mutex;
void* g_na_addr[256] = {};
bool g_na_loaded[256] = {};
thread_local std::string g_na_error;

kkm_status na_fail(kkm_status st, const char* msg) {
  g_na_error = msg;
  return st;
}

// Launches one kernel and returns that launch's own status. A failed launch's
// error is cleared from the thread's last-error record once it is returned
// here; an error left there by someone else's earlier launch is neither
// reported as this call's nor cleared.
template <typename... Params, typename... Args>
cudaError_t na_launch(void (*kern)(Params...), int grid, int block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.stream = st;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, static_cast<Params>(args)...);
  if (e != cudaSuccess) (void)cudaGetLastError();
  return e;
}

// One thread per center (k <= 1024): the tile list of the support segments.
// Offsets that are not non-decreasing within [0, S] (or whose tiles would not
// fit the list, which well-formed offsets under the host's size check never
// do) set `bad` and leave an empty list, so no later kernel reads a tile.
__global__ void __launch_bounds__(1024) k_na_tiles(Scratch* sc, const int32_t* __restrict__ seg_off, int k,
                                                   int S) {
  __shared__ int wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int a = 0, size = 0, nt = 0, bad_here = 0;
  if (tid < k) {
    const int s0 = seg_off[tid], s1 = seg_off[tid + 1];
    bad_here = s0 < 0 || s1 < s0 || s1 > S;
    a = min(max(s0, 0), S);
    size = min(max(s1, a), S) - a;
    nt = (size + NA_TILE - 1) / NA_TILE;
  }
  int x = nt;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  const int any_bad = __syncthreads_or(bad_here);
  if (warp == 0) {
    int t = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  const int total = wsum[31];
  const bool bad = any_bad || total > NA_MAX_TILES;
  const int first = x - nt + (warp > 0 ? wsum[warp - 1] : 0);   // first + nt <= total when !bad
  if (tid == 0) {
    sc->ntiles = bad ? 0 : total;
    sc->bad = bad ? 1 : 0;
  }
  if (tid < k) {
    sc->tile_first[tid] = bad ? 0 : first;
    sc->tile_cnt[tid] = bad ? 0 : nt;
    if (!bad)
      for (int t = 0; t < nt; ++t)
        sc->tiles[first + t] = make_int4(tid, a + t * NA_TILE, min(NA_TILE, size - t * NA_TILE), 0);
  }
}

// One warp per row: FP64 sum of squares, rounded to FP32.
__global__ void k_na_norms(const float* __restrict__ A, int64_t lda, int rows, int d, float* __restrict__ out) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  double acc = 0.0;
  const float* p = A + (int64_t)r * lda;
  for (int c = lane; c < d; c += 32) acc += (double)p[c] * (double)p[c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[r] = (float)acc;
}

// Persistent over (64-row query tile, 64-row support tile): FP32 Gram with
// bounds-checked scalar loads (any leading dimension), then the kernel values
// and the weighted sum of each query row over the tile's support rows.
// DIFF (Laplacian kernel): the tile accumulates ||q - y||^2 from the
// differences instead of <q, y>. Through ||q||^2 + ||y||^2 - 2 <q, y> a query
// equal to a support row would get d2 of the order of the FP32 rounding of
// its norm instead of 0, and the square root magnifies that into an error of
// its square root; the difference form has no such cancellation.
template <bool DIFF>
__global__ void __launch_bounds__(NT) k_na_gram(Scratch* sc, const float* __restrict__ Q, int64_t ldq, int rows,
                                                const float* __restrict__ Y, int64_t ldy,
                                                const float* __restrict__ w, int d, int kind, float negc,
                                                float coef0, int degree) {
  __shared__ float As[BK][64 + 4];
  __shared__ float Bs[BK][64 + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  const int R = (rows + 63) / 64;
  const int ntiles = sc->ntiles;
  for (int item = blockIdx.x; item < R * ntiles; item += gridDim.x) {
    const int t = item / R, rt = item % R;
    const int4 T = sc->tiles[t];
    const int arow = rt * 64 + lr;
    const bool a_ok = arow < rows, b_ok = lr < T.z;
    const float* ap = Q + (int64_t)(a_ok ? arow : 0) * ldq;
    const float* bp = Y + (int64_t)(T.y + (b_ok ? lr : 0)) * ldy;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < d; k0 += BK) {
      float av[4], bv[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = k0 + lk + e;
        av[e] = (a_ok && c < d) ? ap[c] : 0.0f;
        bv[e] = (b_ok && c < d) ? bp[c] : 0.0f;
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        As[lk + e][lr] = av[e];
        Bs[lk + e][lr] = bv[e];
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        float ar[4], br[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) { ar[i] = As[kk][ty * 4 + i]; br[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if constexpr (DIFF) {
              const float t = ar[i] - br[j];
              acc[i][j] = fmaf(t, t, acc[i][j]);
            } else {
              acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
            }
          }
      }
    }
    float yn[4], wy[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = tx * 4 + j;
      const bool ok = c < T.z;
      yn[j] = ok ? sc->yn[T.y + c] : 0.0f;
      wy[j] = ok ? w[T.y + c] : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rt * 64 + ty * 4 + i;
      const float xn = r < rows ? sc->qn[r] : 0.0f;
      float sum = 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float kv = DIFF ? exp2f(sqrtf(acc[i][j]) * negc)
                              : kkm::kernel_from_gram(kind, acc[i][j], xn, yn[j], false, negc, coef0, degree);
        sum += (tx * 4 + j < T.z) ? wy[j] * kv : 0.0f;
      }
      sum += __shfl_xor_sync(0xffffffffu, sum, 8);
      sum += __shfl_xor_sync(0xffffffffu, sum, 4);
      sum += __shfl_xor_sync(0xffffffffu, sum, 2);
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      if (tx == 0 && r < rows) sc->part[(int64_t)t * NA_ROWS + r] = sum;
    }
  }
}

// One thread per query row: Delta(q, C_j) = K(q,q) - 2 <phi(q), C_j> + ||C_j||^2
// and the argmin (ties to the lowest j). Rejected offsets give NaN distances
// and the assignment -1 on every row.
__global__ void k_na_argmin(const Scratch* sc, int rows, int k, const double* __restrict__ cnorm, int kind,
                            double coef0, int degree, float* __restrict__ dist_out,
                            int32_t* __restrict__ assign_out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= rows) return;
  if (sc->bad) {
    if (dist_out)
      for (int j = 0; j < k; ++j) dist_out[(int64_t)x * k + j] = __int_as_float(0x7fc00000);
    if (assign_out) assign_out[x] = -1;
    return;
  }
  const double kxx = kkm::kernel_self(kind, (double)sc->qn[x], coef0, degree);
  double best = 1e300;
  int bj = 0;
  for (int j = 0; j < k; ++j) {
    double inner = 0.0;
    const int t0 = sc->tile_first[j], nt = sc->tile_cnt[j];
    for (int t = 0; t < nt; ++t) inner += (double)sc->part[(int64_t)(t0 + t) * NA_ROWS + x];
    const double dist = kxx - 2.0 * inner + cnorm[j];
    if (dist_out) dist_out[(int64_t)x * k + j] = (float)dist;
    if (dist < best) { best = dist; bj = j; }
  }
  if (assign_out) assign_out[x] = bj;
}

}  // namespace

KKM_API const char* kkm_noalloc_last_error(void) { return g_na_error.c_str(); }

KKM_API kkm_status kkm_distances_noalloc(const float* Q, int64_t m, int64_t ldq, int32_t d, const float* Y,
                                         int64_t S, int64_t ldy, const float* w, const int32_t* seg_off,
                                         const double* cnorm, int32_t k, const kkm_kernel* kernel,
                                         float* dist_out, int32_t* assign_out, void* stream) {
  if (m < 0) return na_fail(KKM_EINVAL, "m must be >= 0");
  if (m > 0) {
    if (!kernel) return na_fail(KKM_EINVAL, "kernel is required");
    if (!Q) return na_fail(KKM_EINVAL, "Q must be given when m > 0");
    if (d < 1 || d > 4096) return na_fail(KKM_EINVAL, "d must be in [1, 4096]");
    if (ldq < d) return na_fail(KKM_EINVAL, "ldq must be >= d");
    if (k < 1 || k > 1024) return na_fail(KKM_EINVAL, "k must be in [1, 1024]");
    if (S < 0 || S > NA_MAX_S)
      return na_fail(KKM_EINVAL, "S exceeds the scratch limit KKM_NOALLOC_MAX_SUPPORT (65536 support rows)");
    if ((S + NA_TILE - 1) / NA_TILE + k > NA_MAX_TILES)
      return na_fail(KKM_EINVAL,
                     "ceil(S/64) + k exceeds the scratch limit KKM_NOALLOC_MAX_TILES (1024 support tiles)");
    if (S > 0 && (!Y || !w || ldy < d)) return na_fail(KKM_EINVAL, "Y and w are required and ldy must be >= d");
    if (!seg_off || !cnorm) return na_fail(KKM_EINVAL, "seg_off and cnorm are required");
    if (kernel->kind < KKM_GAUSSIAN || kernel->kind > KKM_POLY) return na_fail(KKM_EINVAL, "unknown kernel kind");
    if ((kernel->kind == KKM_GAUSSIAN || kernel->kind == KKM_LAPLACIAN) && !(kernel->param > 0.0))
      return na_fail(KKM_EINVAL, "kernel param must be > 0");
    if (kernel->kind == KKM_POLY && (kernel->degree < 1 || kernel->degree > 8))
      return na_fail(KKM_EINVAL, "polynomial degree must be in [1, 8]");
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return na_fail(KKM_ECUDA, "cudaGetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* base = nullptr;
  bool load = false;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, kkm_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return na_fail(KKM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
      g_na_addr[dev] = p;
    }
    base = g_na_addr[dev];
    load = m == 0 && !g_na_loaded[dev];
    if (load) g_na_loaded[dev] = true;
  }
  Scratch* sc = static_cast<Scratch*>(base);
  if (m == 0) {
    // The first empty call on a device launches every kernel of this file on
    // empty work (no row, no center), so that their code is loaded now
    // rather than on the first call with queries.
    cudaError_t e = cudaSuccess;
    if (load) {
      e = na_launch(k_na_tiles, 1, 1024, st, sc, (const int32_t*)nullptr, 0, 0);
      if (e == cudaSuccess) e = na_launch(k_na_norms, 1, 256, st, (const float*)nullptr, (int64_t)0, 0, 1, sc->qn);
      if (e == cudaSuccess)
        e = na_launch(k_na_gram<false>, 1, NT, st, sc, (const float*)nullptr, (int64_t)0, 0, (const float*)nullptr,
                      (int64_t)0, (const float*)nullptr, 1, (int)KKM_LINEAR, 0.0f, 0.0f, 1);
      if (e == cudaSuccess)
        e = na_launch(k_na_gram<true>, 1, NT, st, sc, (const float*)nullptr, (int64_t)0, 0, (const float*)nullptr,
                      (int64_t)0, (const float*)nullptr, 1, (int)KKM_LAPLACIAN, 0.0f, 0.0f, 1);
      if (e == cudaSuccess)
        e = na_launch(k_na_argmin, 1, 128, st, (const Scratch*)sc, 0, 0, (const double*)nullptr, (int)KKM_LINEAR,
                      0.0, 1, (float*)nullptr, (int32_t*)nullptr);
      if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        g_na_loaded[dev] = false;
      }
    }
    return e == cudaSuccess ? KKM_OK : na_fail(KKM_ECUDA, cudaGetErrorString(e));
  }

  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    (void)cudaGetLastError();
    sms = 148;
  }
  const bool normalised = kernel->kind == KKM_GAUSSIAN || kernel->kind == KKM_LAPLACIAN;
  const float negc = normalised ? (float)(-1.4426950408889634 / kernel->param) : 0.0f;
  const int Si = (int)S;
  const int max_tiles = (Si + NA_TILE - 1) / NA_TILE + k;   // bound on the tiles k_na_tiles writes

  cudaError_t e = na_launch(k_na_tiles, 1, 1024, st, sc, seg_off, (int)k, Si);
  if (e == cudaSuccess && Si > 0) e = na_launch(k_na_norms, (Si * 32 + 255) / 256, 256, st, Y, ldy, Si, (int)d, sc->yn);
  for (int64_t r0 = 0; r0 < m && e == cudaSuccess; r0 += NA_ROWS) {
    const int rows = (int)std::min<int64_t>(NA_ROWS, m - r0);
    e = na_launch(k_na_norms, (rows * 32 + 255) / 256, 256, st, Q + r0 * ldq, ldq, rows, (int)d, sc->qn);
    if (e == cudaSuccess && Si > 0) {
      const int items = ((rows + 63) / 64) * max_tiles;
      const int grid = std::max(1, std::min(items, sms * 4));
      e = na_launch(kernel->kind == KKM_LAPLACIAN ? k_na_gram<true> : k_na_gram<false>, grid, NT, st, sc,
                    Q + r0 * ldq, ldq, rows, Y, ldy, w, (int)d, (int)kernel->kind, negc, (float)kernel->coef0,
                    (int)kernel->degree);
    }
    if (e == cudaSuccess)
      e = na_launch(k_na_argmin, (rows + 127) / 128, 128, st, (const Scratch*)sc, rows, (int)k, cnorm,
                    (int)kernel->kind, kernel->coef0, (int)kernel->degree, dist_out ? dist_out + r0 * k : nullptr,
                    assign_out ? assign_out + r0 : nullptr);
  }
  if (e != cudaSuccess) return na_fail(KKM_ECUDA, cudaGetErrorString(e));
  return KKM_OK;
}
