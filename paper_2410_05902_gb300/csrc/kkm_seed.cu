// Kernel k-means++ seeding on the GPU (kkm_kmeanspp).
//
// Secs. 1 and 5 start from k-means++ (Arthur and Vassilvitskii, 2007) run in
// feature space, so every initial center is a data point. D^2 sampling:
//   1. the first center is uniform over X;
//   2. each later center is x with probability proportional to
//      D(x)^2 = min over the chosen c of Delta(x, c),
//      Delta(x, c) = K(x,x) - 2 K(x,c) + K(c,c).
// The uniform variate of draw t is u_t = (h_t >> 11) * 2^-53 with h_t output t
// of SplitMix64 seeded with `seed`; the draw picks the first x whose running
// sum of D^2 exceeds u_t * total. Draw 0 (the first center) maps h_0 onto
// [0, n) by Lemire's multiply-high; so does a draw whose total is 0.
//
// Each draw is two launches: k_pp_update refreshes D^2 against the newest
// center (a warp per point, the distance in FP64 as a sum of squared
// differences, so D^2 matches an FP64 evaluation to rounding) and writes FP64
// block sums; k_pp_select finds the crossing point in one block. The chosen
// index stays on the device, so the k draws need no host round trip.
#include "kkm_internal.cuh"

namespace kkm {
namespace {

constexpr int PP_WARPS = 8;                 // points per update block (a warp each)

__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t counter) {
  return (double)(splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
}

__device__ double kernel_fp64(int kind, double d2, double xy, double param, double coef0, int degree) {
  if (kind == K_GAUSS) return exp(-d2 / param);
  if (kind == K_LAPLACE) return exp(-sqrt(d2) / param);
  if (kind == K_LINEAR) return xy;
  double base = xy + coef0, r = 1.0;
  for (int p = 0; p < degree; ++p) r *= base;
  return r;
}

struct PPArgs {
  const float* X;
  int64_t n, ldx;
  int d, kind, degree;
  double param, coef0;
  uint64_t seed;
  double* d2;          // [n] current D^2
  double* part;        // [nblk] block sums of D^2
  int64_t* chosen;     // [k] chosen indices (device)
};

// D^2(x) = min(D^2(x), Delta(x, c)) for c = chosen[t] (first draw: = Delta).
__global__ void __launch_bounds__(32 * PP_WARPS) k_pp_update(PPArgs a, int t) {
  __shared__ double red[PP_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t x = (int64_t)blockIdx.x * PP_WARPS + w;
  const int64_t c = a.chosen[t];
  double v = 0.0;
  if (x < a.n) {
    const float* xr = a.X + x * a.ldx;
    const float* cr = a.X + c * a.ldx;
    double s2 = 0.0, sxy = 0.0, sxx = 0.0, scc = 0.0;
    for (int i = lane; i < a.d; i += 32) {
      const double xv = xr[i], cv = cr[i], df = xv - cv;
      s2 = fma(df, df, s2);
      sxy = fma(xv, cv, sxy);
      sxx = fma(xv, xv, sxx);
      scc = fma(cv, cv, scc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      sxy += __shfl_xor_sync(0xffffffffu, sxy, o);
      sxx += __shfl_xor_sync(0xffffffffu, sxx, o);
      scc += __shfl_xor_sync(0xffffffffu, scc, o);
    }
    double delta;
    if (a.kind == K_GAUSS || a.kind == K_LAPLACE) {
      delta = 2.0 - 2.0 * kernel_fp64(a.kind, s2, 0.0, a.param, 0.0, 0);
    } else {
      delta = kernel_fp64(a.kind, 0.0, sxx, a.param, a.coef0, a.degree) -
              2.0 * kernel_fp64(a.kind, 0.0, sxy, a.param, a.coef0, a.degree) +
              kernel_fp64(a.kind, 0.0, scc, a.param, a.coef0, a.degree);
    }
    delta = fmax(delta, 0.0);
    v = (t == 0) ? delta : fmin(a.d2[x], delta);
    if (lane == 0) a.d2[x] = v;
  }
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < PP_WARPS; ++q) s += red[q];
    a.part[blockIdx.x] = s;
  }
}

// First index i in [lo, hi) with base + (v[lo] + ... + v[i]) > target, by one
// warp (32 values per round, warp scan, ballot); hi - 1 if none. Returns the
// index and leaves in *before the running sum before it.
template <typename Load>
__device__ int64_t warp_crossing(int64_t lo, int64_t hi, double base, double target, Load load, double* before) {
  const int lane = threadIdx.x & 31;
  for (int64_t i0 = lo; i0 < hi; i0 += 32) {
    const int64_t i = i0 + lane;
    const double v = i < hi ? load(i) : 0.0;
    double incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, i < hi && base + incl > target);
    if (hit) {
      const int l = __ffs(hit) - 1;
      const double inc_l = __shfl_sync(0xffffffffu, incl, l);
      const double v_l = __shfl_sync(0xffffffffu, v, l);
      *before = base + inc_l - v_l;
      return i0 + l;
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
  *before = base;
  return hi - 1;
}

// Draw t: total = sum of the block sums (fixed order); the first point whose
// running sum exceeds u_t * total (points in index order) becomes chosen[t].
// The search narrows run -> block -> point, each step by one warp.
__global__ void __launch_bounds__(1024) k_pp_select(PPArgs a, int nblk, int t) {
  __shared__ double wsum[32];
  __shared__ double pre[1024];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // thread r sums run r of `per` consecutive block sums
  const int per = (nblk + 1023) / 1024;
  const int b0 = min(tid * per, nblk), b1 = min(b0 + per, nblk);
  double mine = 0.0;
  for (int q = b0; q < b1; ++q) mine += a.part[q];
  double v = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    double u = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, u, o);
      if (lane >= o) u += y;
    }
    wsum[lane] = u;
  }
  __syncthreads();
  pre[tid] = mine;                      // run sums, scanned again below in index order
  __syncthreads();
  if (w != 0) return;
  const double total = wsum[31];
  int64_t c;
  if (!(total > 0.0)) {
    c = (int64_t)index_below(splitmix64(a.seed, (uint64_t)t), (uint64_t)a.n);
  } else {
    const double target = uniform01(a.seed, (uint64_t)t) * total;
    double before = 0.0;
    const int64_t r = warp_crossing(0, 1024, 0.0, target, [&](int64_t i) { return pre[i]; }, &before);
    const int64_t q0 = min((int64_t)r * per, (int64_t)nblk), q1 = min(q0 + per, (int64_t)nblk);
    const int64_t q = warp_crossing(q0, q1 > q0 ? q1 : q0 + 1, before, target,
                                    [&](int64_t i) { return i < nblk ? a.part[i] : 0.0; }, &before);
    const int64_t x0 = q * PP_WARPS, x1 = min(x0 + PP_WARPS, a.n);
    const int64_t x = warp_crossing(x0, x1 > x0 ? x1 : x0 + 1, before, target,
                                    [&](int64_t i) { return i < a.n ? a.d2[i] : 0.0; }, &before);
    c = x < a.n ? x : a.n - 1;
  }
  if (lane == 0) a.chosen[t] = c;
}

}  // namespace

cudaError_t launch_kmeanspp(const float* X, int64_t n, int d, int64_t ldx, int k, int kind, double param,
                            double coef0, int degree, uint64_t seed, double* d2, double* part, int64_t* chosen,
                            cudaStream_t st) {
  PPArgs a{X, n, ldx, d, kind, degree, param, coef0, seed, d2, part, chosen};
  const int64_t nblk = (n + PP_WARPS - 1) / PP_WARPS;
  if (nblk > (int64_t)0x7fffffff) return cudaErrorInvalidValue;
  // draw 0: uniform
  const int64_t first = (int64_t)index_below(splitmix64(seed, 0), (uint64_t)n);
  cudaError_t e = cudaMemcpyAsync(chosen, &first, sizeof(first), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  for (int t = 0; t < k; ++t) {
    if (t > 0) {
      k_pp_select<<<1, 1024, 0, st>>>(a, (int)nblk, t);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    if (t + 1 < k) {
      k_pp_update<<<(unsigned)nblk, 32 * PP_WARPS, 0, st>>>(a, t);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace kkm
