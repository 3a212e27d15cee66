// FP32 CUDA-core form of the two Gram passes.
//
// Distance pass: for each (64-row batch tile, 64-row support tile of center j),
// G = X_B Y^T in FP32, then in registers
//   K = kernel(||x||^2 + ||y||^2 - 2G) and part[tile][x] = sum_y w_y K(x, y),
// the per-tile share of <phi(x), C_j> (Sec. 1: <phi(x), c> for a center held
// as a weighted sum of feature vectors; Sec. 4.1 cost O(kb(b+tau))).
//
// Window pass (norm recurrence of Sec. 4 with the drops of Eq. (1)): for each
// center with a new block, the weighted sums
//   A   = sum_{p in D, q in W} w_p w_q K(p, q)   = <C, D>
//   Bdd = sum_{p in D, q in D} w_p w_q K(p, q)   = ||D||^2
//   E   = sum_{p in D, q in B} w_p K(p, q)       = b_j <D, cm(B_j)>
//   M   = sum_{p in B, q in B} K(p, q)           = b_j^2 ||cm(B_j)||^2
// where W is the old window, D its dropped prefix (old weights) and B the new
// block. Each tile writes its four FP64 partial sums; k_finalize adds them in
// tile order.
#include "kkm_internal.cuh"

namespace kkm {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// Four consecutive row values starting at column k, as the Gram product uses them:
// FP32 rows as stored; BF16 rows as hi, or hi + lo for the split form.
template <int F>
__device__ __forceinline__ float4 load4(const void* rowp, int k, int dp) {
  if constexpr (F == FORM_FP32) {
    return *reinterpret_cast<const float4*>((const float*)rowp + k);
  } else {
    const __nv_bfloat16* r = (const __nv_bfloat16*)rowp;
    const uint2 h = *reinterpret_cast<const uint2*>(r + k);
    const __nv_bfloat162 h0 = *reinterpret_cast<const __nv_bfloat162*>(&h.x);
    const __nv_bfloat162 h1 = *reinterpret_cast<const __nv_bfloat162*>(&h.y);
    float4 v = make_float4(__low2float(h0), __high2float(h0), __low2float(h1), __high2float(h1));
    if constexpr (F == FORM_BF16X3) {
      const uint2 l = *reinterpret_cast<const uint2*>(r + dp + k);
      const __nv_bfloat162 l0 = *reinterpret_cast<const __nv_bfloat162*>(&l.x);
      const __nv_bfloat162 l1 = *reinterpret_cast<const __nv_bfloat162*>(&l.y);
      v.x += __low2float(l0); v.y += __high2float(l0); v.z += __low2float(l1); v.w += __high2float(l1);
    }
    return v;
  }
}

// acc[i][j] = sum_k A[ty*4+i][k] * B[tx*4+j][k] for a 64x64 tile. A and B point
// at the tiles' first rows (element type by form); rows are `ld` elements apart
// and the product runs over kend columns (zero padded, a multiple of BK).
// DIFF: acc[i][j] = sum_k (A[ty*4+i][k] - B[tx*4+j][k])^2 instead.
template <int F, bool DIFF = false>
__device__ __forceinline__ void gram_tile(const void* __restrict__ A, const void* __restrict__ B,
                                          int ld, int kend, int dp, float (&acc)[4][4],
                                          float (*As)[BM + 4], float (*Bs)[BN + 4]) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lr = tid >> 2, lk = (tid & 3) * 4;   // loader: row, k offset
  const int esz = (F == FORM_FP32) ? 4 : 2;
  const char* arow = (const char*)A + (int64_t)lr * ld * esz;
  const char* brow = (const char*)B + (int64_t)lr * ld * esz;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (int k0 = 0; k0 < kend; k0 += BK) {
    const float4 a = load4<F>(arow, k0 + lk, dp);
    const float4 b = load4<F>(brow, k0 + lk, dp);
    __syncthreads();
    As[lk + 0][lr] = a.x; As[lk + 1][lr] = a.y; As[lk + 2][lr] = a.z; As[lk + 3][lr] = a.w;
    Bs[lk + 0][lr] = b.x; Bs[lk + 1][lr] = b.y; Bs[lk + 2][lr] = b.z; Bs[lk + 3][lr] = b.w;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 av = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float ar[4] = {av.x, av.y, av.z, av.w};
      const float br[4] = {bv.x, bv.y, bv.z, bv.w};
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
}

template <int F>
__device__ __forceinline__ const void* rows_ptr(const Dev& s, bool support, int64_t row) {
  if constexpr (F == FORM_FP32) return (support ? s.y32 : s.xb32) + row * s.ld;
  else return (support ? s.ybh : s.xbh) + row * s.ld;
}

__device__ __forceinline__ float sum16(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// Item w of a run's distance pass (row tile w % R of support tile w / R).
template <int F>
__device__ __forceinline__ void dist_simt_item(const Dev& s, int rows, int R, int w, float (*As)[BM + 4],
                                               float (*Bs)[BN + 4]) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool lap = s.kind == K_LAPLACE;
  {
    const int t = w / R, rt = w % R;
    const Tile T = s.tiles[t];
    float acc[4][4];
    // Laplacian kernel: ||x - y||^2 from the differences. Through ||x||^2 +
    // ||y||^2 - 2 <x, y> a query row equal to a support row (no data index to
    // recognise it by) keeps d2 ~ eps ||x||^2, which the square root magnifies.
    if (lap)
      gram_tile<F, true>(rows_ptr<F>(s, false, (int64_t)rt * BM), rows_ptr<F>(s, true, T.row0), s.ld,
                         F == FORM_FP32 ? s.ld : s.dp, s.dp, acc, As, Bs);
    else
      gram_tile<F>(rows_ptr<F>(s, false, (int64_t)rt * BM), rows_ptr<F>(s, true, T.row0), s.ld,
                   F == FORM_FP32 ? s.ld : s.dp, s.dp, acc, As, Bs);
    float yn[4], wy[4];
    int yi[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = tx * 4 + j;
      const bool ok = c < T.ncols;
      const int64_t g = (int64_t)T.row0 + (ok ? c : 0);
      yn[j] = s.yn[g];
      yi[j] = s.yi[g];
      wy[j] = ok ? s.w32[g] : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rt * BM + ty * 4 + i;
      const int rr = r < rows ? r : 0;
      const float xn = s.xbn[rr];
      const int xi = s.xbi[rr];
      float sum = 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool same = xi >= 0 && xi == yi[j];
        const float kv = lap ? exp2f(sqrtf(same ? 0.0f : acc[i][j]) * s.negc)
                             : kernel_from_gram(s.kind, acc[i][j], xn, yn[j], same, s.negc, (float)s.coef0,
                                                s.degree);
        sum += (tx * 4 + j < T.ncols) ? wy[j] * kv : 0.0f;
      }
      sum = sum16(sum);
      if (tx == 0 && r < rows) s.part[(int64_t)t * s.bpad + r] = sum;
    }
  }
}

template <int F>
__device__ __forceinline__ void dist_simt_body(const Dev& s, int rows, int bid, int nblk) {
  KKM_GRID_DEP_WAIT();
  KKM_LAUNCH_DEPENDENTS();
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  const int R = (rows + BM - 1) / BM;
  const int total = R * (*s.ntiles);
  for (int w = bid; w < total; w += nblk) dist_simt_item<F>(s, rows, R, w, As, Bs);
}

template <int F>
__global__ void __launch_bounds__(NT) k_dist_simt(Dev s, int rows) { dist_simt_body<F>(s, rows, blockIdx.x, gridDim.x); }

// Pair w of a run's window pass; its four sums go to wpart[w] (slot 0).
template <int F>
__device__ __forceinline__ void wgram_simt_item(const Dev& s, int w, float (*As)[BM + 4], float (*Bs)[BN + 4],
                                                double (*red)[NT / 32]) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;
  {
    const WPair pr = s.wpairs[w];
    const Plan P = s.plan[pr.j];
    const int64_t base = (int64_t)pr.j * s.cap;
    // row and column ranges, as positions inside the center's region
    int r0, rn, c0, cn;
    if (pr.kind == 0) { r0 = P.head_c; rn = P.ndrop; c0 = P.head_c; cn = P.tail_new - P.head_c; }
    else { r0 = P.tail_c; rn = P.cnt; c0 = P.tail_c; cn = P.cnt; }
    const int rs = r0 + pr.rt * BM, cs = c0 + pr.ct * BN;
    float acc[4][4];
    gram_tile<F>(rows_ptr<F>(s, true, base + rs), rows_ptr<F>(s, true, base + cs), s.ld,
                 F == FORM_FP32 ? s.ld : s.dp, s.dp, acc, As, Bs);
    double sA = 0.0, sB = 0.0, sE = 0.0, sM = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int pr_ = pr.rt * BM + ty * 4 + i;         // row offset inside its range
      if (pr_ >= rn) continue;
      const int64_t p = base + rs + ty * 4 + i;
      const float xn = s.yn[p];
      const int xi = s.yi[p];
      const double wp = s.w64[p];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int qc = pr.ct * BN + tx * 4 + j;
        if (qc >= cn) continue;
        const int qpos = cs + tx * 4 + j;                 // position in the region
        const int64_t q = base + qpos;
        const double kv = (double)kernel_from_gram(s.kind, acc[i][j], xn, s.yn[q], xi == s.yi[q],
                                                   s.negc, (float)s.coef0, s.degree);
        if (pr.kind == 0) {
          if (qpos < P.tail_c) {
            const double ww = wp * s.w64[q] * kv;
            sA += ww;
            if (qpos < P.head_new) sB += ww;
          } else {
            sE += wp * kv;
          }
        } else {
          sM += kv;
        }
      }
    }
    // fixed-order block reduction of the four sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sA += __shfl_xor_sync(0xffffffffu, sA, o);
      sB += __shfl_xor_sync(0xffffffffu, sB, o);
      sE += __shfl_xor_sync(0xffffffffu, sE, o);
      sM += __shfl_xor_sync(0xffffffffu, sM, o);
    }
    if (lane == 0) { red[0][warp] = sA; red[1][warp] = sB; red[2][warp] = sE; red[3][warp] = sM; }
    __syncthreads();
    if (tid < 16) {   // slot 0 holds the tile's sums, slots 1-3 are zero
      double v = 0.0;
      if (tid < 4)
        for (int q = 0; q < NT / 32; ++q) v += red[tid][q];
      s.wpart[(int64_t)w * 16 + tid] = v;
    }
    __syncthreads();
  }
}

template <int F>
__device__ __forceinline__ void wgram_simt_body(const Dev& s, int bid, int nblk) {
  KKM_GRID_DEP_WAIT();
  KKM_LAUNCH_DEPENDENTS();
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  __shared__ double red[4][NT / 32];
  const int total = *s.nwpairs;
  for (int w = bid; w < total; w += nblk) wgram_simt_item<F>(s, w, As, Bs, red);
}

template <int F>
__global__ void __launch_bounds__(NT) k_wgram_simt(Dev s) { wgram_simt_body<F>(s, blockIdx.x, gridDim.x); }

// Run groups: the items of all the launch's runs laid end to end (distance
// pass: row tiles x support tiles; window pass: pairs), block-strided, so the
// blocks stay busy until the last item of any run. Item w of the flat space is
// item w - off[r] of run r; every item writes only its own partials, so each
// run computes what its own launch would.
constexpr int GROUP_MAX_RUNS = 1024;

template <int F, int MODE>
__global__ void __launch_bounds__(NT) k_group_simt(GroupPhase g) {
  KKM_GRID_DEP_WAIT();
  KKM_LAUNCH_DEPENDENTS();
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  __shared__ double red[4][NT / 32];
  __shared__ int off[GROUP_MAX_RUNS + 1];
  const int nr = g.nruns < GROUP_MAX_RUNS ? g.nruns : GROUP_MAX_RUNS;
  for (int r = threadIdx.x; r < nr; r += NT) {
    const Dev& s = g.runs[r].s;
    off[r + 1] = MODE == 0 ? ((s.b + BM - 1) / BM) * (*s.ntiles) : *s.nwpairs;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    off[0] = 0;
    for (int r = 0; r < nr; ++r) off[r + 1] += off[r];
  }
  __syncthreads();
  const int total = off[nr];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    int lo = 0, hi = nr;                         // the run r with off[r] <= w < off[r + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (off[mid] <= w) lo = mid;
      else hi = mid;
    }
    const Dev& s = g.runs[lo].s;
    if constexpr (MODE == 0) dist_simt_item<F>(s, s.b, (s.b + BM - 1) / BM, w - off[lo], As, Bs);
    else wgram_simt_item<F>(s, w - off[lo], As, Bs, red);
  }
}

}  // namespace

cudaError_t launch_dist_simt(const Dev& s, int rows, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const int blocks = s.num_sms * 4;
  switch (s.form) {
    case FORM_FP32: return launch_pdl(k_dist_simt<FORM_FP32>, dim3(blocks), dim3(NT), 0, st, s, rows);
    case FORM_BF16: return launch_pdl(k_dist_simt<FORM_BF16>, dim3(blocks), dim3(NT), 0, st, s, rows);
    default: return launch_pdl(k_dist_simt<FORM_BF16X3>, dim3(blocks), dim3(NT), 0, st, s, rows);
  }
  return cudaGetLastError();
}

cudaError_t launch_wgram(const Dev& s, cudaStream_t st) {
  const int blocks = s.num_sms * 4;
  switch (s.form) {
    case FORM_FP32: return launch_pdl(k_wgram_simt<FORM_FP32>, dim3(blocks), dim3(NT), 0, st, s);
    case FORM_BF16: return launch_pdl(k_wgram_simt<FORM_BF16>, dim3(blocks), dim3(NT), 0, st, s);
    default: return launch_pdl(k_wgram_simt<FORM_BF16X3>, dim3(blocks), dim3(NT), 0, st, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_group_simt(const GroupPhase& g, int mode, int form, int blocks, cudaStream_t st) {
  const dim3 grid(blocks > 0 ? blocks : 1), block(NT);
  if (mode == 0) {
    switch (form) {
      case FORM_FP32: return launch_pdl(k_group_simt<FORM_FP32, 0>, grid, block, 0, st, g);
      case FORM_BF16: return launch_pdl(k_group_simt<FORM_BF16, 0>, grid, block, 0, st, g);
      default: return launch_pdl(k_group_simt<FORM_BF16X3, 0>, grid, block, 0, st, g);
    }
  }
  switch (form) {
    case FORM_FP32: return launch_pdl(k_group_simt<FORM_FP32, 1>, grid, block, 0, st, g);
    case FORM_BF16: return launch_pdl(k_group_simt<FORM_BF16, 1>, grid, block, 0, st, g);
    default: return launch_pdl(k_group_simt<FORM_BF16X3, 1>, grid, block, 0, st, g);
  }
}

}  // namespace kkm
