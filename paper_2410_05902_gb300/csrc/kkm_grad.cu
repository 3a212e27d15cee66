// Batch objective at fixed assignments and its adjoint (kkm_objective_fwd /
// kkm_objective_bwd).
//
//   L(Q, s) = (1/m) sum_x Delta(x, C_{a(x)}),
//   Delta(x, C) = 1 - 2 sum_t w_t K(x, y_t) + N_C,  N_C = sum_{t,u} w_t w_u K(y_t, y_u)
//
// with the assignments, support rows and weights held fixed (the f_B
// objective of Sec. 3 at given assignments) and the bandwidth parameterised
// by s = log sigma: Gaussian kappa = 2 e^{2s}, Laplacian sigma = e^s. Both
// kernels have K(x,x) = 1. The support rows are constants, so the query
// gradient flows through the cross term only:
//   dL/dx = (2/m) sum_t c_t (x - y_t),   c_t = w_t g_t K(x, y_t),
//     g = 2/kappa (Gaussian), 1/(sigma ||x - y||) (Laplacian; 0 where x = y)
//   dL/ds = (1/m) sum_x [ -2 sum_t w_t dK(x,y_t)/ds + N'_{a(x)} ],
//     dK/ds = 2 K D^2 / kappa (Gaussian), K D / sigma (Laplacian),
//     N'_C = sum_{t,u} w_t w_u dK(y_t, y_u)/ds.
// Nothing is stored between the two calls: the adjoint recomputes every
// kernel value from the rows (the Gram tile is recomputed, not kept).
// Squared distances are taken as sums of squared differences in FP32 (more
// accurate than the Gram expansion for the D^2 factors of the gradient);
// per-lane sums are FP32, every reduction across rows and blocks is FP64 in
// a fixed order, so results are deterministic.
#include "kkm_internal.cuh"

namespace kkm {
namespace {

constexpr int GW = 8;          // warps per block
constexpr int DCH = 128;       // feature columns staged per pass (pair kernel)

struct BandParams {
  int kind;         // K_GAUSS or K_LAPLACE
  float p;          // kappa or sigma at s
  float negc;       // -log2(e)/kappa or -log2(e)/sigma
  float g_gauss;    // 2/kappa
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The FP32 data row of support row `row`, read from X through its data index
// (exact in every precision form; the BF16 copies of the distance pass are
// not used here).
__device__ __forceinline__ const float* support_row(const Dev& s, int64_t row) {
  return s.X + (int64_t)s.yi[row] * s.ldx;
}

// K, dK/ds and g of one pair from its squared distance.
__device__ __forceinline__ void pair_terms(const BandParams& bp, float d2, float& K, float& dks, float& g) {
  d2 = fmaxf(d2, 0.0f);
  if (bp.kind == K_GAUSS) {
    K = exp2f(d2 * bp.negc);
    dks = K * d2 * bp.g_gauss;
    g = bp.g_gauss;
  } else {
    const float D = sqrtf(d2);
    K = exp2f(D * bp.negc);
    dks = K * D / bp.p;
    g = D > 0.0f ? 1.0f / (bp.p * D) : 0.0f;
  }
}

// N_j and N'_j partials: block (chunk c of 32 window rows of center j) x the
// whole window of j, 32 window rows at a time staged in shared memory, DCH
// feature columns per pass. Warp w takes rows w, w+8, w+16, w+24 of the
// chunk; lane l the l-th row of the staged window slice.
__global__ void __launch_bounds__(32 * GW) k_center_pairs(Dev s, BandParams bp, int nch, double* part) {
  __shared__ __align__(16) float A[32][DCH + 4];   // rows padded to 16 bytes: float4 reads,
  __shared__ __align__(16) float B[32][DCH + 4];   // no bank conflicts within a quarter-warp
  __shared__ int64_t ia[32], ib[32];            // data rows of the chunk's and the staged block's support rows
  __shared__ double red[GW][2];
  const int j = blockIdx.x, c = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int head = s.head[j], size = s.tail[j] - head;
  const int r0 = c * 32;
  if (r0 >= size) return;   // the grid covers the window capacity; k_center_sum reads only chunks < size
  const int64_t base = (int64_t)j * s.cap + head;
  float acc = 0.0f, accs = 0.0f;
  // stages rows idx[0..32) (features k0..k0+kn) into T: every load issued before the stores
  // (features past kn up to the next multiple of 4 are zero: they add nothing)
  auto stage = [&](float (*T)[DCH + 4], const int64_t* idx, int k0, int kn) {
    const int kp = (kn + 3) & ~3;
    float v[(32 * DCH) / (32 * GW)];
#pragma unroll
    for (int q = 0; q < (32 * DCH) / (32 * GW); ++q) {
      const int e = threadIdx.x + q * 32 * GW;
      const int r = e / kp, k = e - r * kp;
      v[q] = e < 32 * kp && k < kn && idx[r] >= 0 ? __ldg(s.X + idx[r] * s.ldx + k0 + k) : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < (32 * DCH) / (32 * GW); ++q) {
      const int e = threadIdx.x + q * 32 * GW;
      const int r = e / kp, k = e - r * kp;
      if (e < 32 * kp) T[r][k] = v[q];
    }
  };
  if (threadIdx.x < 32) ia[threadIdx.x] = r0 + (int)threadIdx.x < size ? (int64_t)s.yi[base + r0 + threadIdx.x] : -1;
  const bool a_once = s.d <= DCH;               // one feature chunk: the chunk's rows are staged once
  {
    float wa[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + w + GW * u;
      wa[u] = r < size ? s.w32[base + r] : 0.0f;
    }
    __syncthreads();
    if (a_once) stage(A, ia, 0, s.d);
    for (int t0 = 0; t0 < size; t0 += 32) {
      float d2[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      __syncthreads();
      if (threadIdx.x < 32) ib[threadIdx.x] = t0 + (int)threadIdx.x < size ? (int64_t)s.yi[base + t0 + threadIdx.x] : -1;
      for (int k0 = 0; k0 < s.d; k0 += DCH) {
        const int kn = min(DCH, s.d - k0);
        __syncthreads();
        if (!a_once) stage(A, ia, k0, kn);
        stage(B, ib, k0, kn);
        __syncthreads();
        const int kp = (kn + 3) & ~3;
        for (int k = 0; k < kp; k += 4) {
          const float4 b4 = *reinterpret_cast<const float4*>(&B[lane][k]);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 a4 = *reinterpret_cast<const float4*>(&A[w + GW * u][k]);
            float sum = d2[u];
            float df = a4.x - b4.x;
            sum = fmaf(df, df, sum);
            df = a4.y - b4.y;
            sum = fmaf(df, df, sum);
            df = a4.z - b4.z;
            sum = fmaf(df, df, sum);
            df = a4.w - b4.w;
            d2[u] = fmaf(df, df, sum);
          }
        }
      }
      const float wb = t0 + lane < size ? s.w32[base + t0 + lane] : 0.0f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float K, dks, g;
        pair_terms(bp, d2[u], K, dks, g);
        const float ww = wa[u] * wb;
        acc = fmaf(ww, K, acc);
        accs = fmaf(ww, dks, accs);
      }
    }
  }
  const double a = warp_sum_d((double)acc), as = warp_sum_d((double)accs);
  if (lane == 0) { red[w][0] = a; red[w][1] = as; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double v = 0.0;
    for (int q = 0; q < GW; ++q) v += red[q][threadIdx.x];
    part[((int64_t)j * nch + c) * 2 + threadIdx.x] = v;
  }
}

// N_j, N'_j from the partials of the chunks that cover the window (fixed order).
__global__ void k_center_sum(Dev s, int nch, const double* part, double* cn) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s.k) return;
  const int used = min(nch, (s.tail[j] - s.head[j] + 31) / 32);
  double a = 0.0, b = 0.0;
  for (int c = 0; c < used; ++c) {
    a += part[((int64_t)j * nch + c) * 2];
    b += part[((int64_t)j * nch + c) * 2 + 1];
  }
  cn[2 * j] = a;
  cn[2 * j + 1] = b;
}

// One warp per query row x against the window of its assigned center, lane =
// window row. Forward: Delta(x). Adjoint (BWD): dL/dx, and the row's share of
// dL/ds. Per-block FP64 partials of sum Delta and of the ds terms. NK = feature
// registers per lane for the query gradient (32 * NK >= d). The warp stages
// each block of 32 window rows in shared memory, RC features at a time, with
// coalesced loads (a lane per feature); each lane then reads its own row there
// (rows padded to RC + 1 floats, no bank conflicts).
constexpr int RC = 64;                           // features per staged chunk
template <bool BWD, int NK>
__global__ void __launch_bounds__(32 * GW) k_rows(Dev s, BandParams bp, const float* __restrict__ Q, int64_t m,
                                                  int64_t ldq, const int32_t* __restrict__ assign,
                                                  const double* __restrict__ cn, float* __restrict__ delta,
                                                  const double* __restrict__ grad_loss, float* __restrict__ grad_q,
                                                  int64_t ldg, double* __restrict__ blk) {
  extern __shared__ float xs[];                 // [GW][d] query rows, then [GW][32][RC + 1] staged window rows
  __shared__ double red[GW][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t x = (int64_t)blockIdx.x * GW + w;
  float* xr = xs + (int64_t)w * s.d;
  float (*ys)[RC + 1] = reinterpret_cast<float (*)[RC + 1]>(xs + (int64_t)GW * s.d + (int64_t)w * 32 * (RC + 1));
  double my_delta = 0.0, my_ds = 0.0;
  if (x < m) {
    int j = assign[x];
    if (j < 0 || j >= s.k) {
      if (lane == 0) atomicOr(s.status, ST_BAD_ASSIGN);
      j = 0;
    }
    for (int k = lane; k < s.d; k += 32) xr[k] = Q[x * ldq + k];
    __syncwarp();
    const int head = s.head[j], size = s.tail[j] - head;
    const int64_t base = (int64_t)j * s.cap + head;
    float inner = 0.0f, dsum = 0.0f, csum = 0.0f;
    float u[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) u[i] = 0.0f;
    for (int t0 = 0; t0 < size; t0 += 32) {
      const int t = t0 + lane;
      const bool live = t < size;
      const int64_t row = base + (live ? t : 0);
      const int nrow = min(32, size - t0);
      const int64_t my_yi = s.yi[row];
      float d2 = 0.0f;
      for (int k0 = 0; k0 < s.d; k0 += RC) {
        const int kn = min(RC, s.d - k0);
        __syncwarp();
        // rows r of the block, a lane per feature: sixteen rows' loads in flight
        // before their stores (read-only loads, so they need not wait for them)
        for (int rb = 0; rb < nrow; rb += 16) {
          float v[16][2];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int r = rb + q;
            const float* src = s.X + __shfl_sync(0xffffffffu, my_yi, r & 31) * s.ldx + k0;
            v[q][0] = (r < nrow && lane < kn) ? __ldg(src + lane) : 0.0f;
            v[q][1] = (r < nrow && lane + 32 < kn) ? __ldg(src + lane + 32) : 0.0f;
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int r = rb + q;
            if (r < nrow) {
              if (lane < kn) ys[r][lane] = v[q][0];
              if (lane + 32 < kn) ys[r][lane + 32] = v[q][1];
            }
          }
        }
        __syncwarp();
        if (live)
          for (int kk = 0; kk < kn; ++kk) {
            const float df = xr[k0 + kk] - ys[lane][kk];
            d2 = fmaf(df, df, d2);
          }
      }
      float K, dks, g;
      pair_terms(bp, d2, K, dks, g);
      const float wt = live ? s.w32[row] : 0.0f;
      inner = fmaf(wt, K, inner);
      if constexpr (BWD) {
        dsum = fmaf(wt, dks, dsum);
        const float c = wt * g * K;
        csum += c;
        // u = sum_t c_t y_t: broadcast each lane's c, lanes over the features
        // (rows from the staged block when it holds all the features)
        const int nt = min(32, size - t0);
        for (int tt = 0; tt < nt; ++tt) {
          const float ct = __shfl_sync(0xffffffffu, c, tt);
          const float* yt = s.d <= RC ? ys[tt] : support_row(s, base + t0 + tt);
#pragma unroll
          for (int i = 0; i < NK; ++i) {
            const int k = lane + 32 * i;
            if (k < s.d) u[i] = fmaf(ct, yt[k], u[i]);
          }
        }
      }
    }
    const double in = warp_sum_d((double)inner);
    my_delta = 1.0 - 2.0 * in + cn[2 * j];
    if (!BWD && lane == 0 && delta) delta[x] = (float)my_delta;
    if constexpr (BWD) {
      const double ds = warp_sum_d((double)dsum);
      my_ds = -2.0 * ds + cn[2 * j + 1];
      const float cs = warp_sum_f(csum);
      const float scale = (float)(2.0 * grad_loss[0] / (double)m);
#pragma unroll
      for (int i = 0; i < NK; ++i) {
        const int k = lane + 32 * i;
        if (k < s.d) grad_q[x * ldg + k] = scale * fmaf(xr[k], cs, -u[i]);
      }
    }
  }
  if (lane == 0) { red[w][0] = my_delta; red[w][1] = my_ds; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double v = 0.0;
    for (int q = 0; q < GW; ++q) v += red[q][threadIdx.x];
    blk[(int64_t)blockIdx.x * 2 + threadIdx.x] = v;
  }
}

// loss = (1/m) sum Delta; ds = grad_loss * (1/m) sum (ds terms). One block, fixed order.
__global__ void k_rows_sum(int nblk, int64_t m, const double* blk, double* loss, const double* grad_loss,
                           double* ds) {
  __shared__ double r0[256], r1[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblk; i += 256) {
    a += blk[2 * i];
    b += blk[2 * i + 1];
  }
  r0[threadIdx.x] = a;
  r1[threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r0[threadIdx.x] += r0[threadIdx.x + o];
      r1[threadIdx.x] += r1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (loss) *loss = r0[0] / (double)m;
    if (ds) *ds = grad_loss[0] * r1[0] / (double)m;
  }
}

template <bool BWD, int NK>
cudaError_t launch_rows(const Dev& s, const BandParams& bp, const float* Q, int64_t m, int64_t ldq,
                        const int32_t* assign, const double* cn, float* delta, const double* grad_loss, float* grad_q,
                        int64_t ldg, double* blk, int64_t nblk, size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_rows<BWD, NK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               GW * (1024 + 32 * (RC + 1)) * 4);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_rows<BWD, NK><<<(unsigned)nblk, 32 * GW, smem, st>>>(s, bp, Q, m, ldq, assign, cn, delta, grad_loss, grad_q, ldg,
                                                         blk);
  return cudaGetLastError();
}

BandParams band_params(const Dev& s, double log_sigma) {
  BandParams bp;
  bp.kind = s.kind;
  const double p = s.kind == K_GAUSS ? 2.0 * exp(2.0 * log_sigma) : exp(log_sigma);
  bp.p = (float)p;
  bp.negc = (float)(-1.4426950408889634 / p);
  bp.g_gauss = (float)(2.0 / p);
  return bp;
}

}  // namespace

int grad_center_chunks(const Dev& s) { return (s.cap + 31) / 32; }

size_t grad_workspace_doubles(const Dev& s, int64_t m) {
  const int64_t nblk = (m + GW - 1) / GW;
  return (size_t)s.k * grad_center_chunks(s) * 2 + (size_t)s.k * 2 + (size_t)nblk * 2;
}

cudaError_t launch_objective(const Dev& s, double log_sigma, const float* Q, int64_t m, int64_t ldq,
                             const int32_t* assign, double* loss, float* delta, const double* grad_loss,
                             float* grad_q, int64_t ldg, double* grad_s, double* ws, cudaStream_t st) {
  const BandParams bp = band_params(s, log_sigma);
  const int nch = grad_center_chunks(s);
  double* part = ws;
  double* cn = part + (size_t)s.k * nch * 2;
  double* blk = cn + (size_t)s.k * 2;
  const int64_t nblk = (m + GW - 1) / GW;
  if (nblk > (int64_t)0x7fffffff) return cudaErrorInvalidValue;
  k_center_pairs<<<dim3(s.k, nch), 32 * GW, 0, st>>>(s, bp, nch, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_center_sum<<<(s.k + 127) / 128, 128, 0, st>>>(s, nch, part, cn);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)GW * (s.d + 32 * (RC + 1)) * sizeof(float);   // query rows + staged window rows
  if (grad_q) {
    if (s.d <= 64) e = launch_rows<true, 2>(s, bp, Q, m, ldq, assign, cn, nullptr, grad_loss, grad_q, ldg, blk, nblk, smem, st);
    else if (s.d <= 128) e = launch_rows<true, 4>(s, bp, Q, m, ldq, assign, cn, nullptr, grad_loss, grad_q, ldg, blk, nblk, smem, st);
    else if (s.d <= 256) e = launch_rows<true, 8>(s, bp, Q, m, ldq, assign, cn, nullptr, grad_loss, grad_q, ldg, blk, nblk, smem, st);
    else if (s.d <= 512) e = launch_rows<true, 16>(s, bp, Q, m, ldq, assign, cn, nullptr, grad_loss, grad_q, ldg, blk, nblk, smem, st);
    else e = launch_rows<true, 32>(s, bp, Q, m, ldq, assign, cn, nullptr, grad_loss, grad_q, ldg, blk, nblk, smem, st);
  } else {
    e = launch_rows<false, 1>(s, bp, Q, m, ldq, assign, cn, delta, nullptr, nullptr, 0, blk, nblk, smem, st);
  }
  if (e != cudaSuccess) return e;
  k_rows_sum<<<1, 256, 0, st>>>((int)nblk, m, blk, loss, grad_loss, grad_s);
  return cudaGetLastError();
}

}  // namespace kkm
