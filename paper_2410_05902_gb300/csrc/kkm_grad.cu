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
// Squared distances of query rows are sums of squared differences in FP32
// (the Laplacian's g = 1/(sigma D) and the D^2 factors of the gradient need
// them exact near D = 0). The Gaussian's window pair sums take D^2 = |a|^2 +
// |b|^2 - 2 a.b instead, with the norms and the dot products accumulated in
// the same order, so identical rows give exactly 0; the cancellation error of
// about eps (|a|^2 + |b|^2) moves K by that over kappa. Per-lane sums are FP32,
// every reduction across rows and blocks is FP64 in a fixed order, so results
// are deterministic.
#include "kkm_internal.cuh"

namespace kkm {
namespace {

constexpr int GW = 8;          // warps per block

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

// 4-byte asynchronous global -> shared copies (staging with every load in flight,
// no registers held).
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Window slabs in shared memory: SR rows of RC features (pitch RP: float4
// reads without bank conflicts), with each row's weight and data-row offset.
constexpr int RC = 64;                           // features per staged chunk
constexpr int RP = RC + 4;                       // staged row pitch
constexpr int NT = 8;                            // 32-row tiles per slab
constexpr int SR = 32 * NT;                      // rows per slab
constexpr size_t SLAB_SMEM = (size_t)(SR * RP + 2 * SR) * sizeof(float) + SR * sizeof(int64_t);

// The query rows grouped by assigned center, by one block: counts, offsets,
// the row list (rows of a center in any order: every per-row result is
// independent of it), and the row items (center, first list position,
// rows <= GW) the row kernel deals one per block. Out-of-range assignments
// raise ST_BAD_ASSIGN and count as center 0. sh: 4 * 1025 ints.
__device__ void group_rows(const Dev& s, const int32_t* __restrict__ assign, int64_t m, int* __restrict__ list,
                           int4* __restrict__ items, int* __restrict__ nitems, int* sh) {
  int* cnt = sh;
  int* cur = sh + 1025;
  int* off = sh + 2 * 1025;
  int* ist = sh + 3 * 1025;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int j = t; j < s.k; j += nt) {
    cnt[j] = 0;
    cur[j] = 0;
  }
  __syncthreads();
  bool bad = false;
  for (int64_t x = t; x < m; x += nt) {
    int j = assign[x];
    if (j < 0 || j >= s.k) {
      bad = true;
      j = 0;
    }
    atomicAdd(&cnt[j], 1);
  }
  if (bad) atomicOr(s.status, ST_BAD_ASSIGN);
  __syncthreads();
  if (t < 32) {
    // exclusive scans of the row counts and of the row items per center: a lane
    // per run of consecutive centers, then a warp scan of the run totals
    const int per = (s.k + 31) / 32, j0 = t * per, j1 = min(s.k, j0 + per);
    int sc = 0, si = 0;
    for (int j = j0; j < j1; ++j) {
      sc += cnt[j];
      si += (cnt[j] + GW - 1) / GW;
    }
    int ic = sc, ii = si;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int vc = __shfl_up_sync(0xffffffffu, ic, o), vi = __shfl_up_sync(0xffffffffu, ii, o);
      if (t >= o) {
        ic += vc;
        ii += vi;
      }
    }
    int ec = ic - sc, ei = ii - si;
    for (int j = j0; j < j1; ++j) {
      off[j] = ec;
      ist[j] = ei;
      ec += cnt[j];
      ei += (cnt[j] + GW - 1) / GW;
    }
    if (t == 31) {
      off[s.k] = ic;
      ist[s.k] = ii;
      *nitems = ii;
    }
  }
  __syncthreads();
  for (int64_t x = t; x < m; x += nt) {
    int j = assign[x];
    if (j < 0 || j >= s.k) j = 0;
    list[off[j] + atomicAdd(&cur[j], 1)] = (int)x;
  }
  const int ni = ist[s.k];
  for (int it = t; it < ni; it += nt) {
    int lo = 0, hi = s.k - 1;                   // the largest center whose items start at or before it
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ist[mid] <= it) lo = mid;
      else hi = mid - 1;
    }
    const int p = off[lo] + (it - ist[lo]) * GW;
    items[it] = make_int4(lo, p, min(GW, off[lo + 1] - p), 0);
  }
}

// N_j and N'_j partials. Block (j, y) takes the 32-row chunks c = y, y + py, ...
// of center j's window; chunk c meets its partners c + dl (mod nc) for
// dl = 0..nc/2, so each unordered pair of chunks is summed once (weight 2 off
// the diagonal; with nc even, the pair at distance nc/2 belongs to the lower
// chunk). A slab holds chunk c in its first tile and up to NT - 1 partners in
// the others, copied with 4-byte asynchronous copies, all in flight at once
// (rows past the window are zero with zero weight). Warp w takes rows w, w+8,
// w+16, w+24 of chunk c, lane l row l of each partner. Every block writes its
// partial (zero when it has no chunk). With py = 16, windows of up to 512 rows
// give each block at most one chunk. Block j * py + y; the one block after
// them groups the query rows (group_rows). GRAM (the Gaussian): D^2 from the
// staged rows' norms (thread r keeps row r's) and the dot products.
template <bool GRAM>
__global__ void __launch_bounds__(32 * GW) k_center_pairs(Dev s, BandParams bp, int py, double* __restrict__ part,
                                                          const int32_t* __restrict__ assign, int64_t m,
                                                          int* __restrict__ list, int4* __restrict__ items,
                                                          int* __restrict__ nitems) {
  extern __shared__ __align__(16) float sm[];
  float* ys = sm;                               // [SR][RP]
  float* yw = ys + SR * RP;                     // [SR] weights, partners' doubled off the diagonal
  int64_t* yx = reinterpret_cast<int64_t*>(yw + SR);   // [SR] data-row offsets, -1 past the window
  float* yn = reinterpret_cast<float*>(yx + SR);        // [SR] squared norms (GRAM)
  __shared__ double red[GW][2];
  KKM_GRID_DEP_WAIT();
  KKM_LAUNCH_DEPENDENTS();
  if ((int)blockIdx.x == s.k * py) {
    group_rows(s, assign, m, list, items, nitems, reinterpret_cast<int*>(sm));
    return;
  }
  const int j = (int)blockIdx.x / py, y = (int)blockIdx.x - j * py;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int head = s.head[j], size = s.tail[j] - head;
  const int nc = (size + 31) / 32, h = nc / 2;
  if (y >= nc) {                                // no chunk for this block
    if (threadIdx.x < 2) part[((int64_t)j * py + y) * 2 + threadIdx.x] = 0.0;
    return;
  }
  const int64_t base = (int64_t)j * s.cap + head;
  float acc = 0.0f, accs = 0.0f;
  for (int c = y; c < nc; c += py) {
    const int nb = ((nc & 1) == 0 && c >= h) ? h : h + 1;   // partners of c
    for (int q0 = 0; q0 < nb; q0 += NT - 1) {
      const int nq = min(NT - 1, nb - q0);
      const int nr = 32 * (1 + nq);
      __syncthreads();                          // the previous slab's readers are done
      for (int r = threadIdx.x; r < nr; r += 32 * GW) {
        int t = c * 32 + r;
        float f = 1.0f;
        if (r >= 32) {
          const int dl = q0 + (r >> 5) - 1;
          t = (c + dl < nc ? c + dl : c + dl - nc) * 32 + (r & 31);
          f = dl == 0 ? 1.0f : 2.0f;
        }
        const bool live = t < size;
        yx[r] = live ? (int64_t)s.yi[base + t] * s.ldx : -1;
        yw[r] = live ? f * s.w32[base + t] : 0.0f;
      }
      __syncthreads();
      float d2[NT - 1][4];                      // squared distances, or dot products (GRAM)
#pragma unroll
      for (int q = 0; q < NT - 1; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) d2[q][u] = 0.0f;
      float nrm = 0.0f;                         // |row threadIdx.x|^2 (GRAM)
      for (int k0 = 0; k0 < s.d; k0 += RC) {
        const int kn = min(RC, s.d - k0), kp = (kn + 3) & ~3;
        if (k0 > 0) __syncthreads();            // the previous feature chunk's readers are done
        for (int r = w; r < nr; r += GW) {
          const int64_t o = yx[r];
          float* dst = ys + r * RP;
          for (int cc = lane; cc < kp; cc += 32) {
            if (o >= 0 && cc < kn) cp_async4(dst + cc, s.X + o + k0 + cc);
            else dst[cc] = 0.0f;
          }
        }
        cp_async_wait_all();
        __syncthreads();
        if (GRAM && (int)threadIdx.x < nr) {
          // the same fmaf sequence as a dot product of the row with itself
          const float* v = ys + threadIdx.x * RP;
          for (int kk = 0; kk < kp; kk += 4) {
            const float4 v4 = *reinterpret_cast<const float4*>(v + kk);
            nrm = fmaf(v4.x, v4.x, nrm);
            nrm = fmaf(v4.y, v4.y, nrm);
            nrm = fmaf(v4.z, v4.z, nrm);
            nrm = fmaf(v4.w, v4.w, nrm);
          }
        }
        for (int kk = 0; kk < kp; kk += 4) {
          float4 a4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) a4[u] = *reinterpret_cast<const float4*>(ys + (w + GW * u) * RP + kk);
#pragma unroll
          for (int q = 0; q < NT - 1; ++q) {
            if (q < nq) {
              const float4 b4 = *reinterpret_cast<const float4*>(ys + (32 + 32 * q + lane) * RP + kk);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                float sum = d2[q][u];
                if constexpr (GRAM) {
                  sum = fmaf(a4[u].x, b4.x, sum);
                  sum = fmaf(a4[u].y, b4.y, sum);
                  sum = fmaf(a4[u].z, b4.z, sum);
                  d2[q][u] = fmaf(a4[u].w, b4.w, sum);
                } else {
                  float df = a4[u].x - b4.x;
                  sum = fmaf(df, df, sum);
                  df = a4[u].y - b4.y;
                  sum = fmaf(df, df, sum);
                  df = a4[u].z - b4.z;
                  sum = fmaf(df, df, sum);
                  df = a4[u].w - b4.w;
                  d2[q][u] = fmaf(df, df, sum);
                }
              }
            }
          }
        }
      }
      if constexpr (GRAM) {
        if ((int)threadIdx.x < nr) yn[threadIdx.x] = nrm;
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < NT - 1; ++q) {
        if (q < nq) {
          const float wb = yw[32 + 32 * q + lane];
          const float nb2 = GRAM ? yn[32 + 32 * q + lane] : 0.0f;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float K, dks, g;
            pair_terms(bp, GRAM ? fmaf(-2.0f, d2[q][u], yn[w + GW * u] + nb2) : d2[q][u], K, dks, g);
            const float ww = yw[w + GW * u] * wb;
            acc = fmaf(ww, K, acc);
            accs = fmaf(ww, dks, accs);
          }
        }
      }
    }
  }
  const double a = warp_sum_d((double)acc), as = warp_sum_d((double)accs);
  if (lane == 0) { red[w][0] = a; red[w][1] = as; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double v = 0.0;
    for (int q = 0; q < GW; ++q) v += red[q][threadIdx.x];
    part[((int64_t)j * py + y) * 2 + threadIdx.x] = v;
  }
}

// One row item per block: up to GW query rows x assigned to the same center j,
// a warp each, against j's window. Forward: Delta(x). Adjoint (BWD): dL/dx and
// the row's share of dL/ds. The window goes through shared memory in slabs of
// SR rows and RC features, copied once per block for all of its rows (4-byte
// asynchronous copies, all in flight at once); lane l takes row l of each
// 32-row tile of the slab. N_j, N'_j: the sum of the center's py pair
// partials (a fixed-order warp sum). Per-row results go to rowv[2x],
// rowv[2x+1] (the Delta and ds terms); the last block to finish sums them in
// row order into loss and ds. NK = feature registers per lane for the query
// gradient (32 * NK >= d). With d <= RC (UG) the adjoint's u_x = sum_t c_xt y_t
// is one product over the block per slab: the warps put their c_xt in shared
// memory, thread (g, k) sums rows t = g (mod 4) at feature k for all GW query
// rows, and the four partial sums are added in order at the end.
template <bool BWD, int NK>
__global__ void __launch_bounds__(32 * GW) k_rows(Dev s, BandParams bp, const float* __restrict__ Q, int64_t m,
                                                  int64_t ldq, const int* __restrict__ list,
                                                  const int4* __restrict__ items, const int* __restrict__ nitems,
                                                  const double* __restrict__ part, int py, float* __restrict__ delta,
                                                  const double* __restrict__ grad_loss, float* __restrict__ grad_q,
                                                  int64_t ldg, double* __restrict__ rowv, int* __restrict__ done,
                                                  double* __restrict__ loss, double* __restrict__ grad_s) {
  // [GW][dq] query rows | [SR][RP] slab | [SR] weights | [SR] row offsets | [SR][GW] c (UG)
  extern __shared__ __align__(16) float sm[];
  constexpr bool UG = BWD && 32 * NK <= RC;
  static_assert(32 * GW == 4 * RC, "UG maps the block to 4 row groups x RC features");
  __shared__ double cnj[2];
  __shared__ int last;
  KKM_GRID_DEP_WAIT();
  KKM_LAUNCH_DEPENDENTS();
  const int dq = (s.d + 3) & ~3;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if ((int)blockIdx.x < *nitems) {
    float* xq = sm;
    float* ys = xq + GW * dq;
    float* yw = ys + SR * RP;
    int64_t* yx = reinterpret_cast<int64_t*>(yw + SR);
    float* csm = reinterpret_cast<float*>(yx + SR);
    const int ug = threadIdx.x / RC, uk = threadIdx.x % RC;
    float ub[GW];
#pragma unroll
    for (int x8 = 0; x8 < GW; ++x8) ub[x8] = 0.0f;
    const int4 item = items[blockIdx.x];
    const int j = item.x, n = item.z;
    const bool mine = w < n;
    const int64_t x = mine ? list[item.y + w] : 0;
    const int head = s.head[j], size = s.tail[j] - head;
    const int64_t base = (int64_t)j * s.cap + head;
    float* xr = xq + w * dq;
    if (w == 0) {
      double pa = 0.0, pb = 0.0;
      if (lane < py) {
        pa = part[((int64_t)j * py + lane) * 2];
        pb = part[((int64_t)j * py + lane) * 2 + 1];
      }
      pa = warp_sum_d(pa);
      pb = warp_sum_d(pb);
      if (lane == 0) {
        cnj[0] = pa;
        cnj[1] = pb;
      }
    }
    if (mine) {
      for (int k = lane; k < dq; k += 32) {
        if (k < s.d) cp_async4(xr + k, Q + x * ldq + k);
        else xr[k] = 0.0f;
      }
    }
    float inner = 0.0f, dsum = 0.0f, csum = 0.0f;
    float u[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) u[i] = 0.0f;
    for (int s0 = 0; s0 < size; s0 += SR) {
      const int nr = min(SR, size - s0);
      const int ntile = (nr + 31) / 32;
      __syncthreads();                          // the previous slab's readers are done
      for (int r = threadIdx.x; r < nr; r += 32 * GW) {
        yx[r] = (int64_t)s.yi[base + s0 + r] * s.ldx;
        yw[r] = s.w32[base + s0 + r];
      }
      __syncthreads();
      float d2[NT];
#pragma unroll
      for (int t8 = 0; t8 < NT; ++t8) d2[t8] = 0.0f;
      for (int k0 = 0; k0 < s.d; k0 += RC) {
        const int kn = min(RC, s.d - k0), kp = (kn + 3) & ~3;
        if (k0 > 0) __syncthreads();            // the previous feature chunk's readers are done
        for (int r = w; r < nr; r += GW) {
          const float* src = s.X + yx[r] + k0;
          float* dst = ys + r * RP;
          for (int c = lane; c < kp; c += 32) {
            if (c < kn) cp_async4(dst + c, src + c);
            else dst[c] = 0.0f;
          }
        }
        cp_async_wait_all();
        __syncthreads();
        if (mine) {
          const float* q = xr + k0;
          for (int kk = 0; kk < kp; kk += 4) {
            const float4 q4 = *reinterpret_cast<const float4*>(q + kk);
#pragma unroll
            for (int t8 = 0; t8 < NT; ++t8) {
              if (t8 < ntile) {
                const float4 y4 = *reinterpret_cast<const float4*>(ys + (t8 * 32 + lane) * RP + kk);
                float sum = d2[t8];
                float df = q4.x - y4.x;
                sum = fmaf(df, df, sum);
                df = q4.y - y4.y;
                sum = fmaf(df, df, sum);
                df = q4.z - y4.z;
                sum = fmaf(df, df, sum);
                df = q4.w - y4.w;
                d2[t8] = fmaf(df, df, sum);
              }
            }
          }
        }
      }
      if (mine) {
        float cv[NT];
#pragma unroll
        for (int t8 = 0; t8 < NT; ++t8) {
          cv[t8] = 0.0f;
          if (t8 < ntile) {
            const int r = t8 * 32 + lane;
            const bool live = r < nr;
            float K, dks, g;
            pair_terms(bp, live ? d2[t8] : 0.0f, K, dks, g);
            const float wt = live ? yw[r] : 0.0f;
            inner = fmaf(wt, K, inner);
            if constexpr (BWD) {
              dsum = fmaf(wt, dks, dsum);
              cv[t8] = wt * g * K;
              csum += cv[t8];
            }
          }
        }
        if constexpr (BWD && !UG) {
          // u = sum_t c_t y_t: broadcast each lane's c, lanes over the features
          // (rows from the slab when it holds all the features, else from X)
#pragma unroll
          for (int t8 = 0; t8 < NT; ++t8) {
            const int nt = min(32, nr - t8 * 32);
            for (int tt = 0; tt < nt; ++tt) {
              const float ct = __shfl_sync(0xffffffffu, cv[t8], tt);
              const float* yt = s.d <= RC ? ys + (t8 * 32 + tt) * RP : s.X + yx[t8 * 32 + tt];
#pragma unroll
              for (int i = 0; i < NK; ++i) {
                const int k = lane + 32 * i;
                if (k < s.d) u[i] = fmaf(ct, yt[k], u[i]);
              }
            }
          }
        }
        if constexpr (UG) {
#pragma unroll
          for (int t8 = 0; t8 < NT; ++t8) {
            const int r = t8 * 32 + lane;
            if (t8 < ntile && r < nr) csm[r * GW + w] = cv[t8];
          }
        }
      }
      if constexpr (UG) {
        __syncthreads();
        for (int t = ug; t < nr; t += 4) {
          const float yv = ys[t * RP + uk];
          const float4 c0 = *reinterpret_cast<const float4*>(csm + t * GW);
          const float4 c1 = *reinterpret_cast<const float4*>(csm + t * GW + 4);
          ub[0] = fmaf(c0.x, yv, ub[0]);
          ub[1] = fmaf(c0.y, yv, ub[1]);
          ub[2] = fmaf(c0.z, yv, ub[2]);
          ub[3] = fmaf(c0.w, yv, ub[3]);
          ub[4] = fmaf(c1.x, yv, ub[4]);
          ub[5] = fmaf(c1.y, yv, ub[5]);
          ub[6] = fmaf(c1.z, yv, ub[6]);
          ub[7] = fmaf(c1.w, yv, ub[7]);
        }
      }
    }
    cp_async_wait_all();                        // an empty window staged nothing: the query row's copies
    __syncthreads();                            // (and cnj)
    float* ured = ys;                           // [4][GW][RC] partial u (UG)
    if constexpr (UG) {
#pragma unroll
      for (int x8 = 0; x8 < GW; ++x8) ured[(ug * GW + x8) * RC + uk] = ub[x8];
      __syncthreads();
    }
    if (mine) {
      const double in = warp_sum_d((double)inner);
      const double my_delta = 1.0 - 2.0 * in + cnj[0];
      double my_ds = 0.0;
      if (!BWD && lane == 0 && delta) delta[x] = (float)my_delta;
      if constexpr (BWD) {
        const double ds = warp_sum_d((double)dsum);
        my_ds = -2.0 * ds + cnj[1];
        const float cs = warp_sum_f(csum);
        const float scale = (float)(2.0 * grad_loss[0] / (double)m);
#pragma unroll
        for (int i = 0; i < NK; ++i) {
          const int k = lane + 32 * i;
          float ui = u[i];
          if constexpr (UG)
            ui = ((ured[(0 * GW + w) * RC + k] + ured[(1 * GW + w) * RC + k]) + ured[(2 * GW + w) * RC + k]) +
                 ured[(3 * GW + w) * RC + k];
          if (k < s.d) grad_q[x * ldg + k] = scale * fmaf(xr[k], cs, -ui);
        }
      }
      if (lane == 0) {
        rowv[2 * x] = my_delta;
        rowv[2 * x + 1] = my_ds;
      }
    }
  }
  // the last block to finish: loss = (1/m) sum Delta, ds = grad_loss * (1/m) sum
  // (ds terms), in row order
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(done, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double* r0 = reinterpret_cast<double*>(sm);
  double* r1 = r0 + 32 * GW;
  double a[4] = {0.0, 0.0, 0.0, 0.0}, b[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i0 = threadIdx.x; i0 < m; i0 += 4 * 32 * GW) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + q * 32 * GW;
      if (i < m) {
        a[q] += __ldcg(rowv + 2 * i);
        b[q] += __ldcg(rowv + 2 * i + 1);
      }
    }
  }
  r0[threadIdx.x] = (a[0] + a[1]) + (a[2] + a[3]);
  r1[threadIdx.x] = (b[0] + b[1]) + (b[2] + b[3]);
  __syncthreads();
  for (int o = 16 * GW; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r0[threadIdx.x] += r0[threadIdx.x + o];
      r1[threadIdx.x] += r1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (loss) *loss = r0[0] / (double)m;
    if (grad_s) *grad_s = grad_loss[0] * r1[0] / (double)m;
    *done = 0;                                  // ready for the next call
  }
}

constexpr size_t ROWS_SMEM_MAX = (size_t)(GW * 1024 + SR * RP + SR + SR * GW) * sizeof(float) + SR * sizeof(int64_t);

template <bool BWD, int NK>
cudaError_t launch_rows(const Dev& s, const BandParams& bp, const float* Q, int64_t m, int64_t ldq, const int* list,
                        const int4* items, const int* nitems, int64_t nblk, const double* part, int py, float* delta,
                        const double* grad_loss, float* grad_q, int64_t ldg, double* rowv, int* done, double* loss,
                        double* grad_s, cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  const cudaError_t e = smem_limit_once(k_rows<BWD, NK>, (int)ROWS_SMEM_MAX, attr);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)(GW * ((s.d + 3) & ~3) + SR * RP + SR + SR * GW) * sizeof(float) + SR * sizeof(int64_t);
  return launch_pdl(k_rows<BWD, NK>, dim3((unsigned)nblk), dim3(32 * GW), smem, st, s, bp, Q, m, ldq, list, items,
                    nitems, part, py, delta, grad_loss, grad_q, ldg, rowv, done, loss, grad_s);
}

// Objective workspace, carved from ws (doubles; cudaMalloc'd, so 16-byte aligned,
// and zeroed when allocated): the row kernel's finished-block counter and the
// item count (first, so the counter stays in place whatever m is; it is back
// to zero after every call) | row items | pair partials | per-row terms | row list.
struct GradWs {
  int4* items;
  double* part;
  double* rowv;
  int* nitems;
  int* done;
  int* list;
};

int pair_blocks(const Dev& s) { return (s.cap + 31) / 32 < 16 ? (s.cap + 31) / 32 : 16; }
int64_t row_items_max(const Dev& s, int64_t m) { return (m + GW - 1) / GW + s.k; }

GradWs carve(const Dev& s, int64_t m, double* ws) {
  GradWs g;
  g.done = reinterpret_cast<int*>(ws);
  g.nitems = g.done + 1;
  g.items = reinterpret_cast<int4*>(ws + 2);
  g.part = ws + 2 + 2 * row_items_max(s, m);
  g.rowv = g.part + (size_t)s.k * pair_blocks(s) * 2;
  g.list = reinterpret_cast<int*>(g.rowv + 2 * m);
  return g;
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

size_t grad_workspace_doubles(const Dev& s, int64_t m) {
  return 2 + (size_t)(2 * row_items_max(s, m)) + (size_t)s.k * pair_blocks(s) * 2 + (size_t)m * 2 + (size_t)(m + 1) / 2;
}

cudaError_t launch_objective(const Dev& s, double log_sigma, const float* Q, int64_t m, int64_t ldq,
                             const int32_t* assign, double* loss, float* delta, const double* grad_loss,
                             float* grad_q, int64_t ldg, double* grad_s, double* ws, cudaStream_t st) {
  if (m > (int64_t)0x3fffffff || s.k > 1024) return cudaErrorInvalidValue;
  const BandParams bp = band_params(s, log_sigma);
  const int py = pair_blocks(s);
  const GradWs g = carve(s, m, ws);
  const int64_t nblk = row_items_max(s, m);
  static std::atomic<uint64_t> attr_g{0}, attr_l{0};
  cudaError_t e = s.kind == K_GAUSS ? smem_limit_once(k_center_pairs<true>, (int)SLAB_SMEM, attr_g)
                                    : smem_limit_once(k_center_pairs<false>, (int)SLAB_SMEM, attr_l);
  if (e != cudaSuccess) return e;
  e = launch_pdl(s.kind == K_GAUSS ? k_center_pairs<true> : k_center_pairs<false>, dim3(s.k * py + 1),
                             dim3(32 * GW), SLAB_SMEM, st, s, bp, py, g.part, assign, m, g.list, g.items, g.nitems);
  if (e != cudaSuccess) return e;
  const double* part = g.part;
  if (grad_q) {
    if (s.d <= 64) e = launch_rows<true, 2>(s, bp, Q, m, ldq, g.list, g.items, g.nitems, nblk, part, py, nullptr, grad_loss, grad_q, ldg, g.rowv, g.done, nullptr, grad_s, st);
    else if (s.d <= 128) e = launch_rows<true, 4>(s, bp, Q, m, ldq, g.list, g.items, g.nitems, nblk, part, py, nullptr, grad_loss, grad_q, ldg, g.rowv, g.done, nullptr, grad_s, st);
    else if (s.d <= 256) e = launch_rows<true, 8>(s, bp, Q, m, ldq, g.list, g.items, g.nitems, nblk, part, py, nullptr, grad_loss, grad_q, ldg, g.rowv, g.done, nullptr, grad_s, st);
    else if (s.d <= 512) e = launch_rows<true, 16>(s, bp, Q, m, ldq, g.list, g.items, g.nitems, nblk, part, py, nullptr, grad_loss, grad_q, ldg, g.rowv, g.done, nullptr, grad_s, st);
    else e = launch_rows<true, 32>(s, bp, Q, m, ldq, g.list, g.items, g.nitems, nblk, part, py, nullptr, grad_loss, grad_q, ldg, g.rowv, g.done, nullptr, grad_s, st);
  } else {
    e = launch_rows<false, 1>(s, bp, Q, m, ldq, g.list, g.items, g.nitems, nblk, part, py, delta, nullptr, nullptr, 0, g.rowv, g.done, loss, nullptr, st);
  }
  return e;
}

}  // namespace kkm
