// Step kernels of truncated mini-batch kernel k-means (Algorithm 2, Appendix A):
// batch sampling, batch gather, argmin assignment, the stable counting sort and
// window plan, row moves, and the finalise step that carries ||C||^2 by the
// Sec. 4 recurrence (FP64) corrected for the rows Eq. (1) drops.
// The distance kernels themselves are in kkm_gram_simt.cu and kkm_gram_tc.cu.
#include <algorithm>

#include "kkm_internal.cuh"

namespace kkm {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Exclusive scan of one int per thread over a block of exactly 1024 threads.
// Returns the exclusive prefix; *total receives the block sum.
__device__ int block_exclusive_scan_1024(int v, int* total) {
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int t = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;   // inclusive warp-total prefix
  }
  __syncthreads();
  int excl = x - v + (warp > 0 ? wsum[warp - 1] : 0);
  if (total) *total = wsum[31];
  __syncthreads();
  return excl;
}

// Exclusive scans of three ints per thread over a block of exactly 1024
// threads, in one pass (two barriers plus one that frees the scratch).
__device__ void block_exclusive_scan3_1024(const int (&v)[3], int (&excl)[3], int (&total)[3]) {
  __shared__ int wsum3[32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x[3] = {v[0], v[1], v[2]};
#pragma unroll
  for (int o = 1; o < 32; o <<= 1)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int y = __shfl_up_sync(0xffffffffu, x[q], o);
      if (lane >= o) x[q] += y;
    }
  if (lane == 31)
    for (int q = 0; q < 3; ++q) wsum3[warp][q] = x[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      int t = wsum3[lane][q];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      wsum3[lane][q] = t;   // inclusive warp-total prefix
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    excl[q] = x[q] - v[q] + (warp > 0 ? wsum3[warp - 1][q] : 0);
    total[q] = wsum3[31][q];
  }
  __syncthreads();
}

// Largest i in [0, n) with a[i] <= v, for a non-decreasing a with a[0] <= v.
__device__ __forceinline__ int last_le(const int* a, int n, int v) {
  int lo = 0, hi = n;                    // answer in [lo, hi)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Stores four consecutive source values at column c of a batch/support row in
// the run's form and returns their contribution to ||row||^2 (the values the
// Gram product will use: FP32, TF32, BF16 hi, or BF16 hi + lo). Per-element work
// stays in FP32: FP64 throughput on GB300 is a small fraction of FP32's.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ float store4(const Dev& s, int64_t dst_row, bool to_support, int c, float4 v) {
  if (s.form == FORM_TF32) {   // the values the TF32 product uses: rounded to nearest, ties away
    v = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
  }
  if (f32_rows(s.form)) {
    float* dst = (to_support ? s.y32 : s.xb32) + dst_row * s.ld + c;
    *reinterpret_cast<float4*>(dst) = v;
    return fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, v.w * v.w)));
  }
  __nv_bfloat16* dst = (to_support ? s.ybh : s.xbh) + dst_row * s.ld + c;
  const float f[4] = {v.x, v.y, v.z, v.w};
  __align__(8) __nv_bfloat16 hi[4], lo[4];
  float acc = 0.0f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    hi[e] = __float2bfloat16_rn(f[e]);
    const float hf = __bfloat162float(hi[e]);
    lo[e] = __float2bfloat16_rn(f[e] - hf);
    const float used = (s.form == FORM_BF16) ? hf : hf + __bfloat162float(lo[e]);
    acc = fmaf(used, used, acc);
  }
  *reinterpret_cast<uint2*>(dst) = *reinterpret_cast<const uint2*>(hi);
  *reinterpret_cast<uint2*>(dst + s.dp) = *reinterpret_cast<const uint2*>(lo);
  return acc;
}

// Writes one FP32 source row (d values) into a batch/support row of the run's
// form and returns ||row||^2 of the values the Gram product will use. Each
// lane sums its columns in FP32 (at most d/32 terms) and the 32 lane sums are
// combined in FP64. Called by a whole warp. Each lane issues up to eight loads
// before it stores, so a row costs about one memory latency.
__device__ double warp_store_row(const Dev& s, const float* src, int64_t dst_row, bool to_support) {
  const int lane = threadIdx.x & 31;
  float acc = 0.0f;
  const int n4 = (s.d + 3) >> 2;
  const bool vec = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && ((s.d & 3) == 0);
  for (int c0 = 0; c0 < n4; c0 += 32 * 8) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + u * 32 + lane;
      if (c < n4) {
        if (vec) {
          v[u] = __ldg(reinterpret_cast<const float4*>(src) + c);
        } else {
          const int b = 4 * c;
          v[u].x = __ldg(src + b);
          v[u].y = b + 1 < s.d ? __ldg(src + b + 1) : 0.0f;
          v[u].z = b + 2 < s.d ? __ldg(src + b + 2) : 0.0f;
          v[u].w = b + 3 < s.d ? __ldg(src + b + 3) : 0.0f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + u * 32 + lane;
      if (c < n4) acc += store4(s, dst_row, to_support, 4 * c, v[u]);
    }
  }
  return warp_sum((double)acc);
}

// Copies a whole row (ld elements) between two rows of the run's row buffers,
// loads first (up to eight 16-byte loads per lane in flight), then stores.
__device__ void warp_copy_row(const Dev& s, bool src_support, int64_t src_row, int64_t dst_row) {
  const int lane = threadIdx.x & 31;
  const bool f32 = f32_rows(s.form);
  const int elem = f32 ? 4 : 2;
  const int n16 = s.ld * elem / 16;
  const char* src = (const char*)(src_support ? (f32 ? (void*)s.y32 : (void*)s.ybh)
                                              : (f32 ? (void*)s.xb32 : (void*)s.xbh));
  char* dst = (char*)(f32 ? (void*)s.y32 : (void*)s.ybh);
  const int4* sp = (const int4*)(src + src_row * (int64_t)s.ld * elem);
  int4* dp = (int4*)(dst + dst_row * (int64_t)s.ld * elem);
  for (int c0 = 0; c0 < n16; c0 += 32 * 8) {
    int4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + u * 32 + lane;
      if (c < n16) v[u] = sp[c];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + u * 32 + lane;
      if (c < n16) dp[c] = v[u];
    }
  }
}

// ------------------------------------------------------------------ kernels
__global__ void k_sample(Dev s) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.b) return;
  const int64_t it = *s.iter;
  const uint64_t c = (uint64_t)(it - 1) * (uint64_t)s.b + (uint64_t)t;
  s.bidx[t] = (int32_t)index_below(splitmix64(s.seed, c), (uint64_t)s.n);
}

// One warp per batch slot: X[idx] -> batch row, norm, data index. With idx
// NULL the slot's index is drawn here: SplitMix64 output (i-1)*b + slot.
__device__ __forceinline__ void gather_one(const Dev& s, const int32_t* __restrict__ idx, int warp) {
  int64_t i;
  if (idx) {
    i = idx[warp];
  } else {
    const uint64_t c = (uint64_t)(*s.iter - 1) * (uint64_t)s.b + (uint64_t)warp;
    i = index_below(splitmix64(s.seed, c), (uint64_t)s.n);
    if ((threadIdx.x & 31) == 0) s.bidx[warp] = (int32_t)i;
  }
  if (i < 0 || i >= s.n) {
    if ((threadIdx.x & 31) == 0) atomicOr(s.status, ST_BAD_BATCH_INDEX);
    i = 0;
  }
  double nrm = warp_store_row(s, s.X + i * s.ldx, warp, false);
  if ((threadIdx.x & 31) == 0) {
    s.xbn[warp] = (float)nrm;
    s.xbi[warp] = (int32_t)i;
  }
}

// Not rotated: waits first, then lets the distance pass stage what it reads
// from earlier steps (the support tiles, their norms and indices, the tile
// list; this kernel writes none of it). Rotated (launched right after the
// previous step's k_finalize): the rows are gathered first, while finalize
// runs (finalize touches none of the batch buffers, the indices or the
// iteration counter), and the distance pass is released at once: its early
// staging reads nothing finalize writes (it loads the weights after its own
// wait, which returns once this kernel, and so finalize, has completed).
// Then the wait and the clear of fin_pending.
__device__ __forceinline__ void gather_body(const Dev& s, const int32_t* __restrict__ idx, int rotated, int bid) {
  if (!rotated) {
    KKM_GRID_DEP_WAIT();
    KKM_LAUNCH_DEPENDENTS();
  }
  const int warp = (bid * blockDim.x + threadIdx.x) >> 5;
  if (warp < s.b) gather_one(s, idx, warp);
  if (rotated) {
    KKM_LAUNCH_DEPENDENTS();
    KKM_GRID_DEP_WAIT();
    if (bid == 0 && threadIdx.x == 0) *s.fin_pending = 0;
  }
}

__global__ void k_gather_batch(Dev s, const int32_t* __restrict__ idx, int rotated) {
  gather_body(s, idx, rotated, blockIdx.x);
}

__global__ void k_gather_query(Dev s, const float* __restrict__ Q, int64_t ldq, int rows) {
  KKM_GRID_DEP_WAIT();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= rows) return;
  double nrm = warp_store_row(s, Q + (int64_t)warp * ldq, warp, false);
  if ((threadIdx.x & 31) == 0) {
    s.xbn[warp] = (float)nrm;
    s.xbi[warp] = -1;
  }
}

// Block of 16 warps per 32 batch rows: lane = row, warp w handles centers
// w, w+16, ... so every load of the per-tile partials is one coalesced
// 128-byte line. <phi(x), C_j> is the sum of center j's per-tile partials (its
// tiles are the consecutive list entries tile_first[j] ..), then
// Delta(x, C_j) = K(x,x) - 2 <phi(x), C_j> + ||C_j||^2 in FP32, and the argmin
// with ties to the lowest j, across the warps in shared memory. A warp takes
// four centers at a time and issues the loads of their first four tiles
// before it adds anything, so a row costs a few memory latencies.
constexpr int AM_WARPS = 16;

__device__ __forceinline__ void argmin_body(const Dev& s, int rows, const int32_t* __restrict__ forced,
                                            int32_t* __restrict__ assign_out, float* __restrict__ mind_out,
                                            float* __restrict__ dist_out, int update, int bid) {
  // Before the wait: the tile tables, the center norms, the batch rows' norms
  // and the forced assignments. They come from kernels that completed before
  // this one was launched (it is launched once the distance pass has passed
  // its own wait): the sort/plan, the weight update and the gather.
  __shared__ float r_best[AM_WARPS][32], r_inner[AM_WARPS][32], r_f[AM_WARPS][32];
  __shared__ int r_j[AM_WARPS][32];
  __shared__ int c_first[1024], c_cnt[1024];
  __shared__ float c_norm[1024];
  for (int j = threadIdx.x; j < s.k; j += 32 * AM_WARPS) {   // a tile holds ppt consecutive partials
    c_first[j] = s.tile_first[j] * s.ppt;
    c_cnt[j] = s.tile_cnt[j] * s.ppt;
    c_norm[j] = s.cnorm32[j];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int x = bid * 32 + lane;
  const bool live = x < rows;
  const int xr = live ? x : 0;
  const float kxx = (float)kernel_self(s.kind, (double)s.xbn[xr], s.coef0, s.degree);
  const int fa = forced ? forced[xr] : -1;
  KKM_GRID_DEP_WAIT();       // the distance pass's partial sums
  KKM_LAUNCH_DEPENDENTS();   // the next kernel waits at its top
  __syncthreads();
  float best = 3.0e38f, best_inner = 0.0f, f_inner = 0.0f;
  int bj = 0x7fffffff;
  const float* part = s.part + xr;
  const int64_t ld = s.bpad;
  for (int j0 = w; j0 < s.k; j0 += 4 * AM_WARPS) {
    float v[4][4];
    int t0[4], nt[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 + u * AM_WARPS;
      t0[u] = j < s.k ? c_first[j] : 0;
      nt[u] = j < s.k ? c_cnt[j] : 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) v[u][t] = t < nt[u] ? part[(int64_t)(t0[u] + t) * ld] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 + u * AM_WARPS;
      if (j >= s.k) break;
      float i0 = v[u][0], i1 = v[u][1], i2 = v[u][2], i3 = v[u][3];
      for (int t = 4; t < nt[u]; t += 4) {
        i0 += part[(int64_t)(t0[u] + t) * ld];
        if (t + 1 < nt[u]) i1 += part[(int64_t)(t0[u] + t + 1) * ld];
        if (t + 2 < nt[u]) i2 += part[(int64_t)(t0[u] + t + 2) * ld];
        if (t + 3 < nt[u]) i3 += part[(int64_t)(t0[u] + t + 3) * ld];
      }
      const float inner = (i0 + i1) + (i2 + i3);
      const float dist = fmaf(-2.0f, inner, kxx + c_norm[j]);
      if (dist_out && live) dist_out[(int64_t)x * s.k + j] = dist;
      if (dist < best) { best = dist; bj = j; best_inner = inner; }   // j increases: ties keep the lowest
      if (j == fa) f_inner = inner;
    }
  }
  r_best[w][lane] = best;
  r_j[w][lane] = bj;
  r_inner[w][lane] = best_inner;
  r_f[w][lane] = f_inner;
  __syncthreads();
  if (w != 0 || !live) return;
  for (int o = 1; o < AM_WARPS; ++o) {
    const float ob = r_best[o][lane];
    const int oj = r_j[o][lane];
    if (ob < best || (ob == best && oj < bj)) { best = ob; bj = oj; best_inner = r_inner[o][lane]; }
    f_inner += r_f[o][lane];   // only the warp owning fa is non-zero
  }
  int a = bj;
  float a_inner = best_inner;
  if (forced) {
    if (fa < 0 || fa >= s.k) {
      atomicOr(s.status, ST_BAD_ASSIGN);
    } else {
      a = fa;
      a_inner = f_inner;
    }
  }
  if (assign_out) assign_out[x] = bj;
  if (mind_out) mind_out[x] = best;
  if (update) {
    s.assign[x] = a;
    s.mind[x] = best;
    s.inner_a[x] = a_inner;
  }
}

__global__ void __launch_bounds__(32 * AM_WARPS) k_argmin(Dev s, int rows, const int32_t* __restrict__ forced,
                                                          int32_t* __restrict__ assign_out,
                                                          float* __restrict__ mind_out,
                                                          float* __restrict__ dist_out, int update) {
  argmin_body(s, rows, forced, assign_out, mind_out, dist_out, update, blockIdx.x);
}

__device__ int tile_count(const Dev& s, int& head, int& size);
__device__ void tiles_write(const Dev& s, int first, int nt, int head, int size, int total);

// Single CTA of 1024 threads. Stable counting sort of the batch by center,
// alpha_i^j, <C_j, cm(B_j)>, and the per-center window plan: compaction,
// block push, the drops of Eq. (1), C_1 retirement, and the tile pairs of the
// norm-recurrence Gram pass.
__device__ __forceinline__ void sort_plan_body(const Dev& s, double* obj_out, int set_pending) {
  KKM_GRID_DEP_WAIT();
  KKM_LAUNCH_DEPENDENTS();   // the next kernel waits at its top (or only stages earlier steps' data)
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = s.k, b = s.b, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Plan* splan = (Plan*)smem;                // [k]   this step's window plans
  int32_t* cnt = (int32_t*)(splan + k);     // [k]
  int32_t* base = cnt + k;                  // [k]
  int32_t* tot = base + k;                  // [k]
  int32_t* coff = tot + k;                  // [k]
  float* sinner = (float*)(coff + k);       // [b]   <phi(x), C_a> at the used assignment
  int16_t* sassign = (int16_t*)(sinner + b);// [b]   assignments (k <= 1024)
  int16_t* sperm = sassign + b;             // [b]   batch rows sorted by center (b <= 8192)
  uint16_t* wtab = (uint16_t*)(sperm + b);  // [32][k] per-warp counts, then their exclusive prefixes
  uint16_t* srank = wtab + 32 * k;          // [b]   rank of a row among its warp's rows of its center
  __shared__ int s_rows;                    // support rows read by this step's distance pass
  if (tid == 0) s_rows = 0;
  // per-center window state, loaded up front together with the assignments
  // (and the two oldest entries of its block ring, so the usual step, which
  // drops at most one block, needs no dependent load later)
  int c_head = 0, c_tail = 0, c_c1 = 0, c_wsum = 0, c_first = 0, c_nb = 0;
  int c_cnt0 = 0, c_cnt1 = 0, c_it0 = 0, c_it1 = 0, c_iter = 0;
  if (tid < k) {
    c_head = s.head[tid];
    c_tail = s.tail[tid];
    c_c1 = s.c1[tid];
    c_wsum = s.wsum[tid];
    c_first = s.blk_first[tid];
    c_nb = s.blk_num[tid];
    c_iter = (int)(*s.iter);
    const int64_t rb = (int64_t)tid * s.nbcap;
    const int f1 = c_first + 1 == s.nbcap ? 0 : c_first + 1;
    c_cnt0 = s.blk_cnt[rb + c_first];
    c_cnt1 = s.blk_cnt[rb + f1];
    c_it0 = s.blk_iter[rb + c_first];
    c_it1 = s.blk_iter[rb + f1];
  }
  float macc = 0.0f;                        // this thread's share of sum_x min_j Delta
  for (int x = tid; x < b; x += 1024) {
    sassign[x] = (int16_t)s.assign[x];
    sinner[x] = s.inner_a[x];
    macc += s.mind[x];
  }
  const int tiles_used = *s.ntiles;         // tiles of this step's distance pass
  for (int e = tid; e < 32 * k; e += 1024) wtab[e] = 0;
  __syncthreads();
  // Stable counting sort of the batch by center in one pass. Warp w ranks the
  // contiguous rows [w seg, (w+1) seg), seg = ceil(b / 32), 32 at a time:
  // match.any gives each row its rank among the step's rows of the same
  // center, and wtab[w][j] (the rows of center j this warp has seen so far)
  // is added to it. No block barrier is needed until every warp is done.
  const int seg = (b + 31) / 32;
  {
    const int r0 = warp * seg, r1 = min(b, r0 + seg);
    uint16_t* wc = wtab + warp * k;
    for (int x0 = r0; x0 < r1; x0 += 32) {
      const int x = x0 + lane;
      const int j = x < r1 ? (int)sassign[x] : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, j);
      const int rank = __popc(peers & ((1u << lane) - 1u));
      const int before = j >= 0 ? (int)wc[j] : 0;
      __syncwarp();
      if (j >= 0 && rank == 0) wc[j] = (uint16_t)(before + __popc(peers));
      if (x < r1) srank[x] = (uint16_t)(before + rank);
      __syncwarp();
    }
  }
  __syncthreads();
  // per center: the exclusive prefix of the 32 warps' counts (a warp per
  // center, a lane per warp) and the center's count
  for (int j = warp; j < k; j += 32) {
    const int v = wtab[lane * k + j];
    int xs = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, xs, o);
      if (lane >= o) xs += y;
    }
    wtab[lane * k + j] = (uint16_t)(xs - v);
    if (lane == 31) cnt[j] = xs;
  }
  __syncthreads();
  // exclusive offsets over centers (k <= 1024: one center per thread)
  const int my = tid < k ? cnt[tid] : 0;
  int total_rows = 0;
  const int off = block_exclusive_scan_1024(my, &total_rows);
  if (tid < k) { coff[tid] = off; s.coff[tid] = off; s.counts[tid] = my; }
  if (tid == 0) s.coff[k] = total_rows;
  __syncthreads();
  for (int x = tid; x < b; x += 1024) {
    const int j = sassign[x];
    sperm[coff[j] + wtab[(x / seg) * k + j] + srank[x]] = (int16_t)x;
  }
  __syncthreads();
  for (int r = tid; r < b; r += 1024) s.perm[r] = sperm[r];
  // per center, the 32 lane partials (FP32) of sum_{x in B_j} <phi(x), C_j>;
  // k_finalize adds them in FP64
  for (int j = warp; j < k; j += 32) {
    const int n = cnt[j], o = coff[j];
    float part = 0.0f;
    for (int r = lane; r < n; r += 32) part += sinner[sperm[o + r]];
    s.cmpart[(int64_t)j * 32 + lane] = part;
  }
  // f_B(C_i) = (1/b) sum_x min_j Delta(x, C_i^j): FP32 partials, FP64 combine in fixed order
  {
    __shared__ float wpartial[32];
    float v = macc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wpartial[warp] = v;
    __syncthreads();
    if (warp == 0) {
      const double t = warp_sum((double)wpartial[lane]);
      if (lane == 0) {
        const double f = t * s.inv_b;
        *s.obj = f;
        if (obj_out) *obj_out = f;
      }
    }
  }
  if (tid < k) atomicAdd(&s_rows, c_tail - c_head);

  // window plan, one thread per center
  int npairs = 0, ncomp = 0;
  int thead = 0, tsize = 0;                 // the window this update leaves (the next tile list)
  if (tid < k) {
    const int j = tid;
    const int n = cnt[j];
    Plan P;
    P.head_c = c_head;
    P.tail_c = c_tail;
    P.head_new = P.head_c;
    P.tail_new = P.tail_c;
    P.src_head = -1;
    P.cnt = n;
    P.ndrop = 0;
    P.c1_new = c_c1;
    if (n > 0) {
      if (P.tail_c + n > s.cap - REGION_PAD) {   // compaction: move the window down to row 0
        P.src_head = P.head_c;
        P.tail_c = P.tail_c - P.head_c;
        P.head_c = 0;
        ncomp = P.tail_c;
      }
      P.tail_new = P.tail_c + n;
      if (P.tail_new > s.cap - REGION_PAD) atomicOr(s.status, ST_CAPACITY);
      int first = c_first, nb = c_nb;
      int32_t* bi = s.blk_iter + (int64_t)j * s.nbcap;
      int32_t* bc = s.blk_cnt + (int64_t)j * s.nbcap;
      const int f1 = c_first + 1 == s.nbcap ? 0 : c_first + 1;
      if (nb >= s.nbcap) {
        atomicOr(s.status, ST_CAPACITY);
      } else {
        const int slot = (first + nb) % s.nbcap;
        bi[slot] = c_iter;
        bc[slot] = n;
        if (slot == first) { c_cnt0 = n; c_it0 = c_iter; }   // the ring was empty
        else if (slot == f1) { c_cnt1 = n; c_it1 = c_iter; }
        ++nb;
      }
      int total = c_wsum + n;
      int drop_rows = 0;
      if (s.tau > 0) {
        // Q_i^j keeps the newest blocks whose counts reach tau: drop the
        // oldest block while the rest still sums to >= tau.
        int oldest = c_cnt0, dropped = 0;          // count of the oldest block in the ring
        while (nb > 1 && total - oldest >= s.tau) {
          drop_rows += oldest;
          total -= oldest;
          first = first + 1 == s.nbcap ? 0 : first + 1;
          --nb;
          ++dropped;
          oldest = dropped == 1 ? c_cnt1 : bc[first];
        }
        const int it_first = dropped == 0 ? c_it0 : (dropped == 1 ? c_it1 : bi[first]);
        // C_1 stays only while min Q_i^j = 1 (Eq. (1), Sec. 4.1).
        if (P.c1_new && total >= s.tau && it_first != 1) {
          P.c1_new = 0;
          P.ndrop += 1;
        }
      }
      P.ndrop += drop_rows;
      P.head_new = P.head_c + P.ndrop;
      s.blk_first[j] = first;
      s.blk_num[j] = nb;
      s.wsum[j] = total;
      // window-pass tiles: the dropped rows D against the old window and the new
      // block, and the new block against itself; tiles start at the range starts
      // rounded down to walign rows
      const int TR = s.pair_rows, TC = s.pair_cols;
      const int hoff = P.head_c & (s.walign - 1), toff = P.tail_c & (s.walign - 1);
      const int nD = P.ndrop, nL = P.tail_new - P.head_c;
      const int rD = nD > 0 ? (nD + hoff + TR - 1) / TR : 0;
      npairs = rD * ((nL + hoff + TC - 1) / TC) + ((n + toff + TR - 1) / TR) * ((n + toff + TC - 1) / TC);
    }
    s.plan[j] = P;
    splan[j] = P;
    thead = P.head_new;
    tsize = P.tail_new - P.head_new;
  }
  // one scan for the compaction offsets, the window-pass tiles and the next
  // step's distance tiles (the distance pass and argmin of this step have
  // already consumed the current tile list)
  const int nt = tile_count(s, thead, tsize);
  int v3[3] = {ncomp, npairs, nt}, ex3[3], tot3[3];
  block_exclusive_scan3_1024(v3, ex3, tot3);
  const int ptotal = tot3[1];
  if (tid < k) {
    s.comp_off[tid] = ex3[0];
    s.wpair_first[tid] = ex3[1];
    s.wpair_cnt[tid] = npairs;
    base[tid] = ex3[1];
    tot[tid] = npairs;
  }
  if (tid == 0) {
    *s.comp_total = tot3[0];
    *s.nwpairs = ptotal <= s.max_pairs ? ptotal : s.max_pairs;
    if (ptotal > s.max_pairs) atomicOr(s.status, ST_CAPACITY);
    s.stats[0] += 1;
    s.stats[1] += s_rows;
    s.stats[2] += tiles_used;
    *s.iter += 1;
    if (set_pending) *s.fin_pending = 1;
  }
  tiles_write(s, ex3[2], nt, thead, tsize, tot3[2]);   // its barrier also publishes base/tot
  // where k_move puts each sorted batch row: after the window's tail (after
  // the compaction, when there is one), in sorted order
  for (int r = tid; r < b; r += 1024) {
    const int x = sperm[r], j = sassign[x];
    const int pos = splan[j].tail_c + (r - coff[j]);
    s.mvdst[r] = pos < s.cap - REGION_PAD ? (int64_t)j * s.cap + pos : -1;   // else flagged ST_CAPACITY
  }
  // the window-pass tile list: a thread per tile, its center by binary search
  const int plim = ptotal <= s.max_pairs ? ptotal : s.max_pairs;
  for (int e = tid; e < plim; e += 1024) {
    const int j = last_le(base, k, e);
    const int i = e - base[j];
    if (i >= tot[j] || base[j] + tot[j] > s.max_pairs) continue;
    const Plan P = splan[j];
    const int TR = s.pair_rows, TC = s.pair_cols;
    const int hoff = P.head_c & (s.walign - 1), toff = P.tail_c & (s.walign - 1);
    const int nD = P.ndrop, nL = P.tail_new - P.head_c, n = P.cnt;
    const int cL = (nL + hoff + TC - 1) / TC, cB = (n + toff + TC - 1) / TC;
    const int n0 = (nD > 0 ? (nD + hoff + TR - 1) / TR : 0) * cL;
    const int f = i - n0;
    s.wpairs[e] = i < n0 ? WPair{j, 0, i / cL, i % cL} : WPair{j, 1, f / cB, f % cB};
  }
}

__global__ void __launch_bounds__(1024) k_sort_plan(Dev s, double* obj_out, int set_pending) {
  sort_plan_body(s, obj_out, set_pending);
}

// The append of the new blocks and the compaction of the windows that need
// it, one warp per row: work items 0..b-1 append batch row perm[w] at the end
// of its center's window; items b.. copy the compacting windows' rows down to
// row 0, all compactions laid end to end (comp_off). Sources and destinations
// never overlap (see the capacity argument in kkm_internal.cuh).
__device__ __forceinline__ void move_body(const Dev& s, int bid, int nblk) {
  KKM_GRID_DEP_WAIT();
  KKM_LAUNCH_DEPENDENTS();   // the next kernel waits at its top (or only stages earlier steps' data)
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int nwarps = nblk * wpb;
  const int items = s.b + *s.comp_total;
  for (int w = bid * wpb + (threadIdx.x >> 5); w < items; w += nwarps) {
    if (w < s.b) {
      const int x = s.perm[w];
      const int64_t dst = s.mvdst[w];              // the sort/plan's destination
      if (dst < 0) continue;                        // flagged ST_CAPACITY in the plan
      warp_copy_row(s, false, x, dst);
      if (lane == 0) {
        s.yn[dst] = s.xbn[x];
        s.yi[dst] = s.xbi[x];
      }
    } else {
      const int f = w - s.b;
      int lo = 0, hi = s.k;                         // last center with comp_off <= f
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s.comp_off[mid] <= f) lo = mid; else hi = mid;
      }
      const Plan P = s.plan[lo];
      const int r = f - s.comp_off[lo];
      const int64_t base = (int64_t)lo * s.cap;
      const int64_t src = base + P.src_head + r, dst = base + r;
      warp_copy_row(s, true, src, dst);
      if (lane == 0) {
        s.yn[dst] = s.yn[src];
        s.yi[dst] = s.yi[src];
        s.w64[dst] = s.w64[src];
        s.w32[dst] = s.w32[src];
      }
    }
  }
}

__global__ void k_move(Dev s) { move_body(s, blockIdx.x, gridDim.x); }

// Tile list of the distance pass (block of 1024, k <= 1024). Thread j < k
// passes the window [head, head + size) of center j. Tiles start at head
// rounded down to a multiple of 4 rows (16-byte aligned metadata); the rows
// before head that this adds carry weight 0.
// Tile counts of one center's window (thread j < k): the window [head,
// head + size) is widened down to a multiple of 4 rows, so every tile starts
// 4-aligned and its metadata copies are 16-byte aligned.
__device__ int tile_count(const Dev& s, int& head, int& size) {
  if (size > 0) {
    size += head & 3;
    head &= ~3;
  }
  return (int)threadIdx.x < s.k ? (size + s.tn - 1) / s.tn : 0;
}

// Writes the tile list given each center's first tile and count (exclusive
// scan over centers, total): tile_first/tile_cnt, ntiles, and one Tile per
// thread, its center found by a binary search over the first tiles.
__device__ void tiles_write(const Dev& s, int first, int nt, int head, int size, int total) {
  __shared__ int t_first[1024], t_nt[1024], t_head[1024], t_size[1024];
  const int tid = threadIdx.x;
  if (tid == 0) {
    *s.ntiles = total <= s.max_tiles ? total : s.max_tiles;
    if (total > s.max_tiles) atomicOr(s.status, ST_CAPACITY);
  }
  if (tid < s.k) {
    const bool fits = first + nt <= s.max_tiles;   // never false by the capacity bound
    s.tile_first[tid] = fits ? first : 0;
    s.tile_cnt[tid] = fits ? nt : 0;
    t_first[tid] = first;
    t_nt[tid] = fits ? nt : 0;
    t_head[tid] = head;
    t_size[tid] = size;
  }
  __syncthreads();
  const int lim = total <= s.max_tiles ? total : s.max_tiles;
  for (int t = tid; t < lim; t += 1024) {
    const int j = last_le(t_first, s.k, t);
    const int i = t - t_first[j];
    if (i < t_nt[j]) {
      const int c = i * s.tn;
      s.tiles[t] = Tile{j, (int32_t)((int64_t)j * s.cap + t_head[j] + c), min(s.tn, t_size[j] - c), 0};
    }
  }
}

__device__ void build_tiles_block(const Dev& s, int head, int size) {
  const int nt = tile_count(s, head, size);
  int total = 0;
  const int first = block_exclusive_scan_1024(nt, &total);
  tiles_write(s, first, nt, head, size, total);
}

__device__ void build_tiles_block(const Dev& s) {
  int head = 0, size = 0;
  if ((int)threadIdx.x < s.k) {
    head = s.head[threadIdx.x];
    size = s.tail[threadIdx.x] - head;
  }
  build_tiles_block(s, head, size);
}

__global__ void __launch_bounds__(1024) k_build_tiles(Dev s) {
  for (int j = threadIdx.x; j < s.k; j += 1024) s.cnorm32[j] = (float)s.cnorm[j];
  build_tiles_block(s);
}

// One block of 256 threads per center j that received points, FP64 where the
// values accumulate over iterations:
//   alpha_j = sqrt(b_j / b) (or eta), <C_j, cm(B_j)> = (1/b_j) sum_x <phi(x), C_j>
//   (from k_sort_plan's 32 FP32 lane partials), the window-pass sums, the
//   Sec. 4 recurrence for ||C_j||^2 corrected for the rows Eq. (1) drops, and
//   the weights: rows [head_new, tail_c) decay by (1 - alpha), rows
//   [tail_c, tail_new) get alpha / b_j, rows that left the window get 0.
// GB300 issues FP64 slowly, so the scalar FP64 work runs on one thread and the
// per-row work is spread over the block, with independent loads in flight.
// The scalar chain has no FP64 division or square root: 1/b_j and the beta
// rate sqrt(b_j / b) come from a table the host fills at kkm_init, and the
// thread's operands are loaded before the window sums so their latency overlaps.
__device__ __forceinline__ void finalize_body(const Dev& s, int if_pending, int bid) {
  // Before the wait: the pending flag, the plan, the running count, the old
  // norm, the rate table, the pair range and the sort/plan's partials of
  // <phi(x), C_j>. Their writers (the sort/plan, the gather, earlier weight
  // updates) completed before this kernel was launched: it is launched once
  // the kernel ahead (the window pass, or a full dependency) has passed its
  // own wait. Only the window-pass sums need the wait, and no block returns
  // before it, so this kernel never completes ahead of the one it follows.
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, j = bid;
  const bool skip = if_pending && *s.fin_pending == 0;   // nothing to apply (the first step, or after a flush)
  const Plan P = s.plan[j];
  double ncum_j = 0.0, cn_old = 0.0, inv_n = 0.0, beta = 0.0;
  if (tid == 0 && !skip && P.cnt > 0) {
    ncum_j = s.ncum[j];
    cn_old = s.cnorm[j];
    inv_n = s.rtab[P.cnt];
    beta = s.rtab[s.b + 1 + P.cnt];
  }
  __shared__ double red[8][4];
  __shared__ double cm_s;
  __shared__ double keep_s, wnew_s;
  const int per = s.wslots * 4;
  const int p0 = s.wpair_first[j];
  const int np = (p0 + s.wpair_cnt[j] <= s.max_pairs) ? s.wpair_cnt[j] : 0;
  if (warp == 0 && !skip && P.cnt > 0) {
    const double v = warp_sum((double)s.cmpart[(int64_t)j * 32 + lane]);
    if (lane == 0) cm_s = v;
  }
  KKM_GRID_DEP_WAIT();
  KKM_LAUNCH_DEPENDENTS();   // the next kernel waits at its top (or, the rotated gather, touches none of this)
  if (skip || P.cnt == 0) return;
  // window-pass sums: element e of a tile's partials is sum e & 3 (A, Bdd, E, M);
  // with a stride of 256 every thread stays on sum tid & 3
  const double* wp = s.wpart + (int64_t)p0 * per;
  double acc = 0.0;
#pragma unroll 8
  for (int e = tid; e < np * per; e += 256) acc += wp[e];
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane < 4) red[warp][lane] = acc;
  __syncthreads();
  const int n = P.cnt;
  if (warp == 0) {
    // lane t < 4 adds sum t over the eight warps, in warp order
    double qt = 0.0;
    if (lane < 4)
      for (int w = 0; w < 8; ++w) qt += red[w][lane];
    const double A = __shfl_sync(0xffffffffu, qt, 0), Bdd = __shfl_sync(0xffffffffu, qt, 1);
    const double E = __shfl_sync(0xffffffffu, qt, 2), M = __shfl_sync(0xffffffffu, qt, 3);
    if (lane == 0) {
      const double dn = (double)n;
      const double N = ncum_j + dn;      // points assigned to j so far, this batch included
      s.ncum[j] = N;
      double a;
      if (s.lr == 0) a = beta;               // sqrt(b_j / b)
      else if (s.lr == 2) a = dn / N;        // sklearn: the running-mean rate
      else a = s.eta;
      const double keep = 1.0 - a;
      s.alpha[j] = a;
      const double cmc = cm_s * inv_n;
      s.cmc[j] = cmc;
      // Sec. 4: ||C'||^2 = (1-a)^2 ||R||^2 + 2a(1-a) <R, m> + a^2 ||m||^2 with
      // m = cm(B_j) and R = C - D, the part of the old center Eq. (1) keeps
      const double m2 = M * inv_n * inv_n;
      const double R2 = cn_old - 2.0 * A + Bdd;
      const double Rm = cmc - E * inv_n;
      const double cn = keep * keep * R2 + 2.0 * a * keep * Rm + a * a * m2;
      s.cnorm[j] = cn;
      s.cnorm32[j] = (float)cn;
      s.head[j] = P.head_new;
      s.tail[j] = P.tail_new;
      s.c1[j] = P.c1_new;
      keep_s = keep;
      wnew_s = a * inv_n;
    }
  }
  __syncthreads();
  const double keep = keep_s, wnew = wnew_s;
  const float wnew32 = (float)wnew;
  const int64_t base = (int64_t)j * s.cap;
  // rows that leave the window get weight 0: the dropped prefix and, after a
  // compaction, the old copies of the moved rows
  for (int r = P.head_c + tid; r < P.head_new; r += 256) {
    s.w64[base + r] = 0.0;
    s.w32[base + r] = 0.0f;
  }
  if (P.src_head >= 0)
    for (int r = P.src_head + tid; r < P.src_head + (P.tail_c - P.head_c); r += 256) {
      s.w64[base + r] = 0.0;
      s.w32[base + r] = 0.0f;
    }
#pragma unroll 4
  for (int r = P.head_new + tid; r < min(P.tail_c, s.cap); r += 256) {
    const double w = s.w64[base + r] * keep;
    s.w64[base + r] = w;
    s.w32[base + r] = (float)w;
  }
  for (int r = P.tail_c + tid; r < min(P.tail_new, s.cap); r += 256) {
    s.w64[base + r] = wnew;
    s.w32[base + r] = wnew32;
  }
}

__global__ void __launch_bounds__(256) k_finalize(Dev s, int if_pending) { finalize_body(s, if_pending, blockIdx.x); }

// Seeds every window with C_1^j = phi(x_{init_idx[j]}), weight 1, ||C||^2 = K(x,x).
__global__ void k_init_centers(Dev s, const int32_t* __restrict__ init_idx) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= s.k) return;
  const int lane = threadIdx.x & 31;
  int64_t i = init_idx[j];
  if (i < 0 || i >= s.n) {
    if (lane == 0) atomicOr(s.status, ST_BAD_BATCH_INDEX);
    i = 0;
  }
  const int64_t row = (int64_t)j * s.cap;
  const float* src = s.X + i * s.ldx;
  double nrm = warp_store_row(s, src, row, true);
  double exact = 0.0;
  for (int c = lane; c < s.d; c += 32) exact += (double)src[c] * (double)src[c];
  exact = warp_sum(exact);
  if (lane == 0) {
    s.yn[row] = (float)nrm;
    s.yi[row] = (int32_t)i;
    s.w64[row] = 1.0;
    s.w32[row] = 1.0f;
    s.head[j] = 0;
    s.tail[j] = 1;
    s.c1[j] = 1;
    s.wsum[j] = 0;
    s.blk_first[j] = 0;
    s.blk_num[j] = 0;
    s.cnorm[j] = kernel_self(s.kind, exact, s.coef0, s.degree);
    s.cnorm32[j] = (float)s.cnorm[j];
  }
}

// Gathers the row data of every window row from X by its data index (restore).
__global__ void k_load_rows(Dev s) {
  const int j = blockIdx.x;
  const int warps = blockDim.x >> 5, wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)j * s.cap;
  for (int r = s.head[j] + wib; r < s.tail[j]; r += warps) {
    const int64_t row = base + r;
    int64_t i = s.yi[row];
    if (i < 0 || i >= s.n) {
      if (lane == 0) atomicOr(s.status, ST_BAD_BATCH_INDEX);
      i = 0;
    }
    double nrm = warp_store_row(s, s.X + i * s.ldx, row, true);
    if (lane == 0) s.yn[row] = (float)nrm;
  }
}

// scale * (FP64 sum of mind[0..rows)) into *out (single CTA, fixed order).
__global__ void __launch_bounds__(1024) k_mind_sum(Dev s, int rows, double scale, double* out) {
  KKM_GRID_DEP_WAIT();
  __shared__ double red[1024];
  double acc = 0.0;
  for (int x = threadIdx.x; x < rows; x += 1024) acc += (double)s.mind[x];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

// ------------------------------------------------------------------------
// Table form of Algorithm 1 (Appendix A, "Runtime analysis of Algorithm 1"):
// the run keeps T[j][x] = <phi(x), C_j> for every x in X and ||C_j||^2. An
// iteration reads the batch distances off the table, sorts the batch by
// center, lays the batch rows out center by center in the support buffer
// (blocks of whole tiles, weight 1/b_j), runs the n x b Gram pass against them
// (S[j][x] = <phi(x), cm(B_j)>), and updates
//   T[j][x] <- (1 - alpha_j) T[j][x] + alpha_j S[j][x],
//   ||C'||^2 = (1-a)^2 ||C||^2 + 2a(1-a) <C, cm(B_j)> + a^2 ||cm(B_j)||^2,
// with <C, cm(B_j)> = (1/b_j) sum_{y in B_j} T[j][y] (old table) and
// ||cm(B_j)||^2 = (1/b_j) sum_{y in B_j} S[j][y].

// Batch distances from the table: a warp per batch row, lanes over centers.
// Same outputs and tie rule as k_argmin.
__global__ void k_tab_batch_dist(Dev s, TabBuf q, int rows, const int32_t* __restrict__ forced,
                                 int32_t* __restrict__ assign_out, float* __restrict__ mind_out,
                                 float* __restrict__ dist_out, int update) {
  KKM_GRID_DEP_WAIT();
  const int x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (x >= rows) return;
  const int64_t i = s.xbi[x];
  const float kxx = (float)kernel_self(s.kind, (double)s.xbn[x], s.coef0, s.degree);
  const int fa = forced ? forced[x] : -1;
  float best = 3.0e38f, best_inner = 0.0f, f_inner = 0.0f;
  int bj = 0x7fffffff;
  for (int j = lane; j < s.k; j += 32) {
    const float inner = q.T[(int64_t)j * s.n + i];
    const float dist = fmaf(-2.0f, inner, kxx + s.cnorm32[j]);
    if (dist_out) dist_out[(int64_t)x * s.k + j] = dist;
    if (dist < best) { best = dist; bj = j; best_inner = inner; }
    if (j == fa) f_inner = inner;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
    const float oi = __shfl_xor_sync(0xffffffffu, best_inner, o);
    if (ob < best || (ob == best && oj < bj)) { best = ob; bj = oj; best_inner = oi; }
    f_inner += __shfl_xor_sync(0xffffffffu, f_inner, o);
  }
  if (lane != 0) return;
  int a = bj;
  float a_inner = best_inner;
  if (forced) {
    if (fa < 0 || fa >= s.k) atomicOr(s.status, ST_BAD_ASSIGN);
    else { a = fa; a_inner = f_inner; }
  }
  if (assign_out) assign_out[x] = bj;
  if (mind_out) mind_out[x] = best;
  if (update) {
    s.assign[x] = a;
    s.mind[x] = best;
    s.inner_a[x] = a_inner;
  }
}

// Single CTA: stable counting sort of the batch by center, <C_j, cm(B_j)>,
// f_B, the support-buffer layout (center j at bs_off[j], blocks of whole
// tiles) and its tile list, weights of every buffer row cleared (k_tab_fill
// sets the used ones).
__global__ void __launch_bounds__(1024) k_tab_plan(Dev s, TabBuf q, double* obj_out) {
  KKM_GRID_DEP_WAIT();
  __shared__ int cnt[1024], coff[1024];
  __shared__ int16_t sassign[8192];
  __shared__ float wpartial[32];
  const int k = s.k, b = s.b, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < k) cnt[tid] = 0;
  float macc = 0.0f;
  for (int x = tid; x < b; x += 1024) {
    macc += s.mind[x];
    sassign[x] = (int16_t)s.assign[x];
  }
  __syncthreads();
  for (int x = tid; x < b; x += 1024) atomicAdd(&cnt[sassign[x]], 1);
  __syncthreads();
  const int my = tid < k ? cnt[tid] : 0;
  int total = 0;
  const int off = block_exclusive_scan_1024(my, &total);
  if (tid < k) { coff[tid] = off; s.coff[tid] = off; s.counts[tid] = my; }
  if (tid == 0) s.coff[k] = total;
  __syncthreads();
  // stable order: row x goes to coff[a] + (rows before x with the same center);
  // one warp per center walks the batch in order (b is small)
  for (int j = warp; j < k; j += 32) {
    int base = coff[j];
    for (int x0 = 0; x0 < b; x0 += 32) {
      const int x = x0 + lane;
      const bool mine = x < b && sassign[x] == j;
      const unsigned m = __ballot_sync(0xffffffffu, mine);
      if (mine) s.perm[base + __popc(m & ((1u << lane) - 1u))] = x;
      base += __popc(m);
    }
    // <C_j, cm(B_j)>: FP32 lane sums of the assigned rows' table entries, FP64 combine
    float part = 0.0f;
    for (int r = coff[j] + lane; r < coff[j] + cnt[j]; r += 32) part += s.inner_a[s.perm[r]];
    const double sum = warp_sum((double)part);
    if (lane == 0) s.cmc[j] = cnt[j] > 0 ? sum / (double)cnt[j] : 0.0;
  }
  // f_B(C_i)
  float v = macc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) wpartial[warp] = v;
  // support-buffer layout and tiles: every center's block is padded to whole
  // tiles, so a tile never reaches the next center's rows (the padding rows
  // carry weight 0)
  const int rowsT = tid < k ? (my + s.tn - 1) / s.tn * s.tn : 0;
  int used = 0;
  const int bo = block_exclusive_scan_1024(rowsT, &used);
  const int nt = tid < k ? (my + s.tn - 1) / s.tn : 0;
  int ntot = 0;
  const int tf = block_exclusive_scan_1024(nt, &ntot);
  if (tid < k) {
    q.bs_off[tid] = bo;
    s.tile_first[tid] = tf;
    s.tile_cnt[tid] = nt;
    for (int t = 0; t < nt; ++t)
      s.tiles[tf + t] = Tile{tid, (int32_t)((int64_t)bo + t * s.tn), min(s.tn, my - t * s.tn), 0};
  }
  if (tid == 0) {
    q.bs_off[k] = used;
    *s.ntiles = ntot;
  }
  for (int r = tid; r < q.bs_rows; r += 1024) {
    s.w32[r] = 0.0f;
    s.w64[r] = 0.0;
  }
  __syncthreads();
  if (warp == 0) {
    const double t = warp_sum((double)wpartial[lane]);
    if (lane == 0) {
      const double f = t * s.inv_b;
      *s.obj = f;
      if (obj_out) *obj_out = f;
      s.stats[0] += 1;
      *s.iter += 1;
    }
  }
}

// The batch rows into the support buffer, center by center (a warp per row),
// with weight 1/b_j.
__global__ void k_tab_fill(Dev s, TabBuf q) {
  KKM_GRID_DEP_WAIT();
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= s.b) return;
  const int x = s.perm[p];
  const int j = s.assign[x];
  const int dst = q.bs_off[j] + (p - s.coff[j]);
  warp_copy_row(s, false, x, dst);
  if ((threadIdx.x & 31) == 0) {
    const double w = 1.0 / (double)s.counts[j];
    s.yn[dst] = s.xbn[x];
    s.yi[dst] = s.xbi[x];
    s.w64[dst] = w;
    s.w32[dst] = (float)w;
  }
}

// Per center with points: ||cm(B_j)||^2 from S at the batch rows, the rate,
// and the FP64 norm recurrence (block of 256 per center).
__global__ void __launch_bounds__(256) k_tab_center(Dev s, TabBuf q) {
  KKM_GRID_DEP_WAIT();
  __shared__ double red[8];
  const int j = blockIdx.x, tid = threadIdx.x;
  const int n = s.counts[j];
  if (n == 0) {
    if (tid == 0) s.alpha[j] = 0.0;
    return;
  }
  const int t0 = s.tile_first[j] * s.ppt, nt = s.tile_cnt[j] * s.ppt;   // ppt partials per tile
  float acc = 0.0f;
  for (int p = s.coff[j] + tid; p < s.coff[j] + n; p += 256) {
    const int64_t i = s.xbi[s.perm[p]];
    float sv = 0.0f;
    for (int t = 0; t < nt; ++t) sv += q.part[(int64_t)(t0 + t) * q.npad + i];
    acc += sv;
  }
  const double w = warp_sum((double)acc);
  if ((tid & 31) == 0) red[tid >> 5] = w;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0.0;
    for (int v = 0; v < 8; ++v) m2 += red[v];
    const double dn = (double)n;
    m2 /= dn;
    const double N = s.ncum[j] + dn;
    s.ncum[j] = N;
    double a;
    if (s.lr == 0) a = sqrt(dn * s.inv_b);
    else if (s.lr == 2) a = dn / N;
    else a = s.eta;
    const double keep = 1.0 - a;
    const double cn = keep * keep * s.cnorm[j] + 2.0 * a * keep * s.cmc[j] + a * a * m2;
    s.alpha[j] = a;
    s.cnorm[j] = cn;
    s.cnorm32[j] = (float)cn;
  }
}

// T[j][x] <- (1 - alpha_j) T[j][x] + alpha_j S[j][x] for the centers with
// points (grid: x in blocks of 1024, y = center). init: T = S for every center.
__global__ void __launch_bounds__(256) k_tab_update(Dev s, TabBuf q, int init) {
  KKM_GRID_DEP_WAIT();
  const int j = blockIdx.y;
  if (!init && s.counts[j] == 0) return;
  const double a = init ? 1.0 : s.alpha[j];
  const float af = (float)a, kf = (float)(1.0 - a);
  const int t0 = s.tile_first[j] * s.ppt, nt = s.tile_cnt[j] * s.ppt;   // ppt partials per tile
  float* T = q.T + (int64_t)j * s.n;
#pragma unroll 4
  for (int64_t x = (int64_t)blockIdx.x * 1024 + threadIdx.x; x < min((int64_t)(blockIdx.x + 1) * 1024, s.n);
       x += 256) {
    float sv = 0.0f;
    for (int t = 0; t < nt; ++t) sv += q.part[(int64_t)(t0 + t) * q.npad + x];
    T[x] = init ? sv : fmaf(kf, T[x], af * sv);
  }
}

// The initial centers C_1^j = phi(x_init_j) as the support buffer (row j*tn,
// weight 1, one tile each), and ||C_1^j||^2 = K(x, x).
__global__ void k_tab_init_rows(Dev s, TabBuf q, const int32_t* __restrict__ init_idx) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= s.k) return;
  const int lane = threadIdx.x & 31;
  int64_t i = init_idx[j];
  if (i < 0 || i >= s.n) {
    if (lane == 0) atomicOr(s.status, ST_BAD_BATCH_INDEX);
    i = 0;
  }
  const int64_t row = (int64_t)j * s.tn;
  const float* src = s.X + i * s.ldx;
  const double nrm = warp_store_row(s, src, row, true);
  double exact = 0.0;
  for (int c = lane; c < s.d; c += 32) exact += (double)src[c] * (double)src[c];
  exact = warp_sum(exact);
  if (lane == 0) {
    s.yn[row] = (float)nrm;
    s.yi[row] = (int32_t)i;
    s.w64[row] = 1.0;
    s.w32[row] = 1.0f;
    s.tiles[j] = Tile{j, (int32_t)row, 1, 0};
    s.tile_first[j] = j;
    s.tile_cnt[j] = 1;
    s.cnorm[j] = kernel_self(s.kind, exact, s.coef0, s.degree);
    s.cnorm32[j] = (float)s.cnorm[j];
    if (j == 0) *s.ntiles = s.k;
  }
}

// Every row of X into the run's operand form (the Gram view's A rows), with
// its norm and its own index (a warp per row).
__global__ void k_tab_convert(Dev g) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= g.n) return;
  const double nrm = warp_store_row(g, g.X + r * g.ldx, r, false);
  if ((threadIdx.x & 31) == 0) {
    g.xbn[r] = (float)nrm;
    g.xbi[r] = (int32_t)r;
  }
}

// f_X = (1/n) sum_x min_j Delta(x, C_j) from the table: FP32 per row, FP64 block sums.
__global__ void __launch_bounds__(256) k_tab_objective(Dev s, TabBuf q, const float* __restrict__ xn,
                                                       double* __restrict__ blk) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int64_t x = (int64_t)blockIdx.x * 256 + threadIdx.x; x < s.n; x += (int64_t)gridDim.x * 256) {
    const float kxx = (float)kernel_self(s.kind, (double)xn[x], s.coef0, s.degree);
    float best = 3.0e38f;
    for (int j = 0; j < s.k; ++j)
      best = fminf(best, fmaf(-2.0f, q.T[(int64_t)j * s.n + x], kxx + s.cnorm32[j]));
    acc += (double)best;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int v = 0; v < 8; ++v) t += red[v];
    blk[blockIdx.x] = t;
  }
}

// ------------------------------------------------------------------------
// Run groups: one launch per step phase for every run of a group. Block b of
// such a launch belongs to the run r with first[r] <= b < first[r + 1] and
// plays block b - first[r] of that run's own launch (the same block count as
// a single-run launch, or any count for the grid-stride phases), so every run
// computes exactly what its own launches would.
__device__ __forceinline__ int group_run(const GroupPhase& g, int& local, int& nblk) {
  const int r = last_le(g.first, g.nruns, (int)blockIdx.x);
  local = (int)blockIdx.x - g.first[r];
  nblk = g.first[r + 1] - g.first[r];
  return r;
}

__global__ void k_group_gather(GroupPhase g) {
  int local, nblk;
  const int r = group_run(g, local, nblk);
  gather_body(g.runs[r].s, nullptr, 0, local);
}

__global__ void __launch_bounds__(32 * AM_WARPS) k_group_argmin(GroupPhase g) {
  int local, nblk;
  const int r = group_run(g, local, nblk);
  const Dev& s = g.runs[r].s;
  argmin_body(s, s.b, nullptr, nullptr, nullptr, nullptr, 1, local);
}

__global__ void __launch_bounds__(1024) k_group_sort_plan(GroupPhase g) {
  int local, nblk;
  const int r = group_run(g, local, nblk);
  sort_plan_body(g.runs[r].s, nullptr, 0);
}

__global__ void k_group_move(GroupPhase g) {
  int local, nblk;
  const int r = group_run(g, local, nblk);
  move_body(g.runs[r].s, local, nblk);
}

__global__ void __launch_bounds__(256) k_group_finalize(GroupPhase g) {
  int local, nblk;
  const int r = group_run(g, local, nblk);
  finalize_body(g.runs[r].s, 0, local);
}

// ------------------------------------------------------------------------
// Full-batch kernel k-means (kernel Lloyd), the baseline of Sec. 6. Every
// iteration assigns all n points to their nearest center, then every center
// with points becomes the mean of its points in feature space,
// C_j = (1/n_j) sum_{x in X_j} phi(x). With T[j][x] = <phi(x), C_j>,
//   Delta(x, C_j) = K(x, x) - 2 T[j][x] + ||C_j||^2,
//   ||C_j||^2 = (1/n_j) sum_{x in X_j} T[j][x],
// and T is the n x n Gram pass of X against X sorted by center, weights
// 1/n_j. A center that gets no points keeps its row of T and its norm.

// Ranking of the counting sort: one warp per chunk of LLOYD_RANK_ROWS rows,
// 32 rows at a time in row order, so a row's rank among its chunk's rows of
// the same center follows row order (the sort is stable).
__global__ void __launch_bounds__(32) k_lloyd_rank(Dev g, LloydBuf L) {
  __shared__ int cnt[1024];
  const int lane = threadIdx.x, c = blockIdx.x;
  for (int j = lane; j < g.k; j += 32) cnt[j] = 0;
  __syncwarp();
  const int64_t base = (int64_t)c * LLOYD_RANK_ROWS;
  for (int p = 0; p < LLOYD_RANK_ROWS; p += 32) {
    const int64_t x = base + p + lane;
    const int a = x < g.n ? (int)min((unsigned)L.assign[x], (unsigned)(g.k - 1)) : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, a);
    const int start = a >= 0 ? cnt[a] : 0;
    __syncwarp();
    if (a >= 0) {
      L.rank[x] = start + __popc(grp & ((1u << lane) - 1u));
      if (lane == __ffs(grp) - 1) cnt[a] = start + __popc(grp);
    }
    __syncwarp();
  }
  for (int j = lane; j < g.k; j += 32) L.ccnt[(int64_t)c * g.k + j] = cnt[j];
}

// Single CTA: per center, the position of every ranking chunk's first row
// (cbase) and n_j; the center offsets of the sorted order; the support-buffer
// layout (center j in whole tiles from its first tile's row) and its tile
// list; weight 0 on the rows that pad a center's last tile.
__global__ void __launch_bounds__(1024) k_lloyd_plan(Dev g, LloydBuf L) {
  const int k = g.k, tid = threadIdx.x;
  int my = 0;
  if (tid < k) {
    for (int c = 0; c < L.nrk; ++c) {
      const int64_t e = (int64_t)c * k + tid;
      const int v = L.ccnt[e];
      L.cbase[e] = my;
      my += v;
    }
  }
  int total = 0;
  const int off = block_exclusive_scan_1024(my, &total);
  const int nt = tid < k ? (my + g.tn - 1) / g.tn : 0;
  int ntot = 0;
  const int tf = block_exclusive_scan_1024(nt, &ntot);
  const int bo = tf * g.tn;
  if (tid < k) {
    g.counts[tid] = my;
    g.coff[tid] = off;
    L.bs_off[tid] = bo;
    g.tile_first[tid] = tf;
    g.tile_cnt[tid] = nt;
    for (int t = 0; t < nt; ++t) g.tiles[tf + t] = Tile{tid, bo + t * g.tn, min(g.tn, my - t * g.tn), 0};
    for (int r = bo + my; r < bo + nt * g.tn; ++r) {
      g.w64[r] = 0.0;
      g.w32[r] = 0.0f;
    }
  }
  if (tid == 0) {
    g.coff[k] = total;
    L.bs_off[k] = ntot * g.tn;
    *g.ntiles = ntot;
  }
}

// Every row of X (the Gram view's operand row) into its place in the support
// buffer, with weight 1/n_j, and its index into the center-sorted order (a
// warp per row).
__global__ void k_lloyd_scatter(Dev g, LloydBuf L) {
  const int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (x >= g.n) return;
  const int a = L.assign[x];
  const int pos = L.cbase[(x / LLOYD_RANK_ROWS) * g.k + a] + L.rank[x];
  const int64_t dst = (int64_t)L.bs_off[a] + pos;
  warp_copy_row(g, false, x, dst);
  if ((threadIdx.x & 31) == 0) {
    const double w = 1.0 / (double)g.counts[a];
    g.yn[dst] = g.xbn[x];
    g.yi[dst] = (int32_t)x;
    g.w64[dst] = w;
    g.w32[dst] = (float)w;
    g.perm[g.coff[a] + pos] = (int32_t)x;
  }
}

// T[j][row0 + x] = the sum of center j's tile partials of the chunk's row x
// (grid: x in blocks of 1024, y = center).
__global__ void __launch_bounds__(256) k_lloyd_reduce(Dev gc, LloydBuf L, int64_t row0, int rows, int all) {
  const int j = blockIdx.y;
  if (!all && gc.counts[j] == 0) return;
  const int t0 = gc.tile_first[j] * gc.ppt, nt = gc.tile_cnt[j] * gc.ppt;   // ppt partials per tile
  float* T = L.T + (int64_t)j * gc.n + row0;
  const int end = min((int)(blockIdx.x + 1) * 1024, rows);
  for (int x = blockIdx.x * 1024 + threadIdx.x; x < end; x += 256) {
    float sv = 0.0f;
    for (int t = 0; t < nt; ++t) sv += gc.part[(int64_t)(t0 + t) * gc.bpad + x];
    T[x] = sv;
  }
}

// ||C_j||^2 = (1/n_j) sum_{x in X_j} T[j][x]: FP32 thread sums, FP64 combine
// (a block of 256 per center with points).
__global__ void __launch_bounds__(256) k_lloyd_cnorm(Dev g, LloydBuf L) {
  __shared__ double red[8];
  const int j = blockIdx.x, tid = threadIdx.x;
  const int nj = g.counts[j];
  if (nj == 0) return;
  const float* T = L.T + (int64_t)j * g.n;
  float acc = 0.0f;
  for (int p = g.coff[j] + tid; p < g.coff[j] + nj; p += 256) acc += T[g.perm[p]];
  const double w = warp_sum((double)acc);
  if ((tid & 31) == 0) red[tid >> 5] = w;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0.0;
    for (int v = 0; v < 8; ++v) m2 += red[v];
    m2 /= (double)nj;
    g.cnorm[j] = m2;
    g.cnorm32[j] = (float)m2;
  }
}

// The nearest center of every row (ties to the lowest j), FP32 distances as
// in the table form, and per block the FP64 sum of the minima and the count
// of rows whose assignment changed.
__global__ void __launch_bounds__(256) k_lloyd_assign(Dev g, LloydBuf L, int first) {
  __shared__ double red[8];
  __shared__ int redc[8];
  double acc = 0.0;
  int ch = 0;
  for (int64_t x = (int64_t)blockIdx.x * 256 + threadIdx.x; x < g.n; x += (int64_t)gridDim.x * 256) {
    const float kxx = (float)kernel_self(g.kind, (double)g.xbn[x], g.coef0, g.degree);
    float best = 3.0e38f;
    int bj = 0;
    for (int j = 0; j < g.k; ++j) {
      const float dist = fmaf(-2.0f, L.T[(int64_t)j * g.n + x], kxx + g.cnorm32[j]);
      if (dist < best) {
        best = dist;
        bj = j;
      }
    }
    if (first || L.assign[x] != bj) ++ch;
    L.assign[x] = bj;
    L.mind[x] = best;
    acc += (double)best;
  }
  acc = warp_sum(acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ch += __shfl_xor_sync(0xffffffffu, ch, o);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = acc;
    redc[threadIdx.x >> 5] = ch;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    int c = 0;
    for (int v = 0; v < 8; ++v) {
      t += red[v];
      c += redc[v];
    }
    L.blk[blockIdx.x] = t;
    L.blk_changed[blockIdx.x] = c;
  }
}

// f_X and the changed count from the block partials, in a fixed order.
__global__ void __launch_bounds__(256) k_lloyd_total(LloydBuf L, double inv_n) {
  __shared__ double red[256];
  __shared__ long long redc[256];
  const int tid = threadIdx.x;
  double t = 0.0;
  long long c = 0;
  for (int i = tid; i < L.nblk; i += 256) {
    t += L.blk[i];
    c += L.blk_changed[i];
  }
  red[tid] = t;
  redc[tid] = c;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) {
      red[tid] += red[tid + w];
      redc[tid] += redc[tid + w];
    }
    __syncthreads();
  }
  if (tid == 0) {
    *L.obj = red[0] * inv_n;
    *L.changed = redc[0];
  }
}

// Delta(x, C_j) for every row and center, the assignment pass's arithmetic.
__global__ void __launch_bounds__(256) k_lloyd_dist(Dev g, LloydBuf L, float* __restrict__ out) {
  const int64_t x = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (x >= g.n) return;
  const float kxx = (float)kernel_self(g.kind, (double)g.xbn[x], g.coef0, g.degree);
  for (int j = 0; j < g.k; ++j) out[x * g.k + j] = fmaf(-2.0f, L.T[(int64_t)j * g.n + x], kxx + g.cnorm32[j]);
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_sample(const Dev& s, cudaStream_t st) {
  k_sample<<<(s.b + 255) / 256, 256, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t launch_gather_batch(const Dev& s, const int32_t* idx, cudaStream_t st, bool rotated) {
  cudaError_t e = launch_pdl(k_gather_batch, dim3((s.b * 32 + 255) / 256), dim3(256), 0, st, s, idx, rotated ? 1 : 0);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_gather_query(const Dev& s, const float* Q, int64_t ldq, int rows, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  cudaError_t e = launch_pdl(k_gather_query, dim3((rows * 32 + 255) / 256), dim3(256), 0, st, s, Q, ldq, rows);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_argmin(const Dev& s, int rows, const int32_t* forced, int32_t* assign_out,
                          float* mind_out, float* dist_out, bool update, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  cudaError_t e = launch_pdl(k_argmin, dim3((rows + 31) / 32), dim3(32 * AM_WARPS), 0, st, s, rows, forced,
                             assign_out, mind_out, dist_out, update ? 1 : 0);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

int sort_plan_smem(int k, int b) { return k * (int)sizeof(Plan) + 4 * k * 4 + b * (4 + 2 + 2 + 2) + 32 * k * 2; }

cudaError_t launch_sort_plan(const Dev& s, double* obj_out, cudaStream_t st, bool set_pending) {
  const int smem = sort_plan_smem(s.k, s.b);
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = smem_limit_once(k_sort_plan, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  e = launch_pdl(k_sort_plan, dim3(1), dim3(1024), smem, st, s, obj_out, set_pending ? 1 : 0);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_move(const Dev& s, cudaStream_t st) {
  const int warps = 8;
  const int blocks = std::max((s.b + warps - 1) / warps, s.num_sms * 2);
  cudaError_t e = launch_pdl(k_move, dim3(blocks), dim3(warps * 32), 0, st, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Dev& s, cudaStream_t st, bool if_pending) {
  cudaError_t e = launch_pdl(k_finalize, dim3(s.k), dim3(256), 0, st, s, if_pending ? 1 : 0);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_build_tiles(const Dev& s, cudaStream_t st) {
  k_build_tiles<<<1, 1024, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t launch_init_centers(const Dev& s, const int32_t* init_idx, cudaStream_t st) {
  k_init_centers<<<(s.k * 32 + 255) / 256, 256, 0, st>>>(s, init_idx);
  return cudaGetLastError();
}

cudaError_t launch_load_rows(const Dev& s, int32_t, cudaStream_t st) {
  k_load_rows<<<s.k, 256, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t launch_mind_sum(const Dev& s, int rows, double scale, double* out, cudaStream_t st) {
  cudaError_t e = launch_pdl(k_mind_sum, dim3(1), dim3(1024), 0, st, s, rows, scale, out);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}


// ------------------------------------------------------------- table form
cudaError_t launch_tab_batch_dist(const Dev& s, const TabBuf& q, int rows, const int32_t* forced,
                                  int32_t* assign_out, float* mind_out, float* dist_out, bool update,
                                  cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  cudaError_t e = launch_pdl(k_tab_batch_dist, dim3((rows * 32 + 255) / 256), dim3(256), 0, st, s, q, rows, forced,
                             assign_out, mind_out, dist_out, update ? 1 : 0);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_tab_plan(const Dev& s, const TabBuf& q, double* obj_out, cudaStream_t st) {
  cudaError_t e = launch_pdl(k_tab_plan, dim3(1), dim3(1024), 0, st, s, q, obj_out);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_tab_fill(const Dev& s, const TabBuf& q, cudaStream_t st) {
  cudaError_t e = launch_pdl(k_tab_fill, dim3((s.b * 32 + 255) / 256), dim3(256), 0, st, s, q);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_tab_center(const Dev& s, const TabBuf& q, cudaStream_t st) {
  cudaError_t e = launch_pdl(k_tab_center, dim3(s.k), dim3(256), 0, st, s, q);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_tab_update(const Dev& s, const TabBuf& q, bool init, cudaStream_t st) {
  const dim3 grid((unsigned)((s.n + 1023) / 1024), (unsigned)s.k);
  cudaError_t e = launch_pdl(k_tab_update, grid, dim3(256), 0, st, s, q, init ? 1 : 0);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_tab_init(const Dev& s, const Dev& g, const TabBuf& q, const int32_t* init_idx, cudaStream_t st) {
  k_tab_convert<<<(unsigned)((g.n * 32 + 255) / 256), 256, 0, st>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_tab_init_rows<<<(s.k * 32 + 255) / 256, 256, 0, st>>>(s, q, init_idx);
  return cudaGetLastError();
}

cudaError_t launch_tab_objective(const Dev& s, const TabBuf& q, const float* xn, double* blk, int nblk,
                                 cudaStream_t st) {
  k_tab_objective<<<nblk, 256, 0, st>>>(s, q, xn, blk);
  return cudaGetLastError();
}

// --------------------------------------------------------- kernel Lloyd
cudaError_t launch_lloyd_sort(const Dev& g, const LloydBuf& L, cudaStream_t st) {
  k_lloyd_rank<<<L.nrk, 32, 0, st>>>(g, L);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_lloyd_plan<<<1, 1024, 0, st>>>(g, L);
  return cudaGetLastError();
}

cudaError_t launch_lloyd_scatter(const Dev& g, const LloydBuf& L, cudaStream_t st) {
  k_lloyd_scatter<<<(unsigned)((g.n * 32 + 255) / 256), 256, 0, st>>>(g, L);
  return cudaGetLastError();
}

cudaError_t launch_lloyd_reduce(const Dev& gc, const LloydBuf& L, int64_t row0, int rows, bool all,
                                cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  k_lloyd_reduce<<<dim3((unsigned)((rows + 1023) / 1024), (unsigned)gc.k), 256, 0, st>>>(gc, L, row0, rows,
                                                                                        all ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_lloyd_cnorm(const Dev& g, const LloydBuf& L, cudaStream_t st) {
  k_lloyd_cnorm<<<g.k, 256, 0, st>>>(g, L);
  return cudaGetLastError();
}

cudaError_t launch_lloyd_assign(const Dev& g, const LloydBuf& L, bool first, cudaStream_t st) {
  k_lloyd_assign<<<L.nblk, 256, 0, st>>>(g, L, first ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_lloyd_total<<<1, 256, 0, st>>>(L, 1.0 / (double)g.n);
  return cudaGetLastError();
}

cudaError_t launch_lloyd_dist(const Dev& g, const LloydBuf& L, float* out, cudaStream_t st) {
  k_lloyd_dist<<<(unsigned)((g.n + 255) / 256), 256, 0, st>>>(g, L, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------- run groups
cudaError_t launch_group_gather(const GroupPhase& g, int blocks, cudaStream_t st) {
  return launch_pdl(k_group_gather, dim3(blocks), dim3(256), 0, st, g);
}

cudaError_t launch_group_argmin(const GroupPhase& g, int blocks, cudaStream_t st) {
  return launch_pdl(k_group_argmin, dim3(blocks), dim3(32 * AM_WARPS), 0, st, g);
}

cudaError_t launch_group_sort_plan(const GroupPhase& g, int smem, cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = smem_limit_once(k_group_sort_plan, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_group_sort_plan, dim3(g.nruns), dim3(1024), smem, st, g);
}

cudaError_t launch_group_move(const GroupPhase& g, int blocks, cudaStream_t st) {
  return launch_pdl(k_group_move, dim3(blocks), dim3(256), 0, st, g);
}

cudaError_t launch_group_finalize(const GroupPhase& g, int blocks, cudaStream_t st) {
  return launch_pdl(k_group_finalize, dim3(blocks), dim3(256), 0, st, g);
}

}  // namespace kkm
