// Step kernels of truncated mini-batch kernel k-means (Algorithm 2, Appendix A):
// batch sampling, batch gather, argmin assignment, the stable counting sort and
// window plan, row moves, and the finalise step that carries ||C||^2 by the
// Sec. 4 recurrence (FP64) corrected for the rows Eq. (1) drops.
// The distance kernels themselves are in kkm_gram_simt.cu and kkm_gram_tc.cu.
#include "kkm_internal.cuh"

namespace kkm {

namespace {

constexpr int kWarp = 32;

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

// Writes one FP32 source row into a batch/support row of the run's form and
// returns ||row||^2 of the values the Gram product will use (FP64 sum).
// Called by a whole warp; columns are strided over lanes.
__device__ double warp_store_row(const Dev& s, const float* src, int64_t dst_row, bool to_support) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  if (s.form == FORM_FP32) {
    float* dst = (to_support ? s.y32 : s.xb32) + dst_row * s.ld;
    for (int c = lane; c < s.d; c += kWarp) {
      float v = src[c];
      dst[c] = v;
      acc += (double)v * (double)v;
    }
  } else {
    __nv_bfloat16* dst = (to_support ? s.ybh : s.xbh) + dst_row * s.ld;
    for (int c = lane; c < s.d; c += kWarp) {
      float v = src[c];
      __nv_bfloat16 hi = __float2bfloat16_rn(v);
      float hf = __bfloat162float(hi);
      __nv_bfloat16 lo = __float2bfloat16_rn(v - hf);
      dst[c] = hi;
      dst[s.dp + c] = lo;
      double used = (s.form == FORM_BF16) ? (double)hf : (double)hf + (double)__bfloat162float(lo);
      acc += used * used;
    }
  }
  return warp_sum(acc);
}

// Copies a whole row (ld elements) between two rows of the run's row buffers.
__device__ void warp_copy_row(const Dev& s, bool src_support, int64_t src_row, int64_t dst_row) {
  const int lane = threadIdx.x & 31;
  const int elem = (s.form == FORM_FP32) ? 4 : 2;
  const int n16 = s.ld * elem / 16;
  const char* src = (const char*)(src_support ? (s.form == FORM_FP32 ? (void*)s.y32 : (void*)s.ybh)
                                              : (s.form == FORM_FP32 ? (void*)s.xb32 : (void*)s.xbh));
  char* dst = (char*)(s.form == FORM_FP32 ? (void*)s.y32 : (void*)s.ybh);
  const int4* sp = (const int4*)(src + src_row * (int64_t)s.ld * elem);
  int4* dp = (int4*)(dst + dst_row * (int64_t)s.ld * elem);
  for (int c = lane; c < n16; c += kWarp) dp[c] = sp[c];
}

// ------------------------------------------------------------------ kernels
__global__ void k_sample(Dev s) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.b) return;
  const int64_t it = *s.iter;
  const uint64_t c = (uint64_t)(it - 1) * (uint64_t)s.b + (uint64_t)t;
  s.bidx[t] = (int32_t)index_below(splitmix64(s.seed, c), (uint64_t)s.n);
}

// One warp per batch slot: X[idx] -> batch row, norm, data index.
__global__ void k_gather_batch(Dev s, const int32_t* __restrict__ idx) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= s.b) return;
  int64_t i = idx[warp];
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

// One warp per query row: Q[r] -> batch row (no data index: K(x,x) is never forced).
__global__ void k_gather_query(Dev s, const float* __restrict__ Q, int64_t ldq, int rows) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= rows) return;
  double nrm = warp_store_row(s, Q + (int64_t)warp * ldq, warp, false);
  if ((threadIdx.x & 31) == 0) {
    s.xbn[warp] = (float)nrm;
    s.xbi[warp] = -1;
  }
}

// One thread per batch row: sum the per-tile weighted kernel sums of each
// center, form Delta(x, C_j) = K(x,x) - 2 <phi(x), C_j> + ||C_j||^2 (FP64
// combine), and take the argmin (strict <, so ties go to the lowest j).
__global__ void k_argmin(Dev s, int rows, const int32_t* __restrict__ forced,
                         int32_t* __restrict__ assign_out, float* __restrict__ mind_out,
                         float* __restrict__ dist_out, int update) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= rows) return;
  const double kxx = kernel_self(s.kind, (double)s.xbn[x], s.coef0, s.degree);
  double best = 1e300, best_inner = 0.0;
  int bj = 0;
  for (int j = 0; j < s.k; ++j) {
    const int t0 = s.tile_first[j], nt = s.tile_cnt[j];
    double inner = 0.0;
    for (int t = 0; t < nt; ++t) inner += (double)s.part[(int64_t)(t0 + t) * s.bpad + x];
    const double dist = kxx - 2.0 * inner + s.cnorm[j];
    if (dist_out) dist_out[(int64_t)x * s.k + j] = (float)dist;
    if (dist < best) { best = dist; bj = j; best_inner = inner; }
  }
  int a = bj;
  double a_inner = best_inner;
  if (forced) {
    a = forced[x];
    if (a < 0 || a >= s.k) {
      atomicOr(s.status, ST_BAD_ASSIGN);
      a = bj;
    } else if (a != bj) {
      const int t0 = s.tile_first[a], nt = s.tile_cnt[a];
      a_inner = 0.0;
      for (int t = 0; t < nt; ++t) a_inner += (double)s.part[(int64_t)(t0 + t) * s.bpad + x];
    }
  }
  if (assign_out) assign_out[x] = bj;
  if (mind_out) mind_out[x] = (float)best;
  if (update) {
    s.assign[x] = a;
    s.mind[x] = (float)best;
    s.inner_a[x] = (float)a_inner;
  }
}

// Single CTA of 1024 threads. Stable counting sort of the batch by center,
// alpha_i^j, <C_j, cm(B_j)>, and the per-center window plan: compaction,
// block push, the drops of Eq. (1), C_1 retirement, and the tile pairs of the
// norm-recurrence Gram pass.
__global__ void __launch_bounds__(1024) k_sort_plan(Dev s, int pair_tile) {
  extern __shared__ unsigned char smem[];
  const int k = s.k, b = s.b, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t* cnt = (int32_t*)smem;      // [k]
  int32_t* base = cnt + k;            // [k]
  int32_t* tot = base + k;            // [k]
  uint16_t* wtab = (uint16_t*)(tot + k);   // [32][k]
  for (int j = tid; j < k; j += 1024) { cnt[j] = 0; base[j] = 0; }
  __syncthreads();
  for (int x = tid; x < b; x += 1024) atomicAdd(&cnt[s.assign[x]], 1);
  __syncthreads();
  // exclusive offsets over centers (k <= 1024: one center per thread)
  const int my = tid < k ? cnt[tid] : 0;
  int total_rows = 0;
  const int off = block_exclusive_scan_1024(my, &total_rows);
  if (tid < k) { s.coff[tid] = off; s.counts[tid] = my; }
  if (tid == 0) s.coff[k] = total_rows;
  __syncthreads();
  // stable ranks in chunks of 1024 rows
  for (int c0 = 0; c0 < b; c0 += 1024) {
    for (int e = tid; e < 32 * k; e += 1024) wtab[e] = 0;
    __syncthreads();
    const int x = c0 + tid;
    const int j = x < b ? s.assign[x] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, j);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (j >= 0 && rank == 0) wtab[warp * k + j] = (uint16_t)__popc(peers);
    __syncthreads();
    for (int jj = tid; jj < k; jj += 1024) {
      int run = 0;
      for (int w = 0; w < 32; ++w) {
        const int v = wtab[w * k + jj];
        wtab[w * k + jj] = (uint16_t)run;
        run += v;
      }
      tot[jj] = run;
    }
    __syncthreads();
    if (j >= 0) s.perm[s.coff[j] + base[j] + wtab[warp * k + j] + rank] = x;
    __syncthreads();
    for (int jj = tid; jj < k; jj += 1024) base[jj] += tot[jj];
    __syncthreads();
  }
  // learning rate and <C_j, cm(B_j)> = (1/b_j) sum_{x in B_j} <phi(x), C_j>
  for (int j = warp; j < k; j += 32) {
    const int n = cnt[j], o = s.coff[j];
    double acc = 0.0;
    for (int r = lane; r < n; r += 32) acc += (double)s.inner_a[s.perm[o + r]];
    acc = warp_sum(acc);
    if (lane == 0) {
      double a = 0.0;
      if (n > 0) a = (s.lr == 0) ? sqrt((double)n / (double)b) : s.eta;
      s.alpha[j] = a;
      s.cmc[j] = n > 0 ? acc / (double)n : 0.0;
    }
  }
  // support rows read by this step's distance pass
  int sz = tid < k ? s.tail[tid] - s.head[tid] : 0;
  int s_total = 0;
  block_exclusive_scan_1024(sz, &s_total);
  if (tid == 0) *s.s_old = s_total;
  // window plan, one thread per center
  int npairs = 0;
  if (tid < k) {
    const int j = tid;
    const int n = cnt[j];
    Plan P;
    P.head_c = s.head[j];
    P.tail_c = s.tail[j];
    P.head_new = P.head_c;
    P.tail_new = P.tail_c;
    P.src_head = -1;
    P.cnt = n;
    P.ndrop = 0;
    P.c1_new = s.c1[j];
    if (n > 0) {
      if (P.tail_c + n > s.cap) {       // compaction: move the window down to row 0
        P.src_head = P.head_c;
        P.tail_c = P.tail_c - P.head_c;
        P.head_c = 0;
      }
      P.tail_new = P.tail_c + n;
      if (P.tail_new > s.cap) atomicOr(s.status, ST_CAPACITY);
      int first = s.blk_first[j], nb = s.blk_num[j];
      int32_t* bi = s.blk_iter + (int64_t)j * s.nbcap;
      int32_t* bc = s.blk_cnt + (int64_t)j * s.nbcap;
      if (nb >= s.nbcap) {
        atomicOr(s.status, ST_CAPACITY);
      } else {
        const int slot = (first + nb) % s.nbcap;
        bi[slot] = (int32_t)(*s.iter);
        bc[slot] = n;
        ++nb;
      }
      int total = s.wsum[j] + n;
      int drop_rows = 0;
      if (s.tau > 0) {
        // Q_i^j keeps the newest blocks whose counts reach tau: drop the
        // oldest block while the rest still sums to >= tau.
        while (nb > 1 && total - bc[first] >= s.tau) {
          drop_rows += bc[first];
          total -= bc[first];
          first = (first + 1) % s.nbcap;
          --nb;
        }
        // C_1 stays only while min Q_i^j = 1 (Eq. (1), Sec. 4.1).
        if (P.c1_new && total >= s.tau && bi[first] != 1) {
          P.c1_new = 0;
          P.ndrop += 1;
        }
      }
      P.ndrop += drop_rows;
      P.head_new = P.head_c + P.ndrop;
      s.blk_first[j] = first;
      s.blk_num[j] = nb;
      s.wsum[j] = total;
      const int T = pair_tile;
      const int nD = P.ndrop, nL = P.tail_new - P.head_c;
      npairs = ((nD + T - 1) / T) * ((nL + T - 1) / T) + ((n + T - 1) / T) * ((n + T - 1) / T);
    }
    s.plan[j] = P;
  }
  __syncthreads();
  int ptotal = 0;
  const int pfirst = block_exclusive_scan_1024(npairs, &ptotal);
  if (tid == 0) {
    *s.nwpairs = ptotal <= s.max_pairs ? ptotal : s.max_pairs;
    if (ptotal > s.max_pairs) atomicOr(s.status, ST_CAPACITY);
  }
  if (tid < k) {
    s.wpair_first[tid] = pfirst;
    s.wpair_cnt[tid] = npairs;
    if (npairs > 0 && pfirst + npairs <= s.max_pairs) {
      const Plan P = s.plan[tid];
      const int T = pair_tile;
      const int nD = P.ndrop, nL = P.tail_new - P.head_c, n = P.cnt;
      const int rD = (nD + T - 1) / T, cL = (nL + T - 1) / T, tB = (n + T - 1) / T;
      int e = pfirst;
      for (int rt = 0; rt < rD; ++rt)
        for (int ct = 0; ct < cL; ++ct) s.wpairs[e++] = WPair{tid, 0, rt, ct};
      for (int rt = 0; rt < tB; ++rt)
        for (int ct = 0; ct < tB; ++ct) s.wpairs[e++] = WPair{tid, 1, rt, ct};
    }
  }
}

// Compaction of the windows that need it (blocks 0..k-1) and the append of the
// new blocks (remaining blocks, one warp per batch row). Sources and
// destinations never overlap (see the capacity argument in kkm_internal.cuh).
__global__ void k_move(Dev s) {
  const int warps = blockDim.x >> 5, wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((int)blockIdx.x < s.k) {
    const int j = blockIdx.x;
    const Plan P = s.plan[j];
    if (P.src_head < 0) return;
    const int64_t base = (int64_t)j * s.cap;
    const int size = P.tail_c - P.head_c;
    for (int r = wib; r < size; r += warps) {
      const int64_t src = base + P.src_head + r, dst = base + r;
      warp_copy_row(s, true, src, dst);
      if (lane == 0) {
        s.yn[dst] = s.yn[src];
        s.yi[dst] = s.yi[src];
        s.w64[dst] = s.w64[src];
        s.w32[dst] = s.w32[src];
      }
    }
    return;
  }
  const int r = (blockIdx.x - s.k) * warps + wib;
  if (r >= s.b) return;
  const int x = s.perm[r];
  const int j = s.assign[x];
  const Plan P = s.plan[j];
  const int pos = P.tail_c + (r - s.coff[j]);
  if (pos >= s.cap) return;                       // flagged ST_CAPACITY in the plan
  const int64_t dst = (int64_t)j * s.cap + pos;
  warp_copy_row(s, false, x, dst);
  if (lane == 0) {
    s.yn[dst] = s.xbn[x];
    s.yi[dst] = s.xbi[x];
  }
}

// Tile list of the distance pass from the current windows (block of 1024, k <= 1024).
__device__ void build_tiles_block(const Dev& s) {
  const int tid = threadIdx.x;
  int nt = 0, size = 0, head = 0;
  if (tid < s.k) {
    head = s.head[tid];
    size = s.tail[tid] - head;
    nt = (size + s.tn - 1) / s.tn;
  }
  int total = 0;
  const int first = block_exclusive_scan_1024(nt, &total);
  if (tid == 0) {
    *s.ntiles = total <= s.max_tiles ? total : s.max_tiles;
    if (total > s.max_tiles) atomicOr(s.status, ST_CAPACITY);
  }
  if (tid < s.k) {
    const bool fits = first + nt <= s.max_tiles;   // never false by the capacity bound
    s.tile_first[tid] = fits ? first : 0;
    s.tile_cnt[tid] = fits ? nt : 0;
    if (fits)
      for (int t = 0; t < nt; ++t) {
        const int c = t * s.tn;
        s.tiles[first + t] = Tile{tid, (int32_t)((int64_t)tid * s.cap + head + c),
                                  min(s.tn, size - c), 0};
      }
  }
}

__global__ void __launch_bounds__(1024) k_build_tiles(Dev s) { build_tiles_block(s); }

// Single CTA of 1024 threads: the FP64 norm recurrence, weight decay/append,
// window bookkeeping, the next tile list, f_B and the iteration counter.
__global__ void __launch_bounds__(1024) k_finalize(Dev s, double* obj_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiles_used = *s.ntiles;   // tiles of this step's distance pass
  for (int j = warp; j < s.k; j += 32) {
    const Plan P = s.plan[j];
    if (P.cnt == 0) continue;
    // window Gram sums of this center, in pair order
    double A = 0.0, Bdd = 0.0, E = 0.0, M = 0.0;
    const int p0 = s.wpair_first[j];
    const int np = (p0 + s.wpair_cnt[j] <= s.max_pairs) ? s.wpair_cnt[j] : 0;
    for (int p = lane; p < np; p += 32) {
      const double* q = s.wpart + (int64_t)(p0 + p) * 4;
      A += q[0]; Bdd += q[1]; E += q[2]; M += q[3];
    }
    A = warp_sum(A); Bdd = warp_sum(Bdd); E = warp_sum(E); M = warp_sum(M);
    const double a = s.alpha[j];
    const double n = (double)P.cnt;
    if (lane == 0) {
      // Sec. 4: ||C'||^2 = (1-a)^2 ||R||^2 + 2a(1-a) <R, m> + a^2 ||m||^2, with
      // m = cm(B_j) and R = C - D the part of the old center that Eq. (1) keeps
      // (D = the dropped rows with their old weights).
      const double m2 = M / (n * n);
      const double R2 = s.cnorm[j] - 2.0 * A + Bdd;
      const double Rm = s.cmc[j] - E / n;
      s.cnorm[j] = (1.0 - a) * (1.0 - a) * R2 + 2.0 * a * (1.0 - a) * Rm + a * a * m2;
    }
    const int64_t base = (int64_t)j * s.cap;
    const double keep = 1.0 - a, wnew = a / n;
    const int tail_new = min(P.tail_new, s.cap);
    for (int r = P.head_new + lane; r < tail_new; r += 32) {
      const int64_t row = base + r;
      const double w = (r < P.tail_c) ? s.w64[row] * keep : wnew;
      s.w64[row] = w;
      s.w32[row] = (float)w;
    }
    if (lane == 0) {
      s.head[j] = P.head_new;
      s.tail[j] = P.tail_new;
      s.c1[j] = P.c1_new;
    }
  }
  __syncthreads();
  build_tiles_block(s);
  // f_B(C_i): mean of the minimum distances, FP64, fixed summation order
  __shared__ double red[1024];
  double acc = 0.0;
  for (int x = tid; x < s.b; x += 1024) acc += (double)s.mind[x];
  red[tid] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) {
    const double f = red[0] / (double)s.b;
    *s.obj = f;
    if (obj_out) *obj_out = f;
    s.stats[0] += 1;
    s.stats[1] += *s.s_old;
    s.stats[2] += tiles_used;
    *s.iter += 1;
  }
}

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

// FP64 sum of mind[0..rows) into *out (single CTA, fixed order).
__global__ void __launch_bounds__(1024) k_mind_sum(Dev s, int rows, double* out) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int x = threadIdx.x; x < rows; x += 1024) acc += (double)s.mind[x];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_sample(const Dev& s, cudaStream_t st) {
  k_sample<<<(s.b + 255) / 256, 256, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t launch_gather_batch(const Dev& s, const int32_t* idx, cudaStream_t st) {
  k_gather_batch<<<(s.b * 32 + 255) / 256, 256, 0, st>>>(s, idx);
  return cudaGetLastError();
}

cudaError_t launch_gather_query(const Dev& s, const float* Q, int64_t ldq, int rows, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  k_gather_query<<<(rows * 32 + 255) / 256, 256, 0, st>>>(s, Q, ldq, rows);
  return cudaGetLastError();
}

cudaError_t launch_argmin(const Dev& s, int rows, const int32_t* forced, int32_t* assign_out,
                          float* mind_out, float* dist_out, bool update, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  k_argmin<<<(rows + 127) / 128, 128, 0, st>>>(s, rows, forced, assign_out, mind_out, dist_out,
                                                update ? 1 : 0);
  return cudaGetLastError();
}

int sort_plan_smem(int k) { return 3 * k * 4 + 32 * k * 2; }

cudaError_t launch_sort_plan(const Dev& s, cudaStream_t st) {
  const int smem = sort_plan_smem(s.k);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_sort_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  k_sort_plan<<<1, 1024, smem, st>>>(s, 64);   // window-pass tile (k_wgram_simt)
  return cudaGetLastError();
}

cudaError_t launch_move(const Dev& s, cudaStream_t st) {
  const int warps = 8;
  const int blocks = s.k + (s.b + warps - 1) / warps;
  k_move<<<blocks, warps * 32, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Dev& s, double* obj_out, cudaStream_t st) {
  k_finalize<<<1, 1024, 0, st>>>(s, obj_out);
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

cudaError_t launch_mind_sum(const Dev& s, int rows, double* out, cudaStream_t st) {
  k_mind_sum<<<1, 1024, 0, st>>>(s, rows, out);
  return cudaGetLastError();
}

}  // namespace kkm
