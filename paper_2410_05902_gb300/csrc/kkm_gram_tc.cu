// tcgen05 / TMA form of the two Gram passes (BF16 and split-BF16 products).
//
// One persistent CTA per SM walks the work items round-robin. In the distance
// pass (mode 0) an item is (128-row batch tile, 128-row support tile of one
// center); in the window pass (mode 1) it is (128 support rows, 64 support
// rows) of one center. For each item:
//   G = X_B Y^T           tcgen05.mma kind::f16 (BF16 x BF16 -> FP32 in TMEM),
//                         operands streamed by TMA through a 6-stage ring of
//                         128B-swizzled shared-memory slices (64 columns each)
//   K = kernel(||x||^2 + ||y||^2 - 2G)     in registers after tcgen05.ld
//   part[tile][x] = sum_y w_y K(x, y)      one partial per row and tile
// The split form (x = hi + lo) runs the K loop three times over the slice
// pairs (hi,hi), (hi,lo), (lo,hi) into the same accumulator.
//
// Roles: warp 0 issues TMA loads, warp 1 issues the MMAs (one elected lane)
// and owns the TMEM allocation (2 accumulators x 128 columns), warps 2-5 are
// the epilogue (one TMEM lane = one batch row per thread). Every mbarrier wait
// is bounded. A wait that runs out sets ST_TIMEOUT and makes the role stop. On
// the way out the producer waits for its last copies to land and the MMA warp
// waits for its last MMAs, so TMEM is freed only once nothing is in flight.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "kkm_internal.cuh"

namespace kkm {
namespace {

constexpr int TM = 128;                         // A rows per tile = TMEM lanes
constexpr int KS = 64;                          // BF16 columns per slice (one 128-byte swizzle row)
constexpr int A_BYTES = TM * KS * 2;            // 16 KB: the A tile of one slice
constexpr int RING_BYTES = 192 * 1024;          // shared memory for the operand ring
constexpr int STAGES = 8;                       // most stages any variant uses
// TNV = support rows per tile (B rows = accumulator columns): 128 or 64.
// BF16:   a stage is one 64-column slice (A, B): 4 MMAs.
// BF16X3: a stage is one 64-column slice of all four operand tiles
//         (A_hi, A_lo, B_hi, B_lo): 12 MMAs (hi.hi, hi.lo, lo.hi), so the hi
//         tiles are fetched once per slice instead of twice.
template <bool X3, int TNV> struct Ring {
  static constexpr int b_bytes = TNV * KS * 2;
  static constexpr int bytes = X3 ? 2 * (A_BYTES + b_bytes) : A_BYTES + b_bytes;
  static constexpr int stages = RING_BYTES / bytes;   // 3, 4, 6 or 8
};
constexpr int NTHREADS = 192;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // 2 s per wait

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int N>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

struct Shared {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t mma_done;
  uint32_t tmem_base;
  uint32_t pad;
  float4 meta[4][128];                          // per epilogue warp: (||y||^2, w, yi, class)
};

constexpr int SMEM_BYTES = 1024 + RING_BYTES + (int)sizeof(Shared);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of parity `parity` to complete; false after WAIT_LIMIT_NS.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(b, parity)) return true;
    if (globaltimer() - t0 > WAIT_LIMIT_NS) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored as rows of
// 128 bytes with the 128-byte swizzle (the layout TMA writes with
// CU_TENSOR_MAP_SWIZZLE_128B): start address >> 4 in bits 0-13, leading byte
// offset 16 (unused by swizzled K-major layouts), stride byte offset 1024
// (8 rows x 128 B) in bits 32-45, descriptor version 1 in bits 46-47,
// swizzle mode 2 (128B) in bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int KIND>
__device__ __forceinline__ float kernel_value(float g, float xn, float yn, bool same, float negc,
                                              float coef0, int degree) {
  if constexpr (KIND == K_GAUSS || KIND == K_LAPLACE) {
    float d2 = fmaxf(fmaf(-2.0f, g, xn + yn), 0.0f);
    d2 = same ? 0.0f : d2;
    const float arg = (KIND == K_GAUSS) ? d2 : sqrtf(d2);
    return ex2_approx(arg * negc);
  } else if constexpr (KIND == K_LINEAR) {
    return g;
  } else {
    const float base = g + coef0;
    float r = 1.0f;
    for (int p = 0; p < degree; ++p) r *= base;
    return r;
  }
}

// A window-pass tile (mode 1): rows of the support store of center j, as
// positions inside its region. Kind 0 pairs the dropped prefix D with the old
// window plus the new block; kind 1 pairs the new block with itself. Row tiles
// are 128 rows (TM), column tiles TNV rows.
struct PairTile {
  int64_t base;      // first row of the center's region
  int rs, rrem;      // first row position, rows left in the row range from rs
  int cs, crem;      // first column position, rows left in the column range from cs
  int kind, head_new, tail_c;
};

template <int TNV>
__device__ __forceinline__ PairTile pair_tile(const Dev& s, int w) {
  const WPair pr = s.wpairs[w];
  const Plan P = s.plan[pr.j];
  PairTile t;
  t.base = (int64_t)pr.j * s.cap;
  int r0, rn, c0, cn;
  if (pr.kind == 0) { r0 = P.head_c; rn = P.ndrop; c0 = P.head_c; cn = P.tail_new - P.head_c; }
  else { r0 = P.tail_c; rn = P.cnt; c0 = P.tail_c; cn = P.cnt; }
  t.rs = r0 + pr.rt * TM;
  t.rrem = rn - pr.rt * TM;
  t.cs = c0 + pr.ct * TNV;
  t.crem = cn - pr.ct * TNV;
  t.kind = pr.kind;
  t.head_new = P.head_new;
  t.tail_c = P.tail_c;
  return t;
}

// MODE 0: distance pass (A = batch tile, B = support tile, one FP32 partial per row).
// MODE 1: window pass (A and B = support rows of one center, four FP64 sums per warp).
// Items are dealt round-robin to the persistent CTAs. Splitting a tile along
// its columns needs no merge because both passes only sum over columns, so
// narrower tiles (TNV = 64) are how the window pass gets enough items.
template <int KIND, int MODE, bool X3, int TNV>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_dist_tc(Dev s, int rows, const __grid_constant__ CUtensorMap tmA,
              const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Shared& sh = *reinterpret_cast<Shared*>(smem + RING_BYTES);
  constexpr int NST = Ring<X3, TNV>::stages;
  constexpr int SB = Ring<X3, TNV>::bytes;
  constexpr int BB = Ring<X3, TNV>::b_bytes;
  constexpr uint32_t TMEM_COLS = 2 * TNV;        // two accumulators (double buffering)
  constexpr uint32_t IDESC = idesc<TNV>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&sh.full[i], 1);
      mbar_init(&sh.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sh.tfull[i], 1);
      mbar_init(&sh.tempty[i], 128);
    }
    mbar_init(&sh.mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&sh.tmem_base)), "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem_base;
  KKM_GRID_DEP_WAIT();   // everything above touches only this CTA's shared memory and TMEM

  const int R = (rows + TM - 1) / TM;
  const int total = (MODE == 0) ? R * (*s.ntiles) : *s.nwpairs;
  const int nks = s.dp / KS;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      bool ok = true;
      uint32_t it = 0;
      for (int item = blockIdx.x; ok && item < total; item += gridDim.x) {
        int ya, yb;
        const CUtensorMap* am;
        if constexpr (MODE == 0) {
          ya = (item % R) * TM;
          yb = s.tiles[item / R].row0;
          am = &tmA;
        } else {
          const PairTile pt = pair_tile<TNV>(s, item);
          ya = (int)(pt.base + pt.rs);
          yb = (int)(pt.base + pt.cs);
          am = &tmA;   // mode 1 gets the 128-row support map as tmA
        }
        for (int sl = 0; sl < nks; ++sl, ++it) {
          const int st = it % NST;
          const uint32_t ph = (it / NST) & 1u;
          if (!mbar_wait(&sh.empty[st], ph ^ 1u)) { ok = false; break; }
          const int x = sl * KS;
          uint8_t* a = smem + st * SB;
          mbar_expect_tx(&sh.full[st], SB);
          if constexpr (X3) {   // stage layout: A_hi | A_lo | B_hi | B_lo
            tma_load_2d(a, am, &sh.full[st], x, ya);
            tma_load_2d(a + A_BYTES, am, &sh.full[st], s.dp + x, ya);
            tma_load_2d(a + 2 * A_BYTES, &tmB, &sh.full[st], x, yb);
            tma_load_2d(a + 2 * A_BYTES + BB, &tmB, &sh.full[st], s.dp + x, yb);
          } else {              // stage layout: A | B
            tma_load_2d(a, am, &sh.full[st], x, ya);
            tma_load_2d(a + A_BYTES, &tmB, &sh.full[st], x, yb);
          }
        }
      }
      // the last fill of every stage must land before the CTA may exit
      for (uint32_t q = (it > (uint32_t)NST ? it - NST : 0u); q < it; ++q)
        if (!mbar_wait(&sh.full[q % NST], (q / NST) & 1u)) ok = false;
      if (!ok) atomicOr(s.status, ST_TIMEOUT);
    }
  } else if (warp == 1) {
    // -------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      bool ok = true;
      uint32_t it = 0, local = 0;
      for (int item = blockIdx.x; ok && item < total; item += gridDim.x, ++local) {
        const uint32_t buf = local & 1u, bph = (local >> 1) & 1u;
        if (!mbar_wait(&sh.tempty[buf], bph ^ 1u)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + buf * TNV;
        for (int sl = 0; sl < nks; ++sl, ++it) {
          const int st = it % NST;
          const uint32_t ph = (it / NST) & 1u;
          if (!mbar_wait(&sh.full[st], ph)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + st * SB);
          if constexpr (X3) {
            const uint32_t alo = a0 + A_BYTES, bhi = a0 + 2 * A_BYTES, blo = bhi + BB;
#pragma unroll
            for (int k = 0; k < KS / 16; ++k) {
              mma_bf16(d, sw128_desc(a0 + 32u * k), sw128_desc(bhi + 32u * k), IDESC, (sl | k) != 0 ? 1u : 0u);
              mma_bf16(d, sw128_desc(a0 + 32u * k), sw128_desc(blo + 32u * k), IDESC, 1u);
              mma_bf16(d, sw128_desc(alo + 32u * k), sw128_desc(bhi + 32u * k), IDESC, 1u);
            }
          } else {
            const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
            for (int k = 0; k < KS / 16; ++k)
              mma_bf16(d, sw128_desc(a0 + 32u * k), sw128_desc(b0 + 32u * k), IDESC, (sl | k) != 0 ? 1u : 0u);
          }
          mma_commit(&sh.empty[st]);
        }
        if (!ok) break;
        mma_commit(&sh.tfull[buf]);
      }
      mma_commit(&sh.mma_done);
      if (!mbar_wait(&sh.mma_done, 0)) ok = false;
      if (!ok) atomicOr(s.status, ST_TIMEOUT);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;                      // TMEM lane quadrant of this warp
    const int rloc = q * 32 + lane;              // this thread's row inside the tile
    float4* meta = sh.meta[warp - 2];
    const float negc = s.negc, coef0 = (float)s.coef0;
    const int degree = s.degree;
    uint32_t local = 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x, ++local) {
      const uint32_t buf = local & 1u, bph = (local >> 1) & 1u;
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + buf * TNV;
      // column metadata and row data first: their global loads overlap the MMAs
      int t = 0, row = 0, ncols = 0;
      float xn;
      int xi;
      PairTile pt;
      double wp = 0.0;
      bool rvalid = true;
      __syncwarp();
      if constexpr (MODE == 0) {
        t = item / R;
        const Tile T = s.tiles[t];
        ncols = T.ncols;
#pragma unroll
        for (int c4 = 0; c4 < TNV / 32; ++c4) {
          const int c = c4 * 32 + lane;
          const bool valid = c < T.ncols;
          const int64_t g = (int64_t)T.row0 + (valid ? c : 0);
          meta[c] = make_float4(s.yn[g], valid ? s.w32[g] : 0.0f, __int_as_float(valid ? s.yi[g] : -2), 0.0f);
        }
        row = (item % R) * TM + rloc;
        const int rr = row < rows ? row : 0;
        xn = s.xbn[rr];
        xi = s.xbi[rr];
      } else {
        pt = pair_tile<TNV>(s, item);
#pragma unroll
        for (int c4 = 0; c4 < TNV / 32; ++c4) {
          const int c = c4 * 32 + lane;
          const int qpos = pt.cs + c;
          const bool valid = c < pt.crem;
          const int64_t g = pt.base + (valid ? qpos : pt.cs);
          // column class: 0 dropped (in D and the old window), 1 old window, 2 new block, 3 none
          const float cls = !valid ? 3.0f : (qpos < pt.head_new ? 0.0f : (qpos < pt.tail_c ? 1.0f : 2.0f));
          meta[c] = make_float4(s.yn[g], valid ? s.w32[g] : 0.0f, __int_as_float(valid ? s.yi[g] : -2), cls);
        }
        rvalid = rloc < pt.rrem;
        const int64_t p = pt.base + pt.rs + (rvalid ? rloc : 0);
        xn = s.yn[p];
        xi = s.yi[p];
        wp = rvalid ? s.w64[p] : 0.0;
      }
      __syncwarp();
      const bool ok = mbar_wait(&sh.tfull[buf], bph);
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) atomicOr(s.status, ST_TIMEOUT);
        break;
      }
      tc_fence_after();
      if constexpr (MODE == 0) {
        float acc = 0.0f;
#pragma unroll
        for (int ch = 0; ch < TNV / 32; ++ch) {
          float g[32];
          tmem_ld32(taddr + ch * 32, g);
          if (ch == TNV / 32 - 1) {
            tc_fence_before();
            mbar_arrive(&sh.tempty[buf]);
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int c = ch * 32 + i;
            const float4 m = meta[c];
            const float kv = kernel_value<KIND>(g[i], xn, m.x, xi == __float_as_int(m.z), negc, coef0, degree);
            acc = (c < ncols) ? fmaf(m.y, kv, acc) : acc;
          }
        }
        if (row < rows) s.part[(int64_t)t * s.bpad + row] = acc;
      } else {
        float fA = 0.0f, fB = 0.0f, fE = 0.0f;
#pragma unroll
        for (int ch = 0; ch < TNV / 32; ++ch) {
          float g[32];
          tmem_ld32(taddr + ch * 32, g);
          if (ch == TNV / 32 - 1) {
            tc_fence_before();
            mbar_arrive(&sh.tempty[buf]);
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float4 m = meta[ch * 32 + i];
            const float kv = kernel_value<KIND>(g[i], xn, m.x, xi == __float_as_int(m.z), negc, coef0, degree);
            const float wk = m.y * kv;
            fA += (m.w < 1.5f) ? wk : 0.0f;
            fB += (m.w < 0.5f) ? wk : 0.0f;
            fE += (m.w > 1.5f && m.w < 2.5f) ? kv : 0.0f;
          }
        }
        // kind 0: A = w_p sum_{q in W} w_q K, Bdd = w_p sum_{q in D} w_q K, E = w_p sum_{q in B} K
        // kind 1: M = sum_{q in B} K (every valid column of a kind-1 tile is in B)
        double sA = 0.0, sB = 0.0, sE = 0.0, sM = 0.0;
        if (rvalid) {
          if (pt.kind == 0) { sA = wp * (double)fA; sB = wp * (double)fB; sE = wp * (double)fE; }
          else sM = (double)fE;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          sA += __shfl_xor_sync(0xffffffffu, sA, o);
          sB += __shfl_xor_sync(0xffffffffu, sB, o);
          sE += __shfl_xor_sync(0xffffffffu, sE, o);
          sM += __shfl_xor_sync(0xffffffffu, sM, o);
        }
        if (lane == 0) {
          double* out = s.wpart + ((int64_t)item * 4 + q) * 4;
          out[0] = sA; out[1] = sB; out[2] = sE; out[3] = sM;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  }
}

template <int KIND, int MODE, bool X3, int TNV>
cudaError_t launch_form(const Dev& s, const CUtensorMap& a, const CUtensorMap& b, int rows, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_dist_tc<KIND, MODE, X3, TNV>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_pdl(k_dist_tc<KIND, MODE, X3, TNV>, dim3(s.num_sms), dim3(NTHREADS), SMEM_BYTES, st, s, rows, a, b);
}

// maps: [0] batch rows, 128-row boxes; [1] support rows, 128-row boxes; [2] support rows, 64-row boxes
template <int MODE, int TNV>
cudaError_t launch_mode(const Dev& s, const void* maps_in, int rows, cudaStream_t st) {
  const CUtensorMap* m = static_cast<const CUtensorMap*>(maps_in);
  const CUtensorMap& a = (MODE == 0) ? m[0] : m[1];
  const CUtensorMap& b = (TNV == 128) ? m[1] : m[2];
  const bool x3 = s.form == FORM_BF16X3;
  switch (s.kind) {
    case K_GAUSS:
      return x3 ? launch_form<K_GAUSS, MODE, true, TNV>(s, a, b, rows, st)
                : launch_form<K_GAUSS, MODE, false, TNV>(s, a, b, rows, st);
    case K_LAPLACE:
      return x3 ? launch_form<K_LAPLACE, MODE, true, TNV>(s, a, b, rows, st)
                : launch_form<K_LAPLACE, MODE, false, TNV>(s, a, b, rows, st);
    case K_LINEAR:
      return x3 ? launch_form<K_LINEAR, MODE, true, TNV>(s, a, b, rows, st)
                : launch_form<K_LINEAR, MODE, false, TNV>(s, a, b, rows, st);
    default:
      return x3 ? launch_form<K_POLY, MODE, true, TNV>(s, a, b, rows, st)
                : launch_form<K_POLY, MODE, false, TNV>(s, a, b, rows, st);
  }
}

}  // namespace

bool tc_available() { return true; }

// Tensor maps of the batch rows and the support store: 2-D BF16 tensors of ld
// columns, boxes of 64 columns x 128 (or 64) rows, 128-byte swizzle.
cudaError_t tc_prepare(Dev& s, void* maps_out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  CUtensorMap* maps = static_cast<CUtensorMap*>(maps_out);
  const int64_t srows = (int64_t)s.k * s.cap + 256;
  struct { void* base; uint64_t rows; uint32_t box_rows; } ops[3] = {
      {s.xbh, (uint64_t)s.bpad, 128u}, {s.ybh, (uint64_t)srows, 128u}, {s.ybh, (uint64_t)srows, 64u}};
  for (int i = 0; i < 3; ++i) {
    cuuint64_t dims[2] = {(cuuint64_t)s.ld, (cuuint64_t)ops[i].rows};
    cuuint64_t strides[1] = {(cuuint64_t)s.ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)KS, ops[i].box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&maps[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ops[i].base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_dist_tc(const Dev& s, const void* maps, int rows, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  return launch_mode<0, 128>(s, maps, rows, st);
}

cudaError_t launch_wgram_tc(const Dev& s, const void* maps, cudaStream_t st) {
  return launch_mode<1, 64>(s, maps, 0, st);
}

}  // namespace kkm
