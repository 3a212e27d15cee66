// tcgen05 / TMA form of the two Gram passes (BF16, split-BF16 and TF32 products).
//
// One persistent CTA per SM walks the work items round-robin. In the distance
// pass (mode 0) an item is (128-row batch tile, TNV-row support tile of one
// center; TNV = 256 by default, 64 or 128 on request); in the window pass
// (mode 1) it is (128 support rows, 64 support rows) of one center. For each
// item:
//   G = X_B Y^T           tcgen05.mma kind::f16 (BF16) or kind::tf32 (TF32),
//                         FP32 in TMEM; operands streamed by TMA through a
//                         192 KB ring of 128B-swizzled shared-memory slices
//   K = kernel(||x||^2 + ||y||^2 - 2G)     in registers after tcgen05.ld
//   part[tile][x] = sum_y w_y K(x, y)      one partial per row and tile
// The split form (x = hi + lo) runs the K loop three times over the slice
// pairs (hi,hi), (hi,lo), (lo,hi) into the same accumulator.
//
// Roles: warp 0 issues TMA loads (and stages each item's metadata), warp 1
// issues the MMAs (one elected lane) and owns the TMEM allocation (2
// accumulators x TNV columns), warps 2-17 are the epilogue (four per TMEM lane
// quadrant). In the distance pass they form two groups that take alternate
// items; in the window pass all sixteen share each item. Every mbarrier wait
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
// operand formats: BF16 (one product), split BF16 (hi.hi + hi.lo + lo.hi), TF32
// (FP32 rows rounded to TF32; a 128-byte slice row holds 32 of them)
constexpr int OP_BF16 = 0, OP_X3 = 1, OP_TF32 = 2;
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
constexpr int NEPI = 16;                         // epilogue warps (four per TMEM lane quadrant)
constexpr int NH = NEPI / 4;                     // column parts of an accumulator
constexpr int NTHREADS = 64 + 32 * NEPI;        // + one TMA warp and one MMA warp
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // 2 s per wait

// Instruction descriptor of tcgen05.mma kind::f16 / kind::tf32: D FP32
// (bits 4-5 = 1), A and B BF16 (type 1) or TF32 (type 2) in bits 7-9 and
// 10-12, both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in
// bits 24-28.
template <int N, int OP>
__host__ __device__ constexpr uint32_t idesc() {
  constexpr uint32_t t = OP == OP_TF32 ? 2u : 1u;
  return (1u << 4) | (t << 7) | (t << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

constexpr int MS = 4;                           // metadata ring slots (items in flight)

// Distance-pass metadata of one item, copied by the producer: col[0] =
// ||y||^2, col[1] = w, col[2] = data index of the 128 support rows; row[0] =
// ||x||^2, row[1] = data index of the 128 batch rows.
struct MetaSlot {
  float col[3][256];
  float row[2][128];
};

struct Shared {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t mfull[MS];
  uint64_t mempty[MS];
  uint64_t mma_done;
  uint32_t tmem_base;
  uint32_t pad;
  union alignas(16) {
    MetaSlot ring[MS];                          // distance pass
    float warp[NEPI][5][32];                    // window pass: per epilogue warp (load_pair_meta)
  } meta;
  float red[768];                                // distance pass: row sums of column parts (dist_epilogue)
  float wred[2][NEPI][4];                       // window pass: per-warp sums (item parity, warp, sum)
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

// One MMA on a 32-byte K step of the 128-byte swizzled rows: K = 16 BF16
// values (kind::f16) or K = 8 TF32 values (kind::tf32).
template <int OP>
__device__ __forceinline__ void mma_op(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accum) {
  if constexpr (OP == OP_TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar))
               : "memory");
}

// tcgen05.ld .16x256b.xNB: 16 TMEM lanes starting at the address's lane, NB
// blocks of 8 consecutive FP32 columns. Thread t receives, for block j,
//   v[4j]   = (lane t/4,     column 8j + 2(t%4)),  v[4j+1] = the next column,
//   v[4j+2] = (lane t/4 + 8, column 8j + 2(t%4)),  v[4j+3] = the next column.
// Each column value is needed by 4 threads instead of 32 (the 32x32b shape
// gives a thread one lane and all columns), which cuts the per-column
// metadata the epilogue reads from shared memory by 4x.
template <int NB>
__device__ __forceinline__ void tmem_ld16x256(uint32_t taddr, float (&v)[4 * NB]) {
  uint32_t r[4 * NB];
  if constexpr (NB == 8) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x8.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
  } else if constexpr (NB == 4) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x4.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  } else {
    static_assert(NB == 2, "tmem_ld16x256: 2, 4 or 8 blocks");
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr));
  }
#pragma unroll
  for (int i = 0; i < 4 * NB; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Kernel values of one row against two columns from their Gram entries g.
// Gaussian: rc = ||x||^2 * negc and cc = ||y||^2 * negc (negc = -log2(e)/kappa),
//           K = 2^(rc + cc - 2 negc g). The exponent is -D^2 log2(e)/kappa with
//           D^2 = ||x||^2 + ||y||^2 - 2g; rounding can leave it a few ulps of
//           ||x||^2 above 0 for near-duplicates, where K = 1 to that accuracy.
// Laplacian: rc = ||x||^2, cc = ||y||^2, K = 2^(negc * sqrt(max(D^2, 0))).
// Both give exactly 1 when the two rows are the same data point (K(x,x) = 1).
// Linear and polynomial values of padding columns (yi = -2) are zeroed, as
// those kernels are unbounded.
template <int KIND>
__device__ __forceinline__ float2 kernel_pair(float2 g, float rc, float2 cc, int xi, int2 yi, float negc,
                                              float coef0, int degree) {
  float2 k;
  if constexpr (KIND == K_GAUSS) {
    const float2 a = __ffma2_rn(g, make_float2(-2.0f * negc, -2.0f * negc), __fadd2_rn(make_float2(rc, rc), cc));
    k.x = xi == yi.x ? 1.0f : ex2_approx(a.x);
    k.y = xi == yi.y ? 1.0f : ex2_approx(a.y);
  } else if constexpr (KIND == K_LAPLACE) {
    const float2 d2 = __ffma2_rn(g, make_float2(-2.0f, -2.0f), __fadd2_rn(make_float2(rc, rc), cc));
    k.x = xi == yi.x ? 1.0f : ex2_approx(sqrt_approx(fmaxf(d2.x, 0.0f)) * negc);
    k.y = xi == yi.y ? 1.0f : ex2_approx(sqrt_approx(fmaxf(d2.y, 0.0f)) * negc);
  } else if constexpr (KIND == K_LINEAR) {
    k.x = yi.x == -2 ? 0.0f : g.x;
    k.y = yi.y == -2 ? 0.0f : g.y;
  } else {
    float rx = 1.0f, ry = 1.0f;
    for (int p = 0; p < degree; ++p) { rx *= g.x + coef0; ry *= g.y + coef0; }
    k.x = yi.x == -2 ? 0.0f : rx;
    k.y = yi.y == -2 ? 0.0f : ry;
  }
  return k;
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

// Window-pass column metadata of one epilogue warp (the C = TNV / NH columns of
// its part of the tile): col[0] = ||y||^2 (times negc for the Gaussian), col[1] = w on the
// old window (A), col[2] = data index (-2 on padding columns), col[3] = w on
// the dropped rows (Bdd), col[4] = 1 on the new block (E). Padding columns
// keep the ||y||^2 of the row the MMA read there, so their kernel values stay
// finite (and their weights are 0).
template <int KIND, int TNV>
__device__ __forceinline__ void load_pair_meta(const Dev& s, const PairTile& pt, int cbase, float (*m)[32],
                                               int lane) {
  constexpr int C = TNV / NH;
  const float sc = (KIND == K_GAUSS) ? s.negc : 1.0f;
#pragma unroll
  for (int c = lane; c < C; c += 32) {
    const int col = cbase + c;
    const int qpos = pt.cs + col;                // inside the region even past the range
    const bool valid = col < pt.crem;
    const int64_t gi = pt.base + qpos;
    const float w = valid ? s.w32[gi] : 0.0f;
    const bool in_d = qpos < pt.head_new, in_old = qpos < pt.tail_c;
    m[0][c] = s.yn[gi] * sc;
    m[1][c] = in_old ? w : 0.0f;
    m[2][c] = __int_as_float(valid ? s.yi[gi] : -2);
    m[3][c] = in_d ? w : 0.0f;
    m[4][c] = (valid && !in_old) ? 1.0f : 0.0f;
  }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Distance-pass epilogue pieces. A chunk is CW accumulator columns of the
// warp's 32 rows: chunk_load reads it from TMEM (two 16-lane loads), and
// chunk_math adds w_y K(x, y) over its columns into the row sums acc[u] (rows
// g4 + 8u of the quadrant, two columns per lane and 8-column block).
template <int NB>
__device__ __forceinline__ void chunk_load(uint32_t taddr, float (&v0)[4 * NB], float (&v1)[4 * NB]) {
  tmem_ld16x256<NB>(taddr, v0);                 // rows g4, g4 + 8
  tmem_ld16x256<NB>(taddr + (16u << 16), v1);   // rows g4 + 16, g4 + 24
  tmem_wait_ld();
}

template <int KIND, int NB>
__device__ __forceinline__ void block_math(const float (&v0)[4 * NB], const float (&v1)[4 * NB], int j, float2 w,
                                           float2 cc, int2 yi, const float (&rc)[4], const int (&xi)[4], float negc,
                                           float coef0, int degree, float2 (&acc)[4]) {
  acc[0] = __ffma2_rn(w, kernel_pair<KIND>(make_float2(v0[4 * j], v0[4 * j + 1]), rc[0], cc, xi[0], yi, negc,
                                                 coef0, degree), acc[0]);
  acc[1] = __ffma2_rn(w, kernel_pair<KIND>(make_float2(v0[4 * j + 2], v0[4 * j + 3]), rc[1], cc, xi[1], yi,
                                                 negc, coef0, degree), acc[1]);
  acc[2] = __ffma2_rn(w, kernel_pair<KIND>(make_float2(v1[4 * j], v1[4 * j + 1]), rc[2], cc, xi[2], yi, negc,
                                                 coef0, degree), acc[2]);
  acc[3] = __ffma2_rn(w, kernel_pair<KIND>(make_float2(v1[4 * j + 2], v1[4 * j + 3]), rc[3], cc, xi[3], yi,
                                                 negc, coef0, degree), acc[3]);
}

template <int KIND, int NB>
__device__ __forceinline__ void chunk_math(const float (&v0)[4 * NB], const float (&v1)[4 * NB], const MetaSlot& m,
                                           int c0, const float (&rc)[4], const int (&xi)[4], float negc, float coef0,
                                           int degree, float2 (&acc)[4]) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const int c = c0 + 8 * j;
    const float2 yn = *reinterpret_cast<const float2*>(&m.col[0][c]);
    const float2 w = *reinterpret_cast<const float2*>(&m.col[1][c]);
    const int2 yi = *reinterpret_cast<const int2*>(&m.col[2][c]);
    const float2 cc = (KIND == K_GAUSS) ? __fmul2_rn(yn, make_float2(negc, negc)) : yn;
    block_math<KIND, NB>(v0, v1, j, w, cc, yi, rc, xi, negc, coef0, degree, acc);
  }
}

// Distance-pass epilogue (warps 2-17): two groups of eight warps, two per TMEM
// lane quadrant. Group g = (warp - 2) / 8 takes this CTA's items of parity g
// (accumulator buffer g, and the metadata slots of those items), so one
// group's TMEM loads, combine and stores overlap the other group's
// arithmetic. Warp part h covers its quadrant's 32 rows and columns
// [h TNV/2, (h+1) TNV/2) in chunks of CW (at most 32, to keep the values in
// registers); it frees the accumulator once the last chunk is in registers.
// A CTA with a single item runs it on both groups instead, each warp on a
// quarter of the columns (part 2g + h). The parts of a row meet in shared
// memory (by the group's item parity), and part 0 writes part[tile][row].
template <int KIND, int TNV>
__device__ __forceinline__ void dist_epilogue(const Dev& s, Shared& sh, uint32_t tmem, int total, int R, int rows,
                                              int warp, int lane) {
  constexpr int CW = TNV / 4 < 32 ? TNV / 4 : 32;   // columns per chunk
  constexpr int NB = CW / 8;                    // 8-column blocks per TMEM load
  const int e = warp - 2, g = e >> 3, h = (e >> 2) & 1, q = warp & 3;
  const int g4 = lane >> 2, c2 = 2 * (lane & 3);
  const int rq = g4 + 8 * (lane & 3);           // the row this thread reports after the lane reduction
  const float negc = s.negc;
  const float coef0 = (float)s.coef0;
  const int degree = s.degree;
  const int mine = total > (int)blockIdx.x ? (total - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const bool solo = mine == 1;
  bool dead = false;                            // a wait ran out: skip the work, keep the barriers
  uint32_t local = 0;
  for (int item = blockIdx.x; item < total; item += gridDim.x, ++local) {
    if (!solo && (int)(local & 1u) != g) continue;
    const uint32_t buf = local & 1u, bph = (local >> 1) & 1u;
    const int ms = local % MS;
    const MetaSlot& m = sh.meta.ring[ms];
    const bool ok = dead || (mbar_wait(&sh.mfull[ms], (local / MS) & 1u) && mbar_wait(&sh.tfull[buf], bph));
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0 && !dead) atomicOr(s.status, ST_TIMEOUT);
      dead = true;
    }
    float f = 0.0f;
    if (!dead) {
      tc_fence_after();
      float rc[4];
      int xi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = q * 32 + g4 + 8 * u;
        rc[u] = (KIND == K_GAUSS) ? m.row[0][r] * negc : m.row[0][r];
        xi[u] = __float_as_int(m.row[1][r]);
      }
      float2 acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = make_float2(0.0f, 0.0f);
      const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + buf * TNV;
      const int pc0 = solo ? (2 * g + h) * (TNV / 4) : h * (TNV / 2);   // first column of this part
      const int nch = (solo ? TNV / 4 : TNV / 2) / CW;
      float v0[4 * NB], v1[4 * NB];
      for (int ch = 0; ch < nch; ++ch) {
        chunk_load<NB>(tq + pc0 + ch * CW, v0, v1);
        if (!solo && ch == nch - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.tempty[buf]);     // the accumulator is free again
        }
        chunk_math<KIND, NB>(v0, v1, m, pc0 + ch * CW + c2, rc, xi, negc, coef0, degree, acc);
      }
      if (!solo) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.mempty[ms]);        // this warp is done with the slot
      }
      // row sums: the four lanes of a group hold the same rows, different columns
      float fr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        fr[u] = acc[u].x + acc[u].y;
        fr[u] += __shfl_xor_sync(0xffffffffu, fr[u], 1);
        fr[u] += __shfl_xor_sync(0xffffffffu, fr[u], 2);
      }
      const int us = lane & 3;
      f = us == 0 ? fr[0] : (us == 1 ? fr[1] : (us == 2 ? fr[2] : fr[3]));   // row rq
    }
    const int row = (item % R) * TM + q * 32 + rq;
    if (solo) {
      const int P = 2 * g + h;
      if (P > 0) sh.red[((P - 1) * 4 + q) * 32 + rq] = f;
      asm volatile("bar.sync %0, 128;" ::"r"(9 + q) : "memory");
      if (P == 0 && !dead && row < rows) {
        f += sh.red[(0 * 4 + q) * 32 + rq];
        f += sh.red[(1 * 4 + q) * 32 + rq];
        f += sh.red[(2 * 4 + q) * 32 + rq];
        s.part[(int64_t)(item / R) * s.bpad + row] = f;
      }
    } else {
      float* slot = sh.red + ((g * 2 + (int)((local >> 1) & 1u)) * 4 + q) * 32;
      if (h == 1) slot[rq] = f;
      asm volatile("bar.sync %0, 64;" ::"r"(1 + g * 4 + q) : "memory");
      if (h == 0 && !dead && row < rows) s.part[(int64_t)(item / R) * s.bpad + row] = f + slot[rq];
    }
  }
}

// MODE 0: distance pass (A = batch tile, B = support tile, one FP32 partial per row).
// MODE 1: window pass (A and B = support rows of one center; four sums per item:
//         FP32 within a warp, FP64 across the eight epilogue warps).
// Items are dealt round-robin to the persistent CTAs. Splitting a tile along
// its columns needs no merge because both passes only sum over columns, so
// narrower tiles (TNV = 64) are how the window pass gets enough items.
//
// Distance pass metadata: a tile starts on a multiple of 4 support rows and
// support weights are 0 outside the windows, so the column metadata of an
// item (||y||^2, w, data index) and its row metadata (||x||^2, data index)
// are plain contiguous ranges. The producer copies them with bulk async
// copies into a 4-slot ring next to the operand ring; nothing on the
// epilogue's path waits on a global load. The tile descriptors themselves are
// fetched 32 items at a time, one per producer lane.
template <int KIND, int MODE, int OP, int TNV>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_dist_tc(Dev s, int rows, const __grid_constant__ CUtensorMap tmA,
              const __grid_constant__ CUtensorMap tmB) {
  constexpr bool X3 = OP == OP_X3;
  constexpr int KSE = OP == OP_TF32 ? 32 : KS;   // operand elements per slice row
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Shared& sh = *reinterpret_cast<Shared*>(smem + RING_BYTES);
  constexpr int NST = Ring<X3, TNV>::stages;
  constexpr int SB = Ring<X3, TNV>::bytes;
  constexpr int BB = Ring<X3, TNV>::b_bytes;
  constexpr uint32_t TMEM_COLS = 2 * TNV;        // two accumulators (double buffering)
  constexpr uint32_t IDESC = idesc<TNV, OP>();
  constexpr uint32_t META_BYTES = 3 * TNV * 4 + 2 * TM * 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&sh.full[i], 1);
      mbar_init(&sh.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sh.tfull[i], 1);
      mbar_init(&sh.tempty[i], MODE == 0 ? NEPI / 2 : NEPI);   // distance pass: one group per buffer
    }
    for (int i = 0; i < MS; ++i) {
      mbar_init(&sh.mfull[i], 1);
      mbar_init(&sh.mempty[i], NEPI / 2);
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
  const int R = (rows + TM - 1) / TM;
  const int nks = s.dp / KSE;

  // Distance pass with s.pre_b (set per launch when the kernel just ahead, the
  // batch gather or this pass itself, writes none of it): before the
  // grid-dependency wait the producer fetches the descriptors of its first 32
  // items (one per lane) and stages the B tiles of its first item's first
  // stages and that item's column norms and indices. They come from the sort,
  // plan and row moves of earlier steps. The column weights (written by the
  // previous step's weight update, which may still be running beside the
  // gather), the batch rows and their metadata follow after the wait.
  int npre = 0;                                  // first-item stages whose B tile is already on its way
  int pya_pre = 0, pyb_pre = 0;                  // this lane's first-round item: its A and B rows
  bool desc_pre = false;
  if constexpr (MODE == 0) {
    if (warp == 0 && s.pre_b) {
      const int tot0 = R * (*s.ntiles);
      const int mine0 = (int)blockIdx.x + lane * (int)gridDim.x;
      if (mine0 < tot0) pyb_pre = s.tiles[mine0 / R].row0;
      desc_pre = true;
      const int yb0 = __shfl_sync(0xffffffffu, pyb_pre, 0);
      if (lane == 0 && (int)blockIdx.x < tot0) {
        MetaSlot& m = sh.meta.ring[0];
        mbar_expect_tx(&sh.mfull[0], META_BYTES);   // covers the row metadata issued after the wait
        bulk_load(m.col[0], s.yn + yb0, TNV * 4, &sh.mfull[0]);
        bulk_load(m.col[2], s.yi + yb0, TNV * 4, &sh.mfull[0]);
        npre = nks < NST ? nks : NST;
        for (int sl = 0; sl < npre; ++sl) {
          uint8_t* a = smem + sl * SB;
          mbar_expect_tx(&sh.full[sl], SB);         // covers the A tile issued after the wait
          if constexpr (X3) {
            tma_load_2d(a + 2 * A_BYTES, &tmB, &sh.full[sl], sl * KSE, yb0);
            tma_load_2d(a + 2 * A_BYTES + BB, &tmB, &sh.full[sl], s.dp + sl * KSE, yb0);
          } else {
            tma_load_2d(a + A_BYTES, &tmB, &sh.full[sl], sl * KSE, yb0);
          }
        }
      }
      npre = __shfl_sync(0xffffffffu, npre, 0);
    }
  } else {
    // window pass: its pair list and plans come from the sort/plan kernel two
    // launches back (the row moves just ahead write neither), so the producer
    // fetches its first 32 pair descriptors before the wait
    if (warp == 0) {
      const int mine0 = (int)blockIdx.x + lane * (int)gridDim.x;
      if (mine0 < *s.nwpairs) {
        const PairTile pt = pair_tile<TNV>(s, mine0);
        pya_pre = (int)(pt.base + pt.rs);
        pyb_pre = (int)(pt.base + pt.cs);
      }
      desc_pre = true;
    }
  }
  KKM_GRID_DEP_WAIT();   // everything above reads only data of earlier steps
  KKM_LAUNCH_DEPENDENTS();   // the next kernel may set itself up; it waits before reading our output


  const int total = (MODE == 0) ? R * (*s.ntiles) : *s.nwpairs;

  if (warp == 0) {
    // ------------------------------------------------------- producer (one warp)
    bool ok = true;
    uint32_t it = 0, local = 0, mi = 0;          // fills issued, items visited, metadata copies issued
    int pya = 0, pyb = 0;                        // this lane's prefetched item: A and B row
    for (int item = blockIdx.x; item < total; item += gridDim.x, ++local) {
      if ((local & 31u) == 0) {                  // descriptors of the next 32 items
        const int mine = item + lane * gridDim.x;
        if (mine < total) {
          if constexpr (MODE == 0) {
            pya = (mine % R) * TM;
            pyb = (local == 0 && desc_pre) ? pyb_pre : s.tiles[mine / R].row0;
          } else if (local == 0 && desc_pre) {
            pya = pya_pre;
            pyb = pyb_pre;
          } else {
            const PairTile pt = pair_tile<TNV>(s, mine);
            pya = (int)(pt.base + pt.rs);
            pyb = (int)(pt.base + pt.cs);
          }
        }
      }
      const int ya = __shfl_sync(0xffffffffu, pya, local & 31u);
      const int yb = __shfl_sync(0xffffffffu, pyb, local & 31u);
      if (lane == 0) {
        if constexpr (MODE == 0) {
          const int ms = local % MS;
          if (!mbar_wait(&sh.mempty[ms], ((local / MS) & 1u) ^ 1u)) ok = false;
          if (ok) {
            MetaSlot& m = sh.meta.ring[ms];
            if (local != 0 || npre == 0) {             // else norms and indices staged before the wait
              mbar_expect_tx(&sh.mfull[ms], META_BYTES);
              bulk_load(m.col[0], s.yn + yb, TNV * 4, &sh.mfull[ms]);
              bulk_load(m.col[2], s.yi + yb, TNV * 4, &sh.mfull[ms]);
            }
            bulk_load(m.col[1], s.w32 + yb, TNV * 4, &sh.mfull[ms]);
            bulk_load(m.row[0], s.xbn + ya, TM * 4, &sh.mfull[ms]);
            bulk_load(m.row[1], s.xbi + ya, TM * 4, &sh.mfull[ms]);
            ++mi;
          }
        }
        for (int sl = 0; ok && sl < nks; ++sl, ++it) {
          const int st = it % NST;
          const uint32_t ph = (it / NST) & 1u;
          if (!mbar_wait(&sh.empty[st], ph ^ 1u)) { ok = false; break; }
          const int x = sl * KSE;
          uint8_t* a = smem + st * SB;
          const bool pre = local == 0 && sl < npre;   // B tile and expected bytes issued before the wait
          if (!pre) mbar_expect_tx(&sh.full[st], SB);
          if constexpr (X3) {   // stage layout: A_hi | A_lo | B_hi | B_lo
            tma_load_2d(a, &tmA, &sh.full[st], x, ya);
            tma_load_2d(a + A_BYTES, &tmA, &sh.full[st], s.dp + x, ya);
            if (!pre) {
              tma_load_2d(a + 2 * A_BYTES, &tmB, &sh.full[st], x, yb);
              tma_load_2d(a + 2 * A_BYTES + BB, &tmB, &sh.full[st], s.dp + x, yb);
            }
          } else {              // stage layout: A | B
            tma_load_2d(a, &tmA, &sh.full[st], x, ya);
            if (!pre) tma_load_2d(a + A_BYTES, &tmB, &sh.full[st], x, yb);
          }
        }
      }
      if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
    }
    if (lane == 0) {
      // the copies in flight must land before the CTA may exit: the last fill
      // of every stage, and the metadata of the last MS items
      for (uint32_t q = (it > (uint32_t)NST ? it - NST : 0u); q < it; ++q)
        if (!mbar_wait(&sh.full[q % NST], (q / NST) & 1u)) ok = false;
      if constexpr (MODE == 0)
        for (uint32_t q = (mi > (uint32_t)MS ? mi - MS : 0u); q < mi; ++q)
          if (!mbar_wait(&sh.mfull[q % MS], (q / MS) & 1u)) ok = false;
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
            for (int k = 0; k < 4; ++k) {
              mma_op<OP>(d, sw128_desc(a0 + 32u * k), sw128_desc(bhi + 32u * k), IDESC, (sl | k) != 0 ? 1u : 0u);
              mma_op<OP>(d, sw128_desc(a0 + 32u * k), sw128_desc(blo + 32u * k), IDESC, 1u);
              mma_op<OP>(d, sw128_desc(alo + 32u * k), sw128_desc(bhi + 32u * k), IDESC, 1u);
            }
          } else {
            const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
            for (int k = 0; k < 4; ++k)   // four 32-byte K steps per 128-byte slice row
              mma_op<OP>(d, sw128_desc(a0 + 32u * k), sw128_desc(b0 + 32u * k), IDESC, (sl | k) != 0 ? 1u : 0u);
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
  } else if constexpr (MODE == 0) {
    // ---------------------------------------------------------------- epilogue
    dist_epilogue<KIND, TNV>(s, sh, tmem, total, R, rows, warp, lane);
  } else {
    // ---------------------------------------------------------------- epilogue
    // NEPI warps, NH per TMEM lane quadrant: warp e = warp - 2 reads lanes
    // 32*(warp % 4).. (the rows of quadrant q) and columns [h*C, h*C + C) of the
    // accumulator, h = e / 4.
    const int e = warp - 2;
    const int q = warp & 3;
    const int h = e >> 2;
    constexpr int C = TNV / NH;                  // accumulator columns of this warp
    constexpr int NB = C / 8;                    // 8-column blocks per TMEM load
    const int cbase = h * C;
    // this thread's rows inside the quadrant: g4 + 8u (u = 0..3); its columns:
    // cbase + 8j + c2 and the next one (j = 0..NB-1)
    const int g4 = lane >> 2, c2 = 2 * (lane & 3);
    const float negc = s.negc;
    const float coef0 = (float)s.coef0;
    const int degree = s.degree;
    bool dead = false;                           // a wait ran out: skip the work, keep the barriers
    uint32_t local = 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x, ++local) {
      const uint32_t buf = local & 1u, bph = (local >> 1) & 1u;
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + buf * TNV + cbase;
      {
        // window pass: this warp loads its own metadata; the loads overlap the MMAs
        float (*mw)[32] = sh.meta.warp[e];
        __syncwarp();
        const PairTile pt = pair_tile<TNV>(s, item);
        load_pair_meta<KIND, TNV>(s, pt, cbase, mw, lane);
        // rows past the range are still rows of the region: their ||y||^2 matches
        // the operand the MMA read, so every kernel value stays finite
        float rc[4], wp[4];
        int xi[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = q * 32 + g4 + 8 * u;
          const int64_t p = pt.base + pt.rs + r;
          rc[u] = (KIND == K_GAUSS) ? s.yn[p] * negc : s.yn[p];
          xi[u] = s.yi[p];
          // kind 0 rows carry their weight, kind 1 rows count once (0 past the range)
          wp[u] = r < pt.rrem ? (pt.kind == 0 ? s.w32[p] : 1.0f) : 0.0f;
        }
        __syncwarp();
        const bool ok = dead || mbar_wait(&sh.tfull[buf], bph);
        if (__any_sync(0xffffffffu, !ok)) {
          if (lane == 0 && !dead) atomicOr(s.status, ST_TIMEOUT);
          dead = true;
        }
        float sA = 0.0f, sB = 0.0f, sE = 0.0f;
        if (!dead) {
          tc_fence_after();
          float v0[4 * NB], v1[4 * NB];
          tmem_ld16x256<NB>(taddr, v0);
          tmem_ld16x256<NB>(taddr + (16u << 16), v1);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.tempty[buf]);
          float2 aA[4], aB[4], aE[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) aA[u] = aB[u] = aE[u] = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int j = 0; j < NB; ++j) {
            const int c = 8 * j + c2;
            const float2 cc = *reinterpret_cast<const float2*>(&mw[0][c]);
            const float2 wa = *reinterpret_cast<const float2*>(&mw[1][c]);
            const int2 yi = *reinterpret_cast<const int2*>(&mw[2][c]);
            const float2 wb = *reinterpret_cast<const float2*>(&mw[3][c]);
            const float2 we = *reinterpret_cast<const float2*>(&mw[4][c]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float* vv = (u < 2) ? v0 : v1;
              const int o = 4 * j + 2 * (u & 1);
              const float2 kv = kernel_pair<KIND>(make_float2(vv[o], vv[o + 1]), rc[u], cc, xi[u], yi, negc,
                                                  coef0, degree);
              aA[u] = __ffma2_rn(wa, kv, aA[u]);
              aB[u] = __ffma2_rn(wb, kv, aB[u]);
              aE[u] = __ffma2_rn(we, kv, aE[u]);
            }
          }
          // kind 0: A = w_p sum_{q in W} w_q K, Bdd = w_p sum_{q in D} w_q K, E = w_p sum_{q in B} K
          // kind 1: M = sum_{q in B} K (every valid column of a kind-1 tile is in B), kept in sE
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            sA = fmaf(wp[u], aA[u].x + aA[u].y, sA);
            sB = fmaf(wp[u], aB[u].x + aB[u].y, sB);
            sE = fmaf(wp[u], aE[u].x + aE[u].y, sE);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            sA += __shfl_xor_sync(0xffffffffu, sA, o);
            sB += __shfl_xor_sync(0xffffffffu, sB, o);
            sE += __shfl_xor_sync(0xffffffffu, sE, o);
          }
        }
        // the warps' sums meet in shared memory (slot by item parity); one
        // thread per sum adds them in a fixed order and writes the item's four sums
        float (*red)[4] = sh.wred[local & 1u];
        if (lane == 0) {
          const bool k0 = pt.kind == 0;
          red[e][0] = k0 ? sA : 0.0f;
          red[e][1] = k0 ? sB : 0.0f;
          red[e][2] = k0 ? sE : 0.0f;
          red[e][3] = k0 ? 0.0f : sE;
        }
        asm volatile("bar.sync 5, %0;" ::"n"(32 * NEPI) : "memory");
        if (e == 0 && lane < 4 && !dead) {
          double v = 0.0;
#pragma unroll
          for (int w = 0; w < NEPI; ++w) v += (double)red[w][lane];
          s.wpart[(int64_t)item * 4 + lane] = v;
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

template <int KIND, int MODE, int OP, int TNV>
cudaError_t launch_form(const Dev& s, const CUtensorMap& a, const CUtensorMap& b, int rows, cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  {
    const cudaError_t e = smem_limit_once(k_dist_tc<KIND, MODE, OP, TNV>, SMEM_BYTES, attr);
    if (e != cudaSuccess) return e;
  }
  // one CTA per SM, but never more CTAs than the most items this launch can
  // have: small runs then leave SMs free for the kernels of other runs
  const int64_t most = MODE == 0 ? (int64_t)((rows + TM - 1) / TM) * s.max_tiles : (int64_t)s.max_pairs;
  const int grid = (int)(most < s.num_sms ? (most > 0 ? most : 1) : s.num_sms);
  return launch_pdl(k_dist_tc<KIND, MODE, OP, TNV>, dim3(grid), dim3(NTHREADS), SMEM_BYTES, st, s, rows, a, b);
}

template <int MODE, int OP, int TNV>
cudaError_t launch_kind(const Dev& s, const CUtensorMap& a, const CUtensorMap& b, int rows, cudaStream_t st) {
  switch (s.kind) {
    case K_GAUSS: return launch_form<K_GAUSS, MODE, OP, TNV>(s, a, b, rows, st);
    case K_LAPLACE: return launch_form<K_LAPLACE, MODE, OP, TNV>(s, a, b, rows, st);
    case K_LINEAR: return launch_form<K_LINEAR, MODE, OP, TNV>(s, a, b, rows, st);
    default: return launch_form<K_POLY, MODE, OP, TNV>(s, a, b, rows, st);
  }
}

// maps: [0] batch rows, 128-row boxes; support rows with [1] 128-row, [2] 64-row, [3] 256-row boxes
template <int MODE, int TNV>
cudaError_t launch_mode(const Dev& s, const void* maps_in, int rows, cudaStream_t st) {
  const CUtensorMap* m = static_cast<const CUtensorMap*>(maps_in);
  const CUtensorMap& a = (MODE == 0) ? m[0] : m[1];
  const CUtensorMap& b = (TNV == 256) ? m[3] : (TNV == 128) ? m[1] : m[2];
  switch (s.form) {
    case FORM_BF16X3: return launch_kind<MODE, OP_X3, TNV>(s, a, b, rows, st);
    case FORM_TF32: return launch_kind<MODE, OP_TF32, TNV>(s, a, b, rows, st);
    default: return launch_kind<MODE, OP_BF16, TNV>(s, a, b, rows, st);
  }
}

}  // namespace

// Tensor maps of the batch rows and the support store: 2-D tensors of ld
// columns (BF16, or FP32 for the TF32 form), boxes of one 128-byte row of
// columns (64 BF16 or 32 FP32) x 128 (64, 256) rows, 128-byte swizzle.
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
  const bool f32 = s.form == FORM_TF32;
  void* xb = f32 ? (void*)s.xb32 : (void*)s.xbh;
  void* yb = f32 ? (void*)s.y32 : (void*)s.ybh;
  const int esz = f32 ? 4 : 2;
  struct { void* base; uint64_t rows; uint32_t box_rows; } ops[4] = {
      {xb, (uint64_t)s.bpad, 128u}, {yb, (uint64_t)srows, 128u}, {yb, (uint64_t)srows, 64u},
      {yb, (uint64_t)srows, 256u}};
  for (int i = 0; i < 4; ++i) {
    cuuint64_t dims[2] = {(cuuint64_t)s.ld, (cuuint64_t)ops[i].rows};
    cuuint64_t strides[1] = {(cuuint64_t)s.ld * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), ops[i].box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&maps[i], f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        ops[i].base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_dist_tc(const Dev& s, const void* maps, int rows, cudaStream_t st, bool stage_early) {
  if (rows <= 0) return cudaSuccess;
  // staging before the grid-dependency wait is only safe when the kernel just
  // ahead writes none of what it stages (the gather, or this pass itself)
  Dev d = s;
  d.pre_b = (stage_early && s.pre_b) ? 1 : 0;
  if (d.tn == 64) return launch_mode<0, 64>(d, maps, rows, st);
  if (d.tn == 256) return launch_mode<0, 256>(d, maps, rows, st);
  return launch_mode<0, 128>(d, maps, rows, st);
}

cudaError_t launch_wgram_tc(const Dev& s, const void* maps, cudaStream_t st) {
  return launch_mode<1, 64>(s, maps, 0, st);
}

}  // namespace kkm
