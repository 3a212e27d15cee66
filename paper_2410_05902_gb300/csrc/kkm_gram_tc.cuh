#pragma once
// tcgen05 / TMA form of the two Gram passes (BF16, split-BF16 and TF32 products).
//
// One persistent CTA per SM walks the work items round-robin. For each item
//   G = A B^T            tcgen05.mma kind::f16 (BF16) or kind::tf32 (TF32),
//                        FP32 in TMEM; operands streamed by TMA through a
//                        192 KB ring of 128B-swizzled shared-memory slices
//   K = kernel(||a||^2 + ||b||^2 - 2G)      in registers after tcgen05.ld
//   weighted row sums of K                  FP32 per row, see below
// The split form (x = hi + lo) runs the K loop three times over the slice
// pairs (hi,hi), (hi,lo), (lo,hi) into the same accumulator.
//
// Distance pass (mode 0): an item is (128-row batch tile, TNV-row support tile
// of one center; TNV = 256 by default, 64 or 128 on request), and it writes
// part[tile][x] = sum_y w_y K(x, y), one partial per row and tile.
// Window pass (mode 1, the norm recurrence of Sec. 4 with the drops of
// Eq. (1)): an item is (128 support rows, 128 support rows) of one center,
// rows from the dropped prefix D (kind 0) or the new block B (kind 1), and it
// writes four sums per TMEM lane quadrant:
//   kind 0: A = sum_{p in D, q in W} w_p w_q K, Bdd = sum_{p, q in D} w_p w_q K,
//           E = sum_{p in D, q in B} w_p K          (W: the old window)
//   kind 1: M = sum_{p, q in B} K.
//
// Roles: warp 0 issues the operand tiles' TMA copies; warp 1 issues the MMAs
// (one elected lane) and owns the TMEM allocation (up to four accumulators);
// warps 2-17 are the epilogue, four groups of four warps, one warp per TMEM
// lane quadrant; warp 18 stages each item's metadata (norms, weights, data
// indices, and for the window pass the item's row and column ranges) into a
// ring of slots with per-lane 16-byte asynchronous copies. A copy through the
// TMA unit costs the issuing thread a few hundred cycles, so an item takes as
// few of them as possible: its B tile, and its A tile only when the row tile
// changes (the batch tile stays resident while consecutive items share it).
//
// Teams: with four accumulators (64- and 128-column tiles) each group is a
// team and takes every fourth item whole; with two (256-column tiles) two
// groups form a team, take every other item and split its columns, each
// writing its own partial. Either way every waiter on a barrier sees each of
// its phases in order. A run with fewer than NTEAM items per SM runs every
// item on all four groups, each on a quarter of the columns, and the groups'
// sums meet in shared memory (chosen per run, so that a run's results do not
// depend on how a launch splits its items).
//
// Gaussian kernel values without a per-element row term: with rc = -log2(e)
// ||x||^2 / kappa and t = (2 log2(e) / kappa) g - log2(e) ||y||^2 / kappa,
//   K(x, y) = 2^(rc + t) = 2^rc 2^t,
// so a row's weighted sum is 2^rc sum_y w_y 2^t: one FMA for t, one MUFU ex2
// and one FMA into the sum per element. t <= -rc, so 2^t stays finite while
// -rc <= 100; a warp whose rows pass that bound uses the full exponent.
//
// Every mbarrier wait is bounded. A wait that runs out sets ST_TIMEOUT and
// makes the role stop. On the way out the producer waits for its last copies
// to land and the MMA warp waits for its last MMAs, so TMEM is freed only once
// nothing is in flight.
#include <cstddef>
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
constexpr int RING_BYTES = 192 * 1024;          // shared memory for the operands
constexpr int STAGES = 16;                      // most stages any layout uses
constexpr int A_RES_MAX = 96 * 1024;            // largest batch tile kept resident (all its slices)
// Operand layout, per launch (Layout below). A slice is 128 bytes of every
// operand row: 64 BF16 or 32 TF32 values. The split form holds hi and lo
// tiles of each operand and runs 12 MMAs per slice (hi.hi, hi.lo, lo.hi).
//   resident A: the A tile's slices stay in shared memory while consecutive
//               items share it (same batch or support row tile); a stage
//               holds one slice of the B tile. A is reloaded only when the
//               row tile changes.
//   streaming:  (A too large to keep) a stage holds one slice of A and B.
constexpr int NEPI = 16;                         // epilogue warps (2 .. 17): four on each scheduler
constexpr int NGRP = 4;                          // epilogue groups, one warp per TMEM lane quadrant each
constexpr int MWARP = 2 + NEPI;                  // the metadata warp
constexpr int NTHREADS = 32 * (MWARP + 1);      // TMA warp, MMA warp, epilogue, metadata warp
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // 2 s per wait
constexpr float ROW_EXP_FLOOR = -100.0f;        // Gaussian: rc at or above it keeps 2^t finite
#ifndef DIST_NB
#define DIST_NB 2                                // distance-pass epilogue: 8-column blocks per TMEM chunk
#endif

// TMEM accumulators (TNV columns each, at most 512 columns), teams of
// groups (one per accumulator), groups per team (= partials per tile), and
// metadata slots
template <int TNV> struct Geo {
  static constexpr int NACC = 512 / TNV < 4 ? 512 / TNV : 4;
  static constexpr int NTEAM = NACC < NGRP ? NACC : NGRP;
  static constexpr int GPT = NGRP / NTEAM;
  static constexpr int MS = TNV == 256 ? 4 : 8;
  static constexpr uint32_t TMEM_COLS = (uint32_t)(NACC * TNV);
};
constexpr uint32_t META_ARRIVALS = 33;           // 32 lanes' asynchronous arrivals + lane 0's release

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y);

// Operand layout of one launch (identical in every role). Byte offsets are
// from the 1024-aligned start of the operand region; every tile starts on a
// multiple of 1024 bytes, as the 128-byte swizzle needs. A tile's slices are
// laid out hi slices first, then (split form) lo slices.
struct Layout {
  bool res;            // A resident; a stage holds one item's whole B tile
  int nsl;             // slices of one operand tile (nks, twice that for the split form)
  int a_bytes;         // resident A region (res), else 0
  int sb;              // bytes per stage
  int nst;             // stages
};
template <bool X3, int TNV>
__device__ __forceinline__ Layout layout(int nks) {
  constexpr int BT = TNV * KS * 2;              // one B slice (TNV rows x 128 bytes)
  Layout L;
  L.nsl = nks * (X3 ? 2 : 1);
  const int a = L.nsl * A_BYTES, sbr = L.nsl * BT;
  // resident only if the A tile fits and at least two whole B tiles fit beside it
  L.res = a <= A_RES_MAX && (RING_BYTES - a) / sbr >= 2;
  L.a_bytes = L.res ? a : 0;
  L.sb = L.res ? sbr : (X3 ? 2 : 1) * (A_BYTES + BT);   // streaming: one slice of A and B
  const int n = (RING_BYTES - L.a_bytes) / L.sb;
  L.nst = n < STAGES ? n : STAGES;
  return L;
}

// Lane t < n issues slice t of a tile (hi slices, then lo slices at column
// dp) into dst + t * tb: the whole tile leaves in one warp instruction.
__device__ __forceinline__ void tile_issue(int lane, int n, int nks, int dp, int kse, uint8_t* dst, int tb,
                                           const CUtensorMap* tm, uint64_t* bar, int y) {
  if (lane < n) {
    const int x = lane < nks ? lane * kse : dp + (lane - nks) * kse;
    tma_load_2d(dst + lane * tb, tm, bar, x, y);
  }
}

// Instruction descriptor of tcgen05.mma kind::f16 / kind::tf32: D FP32
// (bits 4-5 = 1), A and B BF16 (type 1) or TF32 (type 2) in bits 7-9 and
// 10-12, both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in
// bits 24-28.
template <int N, int OP>
__host__ __device__ constexpr uint32_t idesc() {
  constexpr uint32_t t = OP == OP_TF32 ? 2u : 1u;
  return (1u << 4) | (t << 7) | (t << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// Window-pass item: row and column ranges relative to the item's first row
// and column (both 4-aligned positions of the center's region).
struct ItemDesc {
  int32_t kind;        // 0: rows of D against W and B; 1: rows of B against B
  int32_t rlo, rhi;    // rows [rlo, rhi) of the tile are in the row range
  int32_t dnew;        // columns below dnew are dropped rows (D)
  int32_t told;        // columns below told are the old window W (D included)
  int32_t tnew;        // columns in [told, tnew) are the new block B
  int32_t pad0, pad1;
};

// Metadata of one item, copied by the producer. col[0] = ||y||^2, col[1] = w,
// col[2] = data index (bits) of the TNV B rows; row[0] = ||a||^2, row[1] =
// data index, row[2] = w (window pass) of the 128 A rows.
template <int TNV> struct MetaSlot {
  float col[3][TNV];
  float row[3][TM];
  ItemDesc desc;
};

template <int TNV> struct Shared {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t afull;                // resident A tile landed
  uint64_t afree;                // the MMAs on the previous resident A tile are done
  uint32_t anew[STAGES];         // resident A: the stage's item brings a new A tile
  uint64_t tfull[4];
  uint64_t tempty[4];
  uint64_t mfull[8];
  uint64_t mempty[8];
  uint64_t mma_done;
  uint32_t tmem_base;
  uint32_t pad;
  long long gtot;                // run groups: the class's weighted item total
  int gseg[4];                   // run groups: the next segment (run, first item, end item)
  alignas(16) Dev gdev;          // run groups: the segment's run (a shared copy: no reloads after global stores)
  alignas(16) MetaSlot<TNV> ring[Geo<TNV>::MS];   // 16-byte asynchronous copies land here
  union alignas(16) {
    float red[2][NGRP][4][32];     // distance pass, all groups on one item: row sums (item parity, group, quadrant, row)
    double wred[2][NGRP][4][4];    // window pass, the same: the four sums
    double wq[NGRP][2][4][4];      // window pass, a group per item: (group, buffer, quadrant, sum)
  } x;
};

template <int TNV> constexpr int smem_bytes() { return 1024 + RING_BYTES + (int)sizeof(Shared<TNV>); }
// the metadata slots take 16-byte cp.async copies: each slot, and every array in it, on a 16-byte boundary
static_assert(offsetof(Shared<64>, ring) % 16 == 0 && offsetof(Shared<128>, ring) % 16 == 0 &&
                  offsetof(Shared<256>, ring) % 16 == 0 && sizeof(MetaSlot<64>) % 16 == 0 &&
                  sizeof(MetaSlot<128>) % 16 == 0 && sizeof(MetaSlot<256>) % 16 == 0,
              "metadata ring misaligned for 16-byte copies");
static_assert(smem_bytes<128>() <= 232448 && smem_bytes<256>() <= 232448 && smem_bytes<64>() <= 232448,
              "shared memory per CTA");

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

__device__ __forceinline__ void mbar_inval(uint64_t* b) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}

// dist_tc_body's lifecycle flags: allocate TMEM on entry, free it on exit,
// invalidate the barriers before initialising them (a later segment)
constexpr int TC_ALLOC = 1, TC_FREE = 2, TC_REINIT = 4;

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
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns = WAIT_LIMIT_NS) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(b, parity)) return true;
    if (globaltimer() - t0 > limit_ns) return false;
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

// Kernel values of one row against two columns from their Gram entries g, for
// the kernels without the factored Gaussian form: the Laplacian, the linear
// and the polynomial kernel, and the Gaussian with its full exponent.
// Gaussian: rc = ||x||^2 * negc and cc = ||y||^2 * negc (negc = -log2(e)/kappa),
//           K = 2^(rc + cc - 2 negc g).
// Laplacian: rc = ||x||^2, cc = ||y||^2, K = 2^(negc * sqrt(max(D^2, 0))).
// Both give exactly 1 when the two rows are the same data point (K(x,x) = 1).
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


// 16-byte asynchronous copy global -> shared through the LSU (not the TMA
// unit), and the asynchronous arrive that follows this thread's earlier ones.
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// A chunk is 8 NB accumulator columns of a warp's 32 rows: two 16-lane loads.
// Thread t receives, for block j (8 columns), rows g4 = t/4 and g4 + 8 from
// the first load (v0[4j..4j+3]) and g4 + 16, g4 + 24 from the second (v1),
// columns 8j + 2(t%4) and the next one. Row u of the thread (0..3) is
// g4 + 8u: u = 0, 1 in v0 at offset 4j + 2u, u = 2, 3 in v1 at 4j + 2(u-2).
template <int NB>
__device__ __forceinline__ void chunk_load(uint32_t taddr, float (&v0)[4 * NB], float (&v1)[4 * NB]) {
  tmem_ld16x256<NB>(taddr, v0);                 // rows g4, g4 + 8
  tmem_ld16x256<NB>(taddr + (16u << 16), v1);   // rows g4 + 16, g4 + 24
  tmem_wait_ld();
}

// The two loads of a chunk without the wait (the caller waits before reading).
template <int NB>
__device__ __forceinline__ void chunk_issue(uint32_t taddr, float (&v0)[4 * NB], float (&v1)[4 * NB]) {
  tmem_ld16x256<NB>(taddr, v0);
  tmem_ld16x256<NB>(taddr + (16u << 16), v1);
}

template <int NB>
__device__ __forceinline__ float2 gram2(const float (&v0)[4 * NB], const float (&v1)[4 * NB], int j, int u) {
  const int o = 4 * j + 2 * (u & 1);
  return u < 2 ? make_float2(v0[o], v0[o + 1]) : make_float2(v1[o], v1[o + 1]);
}

// Distance pass, Gaussian: acc[u] += w_y 2^t over the chunk's columns, with
// t = C2 g + cc (FAST, the row term 2^rc applied to the row sum later) or
// t = C2 g + cc + rc (full exponent). c is this thread's first column.
template <int NB, bool FAST>
__device__ __forceinline__ void gauss_chunk(const float (&v0)[4 * NB], const float (&v1)[4 * NB],
                                            const float* __restrict__ yn, const float* __restrict__ w, int c,
                                            float negc, float2 C2, const float (&rc)[4], float2 (&acc)[4]) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const float2 y2 = *reinterpret_cast<const float2*>(yn + c + 8 * j);
    const float2 w2 = *reinterpret_cast<const float2*>(w + c + 8 * j);
    const float2 cc = __fmul2_rn(y2, make_float2(negc, negc));
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 bias = FAST ? cc : __fadd2_rn(cc, make_float2(rc[u], rc[u]));
      const float2 t = __ffma2_rn(gram2<NB>(v0, v1, j, u), C2, bias);
      acc[u] = __ffma2_rn(w2, make_float2(ex2_approx(t.x), ex2_approx(t.y)), acc[u]);
    }
  }
}

// Distance pass, other kernels: acc[u] += w_y K(x_u, y) by kernel_pair.
template <int KIND, int NB>
__device__ __forceinline__ void generic_chunk(const float (&v0)[4 * NB], const float (&v1)[4 * NB],
                                              const float* __restrict__ yn, const float* __restrict__ w,
                                              const float* __restrict__ yi, int c, float negc, float coef0,
                                              int degree, const float (&rc)[4], const int (&xi)[4],
                                              float2 (&acc)[4]) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const float2 y2 = *reinterpret_cast<const float2*>(yn + c + 8 * j);
    const float2 w2 = *reinterpret_cast<const float2*>(w + c + 8 * j);
    const int2 i2 = *reinterpret_cast<const int2*>(yi + c + 8 * j);
    const float2 cc = (KIND == K_GAUSS) ? __fmul2_rn(y2, make_float2(negc, negc)) : y2;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      acc[u] = __ffma2_rn(w2, kernel_pair<KIND>(gram2<NB>(v0, v1, j, u), rc[u], cc, xi[u], i2, negc, coef0,
                                                degree), acc[u]);
  }
}

__device__ __forceinline__ float pick4(const float (&v)[4], int u) {
  return u == 0 ? v[0] : (u == 1 ? v[1] : (u == 2 ? v[2] : v[3]));
}

// Sum of a row's values over the four lanes that hold it (lanes 4r .. 4r+3).
__device__ __forceinline__ float quad_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Range {
  int lo, hi;
};

// Distance-pass epilogue (warps 2-17). Group g = (warp - 2) / 4 takes the
// items of local index = g (mod 4), or, when the CTA has fewer than four
// items, a quarter of the columns of every item. A warp covers its quadrant's
// 32 rows; it releases the accumulator once its last chunk is in registers
// and the metadata slot once its arithmetic is done. Part 0 (the only part,
// or group 0 after the groups' sums meet) writes part[tile][row].
template <int KIND, int TNV>
__device__ __forceinline__ void dist_epilogue(const Dev& s, Shared<TNV>& sh, uint32_t tmem, Range rg, int T,
                                              int rows, int warp, int lane, bool all) {
  constexpr int NACC = Geo<TNV>::NACC, MS = Geo<TNV>::MS, NTEAM = Geo<TNV>::NTEAM, GPT = Geo<TNV>::GPT;
  const int g = (warp - 2) >> 2, q = warp & 3;
  const int g4 = lane >> 2, us = lane & 3, c2 = 2 * us;
  const int rq = g4 + 8 * us;                   // the row this lane reports
  const float negc = s.negc;
  const float2 C2 = make_float2(-2.0f * negc, -2.0f * negc);
  const float coef0 = (float)s.coef0;
  const int degree = s.degree;
  // Team team = g / GPT takes the items of local index = team (mod NTEAM),
  // using accumulator `team` on each, and its group h = g % GPT the columns
  // [h TNV / GPT, (h+1) TNV / GPT), written as partial h of the tile. In the
  // all-groups mode (a run with fewer than NTEAM items per SM) every group
  // takes every item (a quarter of the columns) and the quarters of each
  // partial meet in shared memory.
  const int team = g / GPT, h = g % GPT;
  const int ncols = all ? TNV / NGRP : TNV / GPT;
  const int cbeg = all ? g * ncols : h * ncols;
  constexpr int QPP = NGRP / GPT;                // all-mode quarters per partial
  const int ph = all ? g / QPP : h;             // this group's partial
  const bool lead = !all || g % QPP == 0;        // writes the partial and frees the slot and accumulator
  // part[] must hold GPT partials per tile, as the host sized it (Dev::ppt)
  bool dead = s.ppt != GPT;                     // a wait ran out (or bad layout): skip the work, keep the barriers
  if (dead && lane == 0 && warp == 2) atomicOr(s.status, ST_CAPACITY);
  uint32_t local = 0;
  for (int item = rg.lo; item < rg.hi; ++item, ++local) {
    if (!all && (int)(local % NTEAM) != team) continue;
    const uint32_t buf = local % NACC, bph = (local / NACC) & 1u;
    const uint32_t ms = local % MS, mph = (local / MS) & 1u;
    const MetaSlot<TNV>& m = sh.ring[ms];
    const bool ok = dead || (mbar_wait(&sh.mfull[ms], mph) && mbar_wait(&sh.tfull[buf], bph));
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
      const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + buf * TNV + cbeg;
      bool fast = false;
      if constexpr (KIND == K_GAUSS)
        fast = __all_sync(0xffffffffu, fminf(fminf(rc[0], rc[1]), fminf(rc[2], rc[3])) >= ROW_EXP_FLOOR);
      // chunks of CW columns, two in flight: the next chunk's TMEM loads are
      // issued before the current chunk's arithmetic and waited for after it
      // (tcgen05.wait::ld waits for every load in flight, so a chunk's
      // arithmetic is what hides the next chunk's load latency)
      auto release = [&]() {                    // the accumulator is free again
        if (!all) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.tempty[buf]);
        }
      };
      auto run = [&](auto nbt) {
        constexpr int NB = decltype(nbt)::value, CW = 8 * NB;
        const int nch = ncols / CW;
        auto math = [&](const float (&w0)[4 * NB], const float (&w1)[4 * NB], int ch) {
          const int c = cbeg + ch * CW + c2;
          if constexpr (KIND == K_GAUSS) {
            if (fast) gauss_chunk<NB, true>(w0, w1, m.col[0], m.col[1], c, negc, C2, rc, acc);
            else gauss_chunk<NB, false>(w0, w1, m.col[0], m.col[1], c, negc, C2, rc, acc);
          } else {
            generic_chunk<KIND, NB>(w0, w1, m.col[0], m.col[1], m.col[2], c, negc, coef0, degree, rc, xi, acc);
          }
        };
        float a0[4 * NB], a1[4 * NB], b0[4 * NB], b1[4 * NB];
        chunk_issue<NB>(tq, a0, a1);
        tmem_wait_ld();
        for (int ch = 0; ch < nch; ch += 2) {
          if (ch + 1 < nch) chunk_issue<NB>(tq + (ch + 1) * CW, b0, b1);
          else release();
          math(a0, a1, ch);
          if (ch + 1 < nch) {
            tmem_wait_ld();
            if (ch + 2 < nch) chunk_issue<NB>(tq + (ch + 2) * CW, a0, a1);
            else release();
            math(b0, b1, ch + 1);
            if (ch + 2 < nch) tmem_wait_ld();
          }
        }
      };
      if (ncols % (8 * DIST_NB) == 0) run(std::integral_constant<int, DIST_NB>{});
      else if (ncols % 32 == 0) run(std::integral_constant<int, 4>{});
      else run(std::integral_constant<int, 2>{});
      float fr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) fr[u] = quad_sum(acc[u].x + acc[u].y);
      f = pick4(fr, us);
      if (KIND == K_GAUSS && fast) f *= ex2_approx(pick4(rc, us));   // the row term 2^rc
    }
    const int row = (item / T) * TM + q * 32 + rq;
    float* out = s.part + ((int64_t)(item % T) * GPT + ph) * s.bpad + row;
    if (!all) {
      if (!dead) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.mempty[ms]);        // this warp is done with the slot
        if (row < rows) *out = f;
      }
    } else {
      float (*red)[4][32] = sh.x.red[local & 1u];
      red[g][q][rq] = f;
      tc_fence_before();
      asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
      if (lead) {
        if (!dead && row < rows) {
          float v = red[g][q][rq];
          for (int o = 1; o < QPP; ++o) v += red[g + o][q][rq];
          *out = v;
        }
        __syncwarp();
        if (lane == 0 && !dead) {
          mbar_arrive(&sh.tempty[buf]);
          mbar_arrive(&sh.mempty[ms]);
        }
      }
    }
  }
}

// Window-pass epilogue: per element K(a, b) once, three weighted column sums
// per row (A: w_q on W, Bdd: w_q on D, E: 1 on B), then per row the weight
// w_p (kind 0) or 1 (kind 1) and an FP64 sum over the warp's 32 rows. A row
// meeting its own copy (same data index) gets K = 1.
template <int KIND, int TNV>
__device__ __forceinline__ void pair_epilogue(const Dev& s, Shared<TNV>& sh, uint32_t tmem, Range rg, int warp,
                                              int lane, bool all) {
  constexpr int NACC = Geo<TNV>::NACC, MS = Geo<TNV>::MS, NTEAM = Geo<TNV>::NTEAM, GPT = Geo<TNV>::GPT;
  const int g = (warp - 2) >> 2, q = warp & 3;
  const int g4 = lane >> 2, us = lane & 3, c2 = 2 * us;
  const float negc = s.negc;
  const float2 C2 = make_float2(-2.0f * negc, -2.0f * negc);
  const float coef0 = (float)s.coef0;
  const int degree = s.degree;
  // teams, halves and the all-groups mode as in dist_epilogue; partial ph
  // of an item is its slot set ((item GPT + ph) 4 + quadrant) of wpart
  const int team = g / GPT, h = g % GPT;
  const int ncols = all ? TNV / NGRP : TNV / GPT;
  const int cbeg = all ? g * ncols : h * ncols;
  constexpr int QPP = NGRP / GPT;
  const int ph = all ? g / QPP : h;
  const bool lead = !all || g % QPP == 0;
  // wpart[] must hold GPT slots of four sums per item, as the host sized it (Dev::wslots)
  bool dead = s.wslots != GPT;
  uint32_t gi = 0;                               // items this group has taken (shared-memory buffer parity)
  if (dead && lane == 0 && warp == 2) atomicOr(s.status, ST_CAPACITY);
  uint32_t local = 0;
  for (int item = rg.lo; item < rg.hi; ++item, ++local) {
    if (!all && (int)(local % NTEAM) != team) continue;
    const uint32_t buf = local % NACC, bph = (local / NACC) & 1u;
    const uint32_t ms = local % MS, mph = (local / MS) & 1u;
    const MetaSlot<TNV>& m = sh.ring[ms];
    const bool ok = dead || (mbar_wait(&sh.mfull[ms], mph) && mbar_wait(&sh.tfull[buf], bph));
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0 && !dead) atomicOr(s.status, ST_TIMEOUT);
      dead = true;
    }
    double tA = 0.0, tB = 0.0, tE = 0.0;
    int kind = 0;
    if (!dead) {
      tc_fence_after();
      const ItemDesc dsc = m.desc;
      kind = dsc.kind;
      float rc[4], wp[4], self[4];
      int xi[4];
      bool fast = false;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = q * 32 + g4 + 8 * u;
        rc[u] = (KIND == K_GAUSS) ? m.row[0][r] * negc : m.row[0][r];
        xi[u] = __float_as_int(m.row[1][r]);
        const bool in = r >= dsc.rlo && r < dsc.rhi;
        wp[u] = in ? (dsc.kind == 0 ? m.row[2][r] : 1.0f) : 0.0f;
      }
      if constexpr (KIND == K_GAUSS)
        fast = __all_sync(0xffffffffu, fminf(fminf(rc[0], rc[1]), fminf(rc[2], rc[3])) >= ROW_EXP_FLOOR);
#pragma unroll
      for (int u = 0; u < 4; ++u) self[u] = fast ? ex2_approx(-rc[u]) : 1.0f;   // 2^t of K = 1
      float2 aA[4], aB[4], aE[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) aA[u] = aB[u] = aE[u] = make_float2(0.0f, 0.0f);
      const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + buf * TNV + cbeg;
      auto run = [&](auto nbt) {
        constexpr int NB = decltype(nbt)::value;
        constexpr int CW = 8 * NB;
        const int nch = ncols / CW;
        float v0[4 * NB], v1[4 * NB];
        for (int ch = 0; ch < nch; ++ch) {
          chunk_load<NB>(tq + ch * CW, v0, v1);
          if (!all && ch == nch - 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.tempty[buf]);
          }
#pragma unroll
          for (int j = 0; j < NB; ++j) {
            const int c = cbeg + ch * CW + 8 * j + c2;
            const float2 y2 = *reinterpret_cast<const float2*>(&m.col[0][c]);
            const float2 w2 = *reinterpret_cast<const float2*>(&m.col[1][c]);
            const int2 i2 = *reinterpret_cast<const int2*>(&m.col[2][c]);
            const float2 cc = (KIND == K_GAUSS) ? __fmul2_rn(y2, make_float2(negc, negc)) : y2;
            const float2 wa = make_float2(c < dsc.told ? w2.x : 0.0f, c + 1 < dsc.told ? w2.y : 0.0f);
            const float2 wb = make_float2(c < dsc.dnew ? w2.x : 0.0f, c + 1 < dsc.dnew ? w2.y : 0.0f);
            const float2 we = make_float2(c >= dsc.told && c < dsc.tnew ? 1.0f : 0.0f,
                                          c + 1 >= dsc.told && c + 1 < dsc.tnew ? 1.0f : 0.0f);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float2 gg = gram2<NB>(v0, v1, j, u);
              float2 kv;
              if (KIND == K_GAUSS && fast) {
                const float2 t = __ffma2_rn(gg, C2, cc);
                kv.x = xi[u] == i2.x ? self[u] : ex2_approx(t.x);
                kv.y = xi[u] == i2.y ? self[u] : ex2_approx(t.y);
              } else {
                kv = kernel_pair<KIND>(gg, rc[u], cc, xi[u], i2, negc, coef0, degree);
                // columns outside every range contribute nothing (unbounded kernels included)
                kv.x = (wa.x != 0.0f || wb.x != 0.0f || we.x != 0.0f) ? kv.x : 0.0f;
                kv.y = (wa.y != 0.0f || wb.y != 0.0f || we.y != 0.0f) ? kv.y : 0.0f;
              }
              aA[u] = __ffma2_rn(wa, kv, aA[u]);
              aB[u] = __ffma2_rn(wb, kv, aB[u]);
              aE[u] = __ffma2_rn(we, kv, aE[u]);
            }
          }
        }
      };
      run(std::integral_constant<int, 2>{});     // 16-column chunks: three sets of row sums stay in registers
      float fa[4], fb[4], fe[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        fa[u] = quad_sum(aA[u].x + aA[u].y);
        fb[u] = quad_sum(aB[u].x + aB[u].y);
        fe[u] = quad_sum(aE[u].x + aE[u].y);
      }
      // this lane's row rq = g4 + 8 us: its row term and row weight, summed over the warp in FP64
      const float fac = (KIND == K_GAUSS && fast) ? ex2_approx(pick4(rc, us)) : 1.0f;
      const double wr = (double)pick4(wp, us) * (double)fac;
      tA = warp_sum64(wr * (double)pick4(fa, us));
      tB = warp_sum64(wr * (double)pick4(fb, us));
      tE = warp_sum64(wr * (double)pick4(fe, us));
    }
    // The item's four sums (A, Bdd, E for kind 0; M for kind 1) over its 128
    // rows: the quadrant warps' FP64 sums meet in shared memory and one warp
    // adds them in quadrant order (group by group in the all-groups mode).
    double* out = s.wpart + ((int64_t)item * GPT + ph) * 4;
    const bool first = ((warp - 2) & 3) == 0;   // the group's first warp
    if (!all) {
      double (*wq)[4] = sh.x.wq[g][gi & 1u];
      if (lane == 0) {
        wq[q][0] = tA;
        wq[q][1] = tB;
        wq[q][2] = tE;
      }
      __syncwarp();
      if (lane == 0 && !dead) mbar_arrive(&sh.mempty[ms]);
      asm volatile("bar.sync %0, 128;" ::"r"(2 + g) : "memory");   // every warp of the group, dead or not
      if (first && !dead && lane < 4) {
        const int src = lane == 3 ? 2 : lane;   // M is the E sum of a kind-1 item
        const bool keep = (lane < 3) == (kind == 0);
        const double v = ((wq[0][src] + wq[1][src]) + wq[2][src]) + wq[3][src];
        out[lane] = keep ? v : 0.0;
      }
      ++gi;
    } else {
      double (*wr)[4][4] = sh.x.wred[local & 1u];
      if (lane == 0) {
        wr[g][q][0] = tA;
        wr[g][q][1] = tB;
        wr[g][q][2] = tE;
        wr[g][q][3] = (double)kind;
      }
      tc_fence_before();
      asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
      if (lead) {
        if (first && !dead && lane < 4) {
          const int k0 = (int)wr[g][0][3];
          const int src = lane == 3 ? 2 : lane;
          const bool keep = (lane < 3) == (k0 == 0);
          double v = 0.0;
          for (int o = 0; o < QPP; ++o)
            v += ((wr[g + o][0][src] + wr[g + o][1][src]) + wr[g + o][2][src]) + wr[g + o][3][src];
          out[lane] = keep ? v : 0.0;
        }
        __syncwarp();
        if (lane == 0 && !dead) {
          mbar_arrive(&sh.tempty[buf]);
          mbar_arrive(&sh.mempty[ms]);
        }
      }
    }
  }
}

// A window-pass item from the pair list: the first rows of its A and B tiles
// (global support rows, both 4-aligned) and its ranges. Row and column tiles
// start at the range starts rounded down to a multiple of 4 rows; rows and
// columns outside the ranges are masked by position.
template <int TNV>
__device__ __forceinline__ void pair_item(const Dev& s, int w, int& ya, int& yb, ItemDesc& d) {
  const WPair pr = s.wpairs[w];
  const Plan P = s.plan[pr.j];
  int r0, r1, c0;
  if (pr.kind == 0) { r0 = P.head_c; r1 = P.head_c + P.ndrop; c0 = P.head_c; }
  else { r0 = P.tail_c; r1 = P.tail_new; c0 = P.tail_c; }
  const int ra = (r0 & ~3) + pr.rt * TM;
  const int ca = (c0 & ~3) + pr.ct * TNV;
  const int base = pr.j * s.cap;
  ya = base + ra;
  yb = base + ca;
  d.kind = pr.kind;
  d.rlo = r0 - ra;
  d.rhi = r1 - ra;
  d.dnew = P.head_new - ca;
  d.told = P.tail_c - ca;
  d.tnew = P.tail_new - ca;
  d.pad0 = d.pad1 = 0;
}

// This CTA's items: a contiguous range of the launch's items, in row-tile-
// major order (distance pass: item = row tile * tiles + support tile; window
// pass: the pair list's order, row tiles outer within each center), so that
// consecutive items mostly share their A tile.
__device__ __forceinline__ Range my_range(int total, int cta, int ncta) {
  Range r;
  r.lo = (int)((int64_t)cta * total / ncta);
  r.hi = (int)((int64_t)(cta + 1) * total / ncta);
  return r;
}

// MODE 0: distance pass (A = batch tile, B = support tile, one FP32 partial per row).
// MODE 1: window pass (A and B = support rows of one center, four FP64 sums per
//         TMEM lane quadrant).
// Both passes only sum over columns, so a tile can be split along its
// columns with no merge.
//
// Metadata: distance-pass tiles start on a multiple of 4 support rows and
// support weights are 0 outside the windows, so an item's column metadata
// (||y||^2, w, data index) and row metadata (||x||^2, data index) are plain
// contiguous, 16-byte aligned ranges; window-pass tiles start 4-aligned by
// construction. The producer copies them with bulk async copies into a ring
// of slots next to the operands, so nothing on the epilogue's path waits on a
// global load. Tile descriptors are fetched 32 items at a time, one per
// producer lane.
template <int KIND, int MODE, int OP, int TNV>
__device__ __forceinline__ void dist_tc_body(const Dev& s, int rows, const CUtensorMap* tmA,
                                             const CUtensorMap* tmB, int cta, int ncta,
                                             Range ovr = Range{-1, -1}, int flags = TC_ALLOC | TC_FREE) {
  constexpr bool X3 = OP == OP_X3;
  constexpr int KSE = OP == OP_TF32 ? 32 : KS;   // operand elements per slice row
  constexpr int NACC = Geo<TNV>::NACC, MS = Geo<TNV>::MS;
  constexpr int BT = TNV * KS * 2;               // one B slice (TNV rows x 128 bytes)
  constexpr int AH = X3 ? 2 : 1;                 // hi (and lo) tiles per operand
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Shared<TNV>& sh = *reinterpret_cast<Shared<TNV>*>(smem + RING_BYTES);
  constexpr uint32_t TMEM_COLS = Geo<TNV>::TMEM_COLS;
  constexpr uint32_t IDESC = idesc<TNV, OP>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nks = s.dp / KSE;
  const Layout L = layout<X3, TNV>(nks);
  uint8_t* const ring = smem + L.a_bytes;        // stages (resident A sits below them)

  if (threadIdx.x == 0) {
    if (flags & TC_REINIT) {
      // a later segment of a group CTA: every barrier initialised below is
      // quiescent (the previous segment ended on a CTA barrier after all its
      // waits), so it is invalidated before it is initialised again
      for (int i = 0; i < STAGES; ++i) {
        mbar_inval(&sh.full[i]);
        mbar_inval(&sh.empty[i]);
      }
      mbar_inval(&sh.afull);
      mbar_inval(&sh.afree);
      for (int i = 0; i < NACC; ++i) {
        mbar_inval(&sh.tfull[i]);
        mbar_inval(&sh.tempty[i]);
      }
      for (int i = 0; i < MS; ++i) {
        mbar_inval(&sh.mfull[i]);
        mbar_inval(&sh.mempty[i]);
      }
      mbar_inval(&sh.mma_done);
    }
    // every stage's pair, not only the layout's L.nst: a later segment may use more
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&sh.full[i], 1);
      mbar_init(&sh.empty[i], 1);
    }
    mbar_init(&sh.afull, 1);
    mbar_init(&sh.afree, 1);
    for (int i = 0; i < NACC; ++i) {
      mbar_init(&sh.tfull[i], 1);
      mbar_init(&sh.tempty[i], 4 * Geo<TNV>::GPT);   // the warps of one team
    }
    for (int i = 0; i < MS; ++i) {
      mbar_init(&sh.mfull[i], META_ARRIVALS);
      mbar_init(&sh.mempty[i], 4 * Geo<TNV>::GPT);
    }
    mbar_init(&sh.mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1 && (flags & TC_ALLOC)) {
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

  // Streaming stage for slice sl: lanes issue A_hi, A_lo (split form), B_hi,
  // B_lo in one instruction; with b_only, only the B tiles.
  auto stream_issue = [&](uint8_t* st, uint64_t* bar, int sl, int ya, int yb, bool b_only) {
    const int nl = 2 * AH;
    if (lane < nl) {
      const bool isb = lane >= AH;
      const int hl = X3 ? (lane & 1) : 0;
      if (isb || !b_only) {
        const int x = hl ? s.dp + sl * KSE : sl * KSE;
        uint8_t* dst = st + (isb ? AH * A_BYTES + hl * BT : hl * A_BYTES);
        tma_load_2d(dst, isb ? tmB : tmA, bar, x, isb ? yb : ya);
      }
    }
  };

  // Metadata of one item as 16-byte chunks: the column arrays (TNV floats
  // each: ||y||^2, w, data index) then the row arrays (128 each: distance
  // pass ||x||^2, data index; window pass ||y||^2, data index, w).
  constexpr int NCC = TNV / 4, NRA = MODE == 0 ? 2 : 3;
  constexpr int NCHUNK = 3 * NCC + 32 * NRA;
  constexpr uint32_t META_ALL = (1u << (3 + NRA)) - 1u;
  constexpr uint32_t META_PRE = (1u << 0) | (1u << 2);   // column norms and data indices: earlier steps' data
  // arrays: bit a of `which` selects array a (0-2 columns, 3.. rows)
  auto meta_copy = [&](MetaSlot<TNV>& m, int ya, int yb, uint32_t which) {
    for (int c = lane; c < NCHUNK; c += 32) {
      const int a = c < 3 * NCC ? c / NCC : 3 + (c - 3 * NCC) / 32;
      const int o = 4 * (c < 3 * NCC ? c % NCC : (c - 3 * NCC) % 32);
      if (!((which >> a) & 1u)) continue;
      float* dst = a < 3 ? m.col[a] : m.row[a - 3];
      const float* src;
      if (a == 0) src = s.yn + yb;
      else if (a == 1) src = s.w32 + yb;
      else if (a == 2) src = (const float*)s.yi + yb;
      else if (MODE == 0) src = a == 3 ? s.xbn + ya : (const float*)s.xbi + ya;
      else src = a == 3 ? s.yn + ya : (a == 4 ? (const float*)s.yi + ya : s.w32 + ya);
      cp16(dst + o, src + o);
    }
  };

  // Distance pass with s.pre_b (set per launch when the kernel just ahead, the
  // batch gather or this pass itself, writes none of it): before the
  // grid-dependency wait the producer fetches the descriptors of its first 32
  // items (one per lane) and stages the B tile of its first item, and the
  // metadata warp stages that item's column norms and indices. They come from
  // the sort, plan and row moves of earlier steps. The column weights (written
  // by the previous step's weight update, which may still be running beside
  // the gather), the batch rows and their metadata follow after the wait.
  int npre = 0;                                  // first-item stages already on their way
  bool meta_pre = false;                         // first item's column norms and indices on their way
  int pya_pre = 0, pyb_pre = 0;                  // this lane's first-round item: its A and B rows
  ItemDesc pd_pre{};
  bool desc_pre = false;
  if constexpr (MODE == 0) {
    if ((warp == 0 || warp == MWARP) && s.pre_b) {
      const int T0 = *s.ntiles;
      const Range r0 = my_range(R * T0, cta, ncta);
      const int mine0 = r0.lo + lane;
      if (mine0 < r0.hi) {
        pya_pre = (mine0 / T0) * TM;
        pyb_pre = s.tiles[mine0 % T0].row0;
      }
      desc_pre = true;
      const int yb0 = __shfl_sync(0xffffffffu, pyb_pre, 0);
      if (r0.lo < r0.hi) {
        if (warp == MWARP) {
          meta_copy(sh.ring[0], 0, yb0, META_PRE);   // column norms and indices
          meta_pre = true;
        } else if (L.res) {
          if (lane == 0) {
            sh.anew[0] = 1u;                          // the first item brings the first A tile
            mbar_expect_tx(&sh.full[0], L.sb);
          }
          __syncwarp();
          tile_issue(lane, L.nsl, nks, s.dp, KSE, ring, BT, tmB, &sh.full[0], yb0);
          npre = 1;
        } else {
          npre = nks < L.nst ? nks : L.nst;
          for (int sl = 0; sl < npre; ++sl) {
            if (lane == 0) mbar_expect_tx(&sh.full[sl], L.sb);   // covers the A slice issued after the wait
            __syncwarp();
            stream_issue(ring + sl * L.sb, &sh.full[sl], sl, 0, yb0, true);
          }
        }
      }
    }
  } else {
    // window pass: its pair list and plans come from the sort/plan kernel two
    // launches back (the row moves just ahead write neither), so the producer
    // and the metadata warp fetch their first 32 pair descriptors before the wait
    if (warp == 0 || warp == MWARP) {
      const Range r0 = ovr.lo >= 0 ? ovr : my_range(*s.nwpairs, cta, ncta);
      const int mine0 = r0.lo + lane;
      if (mine0 < r0.hi) pair_item<TNV>(s, mine0, pya_pre, pyb_pre, pd_pre);
      desc_pre = true;
    }
  }
  KKM_GRID_DEP_WAIT();   // everything above reads only data of earlier steps
  KKM_LAUNCH_DEPENDENTS();   // the next kernel may set itself up; it waits before reading our output

  const int T = MODE == 0 ? *s.ntiles : 1;
  const int total = (MODE == 0) ? R * T : *s.nwpairs;
  const Range rg = ovr.lo >= 0 ? ovr : my_range(total, cta, ncta);
  // All epilogue groups on each item (instead of a team per item) when the
  // run has fewer than NTEAM items per SM. The choice depends on the run
  // alone, never on how a launch splits its items, so an item's sums come out
  // the same in a run's own launch and in a run group's.
  const bool all_groups = total < Geo<TNV>::NTEAM * s.num_sms;

  // descriptors of the next 32 items, one per lane (producer and metadata warp)
  auto fetch_desc = [&](int item, uint32_t local, int& pya, int& pyb, ItemDesc& pd) {
    const int mine = item + lane;
    if (mine >= rg.hi) return;
    if (local == 0 && desc_pre) {
      pya = pya_pre;
      pyb = pyb_pre;
      pd = pd_pre;
    } else if constexpr (MODE == 0) {
      pya = (mine / T) * TM;
      pyb = s.tiles[mine % T].row0;
    } else {
      pair_item<TNV>(s, mine, pya, pyb, pd);
    }
  };

  if (warp == 0) {
    // ------------------------------------------------- operand producer (one warp)
    // Lane 0 waits on the barriers and posts the expected bytes; the slices of
    // a tile are issued by several lanes at once.
    bool ok = true;
    uint32_t it = 0, local = 0, na = 0;          // stage fills, items visited, A tiles
    int cur_ya = -1;                             // the resident A tile's first row
    int pya = 0, pyb = 0;                        // this lane's prefetched item: A and B row
    ItemDesc pd{};
    for (int item = rg.lo; item < rg.hi; ++item, ++local) {
      if ((local & 31u) == 0) fetch_desc(item, local, pya, pyb, pd);
      const int src = (int)(local & 31u);
      const int ya = __shfl_sync(0xffffffffu, pya, src);
      const int yb = __shfl_sync(0xffffffffu, pyb, src);
      const bool new_a = L.res && ya != cur_ya;
      if (L.res) {
        // one stage: the item's whole B tile
        const int st = it % L.nst;
        const uint32_t ph = (it / L.nst) & 1u;
        const bool pre = MODE == 0 && local == 0 && npre > 0;
        if (!pre) {
          if (lane == 0) {
            if (!mbar_wait(&sh.empty[st], ph ^ 1u)) ok = false;
            sh.anew[st] = new_a ? 1u : 0u;             // published by the arrive below
            if (ok) mbar_expect_tx(&sh.full[st], L.sb);
          }
          if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
          tile_issue(lane, L.nsl, nks, s.dp, KSE, ring + st * L.sb, BT, tmB, &sh.full[st], yb);
        }
        ++it;
        if (new_a) {
          // the item's B tile is queued (the MMA warp sees the new-A mark on it
          // and releases the old A tile); then the new A tile
          if (lane == 0) {
            if (na > 0 && !mbar_wait(&sh.afree, (na - 1) & 1u)) ok = false;
            if (ok) mbar_expect_tx(&sh.afull, (uint32_t)L.a_bytes);
          }
          if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
          tile_issue(lane, L.nsl, nks, s.dp, KSE, smem, A_BYTES, tmA, &sh.afull, ya);
          ++na;
          cur_ya = ya;
        }
      } else {
        for (int sl = 0; sl < nks; ++sl, ++it) {
          const int st = it % L.nst;
          const uint32_t ph = (it / L.nst) & 1u;
          const bool pre = MODE == 0 && local == 0 && sl < npre;   // B slices and expected bytes sent before the wait
          if (lane == 0) {
            if (!mbar_wait(&sh.empty[st], ph ^ 1u)) ok = false;
            if (ok && !pre) mbar_expect_tx(&sh.full[st], L.sb);
          }
          if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
          if (pre) {   // the A slice only
            if (lane < AH) {
              const int x = lane ? s.dp + sl * KSE : sl * KSE;
              tma_load_2d(ring + st * L.sb + lane * A_BYTES, tmA, &sh.full[st], x, ya);
            }
          } else {
            stream_issue(ring + st * L.sb, &sh.full[st], sl, ya, yb, false);
          }
        }
        if (!ok) break;
      }
    }
    if (lane == 0) {
      // the copies in flight must land before the CTA may exit: the last fill
      // of every stage and the last A tile
      for (uint32_t q = (it > (uint32_t)L.nst ? it - L.nst : 0u); q < it; ++q)
        if (!mbar_wait(&sh.full[q % L.nst], (q / L.nst) & 1u)) ok = false;
      if (na > 0 && !mbar_wait(&sh.afull, (na - 1) & 1u)) ok = false;
      if (!ok) atomicOr(s.status, ST_TIMEOUT);
    }
  } else if (warp == MWARP) {
    // ------------------------------------------------------ metadata (one warp)
    // Every lane copies its share of an item's metadata and arrives on the
    // slot's barrier once its copies have landed; lane 0 also arrives after
    // writing the window-pass ranges, which publishes them.
    bool ok = true;
    uint32_t local = 0;
    int pya = 0, pyb = 0;
    ItemDesc pd{};
    for (int item = rg.lo; item < rg.hi; ++item, ++local) {
      if ((local & 31u) == 0) fetch_desc(item, local, pya, pyb, pd);
      const int src = (int)(local & 31u);
      const int ya = __shfl_sync(0xffffffffu, pya, src);
      const int yb = __shfl_sync(0xffffffffu, pyb, src);
      const int ms = local % MS;
      if (lane == 0 && !mbar_wait(&sh.mempty[ms], ((local / MS) & 1u) ^ 1u)) ok = false;
      if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
      MetaSlot<TNV>& m = sh.ring[ms];
      if constexpr (MODE == 1) {
        ItemDesc d;
        d.kind = __shfl_sync(0xffffffffu, pd.kind, src);
        d.rlo = __shfl_sync(0xffffffffu, pd.rlo, src);
        d.rhi = __shfl_sync(0xffffffffu, pd.rhi, src);
        d.dnew = __shfl_sync(0xffffffffu, pd.dnew, src);
        d.told = __shfl_sync(0xffffffffu, pd.told, src);
        d.tnew = __shfl_sync(0xffffffffu, pd.tnew, src);
        d.pad0 = d.pad1 = 0;
        if (lane == 0) m.desc = d;
      }
      meta_copy(m, ya, yb, (local == 0 && meta_pre) ? META_ALL & ~META_PRE : META_ALL);
      cp_arrive_noinc(&sh.mfull[ms]);
      if (lane == 0) mbar_arrive(&sh.mfull[ms]);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");   // nothing in flight when the CTA exits
    if (lane == 0 && !ok) atomicOr(s.status, ST_TIMEOUT);
  } else if (warp == 1) {
    // -------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      bool ok = true;
      uint32_t it = 0, local = 0, na = 0;
      const uint32_t abase = smem_u32(smem), rbase = smem_u32(ring);
      // descriptors of a slice's tiles; a 32-byte K step adds 2 to the address field
      auto mma_slice = [&](uint32_t d, uint32_t ahi, uint32_t alo, uint32_t bhi, uint32_t blo, bool first) {
        const uint64_t dah = sw128_desc(ahi), dbh = sw128_desc(bhi);
        if constexpr (X3) {
          const uint64_t dal = sw128_desc(alo), dbl = sw128_desc(blo);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            mma_op<OP>(d, dah + 2u * k, dbh + 2u * k, IDESC, (first && k == 0) ? 0u : 1u);
            mma_op<OP>(d, dah + 2u * k, dbl + 2u * k, IDESC, 1u);
            mma_op<OP>(d, dal + 2u * k, dbh + 2u * k, IDESC, 1u);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)   // four 32-byte K steps per 128-byte slice row
            mma_op<OP>(d, dah + 2u * k, dbh + 2u * k, IDESC, (first && k == 0) ? 0u : 1u);
        }
      };
      for (int item = rg.lo; ok && item < rg.hi; ++item, ++local) {
        const uint32_t buf = local % NACC, bph = (local / NACC) & 1u;
        if (!mbar_wait(&sh.tempty[buf], bph ^ 1u)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + buf * TNV;
        if (L.res) {
          const int st = it % L.nst;
          if (!mbar_wait(&sh.full[st], (it / L.nst) & 1u)) { ok = false; break; }
          tc_fence_after();
          if (sh.anew[st]) {
            // a new resident A tile: release the old one once its MMAs are done, wait for the new one
            if (na > 0) mma_commit(&sh.afree);
            if (!mbar_wait(&sh.afull, na & 1u)) { ok = false; break; }
            tc_fence_after();
            ++na;
          }
          const uint32_t b0 = rbase + (uint32_t)(st * L.sb);
          for (int sl = 0; sl < nks; ++sl)
            mma_slice(d, abase + sl * A_BYTES, abase + (nks + sl) * A_BYTES, b0 + sl * BT, b0 + (nks + sl) * BT,
                      sl == 0);
          mma_commit(&sh.empty[st]);
          ++it;
        } else {
          for (int sl = 0; sl < nks; ++sl, ++it) {
            const int st = it % L.nst;
            if (!mbar_wait(&sh.full[st], (it / L.nst) & 1u)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a0 = rbase + (uint32_t)(st * L.sb), b0 = a0 + AH * A_BYTES;
            mma_slice(d, a0, a0 + A_BYTES, b0, b0 + BT, sl == 0);
            mma_commit(&sh.empty[st]);
          }
          if (!ok) break;
        }
        mma_commit(&sh.tfull[buf]);
      }
      mma_commit(&sh.mma_done);
      if (!mbar_wait(&sh.mma_done, 0)) ok = false;
      if (!ok) atomicOr(s.status, ST_TIMEOUT);
    }
  } else if constexpr (MODE == 0) {
    dist_epilogue<KIND, TNV>(s, sh, tmem, rg, T, rows, warp, lane, all_groups);
  } else {
    pair_epilogue<KIND, TNV>(s, sh, tmem, rg, warp, lane, all_groups);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1 && (flags & TC_FREE)) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  }
}

template <int KIND, int MODE, int OP, int TNV>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_dist_tc(Dev s, int rows, const __grid_constant__ CUtensorMap tmA,
              const __grid_constant__ CUtensorMap tmB) {
  dist_tc_body<KIND, MODE, OP, TNV>(s, rows, &tmA, &tmB, blockIdx.x, gridDim.x);
}

// Run groups. A launch covers the runs of one class (same form, kernel kind
// and tile width; their d may differ). Each run's items (distance pass:
// row tiles x support tiles; window pass: its pair list) are laid end to end
// in one weighted item space, an item of run r weighing
// max(5, 2 nks_r m_r) (m = 3 for the split form: the MMA share next to the
// epilogue's fixed share), and CTA c takes the items whose start falls in
// [c W / G, (c + 1) W / G). It walks its range run by run: each stretch of
// one run's items is a segment, run with that run's Dev and TMA descriptors
// (read from device memory; the host wrote them before the group's first
// launch, and the acquire fence orders that write before the tensor-map
// proxy's reads). TMEM is allocated for the first segment and freed after the
// last; the barriers are invalidated and initialised again between segments.
// Item counts are read after the grid-dependency wait, so no data of this
// step is staged before it (the runs' copies carry pre_b = 0).
template <int MODE>
__device__ __forceinline__ int group_items(const Dev& s) {
  return MODE == 0 ? ((s.b + TM - 1) / TM) * (*s.ntiles) : *s.nwpairs;
}

__device__ __forceinline__ int group_weight(const Dev& s) {
  const int kse = s.form == FORM_TF32 ? 32 : KS;
  const int m = s.form == FORM_BF16X3 ? 3 : 1;
  const int w = 2 * (s.dp / kse) * m;
  return w > 5 ? w : 5;
}

__device__ __forceinline__ long long ceil_div_ll(long long a, long long b) {
  return a >= 0 ? (a + b - 1) / b : -((-a) / b);
}

// Warp-wide: the first run r >= rnext whose items intersect the weighted
// range [A, B), with that intersection [lo, hi) of its items; -1 if none.
// With A = B = -1, returns -1 and sets lo to the low and hi to the high word
// of the total weight instead.
template <int MODE>
__device__ __forceinline__ int group_find(const GroupPhase& g, long long A, long long B, int rnext, int& lo,
                                          int& hi, long long& total) {
  const int lane = threadIdx.x & 31;
  long long carry = 0;
  for (int base = 0; base < g.nruns; base += 32) {
    const int r = base + lane;
    int n = 0, om = 1;
    if (r < g.nruns) {
      const Dev& s = g.runs[r].s;
      n = group_items<MODE>(s);
      om = group_weight(s);
    }
    const long long W = (long long)n * om;
    long long incl = W;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const long long P = carry + incl - W;
    int mlo = 0, mhi = 0;
    if (A >= 0 && r < g.nruns && r >= rnext && n > 0) {
      mlo = (int)min((long long)n, max(0LL, ceil_div_ll(A - P, om)));
      mhi = (int)min((long long)n, max(0LL, ceil_div_ll(B - P, om)));
    }
    const unsigned hit = __ballot_sync(0xffffffffu, mlo < mhi);
    if (hit) {
      const int src = __ffs(hit) - 1;
      lo = __shfl_sync(0xffffffffu, mlo, src);
      hi = __shfl_sync(0xffffffffu, mhi, src);
      return base + src;
    }
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  total = carry;
  return -1;
}

template <int KIND, int MODE, int OP, int TNV>
__global__ void __launch_bounds__(NTHREADS, 1) k_group_tc(GroupPhase g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Shared<TNV>& sh = *reinterpret_cast<Shared<TNV>*>(smem + RING_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  KKM_GRID_DEP_WAIT();
  KKM_LAUNCH_DEPENDENTS();
  if (warp == 0) {
    int lo = 0, hi = 0;
    long long total = 0;
    group_find<MODE>(g, -1, -1, 0, lo, hi, total);
    if (lane == 0) sh.gtot = total;
  }
  __syncthreads();
  const long long W = sh.gtot;
  const long long A = W * (long long)blockIdx.x / gridDim.x, B = W * (long long)(blockIdx.x + 1) / gridDim.x;
  int flags = TC_ALLOC, rnext = 0;
  for (;;) {
    if (warp == 0) {
      int lo = 0, hi = 0;
      long long total = 0;
      const int r = A < B ? group_find<MODE>(g, A, B, rnext, lo, hi, total) : -1;
      if (lane == 0) {
        sh.gseg[0] = r;
        sh.gseg[1] = lo;
        sh.gseg[2] = hi;
      }
    }
    __syncthreads();
    const int r = sh.gseg[0];
    if (r < 0) break;
    const Range seg{sh.gseg[1], sh.gseg[2]};
    const GroupRun& gr = g.runs[r];
    {
      // the run's Dev into shared memory (the previous segment ended on a CTA
      // barrier, so nobody reads the old copy any more)
      static_assert(sizeof(Dev) % 16 == 0, "Dev copied in 16-byte words");
      const int4* src = reinterpret_cast<const int4*>(&gr.s);
      int4* dst = reinterpret_cast<int4*>(&sh.gdev);
      for (int i = threadIdx.x; i < (int)(sizeof(Dev) / 16); i += NTHREADS) dst[i] = src[i];
    }
    __syncthreads();
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(gr.maps);
    const CUtensorMap* a = MODE == 0 ? &m[0] : &m[1];
    const CUtensorMap* b = TNV == 256 ? &m[3] : (TNV == 128 ? &m[1] : &m[2]);
    if (warp == 0) {
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)a) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)b) : "memory");
    }
    // the body starts and ends on CTA barriers, so gseg is read by every
    // thread before warp 0 writes the next segment
    dist_tc_body<KIND, MODE, OP, TNV>(sh.gdev, sh.gdev.b, a, b, 0, 1, seg, flags);
    flags = TC_REINIT;
    rnext = r + 1;
  }
  if (flags == TC_REINIT && warp == 1) {   // TMEM was allocated by the first segment
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh.tmem_base),
                 "r"(Geo<TNV>::TMEM_COLS)
                 : "memory");
  }
}

}  // namespace
}  // namespace kkm
