// Internal declarations shared by the libkkm translation units.
//
// Device state of one run. Everything lives in HBM and is sized at kkm_init;
// nothing is allocated per step.
//
//   support store  k regions of `cap` rows, one per center. Center j's
//                  window (Eq. (1)) occupies rows [head_j, tail_j) of region j,
//                  laid out as C_1 (while kept), then blocks oldest -> newest,
//                  each block in batch order. Appends go at tail. Drops advance
//                  head. When an append would pass the region's end, the
//                  window is first copied down to row 0 ("compaction"). With
//                  cap - REGION_PAD = 2*tau + 4*b + 8 usable rows the source
//                  and destination rows of that copy never overlap, because a
//                  window holds at most tau + b rows. The last REGION_PAD rows
//                  of a region are never used, so a tile (at most 256 rows)
//                  that starts inside the window never reaches the next region.
//   row data       FP32 form: FP32 rows, ld = round_up(d, 16), zero padded.
//                  TF32 form: FP32 rows rounded to TF32, ld = dp = round_up(d, 32).
//                  BF16 forms: BF16 rows [hi(0..dp) | lo(0..dp)], dp =
//                  round_up(d, 64), zero padded; ld = 2*dp.
//   yn             FP32 ||y||^2 of the values the Gram product actually uses
//   yi             int32 data index of the row (the key that forces K(x,x)=1
//                  when a batch point meets its own support copy)
//   w64 / w32      FP64 master weight and its FP32 copy for the distance kernel.
//                  Invariant: both are 0 on every row outside its window, so a
//                  tile may cover rows on either side of a window and read
//                  their weights as they are.
//
// Per-center block ring: (iteration, count) of the window's blocks, oldest
// first, at most tau + 2 entries. C_1 is not in the ring; c1[j] flags it.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <atomic>
#include <type_traits>

namespace kkm {

enum Form : int { FORM_FP32 = 0, FORM_BF16 = 1, FORM_BF16X3 = 2, FORM_TF32 = 3 };

// forms whose row buffers hold FP32 values (xb32 / y32)
__host__ __device__ inline bool f32_rows(int form) { return form == FORM_FP32 || form == FORM_TF32; }
enum KernelKind : int { K_GAUSS = 0, K_LAPLACE = 1, K_LINEAR = 2, K_POLY = 3 };

// device status bits (sticky until the context is destroyed)
constexpr int ST_BAD_BATCH_INDEX = 1;
constexpr int ST_BAD_ASSIGN = 2;
constexpr int ST_CAPACITY = 4;
constexpr int ST_TIMEOUT = 8;

constexpr int REGION_PAD = 256;   // unused rows at the end of each support region (the widest tile)
constexpr int WPASS_TNV = 128;    // tcgen05 window pass: support rows per column tile

// Column tile of the distance pass: support rows [row0, row0 + ncols) of center j.
struct Tile {
  int32_t j;
  int32_t row0;   // global support row
  int32_t ncols;
  int32_t pad;
};

// Tile pair of the window Gram pass (norm recurrence terms), see kkm_step.cu.
struct WPair {
  int32_t j;
  int32_t kind;   // 0: dropped rows x (old window + new block); 1: new block x new block
  int32_t rt;     // row tile index within the row range
  int32_t ct;     // column tile index within the column range
};

// Per-center plan of one update, written by the sort/plan kernel.
struct Plan {
  int32_t head_c;    // window start after compaction
  int32_t tail_c;    // window end after compaction (= start of the new block)
  int32_t head_new;  // window start after the drops
  int32_t tail_new;  // window end after the append
  int32_t src_head;  // compaction source start (-1 when not compacting)
  int32_t cnt;       // b_i^j
  int32_t ndrop;     // rows dropped (C_1 included)
  int32_t c1_new;    // C_1 kept after this update
};

struct Dev {
  // problem
  int64_t n;
  int32_t d, k, b, tau, cap, nbcap;
  int64_t ldx;
  int32_t ld;        // row stride of batch and support rows, in elements
  int32_t dp;        // BF16 forms: padded d (hi part length)
  int32_t form, kind, degree, lr;
  double param, coef0, eta;
  double inv_b;      // 1 / b
  float negc;        // -log2(e) / param (Gaussian, Laplacian)
  int32_t num_sms;
  uint64_t seed;
  int32_t tn;        // support rows per distance tile
  int32_t ppt;       // partials per distance tile in part[] (2 for 256-row tcgen05 tiles: one per column half)
  int32_t pre_b;     // distance pass: stage the support operand, its metadata and the tile list before
                     // the grid-dependency wait (launch_dist_tc sets it per launch, only after the gather)
  int32_t pair_rows, pair_cols; // window-pass tile: row and column counts (64x64 SIMT, 128x128 tcgen05)
  int32_t walign;    // window-pass tiles start at range starts rounded down to this many rows (1 SIMT, 4 tcgen05)
  int32_t bpad;      // rows of the batch buffers (>= b, multiple of 128)
  int32_t max_tiles, max_pairs;
  const float* X;
  // batch
  int32_t* bidx;     // [b] indices of the batch being processed
  float* xb32;       // [bpad * ld]   FP32 form
  __nv_bfloat16* xbh;// [bpad * ld]   BF16 forms
  float* xbn;        // [bpad]
  int32_t* xbi;      // [bpad] data index, -1 for query rows
  // support store
  float* y32;
  __nv_bfloat16* ybh;
  float* yn;
  int32_t* yi;
  double* w64;
  float* w32;
  // per center
  int32_t* head;
  int32_t* tail;
  int32_t* c1;
  int32_t* wsum;     // sum of block counts in the window (C_1 excluded)
  double* cnorm;
  float* cnorm32;    // FP32 copy of cnorm for the argmin
  int32_t* blk_iter; // [k * nbcap]
  int32_t* blk_cnt;  // [k * nbcap]
  int32_t* blk_first;
  int32_t* blk_num;
  // step workspaces
  int32_t* assign;   // [bpad] assignment used by the update
  float* mind;       // [bpad]
  float* inner_a;    // [bpad] <phi(x), C_a> at the used assignment a
  int32_t* counts;   // [k]
  double* alpha;     // [k]
  int32_t* coff;     // [k + 1] exclusive offsets of the center-sorted batch
  int32_t* perm;     // [b] batch rows sorted by center (stable)
  int64_t* mvdst;    // [b] support row that sorted batch row w moves to (k_sort_plan), -1 past capacity
  double* cmc;       // [k] <C_j, cm(B_j)>
  Plan* plan;        // [k]
  int32_t* comp_off; // [k] first flat row of each center's compaction copy
  int32_t* comp_total; // [1] rows copied by this step's compactions
  Tile* tiles;       // [max_tiles]
  int32_t* ntiles;   // [1]
  int32_t* tile_first; // [k]
  int32_t* tile_cnt;   // [k]
  float* part;       // [max_tiles * ppt * bpad] per-tile weighted kernel sums (ppt partials per tile)
  WPair* wpairs;     // [max_pairs]
  int32_t* nwpairs;  // [1]
  int32_t* wpair_first; // [k]
  int32_t* wpair_cnt;   // [k]
  double* ncum;      // [k] points assigned to each center so far (N^j of the sklearn rate)
  const double* rtab; // [2 (b + 1)]: 1/n at [n] and sqrt(n / b) at [b + 1 + n], n = 0..b (host-computed)
  double* wpart;     // [max_pairs][wslots][4 sums]: A, Bdd, E, M partials per tile
  int32_t wslots;    // partial slots per window-pass tile (SIMT: 4, slot 0 used; tcgen05: one per team group)
  int64_t* iter;     // [1] next iteration number
  int32_t* status;   // [1] sticky device status bits
  int32_t* fin_pending;   // [1] 1 while a step's weight update (k_finalize) is still to run
  int64_t* stats;    // [3] steps, support rows, tiles
  double* obj;       // [1] last batch objective
  float* cmpart;     // [k][32] FP32 lane partials of sum_{x in B_j} <phi(x), C_j>
};

// Programmatic dependent launch: every step kernel is launched so that it may
// be scheduled while its predecessor drains. It must wait here before it reads
// anything the predecessor writes (a no-op when launched without the attribute).
#define KKM_GRID_DEP_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")
// Lets the next kernel in the stream start its pre-wait part. Issued only after
// this kernel's own wait, so every kernel before it has completed by then,
// with one exception: the rotated gather (which follows the previous step's
// k_finalize) issues it before its wait. The distance pass it releases reads
// before its own wait only what the previous step's sort, plan and row moves
// wrote, and those completed before the gather was launched. The step kernels
// all issue it; each of them waits at its first statement, except the
// tcgen05 passes, whose pre-wait part sets up shared memory and TMEM and
// (distance pass after the gather only) stages data of earlier steps, and
// the rotated gather.
#define KKM_LAUNCH_DEPENDENTS() asm volatile("griddepcontrol.launch_dependents;" ::: "memory")

// Raises `kern`'s dynamic shared-memory limit to `bytes` on the current device,
// once per device: the attribute belongs to the function on that device.
// `done` is the caller's per-kernel mask of devices already set.
template <typename Kern>
inline cudaError_t smem_limit_once(Kern kern, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (uint64_t)1 << dev : 0;
  if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_relaxed);
  return e;
}

// Launches `kern` with the programmatic-stream-serialization attribute.
template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Params>(args)...);
}

// ---------------------------------------------------------------- helpers
__host__ __device__ inline int64_t round_up(int64_t a, int64_t m) { return (a + m - 1) / m * m; }

// SplitMix64 (Steele, Lea, Flood 2014): output `counter` of the sequential
// generator seeded with `seed`, i.e. the finaliser applied to
// seed + (counter + 1) * golden gamma.
__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Lemire's multiply-high reduction of a 64-bit value onto [0, n).
__host__ __device__ inline int64_t index_below(uint64_t h, uint64_t n) {
#ifdef __CUDA_ARCH__
  return (int64_t)__umul64hi(h, n);
#else
  return (int64_t)(((unsigned __int128)h * n) >> 64);
#endif
}

// Kernel value from the Gram entry g = <x,y> and the squared norms, in FP32.
// `same` forces ||x - y|| = 0 when x and y are the same data point.
__device__ __forceinline__ float kernel_from_gram(int kind, float g, float xn, float yn, bool same,
                                                  float negc, float coef0, int degree) {
  if (kind == K_GAUSS || kind == K_LAPLACE) {
    float d2 = fmaxf(fmaf(-2.0f, g, xn + yn), 0.0f);
    if (same) d2 = 0.0f;
    float arg = (kind == K_GAUSS) ? d2 : sqrtf(d2);
    return exp2f(arg * negc);       // negc = -log2(e) / param
  }
  if (kind == K_LINEAR) return g;
  float base = g + coef0, r = 1.0f;
  for (int p = 0; p < degree; ++p) r *= base;
  return r;
}

// K(x, x) from ||x||^2 (FP64, for the distance formula).
__host__ __device__ inline double kernel_self(int kind, double xn, double coef0, int degree) {
  if (kind == K_GAUSS || kind == K_LAPLACE) return 1.0;
  if (kind == K_LINEAR) return xn;
  double base = xn + coef0, r = 1.0;
  for (int p = 0; p < degree; ++p) r *= base;
  return r;
}

// Table form of Algorithm 1 (kkm_config.algo = KKM_ALGO_TABLE).
struct TabBuf {
  float* T;            // [k][n] <phi(x), C_j>, center-major
  int32_t* bs_off;     // [k+1] start of each center's rows in the support buffer (whole tiles)
  const float* part;   // the Gram view's per-tile partials, [tiles][npad]
  int64_t npad;        // row stride of part (round_up(n, 128))
  int32_t bs_rows;     // rows of the support buffer (k * cap + 256)
};

// ------------------------------------------------------------ launchers
// All return cudaGetLastError() of their launches.
cudaError_t launch_sample(const Dev& s, cudaStream_t st);
// rotated: the gather follows the previous step's k_finalize, does its work
// and releases the distance pass before its grid-dependency wait (neither
// touches before its wait what finalize writes), then clears fin_pending
cudaError_t launch_gather_batch(const Dev& s, const int32_t* idx, cudaStream_t st, bool rotated = false);
cudaError_t launch_gather_query(const Dev& s, const float* Q, int64_t ldq, int rows, cudaStream_t st);
cudaError_t launch_dist_simt(const Dev& s, int rows, cudaStream_t st);
cudaError_t launch_argmin(const Dev& s, int rows, const int32_t* forced, int32_t* assign_out,
                          float* mind_out, float* dist_out, bool update, cudaStream_t st);
// set_pending: the step's k_finalize runs at the start of the next step (or a flush)
cudaError_t launch_sort_plan(const Dev& s, double* obj_out, cudaStream_t st, bool set_pending = false);
cudaError_t launch_move(const Dev& s, cudaStream_t st);
cudaError_t launch_wgram(const Dev& s, cudaStream_t st);
// if_pending: a no-op unless fin_pending is set
cudaError_t launch_finalize(const Dev& s, cudaStream_t st, bool if_pending = false);
// batch objective at fixed assignments and its adjoint (kkm_grad.cu): two
// launches. ws holds grad_workspace_doubles(s, m) doubles, zeroed when it is
// allocated (its first int is the row kernel's finished-block counter, which
// every call leaves at zero). With grad_q == NULL only the forward runs
// (loss, delta); otherwise the adjoint (grad_q, grad_s).
// kernel k-means++ seeding (kkm_seed.cu): chosen[0..k) on the device;
// d2 holds n doubles, part ceil(n/8) doubles
cudaError_t launch_kmeanspp(const float* X, int64_t n, int d, int64_t ldx, int k, int kind, double param,
                            double coef0, int degree, uint64_t seed, double* d2, double* part, int64_t* chosen,
                            cudaStream_t st);
size_t grad_workspace_doubles(const Dev& s, int64_t m);
cudaError_t launch_objective(const Dev& s, double log_sigma, const float* Q, int64_t m, int64_t ldq,
                             const int32_t* assign, double* loss, float* delta, const double* grad_loss,
                             float* grad_q, int64_t ldg, double* grad_s, double* ws, cudaStream_t st);
cudaError_t launch_build_tiles(const Dev& s, cudaStream_t st);
cudaError_t launch_init_centers(const Dev& s, const int32_t* init_idx, cudaStream_t st);
cudaError_t launch_load_rows(const Dev& s, int32_t rows_total, cudaStream_t st);
cudaError_t launch_tab_batch_dist(const Dev& s, const TabBuf& q, int rows, const int32_t* forced,
                                  int32_t* assign_out, float* mind_out, float* dist_out, bool update, cudaStream_t st);
cudaError_t launch_tab_plan(const Dev& s, const TabBuf& q, double* obj_out, cudaStream_t st);
cudaError_t launch_tab_fill(const Dev& s, const TabBuf& q, cudaStream_t st);
cudaError_t launch_tab_center(const Dev& s, const TabBuf& q, cudaStream_t st);
cudaError_t launch_tab_update(const Dev& s, const TabBuf& q, bool init, cudaStream_t st);
cudaError_t launch_tab_init(const Dev& s, const Dev& g, const TabBuf& q, const int32_t* init_idx, cudaStream_t st);
cudaError_t launch_tab_objective(const Dev& s, const TabBuf& q, const float* xn, double* blk, int nblk,
                                 cudaStream_t st);
cudaError_t launch_mind_sum(const Dev& s, int rows, double scale, double* out, cudaStream_t st);  // scale * sum of mind

// --------------------------------------------------------------- run groups
// A run of a group as the group's launches see it: its four TMA descriptors
// (tc_prepare's layout, used in place by the tcgen05 passes) and its Dev.
struct alignas(64) GroupRun {
  unsigned char maps[512];
  Dev s;
};
static_assert(sizeof(GroupRun) % 64 == 0, "descriptors of consecutive runs stay 64-byte aligned");
// One launch over several runs. The step phases: runs[r] owns blocks
// [first[r], first[r + 1]) and each of them plays one block of that run's own
// launch. The Gram passes read no `first`: they spread the runs' items over
// the launch on the device (kkm_gram_tc.cuh, kkm_gram_simt.cu).
struct GroupPhase {
  const GroupRun* runs;   // device
  const int32_t* first;   // device, nruns + 1 entries, non-decreasing, first[0] = 0
  int32_t nruns;
};
cudaError_t launch_group_gather(const GroupPhase& g, int blocks, cudaStream_t st);
cudaError_t launch_group_argmin(const GroupPhase& g, int blocks, cudaStream_t st);
cudaError_t launch_group_sort_plan(const GroupPhase& g, int smem, cudaStream_t st);   // one block per run
cudaError_t launch_group_move(const GroupPhase& g, int blocks, cudaStream_t st);
cudaError_t launch_group_finalize(const GroupPhase& g, int blocks, cudaStream_t st);
// distance pass (mode 0) or window pass (mode 1) of runs that share the form,
// kernel kind and distance tile: tcgen05 (ctas persistent CTAs) ...
cudaError_t launch_group_tc(const GroupPhase& g, int mode, int form, int kind, int tn, int ctas, cudaStream_t st);
// ... or the FP32 CUDA-core passes
cudaError_t launch_group_simt(const GroupPhase& g, int mode, int form, int blocks, cudaStream_t st);
int sort_plan_smem(int k, int b);

// ------------------------------------------------ full-batch kernel Lloyd
// The Gram view's Dev (xb*: every row of X in the operand form, y*: the
// support buffer of X sorted by center) plus these buffers (kkm_lloyd.cu).
constexpr int LLOYD_RANK_ROWS = 1024;   // rows per chunk of the counting sort's ranking
struct LloydBuf {
  float* T;               // [k][n] <phi(x), C_j>, center-major
  int32_t* assign;        // [n] assignment at the current centers
  float* mind;            // [n] min_j Delta(x, C_j) at the current centers
  int32_t* rank;          // [n] rank of x among the rows of its center within its ranking chunk
  int32_t* ccnt;          // [nrk][k] rows of center j in ranking chunk c (chunk-major)
  int32_t* cbase;         // [nrk][k] position of chunk c's first row of center j within center j
  int32_t* bs_off;        // [k + 1] first support-buffer row of each center (blocks of whole tiles)
  double* blk;            // [nblk] objective partials of the assignment pass
  int32_t* blk_changed;   // [nblk] changed-assignment partials
  double* obj;            // [1] f_X at the current centers
  int64_t* changed;       // [1] rows whose assignment the last assignment pass changed
  int32_t nrk;            // ranking chunks, ceil(n / LLOYD_RANK_ROWS)
  int32_t nblk;           // blocks of the assignment pass
};
// counting sort of X by assignment: ranks, then offsets, tiles and weights 1/n_j
cudaError_t launch_lloyd_sort(const Dev& g, const LloydBuf& L, cudaStream_t st);
// the center-sorted rows into the support buffer
cudaError_t launch_lloyd_scatter(const Dev& g, const LloydBuf& L, cudaStream_t st);
// T[j][row0 + r] from the Gram pass partials of one chunk of rows (gc: the chunk's view);
// all: every center (initial centers), else only centers with rows
cudaError_t launch_lloyd_reduce(const Dev& gc, const LloydBuf& L, int64_t row0, int rows, bool all, cudaStream_t st);
// ||C_j||^2 = (1/n_j) sum_{x in X_j} T[j][x] for the centers with rows
cudaError_t launch_lloyd_cnorm(const Dev& g, const LloydBuf& L, cudaStream_t st);
// argmin over the centers for every row, f_X and the changed count; first: every row counts as changed
cudaError_t launch_lloyd_assign(const Dev& g, const LloydBuf& L, bool first, cudaStream_t st);
// Delta(x, C_j) for every row and center, FP32 (n x k row-major)
cudaError_t launch_lloyd_dist(const Dev& g, const LloydBuf& L, float* out, cudaStream_t st);

// tensor-core passes (BF16, split-BF16 and TF32 forms)
// maps: 512 bytes, 64-byte aligned, holding the four CUtensorMap of the passes
cudaError_t tc_prepare(Dev& s, void* maps);
// one bounded mbarrier wait (the passes' own), limited to limit_ns; out[0] = 1 when it ran out
cudaError_t launch_wait_probe(uint64_t limit_ns, int arrive, int* out, cudaStream_t st);
// partials the distance pass writes per tile of tn support rows (Dev::ppt)
int tc_parts_per_tile(int tn);
// stage_early: the kernel just ahead on `st` (the batch gather, or this pass
// itself) writes none of the support tiles, their metadata or the tile list,
// so the pass may stage them before its grid-dependency wait.
cudaError_t launch_dist_tc(const Dev& s, const void* maps, int rows, cudaStream_t st, bool stage_early = false);
// The window pass reads its pair list and plans before its grid-dependency
// wait: launch it only right after k_move (which writes neither).
cudaError_t launch_wgram_tc(const Dev& s, const void* maps, cudaStream_t st);

}  // namespace kkm
