/*
 * kkm.h -- C ABI of libkkm, truncated mini-batch kernel k-means on NVIDIA GB300
 * (sm_103a). Jourdan & Schwartzman, "Mini-batch kernel k-means".
 *
 * One context holds one clustering run. The run covers the dataset X, the
 * number of centers k, the kernel K and the batch size b of the problem
 * statement (Sec. 1) and of the inputs of Algorithms 1/2, together with the
 * truncation parameter tau of Sec. 4.1. Each center j is held implicitly, as
 * Eq. (1) defines it: a weighted sum of feature vectors phi(y_s) over a sliding
 * window of support rows, plus the FP64 norm ||C_j||^2.
 *
 * Conventions shared by every call:
 *  - Pointers marked "device" must be CUDA device (or managed) memory that the
 *    calling process can reach on the context's device. Pointers marked "host"
 *    are ordinary CPU memory.
 *  - Matrices are row-major. A "leading dimension" counts elements between the
 *    starts of consecutive rows.
 *  - Unless stated otherwise a call only enqueues work on the context's stream
 *    and returns. Results are ready once that stream has been synchronised.
 *  - The caller keeps ownership of every buffer it passes in. The library owns
 *    only what it allocates inside a context, and kkm_destroy frees all of it.
 *  - Every call returns a kkm_status, and no C++ exception crosses the ABI.
 *    Arguments are validated on the host before any work is queued, and an
 *    invalid call changes no state. Faults found on the device (an
 *    out-of-range batch or assignment index) are recorded in a sticky device
 *    status word. They are reported as KKM_EINVAL by the next call that
 *    synchronises (kkm_sync, kkm_objective, kkm_get_state, kkm_step_host).
 *    Once that happens the context is poisoned: every later call returns
 *    KKM_ESTATE.
 *  - kkm_last_error(ctx) gives a message for the last failure on that
 *    context. kkm_last_error(NULL) gives the calling thread's last failure of
 *    kkm_init.
 *  - A context may be used by one host thread at a time.
 */
#ifndef KKM_H
#define KKM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KKM_ABI_VERSION 2

typedef enum kkm_status {
  KKM_OK = 0,
  KKM_EINVAL = 1,   /* invalid argument, or invalid index data found on the device */
  KKM_ENOMEM = 2,   /* a device or pinned-host allocation failed */
  KKM_ECUDA = 3,    /* a CUDA runtime or driver call failed */
  KKM_ETIMEOUT = 4, /* a bounded device wait gave up */
  KKM_ESTATE = 5,   /* the context is poisoned, or the call does not fit its state */
  KKM_ENOTSUP = 6   /* the combination of options is not supported */
} kkm_status;

/* Kernel functions K(x, y). Sec. 6 prints the Gaussian kernel. Sec. 1 names
 * the Laplacian kernel as normalised (gamma = 1) but prints no formula; the
 * library reads it as exp(-||x - y||_2 / sigma). The linear and polynomial
 * kernels are the textbook ones. */
typedef enum kkm_kernel_kind {
  KKM_GAUSSIAN = 0,  /* K = exp(-||x - y||^2 / param), param = kappa > 0      */
  KKM_LAPLACIAN = 1, /* K = exp(-||x - y||_2 / param), param = sigma > 0      */
  KKM_LINEAR = 2,    /* K = <x, y>                                            */
  KKM_POLY = 3       /* K = (<x, y> + coef0)^degree, 1 <= degree <= 8         */
} kkm_kernel_kind;

typedef struct kkm_kernel {
  int32_t kind;   /* kkm_kernel_kind */
  double param;   /* kappa (Gaussian) or sigma (Laplacian) */
  double coef0;   /* polynomial offset */
  int32_t degree; /* polynomial degree */
} kkm_kernel;

/* Learning rates. KKM_LR_BETA is alpha_i^j = sqrt(b_i^j / b), the rate of
 * Schwartzman (2023) that the truncation lemma's proof in Sec. 4.1 uses.
 * KKM_LR_CONST is alpha = eta. KKM_LR_SKLEARN is alpha_i^j = b_i^j / N^j with
 * N^j the points assigned to center j over all iterations, this batch
 * included (the running-mean rate Sec. 6 compares against; N^j is part of
 * the state, see kkm_get_cum_counts). Every rate gives an empty cluster
 * (b_i^j = 0) alpha = 0, so its center does not change. */
typedef enum kkm_lr { KKM_LR_BETA = 0, KKM_LR_CONST = 1, KKM_LR_SKLEARN = 2 } kkm_lr;

/* Arithmetic of the batch-by-support Gram products x.y (Sec. 4.1, "Algorithm
 * implementation and runtime"). Norms, kernel values and weighted sums are
 * FP32 in every form. Center norms and weights are FP64 in every form.
 *   FP32   : CUDA-core FP32 FMA products.
 *   BF16   : tcgen05 tensor cores, BF16 operands, FP32 accumulation.
 *   BF16X3 : tcgen05, split operands x = hi + lo (both BF16); the product is
 *            hi.hi + hi.lo + lo.hi, accumulated in FP32.
 *   TF32   : tcgen05 kind::tf32, operands rounded to TF32 (10 explicit
 *            mantissa bits, round to nearest with ties away), FP32
 *            accumulation.
 * The tensor-core forms need a compute capability 10.3 device: kkm_init
 * returns KKM_ENOTSUP for them on any other device (no CUDA-core stand-in). */
typedef enum kkm_precision {
  KKM_PREC_FP32 = 0,
  KKM_PREC_BF16 = 1,
  KKM_PREC_BF16X3 = 2,
  KKM_PREC_TF32 = 3
} kkm_precision;

/* How the centers are held.
 *   KKM_ALGO_WINDOWS : as weighted support rows (the truncated centers of
 *                      Eq. (1); with tau <= 0 every block is kept).
 *   KKM_ALGO_TABLE   : Algorithm 1 (untruncated; tau must be <= 0) through the
 *                      table <phi(x), C_j> for every x in X and every j, the
 *                      O(n(b+k))-per-iteration scheme of Appendix A: each step
 *                      is an n x b Gram pass against the center-sorted batch
 *                      and a table update. Needs n*k FP32 of table; support
 *                      rows are never stored, so kkm_get_state / set_state,
 *                      kkm_assign of arbitrary rows and the objective adjoint
 *                      return KKM_ENOTSUP (kkm_objective over X works). */
typedef enum kkm_algo { KKM_ALGO_WINDOWS = 0, KKM_ALGO_TABLE = 1 } kkm_algo;

typedef struct kkm_config {
  int32_t tau;       /* truncation parameter tau of Sec. 4.1; <= 0 runs Algorithm 1 untruncated */
  int32_t lr;        /* kkm_lr */
  double eta;        /* rate for KKM_LR_CONST, in (0, 1] */
  int32_t precision; /* kkm_precision */
  int32_t max_iters; /* untruncated runs only: iterations the support store must hold (>= 1) */
  uint64_t seed;     /* SplitMix64 seed of the built-in batch sampler */
  int32_t dist_tile; /* tensor-core forms: support rows per distance-pass tile, 64, 128 or 256; 0 = 256 */
  int32_t algo;      /* kkm_algo */
} kkm_config;

typedef struct kkm_ctx kkm_ctx;

/* ABI version of the loaded library (KKM_ABI_VERSION). */
int32_t kkm_version(void);

/* kkm_kmeanspp -- kernel k-means++ seeding (D^2 sampling in feature space,
 * the initialisation of Secs. 1 and 5): k data indices, the first uniform,
 * each later one with probability proportional to min over the chosen c of
 * Delta(x, c) = K(x,x) - 2K(x,c) + K(c,c), evaluated in FP64. Draw t uses
 * output t of SplitMix64 seeded with `seed`: the first as an index by
 * Lemire's multiply-high, the others as u = (h >> 11) 2^-53, picking the first
 * x whose running sum of D^2 exceeds u times the total.
 *   X       : device, n x d FP32, leading dimension ldx >= d.
 *   k       : 1 <= k <= n.
 *   kernel  : host; as for kkm_init.
 *   out_idx : host, k int64 (the indices kkm_init's init_idx takes).
 *   stream  : cudaStream_t or NULL. The call allocates n + n/8 + k words of
 *             device scratch, frees it, and synchronises the stream.
 * kkm_last_error(NULL) reports failures. */
kkm_status kkm_kmeanspp(const float* X, int64_t n, int32_t d, int64_t ldx, int32_t k, const kkm_kernel* kernel,
                        uint64_t seed, int64_t* out_idx, void* stream);

/* kkm_form_supported -- whether a precision form (kkm_precision) runs on a
 * device of compute capability cc_major.cc_minor: KKM_OK, or KKM_ENOTSUP for
 * the tensor-core forms (BF16, split-BF16, TF32) on anything but 10.3, where
 * the library has only its tcgen05 passes built for sm_103a and no CUDA-core
 * stand-in. KKM_EINVAL for an unknown form. Host only, no CUDA call; kkm_init
 * applies the same rule to the current device. The paper has no counterpart
 * (its precision is not stated). */
kkm_status kkm_form_supported(int32_t precision, int32_t cc_major, int32_t cc_minor);

/* kkm_init -- creates a run (the inputs of Algorithms 1/2).
 *   out        : host; receives the new context, or NULL on failure.
 *   X          : device, n x d FP32 dataset, leading dimension ldx >= d.
 *                Caller-owned. It must stay alive and unchanged until
 *                kkm_destroy, because batches and support rows are read
 *                from it.
 *   n, d       : 1 <= n < 2^31, 1 <= d <= 4096.
 *   k          : number of centers, 1 <= k <= min(n, 1024).
 *   kernel     : host; copied.
 *   b          : batch size, 1 <= b <= 8192.
 *   cfg        : host; copied.
 *   init_idx   : host, k data indices in [0, n): C_1^j = phi(x_{init_idx[j]}),
 *                for example from kernel k-means++ (Secs. 1 and 5). NULL picks
 *                k distinct indices with the library's own seeded sampler.
 *   stream     : cudaStream_t on which every later call of this context
 *                queues its work. NULL means the legacy default stream.
 * KKM_ENOTSUP when cfg->precision is not FP32 and the device is not compute
 * capability 10.3 (see kkm_form_supported).
 * Allocates all device state up front: the support store of k*(2*tau + 4*b + 8)
 * rows (k*(1 + b*max_iters) when untruncated) and the step workspaces. No
 * later call allocates. Sets ||C_1^j||^2 = K(x, x). */
kkm_status kkm_init(kkm_ctx** out, const float* X, int64_t n, int32_t d, int64_t ldx, int32_t k,
                    const kkm_kernel* kernel, int32_t b, const kkm_config* cfg,
                    const int64_t* init_idx, void* stream);

/* kkm_step -- one iteration i of Algorithm 2 (Algorithm 1 when untruncated),
 * Appendix A. It samples or takes the batch B_i, computes the distances
 * Delta(x, C_i^j) = K(x,x) - 2 sum_s w_s K(x, y_s) + ||C_i^j||^2 (Sec. 1 and
 * Sec. 4), assigns each x to the argmin (ties go to the lowest j), forms
 * b_i^j and alpha_i^j, and updates every window as Eq. (1) and the sliding
 * window of Sec. 4.1 describe: decay the old weights by (1 - alpha), append
 * B_i^j with weight alpha / b_i^j per row, drop the oldest blocks that fall
 * out of Q_i^j, and drop C_1 once min Q_i^j > 1. It then carries ||C^j||^2 by
 * the Sec. 4 recurrence, corrected for the dropped rows, in FP64.
 *   batch_idx     : device, b int32 indices in [0, n), or NULL to draw them
 *                   with SplitMix64: output (i-1)*b + s of the generator
 *                   seeded with cfg->seed, mapped to [0, n) by floor(h*n/2^64).
 *   forced_assign : device, b centers in [0, k) that replace the argmin in the
 *                   update, or NULL. This is teacher forcing for tests; the
 *                   distances are still computed.
 *   assign_out    : device, b int32, or NULL. Receives argmin_j Delta(x, C_i^j).
 *   dist_out      : device, b x k FP32 row-major, or NULL. Receives Delta(x, C_i^j).
 *   batch_obj_out : device, one double, or NULL. Receives
 *                   f_{B_i}(C_i) = (1/b) sum_x min_j Delta(x, C_i^j) (Sec. 3).
 * An index out of range is found on the device, and it poisons the context.
 * The last kernel of the weight update (k_finalize) is queued at the start of
 * the next kkm_step, where it runs beside the next batch's gather, or by the
 * next call that reads or replaces the centers (every call below but
 * kkm_stats and the timing and launch counters), or by kkm_flush. The
 * outputs above do not depend on it. */
kkm_status kkm_step(kkm_ctx* ctx, const int32_t* batch_idx, const int32_t* forced_assign,
                    int32_t* assign_out, float* dist_out, double* batch_obj_out);

/* kkm_flush -- queues the weight update the last kkm_step left pending, if
 * any, on the context's stream (asynchronous; nothing to do otherwise). */
kkm_status kkm_flush(kkm_ctx* ctx);

/* kkm_steps -- n iterations of kkm_step with the built-in sampler and no
 * outputs: the fixed-iteration loop of the experiments (Sec. 6). With graphs
 * enabled (kkm_graph_enable) it replays a captured graph of 16 iterations,
 * inside which consecutive iterations meet through programmatic dependent
 * launch, and runs the remainder one step at a time. The result is the same,
 * bit for bit, as n calls of kkm_step(ctx, NULL, NULL, NULL, NULL, NULL).
 * Asynchronous; n >= 0. */
kkm_status kkm_steps(kkm_ctx* ctx, int64_t n);

/* kkm_step_eval -- kkm_step (device sampler when batch_idx is NULL) that
 * also evaluates the updated centers on the same batch: obj_before_dev
 * receives f_{B_i}(C_i) and obj_after_dev f_{B_i}(C_{i+1}) (device doubles,
 * both required). Their difference is the improvement the early-stopping
 * rule of Sec. 5 tests. Asynchronous. */
kkm_status kkm_step_eval(kkm_ctx* ctx, const int32_t* batch_idx, double* obj_before_dev, double* obj_after_dev);

/* kkm_fit -- up to max_iters iterations with early stopping (Sec. 5): it
 * stops after the first iteration whose improvement
 * f_{B_i}(C_i) - f_{B_i}(C_{i+1}) is below eps. Writes the iterations done
 * and the last improvement (host; either may be NULL). Synchronises every
 * iteration. */
kkm_status kkm_fit(kkm_ctx* ctx, int64_t max_iters, double eps, int64_t* iters_done, double* last_improvement);

/* kkm_get_cum_counts / kkm_set_cum_counts -- the cumulative counts N^j of
 * the sklearn rate (k int64, host). Part of a checkpoint of such a run;
 * kkm_init starts them at 0. Both synchronise. */
kkm_status kkm_get_cum_counts(kkm_ctx* ctx, int64_t* counts);
kkm_status kkm_set_cum_counts(kkm_ctx* ctx, const int64_t* counts);

/* kkm_graph_enable -- with enable != 0, kkm_step captures its kernel sequence
 * in a CUDA graph and replays that graph. The graph is built once for each
 * combination of kkm_step pointer arguments (rebuilt when they change) and
 * launched on the context's stream. Replays give results identical to eager
 * steps. Capture starts only after one eager step, and never while event
 * timing is enabled. Reuse the same buffers to keep replaying one graph. */
kkm_status kkm_graph_enable(kkm_ctx* ctx, int32_t enable);

/* kkm_step_host -- kkm_step with host buffers, for callers that keep the
 * batch on the CPU. batch_idx (b indices; NULL for the built-in sampler),
 * assign_out (b) and batch_obj_out (f_{B_i}(C_i)) are ordinary host memory;
 * either output may be NULL. The values pass through a staging area of the
 * context in page-locked, device-mapped host memory: the call copies the
 * indices into it, the step's kernels read them and write the results there
 * across the CPU-GPU link (no copy-engine transfer), and after the stream
 * synchronises the call copies the results out. It returns once the step is
 * done. */
kkm_status kkm_step_host(kkm_ctx* ctx, const int32_t* batch_idx, int32_t* assign_out,
                         double* batch_obj_out);

/* kkm_steps_host -- n iterations of Algorithm 2 with host buffers, as n calls
 * of kkm_step_host would run them, without a host round trip per step.
 *   batch_idx     : host, n x b indices (step i's batch at i*b), or NULL for
 *                   the built-in sampler.
 *   assign_out    : host, n x b int32 (step i's assignments at i*b), or NULL.
 *   batch_obj_out : host, n doubles f_{B_i}(C_i), or NULL.
 * Steps go in chunks of 16 through two staging slots of the context in
 * page-locked, device-mapped host memory: while the device runs one chunk
 * (one CUDA graph replay when graphs are enabled), the call copies the next
 * chunk's indices in and the previous chunk's results out. Every step's
 * indices and results still cross the CPU-GPU link. A context's first step,
 * and every step while timing is enabled, go through kkm_step_host. Returns
 * once all n steps are done, after the device status check. n < 0 is
 * KKM_EINVAL; an untruncated run (tau = 0) may not pass max_iters. On a
 * failure the outputs are unspecified, and no staged work is left in flight. */
kkm_status kkm_steps_host(kkm_ctx* ctx, int64_t n, const int32_t* batch_idx, int32_t* assign_out,
                          double* batch_obj_out);

/* kkm_assign -- nearest centers of arbitrary query points (the assignment
 * rule of Algorithms 1/2, applied to the current centers without updating
 * them).
 *   Q          : device, m x d FP32, leading dimension ldq >= d; m >= 0.
 *   assign_out : device, m int32, or NULL.
 *   mind_out   : device, m FP32 min_j Delta(q, C_j), or NULL.
 *   dist_out   : device, m x k FP32, or NULL.
 * Work goes in chunks of at most b rows through the same kernels as kkm_step. */
kkm_status kkm_assign(kkm_ctx* ctx, const float* Q, int64_t m, int64_t ldq, int32_t* assign_out,
                      float* mind_out, float* dist_out);

/* kkm_objective -- f_A(C) = (1/|A|) sum_{a in A} min_j Delta(a, C_j) (Sec. 3)
 * for A = the rows of Q (device, m x d, ldq), or for A = X when Q is NULL.
 * The sum is taken in FP64. Synchronises the stream and writes the value to
 * *out (host). */
kkm_status kkm_objective(kkm_ctx* ctx, const float* Q, int64_t m, int64_t ldq, double* out);

/* kkm_objective_fwd / kkm_objective_bwd -- the batch objective of Sec. 3,
 * f_A(C) = (1/|A|) sum_a Delta(a, C_{assign(a)}), at GIVEN assignments, as a
 * differentiable function of the query rows and of the bandwidth, and its
 * adjoint. The centers (support rows, weights) are held fixed and the
 * bandwidth is parameterised by s = log_sigma: Gaussian kappa = 2 e^{2s},
 * Laplacian sigma = e^s (the context's own kernel parameter is not used or
 * changed). Only the Gaussian and Laplacian kernels qualify (KKM_ENOTSUP
 * otherwise), with d <= 1024.
 *   Q        : device, m x d FP32, leading dimension ldq >= d; 1 <= m < 2^30.
 *   assign   : device, m int32 centers in [0, k) (an index outside sets the
 *              device status; the next synchronising call returns KKM_EINVAL).
 *   loss_out : device, 1 double: the objective.
 *   delta_out: device, m FP32 Delta(q, C_{assign(q)}), or NULL.
 * The adjoint recomputes every kernel value (nothing is kept between calls):
 *   grad_loss      : device, 1 double, dObjective of the caller's loss.
 *   grad_q         : device, m x d FP32 (leading dimension ldg >= d):
 *                    grad_loss * d objective / d Q. Support rows are constants.
 *   grad_log_sigma : device, 1 double: grad_loss * d objective / d s.
 * Both calls are asynchronous on the context's stream (two kernel launches
 * each) and allocate a workspace that grows with m and lives until
 * kkm_destroy. Results are deterministic: every sum across rows and blocks
 * runs in a fixed order. */
kkm_status kkm_objective_fwd(kkm_ctx* ctx, const float* Q, int64_t m, int64_t ldq, const int32_t* assign,
                             double log_sigma, double* loss_out, float* delta_out);
kkm_status kkm_objective_bwd(kkm_ctx* ctx, const float* Q, int64_t m, int64_t ldq, const int32_t* assign,
                             double log_sigma, const double* grad_loss, float* grad_q, int64_t ldg,
                             double* grad_log_sigma);

/* kkm_sync -- synchronises the context's stream and reports device-side faults. */
kkm_status kkm_sync(kkm_ctx* ctx);

/* Checkpoint / restore of the centers (Eq. (1) window layout). It is also
 * how tests load a state computed elsewhere ("teacher forcing").
 * kkm_get_state_sizes writes the total support rows S and the total block
 * count; both are host outputs. kkm_get_state fills host arrays:
 *   iteration         : the next iteration number i (1-based)
 *   rows_per_center   : k int32, support rows of each center
 *   row_idx, row_w    : S entries, center-major, window order. For each
 *                       center this is C_1 first (when kept), then the blocks
 *                       from oldest to newest, each in batch order. row_idx
 *                       holds data indices, row_w the FP64 weights.
 *   blocks_per_center : k int32
 *   block_iter        : per block, the iteration that appended it (0 = C_1)
 *   block_count       : per block, its rows
 *   c1_kept           : k bytes, 1 while C_1 is part of the center
 *   cnorm             : k doubles, ||C_j||^2
 * Both calls synchronise. kkm_set_state takes the same arrays. It checks
 * them against each other and the capacities (KKM_EINVAL on any mismatch),
 * then gathers the support rows from X. */
kkm_status kkm_get_state_sizes(kkm_ctx* ctx, int64_t* total_rows, int64_t* total_blocks);
kkm_status kkm_get_state(kkm_ctx* ctx, int64_t* iteration, int32_t* rows_per_center,
                         int64_t* row_idx, double* row_w, int32_t* blocks_per_center,
                         int64_t* block_iter, int32_t* block_count, uint8_t* c1_kept,
                         double* cnorm);
kkm_status kkm_set_state(kkm_ctx* ctx, int64_t iteration, const int32_t* rows_per_center,
                         const int64_t* row_idx, const double* row_w,
                         const int32_t* blocks_per_center, const int64_t* block_iter,
                         const int32_t* block_count, const uint8_t* c1_kept,
                         const double* cnorm);

/* kkm_stats -- counters accumulated on the device since kkm_init or the last
 * reset (reset != 0 clears them after reading). Synchronises. Host outputs:
 *   steps        : kkm_step calls
 *   support_rows : sum over steps of S, the support rows the distance pass
 *                  read (the algorithmic size of the b x S Gram product)
 *   gram_tiles   : sum over steps of the support tiles the distance kernel ran
 * Any output may be NULL. */
kkm_status kkm_stats(kkm_ctx* ctx, int64_t* steps, int64_t* support_rows, int64_t* gram_tiles,
                     int32_t reset);

/* kkm_timing -- CUDA-event timing of the distance kernel (the b x S Gram
 * product with its kernel and weighted-sum epilogue). While it is enabled
 * (enable != 0), every eager kkm_step records a pair of events on the
 * context's stream around that kernel, for up to 4096 steps. With enable = R
 * > 1 the step launches the kernel R times back to back between the two
 * events (it is idempotent: it rewrites the same partial sums from the same
 * inputs) and the record is the average, which leaves out the launch gap
 * that a single launch between two events includes. enable must be in
 * [0, 1000] (KKM_EINVAL otherwise). kkm_timing_read synchronises and writes
 * the launches recorded and the sum of their per-launch milliseconds (host).
 * reset != 0 clears the record. */
kkm_status kkm_timing_enable(kkm_ctx* ctx, int32_t enable);
kkm_status kkm_timing_read(kkm_ctx* ctx, int64_t* launches, double* total_ms, int32_t reset);

/* kkm_launches -- number of CUDA kernels this context has launched (counted on
 * the host at each launch) since kkm_init or the last reset. Host output. */
kkm_status kkm_launches(kkm_ctx* ctx, int64_t* launches, int32_t reset);

/* ------------------------------------------------------------------------
 * Full-batch kernel k-means (kernel Lloyd) -- the baseline the paper
 * compares its mini-batch algorithm with (Sec. 6; its O(n^2) cost per
 * iteration is the motivation of Sec. 1).
 *
 * Every iteration assigns all n points to their nearest center and moves
 * every center that got points to the mean of its points in feature space,
 * C_j = (1/n_j) sum_{x in X_j} phi(x). This equals Algorithm 1 with the whole
 * data set as the batch and learning rate 1; a center with no points keeps
 * its value. The run keeps T[j][x] = <phi(x), C_j> (k x n FP32) and
 * ||C_j||^2 = (1/n_j) sum_{x in X_j} T[j][x]; T comes from the n x n Gram
 * pass of X against X sorted by center, in the chosen precision form.
 * Distances and the argmin use Delta(x, C_j) = K(x,x) - 2 T[j][x] + ||C_j||^2
 * in FP32 (ties go to the lowest j); f_X sums the minima in FP64.
 * ------------------------------------------------------------------------ */
typedef struct kkm_lloyd kkm_lloyd;

/* kkm_lloyd_init -- a run on X and k initial points; assigns every point to
 * its nearest initial point before it returns (f_X at the initial centers).
 *   X         : device, n x d FP32, leading dimension ldx >= d. Read only
 *               during this call (the run keeps its own operand copy).
 *   k         : 1 <= k <= min(n, 1024)
 *   kernel    : host, as in kkm_init
 *   precision : kkm_precision; the BF16, split-BF16 and TF32 forms need a
 *               compute capability 10.3 device (else KKM_ENOTSUP)
 *   init_idx  : host, k indices into X (the initial centers phi(x_i))
 *   chunk_rows: rows of X per Gram-pass launch, a multiple of 128, or 0 for
 *               the largest chunk whose partial sums fit in 1 GiB
 *   stream    : cudaStream_t the run queues its work on
 * Device memory: about (2 n + k tn) ld operand elements, k n floats for T and
 * the chunk's partial sums. Synchronises the stream before returning. */
kkm_status kkm_lloyd_init(kkm_lloyd** out, const float* X, int64_t n, int32_t d, int64_t ldx, int32_t k,
                          const kkm_kernel* kernel, int32_t precision, const int64_t* init_idx,
                          int64_t chunk_rows, void* stream);
/* kkm_lloyd_iterate -- queues `iters` iterations (center update from the
 * current assignment, then the new assignment). Does not synchronise. */
kkm_status kkm_lloyd_iterate(kkm_lloyd* run, int32_t iters);
/* kkm_lloyd_read -- synchronises; host outputs (each may be NULL): f_X at the
 * current centers, the number of points whose assignment the last
 * assignment changed (all n after kkm_lloyd_init; 0 at Lloyd's fixed point),
 * and the iterations run. Reports device-side errors (KKM_ETIMEOUT for a
 * bounded wait in the Gram pass that gave up). */
kkm_status kkm_lloyd_read(kkm_lloyd* run, double* obj, int64_t* changed, int64_t* iters_done);
/* kkm_lloyd_assignments -- device outputs (each may be NULL): the n
 * assignments at the current centers, and min_j Delta(x, C_j). Queued on the
 * run's stream. */
kkm_status kkm_lloyd_assignments(kkm_lloyd* run, int32_t* assign_out, float* mind_out);
/* kkm_lloyd_distances -- device output: Delta(x, C_j), n x k FP32 row-major,
 * the values the assignment compares. Queued on the run's stream. */
kkm_status kkm_lloyd_distances(kkm_lloyd* run, float* dist_out);
/* kkm_lloyd_center_norms -- host output: ||C_j||^2 (k doubles). Synchronises. */
kkm_status kkm_lloyd_center_norms(kkm_lloyd* run, double* out);
/* kkm_lloyd_info -- host outputs (each may be NULL): kernels launched so far
 * (host count), Gram-pass chunks per iteration and rows per chunk. */
kkm_status kkm_lloyd_info(const kkm_lloyd* run, int64_t* launches, int32_t* chunks, int64_t* chunk_rows);
/* kkm_lloyd_destroy -- synchronises the stream and frees the run (NULL is a no-op). */
kkm_status kkm_lloyd_destroy(kkm_lloyd* run);
/* kkm_lloyd_last_error -- the message of the run's last failure, or, for
 * NULL, of this thread's last failed kkm_lloyd_init. */
const char* kkm_lloyd_last_error(const kkm_lloyd* run);

/* kkm_distances_noalloc -- distances and nearest centers with no allocation.
 *
 * The paper has no counterpart to this call. It exists for callers that
 * cannot call cudaMalloc. One kind is a process whose device memory a
 * framework's caching allocator or a pre-sized arena owns completely (a
 * serving process that reserved the free memory at start-up). There, a stray
 * cudaMalloc fails or fragments the reservation. The other kind is a loop on a
 * latency-critical path, where cudaMalloc and cudaFree can synchronise the
 * device. Such a caller keeps its centers itself, as weighted support rows in
 * the window layout that kkm_get_state exports. The call needs no context.
 *
 * It computes Delta(q, C_j) = K(q,q) - 2 sum_s w_s K(q, y_s) + ||C_j||^2 for
 * every query row q and center j, in FP32 arithmetic with FP64 combination,
 * and the argmin over j (ties go to the lowest j).
 *   Q        : device, m x d FP32, leading dimension ldq >= d; m >= 0
 *   Y        : device, S x d FP32 support rows, leading dimension ldy >= d
 *   w        : device, S FP32 weights
 *   seg_off  : device, k + 1 int32 offsets. Center j owns the rows
 *              [seg_off[j], seg_off[j+1]) of Y; an empty range is a center
 *              with no support row (its inner products are 0). The offsets
 *              must be non-decreasing within [0, S]. Offsets that are not are
 *              found on the device: every distance of the call is then NaN
 *              and every assignment -1.
 *   cnorm    : device, k doubles, ||C_j||^2
 *   kernel   : host, as in kkm_init
 *   dist_out : device, m x k FP32 row-major, or NULL
 *   assign_out: device, m int32, or NULL
 *   stream   : cudaStream_t, NULL for the legacy default stream
 * Limits: k <= 1024, d <= 4096, S <= KKM_NOALLOC_MAX_SUPPORT and
 * ceil(S / 64) + k <= KKM_NOALLOC_MAX_TILES. Larger sizes are rejected with
 * KKM_EINVAL before any work is queued. Query rows go through in passes of
 * KKM_NOALLOC_MAX_ROWS_PER_PASS.
 *
 * Memory: the only scratch is one fixed array of KKM_NOALLOC_SCRATCH_BYTES
 * inside the library. CUDA loads modules lazily by default, so the array and
 * the call's kernels come onto a device at the first call made with that
 * device current: that call looks up the array's address
 * (cudaGetSymbolAddress) and launches the kernels, and so reserves the
 * scratch and the code. A call with m = 0 does only that (launching each
 * kernel once on empty work) and reads no other argument. Make the first
 * call on each device, for example with m = 0, before reserving the rest of
 * the device memory and before any stream capture. After it the call never
 * allocates or frees, neither directly nor through a library, and the device
 * keeps the array until the process exits. Every call shares the array:
 * calls whose work overlaps on the GPU (two streams with no ordering between
 * them) race on it, while calls queued one after another on one stream are
 * safe. The call only queues work on `stream`; a failed launch is reported
 * from that launch's own status, not from an error left by earlier work.
 * Errors are reported through kkm_noalloc_last_error(), a per-thread
 * message. */
#define KKM_NOALLOC_MAX_ROWS_PER_PASS 1024
#define KKM_NOALLOC_MAX_TILES 1024
#define KKM_NOALLOC_MAX_SUPPORT 65536
#define KKM_NOALLOC_SCRATCH_BYTES (4718592) /* 4.5 MiB */
kkm_status kkm_distances_noalloc(const float* Q, int64_t m, int64_t ldq, int32_t d, const float* Y,
                                 int64_t S, int64_t ldy, const float* w, const int32_t* seg_off,
                                 const double* cnorm, int32_t k, const kkm_kernel* kernel,
                                 float* dist_out, int32_t* assign_out, void* stream);
const char* kkm_noalloc_last_error(void);

/* kkm_probe_bounded_wait -- the failure-detection path of the tcgen05 passes
 * on the current device. The paper has no counterpart. One thread waits on a
 * shared-memory mbarrier (the kind every role of the passes waits on) with the
 * passes' bounded wait, limited to limit_ns (1e3 .. 5e9). With arrive = 0
 * nothing arrives, so the wait runs out and the call returns KKM_ETIMEOUT, as
 * a step whose pass gave up reports through the context's status; with
 * arrive = 1 the thread arrives first and the call returns KKM_OK. Allocates
 * and frees one int of device memory and synchronises the stream. KKM_EINVAL
 * for arguments out of range (checked before any CUDA call). */
kkm_status kkm_probe_bounded_wait(int64_t limit_ns, int32_t arrive, void* stream);

/* kkm_probe_unit_rate -- measured issue rate of one arithmetic unit on the
 * current device. The paper has no counterpart: it supplies the denominators
 * of the distance pass's roofline (the pass's epilogue spends one MUFU
 * exponential and a few FP32 FMAs per kernel value).
 *   op         : 0 ex2.approx.ftz.f32 (MUFU), 1 scalar FP32 fma, 2 packed
 *                f32x2 fma (counted as two FP32 FMAs)
 *   iters      : loop trips per thread, 1 .. 2^24 (eight operations each)
 *   per_clk_sm : host out, operations per SM per SM clock (median over the
 *                SMs' own cycle counters, so independent of the clock rate)
 *   per_second : host out, operations per second over the whole device
 *   stream     : cudaStream_t, NULL for the legacy default stream
 * One block of 1024 threads runs on every SM. The call allocates and frees
 * two small device buffers, and it synchronises. KKM_EINVAL for a bad op or
 * iters, KKM_ECUDA when a CUDA call fails. */
kkm_status kkm_probe_unit_rate(int32_t op, int64_t iters, double* per_clk_sm, double* per_second, void* stream);

/* Frees everything the context allocated. NULL is accepted. It synchronises first. */
kkm_status kkm_destroy(kkm_ctx* ctx);

/* Run groups: many independent runs (restarts, bandwidth or k sweeps, runs
 * of different n, d, k, b) stepped together.
 * kkm_group_create -- groups n distinct contexts of one device. stream (a
 *   cudaStream_t, or NULL for a stream of the group's own) orders the
 *   group's work. The runs' own streams are synchronised once here; while
 *   grouped, a run must not be stepped on its own, and kkm_group_sync must
 *   precede any other call on a run. The group does not own the runs.
 *   The runs' device buffers and settings are captured here: a group of
 *   windows-form runs steps them with one launch per step phase over all
 *   runs (gather, argmin, sort/plan, row moves, weight update) and one launch
 *   per Gram pass and class of runs sharing form, kernel kind and distance
 *   tile; each block of such a launch does what one block of one run's own
 *   launch would, so every run's results equal its single-run steps. A group
 *   with table-form runs steps each run on a branch of its own.
 * kkm_group_step -- one iteration of every run (each with its built-in
 *   sampler), asynchronous. From the second call on, the iteration of all
 *   runs is one CUDA graph launch.
 * kkm_group_sync -- synchronises and reports each run's device status.
 * kkm_group_set_chains -- before the first group step: deal the runs to
 *   `chains` chains (1 <= chains <= n), each stepped by its own per-phase
 *   launches on a graph branch of its own with a share of the SMs by
 *   estimated work, so one chain's short phases overlap another's Gram
 *   passes. chains = 0 steps every run on a graph branch of its own with its
 *   own kernels (the launch structure of a group with table-form runs, which
 *   accept no other value: KKM_ENOTSUP). The default is 2 for 16 runs or
 *   more, else 1. Which is fastest depends on the mix of runs; measure.
 * kkm_group_launches -- host outputs (each may be NULL): kernels the group's
 *   steps have launched and kernels per step; reset != 0 clears the count.
 * kkm_group_last_error(NULL) gives the calling thread's last create failure. */
typedef struct kkm_group kkm_group;
kkm_status kkm_group_create(kkm_group** out, kkm_ctx* const* runs, int32_t n, void* stream);
kkm_status kkm_group_step(kkm_group* group);
kkm_status kkm_group_set_chains(kkm_group* group, int32_t chains);
kkm_status kkm_group_launches(kkm_group* group, int64_t* launches, int32_t* per_step, int32_t reset);
kkm_status kkm_group_sync(kkm_group* group);
const char* kkm_group_last_error(kkm_group* group);
kkm_status kkm_group_destroy(kkm_group* group);

/* Message of the last failure (see the conventions above). Never NULL. */
const char* kkm_last_error(const kkm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* KKM_H */
