/*
 * opevo.h - C ABI of the GB300 orthogonality-preserving eigensolver.
 *
 * Method: Chu, Dai, Wang, Zhou, "An orthogonality-preserving approach for
 * eigenvalue problems" (arXiv 2511.06788).  Given a potential V on a box, the
 * library computes the lowest p eigenpairs of H = -1/2 Delta_h + V (problem
 * (2.2) of §2.2, finite differences instead of the paper's finite elements)
 * by the midpoint time stepping (4.1) of §4.1, carried out as Steps 1-4:
 *
 *   Step 1  W = G U,  G = (H + sigma)^-1     p independent source problems
 *   Step 2  B = (I + tau^2/4 <W,W> - tau^2/4 <W,U><W,U>)^-1
 *   Step 3  tau/2 A = I - B + tau/2 <W,U> B
 *   Step 4  U <- U - tau U A + tau W B
 *
 * iterated by Algorithm 1 of §4.1.  <X,Y> is the inner matrix of §2.1
 * (<X,Y>_ij = x_i . y_j).
 *
 * Conventions shared by every entry point
 *   - Return value: an op_status; no exception, abort or exit crosses the ABI.
 *     On error, op_last_error() returns a message for the calling thread.
 *   - Grid ordering: point (ix, iy, iz) of an nx x ny x nz interior grid has
 *     index ix + nx*(iy + ny*iz); its coordinate on axis d is
 *     lo[d] + (i_d + 1) h_d with h_d = (hi[d] - lo[d]) / (n_d + 1); the
 *     boundary of the box carries zero values (Dirichlet).
 *   - Orbital blocks are row-major n x ld (ld >= p; the p values of one grid
 *     point are contiguous; columns p..ld-1 are padding and are kept zero).
 *   - Host pointers are caller-owned and only read or written during the call.
 *     Device pointers are caller-owned, must stay valid until the work queued
 *     on `stream` has finished, and must be 16-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Kernel-level calls only enqueue work; context-level calls
 *     synchronise the context's stream where they say so.
 *   - Inputs and outputs in FP64 unless stated; blocks of a context in
 *     OP_FP32 or a mixed mode are stored in FP32 on the device.
 */
#ifndef OPEVO_H
#define OPEVO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OP_OK = 0,
  OP_ERR_ARG = -1,       /* invalid argument (null pointer, size, alignment, mode) */
  OP_ERR_CUDA = -2,      /* a CUDA runtime call failed (message has the detail)   */
  OP_ERR_NOTSPD = -3,    /* factorisation breakdown: zero/non-finite Step-2 pivot, or a
                            non-positive Cholesky-QR pivot                           */
  OP_ERR_DIVERGED = -4,  /* non-finite energy / residual, or energy increase beyond roundoff */
  OP_ERR_TIMEOUT = -5,   /* a bounded device wait gave up                           */
  OP_ERR_OOM = -6,       /* device allocation failed                               */
  OP_ERR_STATE = -7      /* call not valid in the context's current state          */
} op_status;

typedef enum {
  OP_FP64 = 0,           /* blocks, stencil, CG, Gram and update in FP64 (the Gram and
                            update by op_problem.fp64_gemm)                          */
  OP_FP32 = 1,           /* blocks, stencil and CG in FP32; Gram and update on the
                            tensor cores with a TF32 hi/lo split (FP32-class accuracy),
                            Gram chunk sums in FP64; Step 2-3 core in FP64           */
  OP_MIX_TF32 = 2,       /* as OP_FP32 but one TF32 MMA per product (operands rounded
                            to TF32, 10-bit mantissa); context-level API only        */
  OP_MIX_BF16X3 = 3,     /* as OP_FP32 but the Gram and update take BF16 operands split
                            in three (x = b0 + b1 + b2 to 2^-24) and six kind::f16 MMAs
                            per product (piece index sum <= 2), FP32 accumulation    */
  OP_MIX_BF16 = 4        /* as OP_MIX_BF16X3 with one piece and one MMA per product
                            (operands rounded to BF16, 8-bit mantissa); context-level
                            API only                                                 */
} op_prec;

/* Solver of the source problems (H + sigma) w = u of Step 1 (the paper does not say how
 * they are solved; every choice stops on the same unpreconditioned residual test). */
typedef enum {
  OP_PRECOND_NONE = 0,   /* conjugate gradients                                       */
  OP_PRECOND_JACOBI = 1  /* conjugate gradients preconditioned with d = diag(H + sigma)
                            (z = r / d; the residual buffer holds z)                   */
} op_precond;

/* The evolution the scheme discretises.  OP_FLOW_G is the paper's model (§2.2):
 * dU/dt = G U <U,U> - U <G U,U>, Step 1 solving W = (H + sigma)^-1 U.  OP_FLOW_L2 is the
 * L2 gradient flow of the earlier orthogonality-preserving schemes the paper contrasts
 * itself with (§1): the midpoint step with W = -(H + sigma) U (a stencil apply, no
 * solve; sigma drops out of U+), taken as the exact Cayley transform (a 2p x 2p solve
 * with the joint Gram of [U W], p <= 256) because this W amplifies any drift of <U,U>
 * through the p x p Steps 2-3.  Its useful time step shrinks with the mesh width like
 * h^2 (the CFL restriction the paper's model removes). */
typedef enum {
  OP_FLOW_G = 0,
  OP_FLOW_L2 = 1
} op_flow;

/* How FP64 contexts form their FP64 products of n x p blocks (the Grams of §2.1 and the
 * Step-4 update, also the set-up Cholesky-QR of every mode and, for p > 128, the
 * Newton-Schulz inverse of the Step-2 matrix).  OP_GEMM_TC: every FP64 operand is written
 * exactly as balanced base-256 integer digits (one power-of-two exponent per row of the
 * contraction; seven digits for the Gram, eight for the update), the digit products with
 * digit index sum below the digit count (28 or 36) run on the tensor cores (tcgen05
 * kind::f16) with exact integer level sums over runs of 256 terms, added in int64 and
 * scaled back in FP64: each product term is exact up to 2^-53.4 (Gram) or 2^-61.4
 * (update) of |a| |b| for the largest |a|, |b| of their rows, so the result carries an
 * error of the class of an FP64 dot product.  OP_GEMM_FMA: FP64 FMA on the FP64 pipe
 * (about 2 per clock per SM on GB300). */
typedef enum {
  OP_GEMM_TC = 0,
  OP_GEMM_FMA = 1
} op_fp64_gemm;

/* Solver of Step 1 in a context.  OP_STEP1_CG: conjugate gradients in the block precision.
 * OP_STEP1_REFINE (FP64 contexts): iterative refinement in FP64 around an FP32 CG; every
 * cycle forms the FP64 residual, stops when each column meets the FP64 residual test of
 * cg_rtol, and otherwise adds the FP32 CG's solution of the scaled residual equation.
 * OP_STEP1_AUTO: OP_STEP1_REFINE for FP64 contexts with fp64_gemm = OP_GEMM_TC, else CG. */
typedef enum {
  OP_STEP1_AUTO = 0,
  OP_STEP1_CG = 1,
  OP_STEP1_REFINE = 2
} op_step1;

typedef enum {
  OP_STOP_RESIDUAL = 0,  /* r <= tol, r = ||H U - U Theta||_F / (||H+sigma||_G sqrt(p)) */
  OP_STOP_ERR_E = 1,     /* Algorithm 1: |E(U^{n+1}) - E(U^n)| / |E(U^n)| <= tol   */
  OP_STOP_STEPS = 2      /* exactly max_steps steps                               */
} op_stop;

typedef enum {
  OP_EIG_RITZ = 0,       /* eigenvalues of Theta = U^T H U (ascending)             */
  OP_EIG_PAPER = 1       /* eigenvalues of <GU,U>^-1 minus sigma (error measures of §5) */
} op_eig_kind;

/* Problem description (the data of problem (2.2) plus the scheme's parameters). */
typedef struct {
  int dim;               /* 2 or 3                                                  */
  int shape[3];          /* interior points per axis (shape[2] ignored for dim 2)   */
  double lo[3], hi[3];   /* box                                                     */
  int p;                 /* number of eigenpairs N (>= 1)                           */
  double sigma;          /* shift of G = (H+sigma)^-1; NaN: max(0, 1 - L) with L =
                            sum_d (2/h_d^2) sin^2(pi/(2(n_d+1))) + min V            */
  double tau;            /* uniform time step; NaN: 1.5 (L + sigma), or for OP_FLOW_L2
                            1 / ||H + sigma||_G (Gershgorin bound 2 sum_d 1/h_d^2 +
                            max |V + sigma|)                                         */
  int prec;              /* op_prec                                                 */
  double cg_rtol;        /* Step-1 CG: relative residual per column; <= 0 selects
                            max(floor, min(1e-2, 0.1 g)) with g the relative
                            G-residual sqrt(g_residual / tr<W,W>) of the previous
                            step, floor 1e-13 (FP64) or 1e-6 (FP32); inside op_solve
                            also <= 0.1 tol (residual rule) or 0.1 sqrt(tol) (err_E) */
  int cg_max_iter;       /* Step-1 CG iteration cap per step (<= 0: 2000)           */
  int check_every;       /* op_solve: residual evaluated every this many steps (<= 0: 10) */
  int adapt_every;       /* op_solve: <= 0 keeps sigma and tau fixed; > 0 re-tunes them
                            (inside op_solve, before a step whose context step count
                            is a multiple of this) from the Ritz values lambda_1 <= ..
                            <= lambda_p of the current U: sigma = max(sigma_0,
                            lambda_p - 2 lambda_1) (the shift that maximises the
                            per-step contraction (lambda_1 + sigma) / (lambda_p +
                            sigma)^2 of the slowest directions), tau = 1.5 (L + sigma);
                            a re-tune that is followed by an energy increase is undone
                            and adaptation stops.  sigma_0 is the initial sigma; the
                            residual normalisation keeps sigma_0.  Algorithm 1 allows
                            a variable tau_n; the fixed points do not depend on sigma
                            or tau. */
  int cg_precond;        /* op_precond of the Step-1 CG                              */
  int flow;              /* op_flow (contexts; the batched solver and the adaptive
                            shift take OP_FLOW_G only)                               */
  int fp64_gemm;         /* op_fp64_gemm: FP64 Gram and update of OP_FP64 contexts and
                            the set-up Cholesky-QR of every context                  */
  int step1;             /* op_step1: the Step-1 solver of a context (G flow)        */
} op_problem;

/* Per-context statistics, filled by op_step / op_solve. */
typedef struct {
  int steps;             /* time steps taken since op_init                         */
  int last_cg_iters;     /* CG iterations of the last step                          */
  long long cg_iters;    /* CG iterations since op_init                             */
  double energy;         /* E(U) = 1/2 tr(U^T H U) of the current U (unshifted)     */
  double err_E;          /* |E(U^n) - E(U^{n-1})| / |E(U^{n-1})| of the last step   */
  double residual;       /* last evaluated r (see OP_STOP_RESIDUAL), NaN if none    */
  double g_residual;     /* tr(<W,W>) - ||<W,U>||_F^2 of the last step (G-residual^2) */
  double orth;           /* ||<U,U> - I||_F of the U entering the last step         */
  double sigma, tau;     /* parameters in use                                       */
  double ms;             /* wall time of the last op_step / op_solve call (ms)      */
} op_stats;

typedef struct op_ctx op_ctx;

/* ---------------------------------------------------------------------------
 * Context-level API (problem statement (2.2); scheme (4.1); Algorithm 1)
 * ------------------------------------------------------------------------- */

/* Library version string (static storage). */
const char *op_version(void);

/* Message of the last failed call on this thread ("" if none). Static per thread. */
const char *op_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all contexts). */
long long op_kernel_launches(void);

/* Create a context: validates `pb`, allocates the device blocks (cudaMalloc on the
 * current device; the context owns them), uploads V (n FP64 values, host) and the
 * raw initial block U0 (n x p FP64, host, row-major, ld = p), and orthonormalises
 * U0 by Cholesky-QR in FP64 on the device (§5 starts from random orthonormal data).
 * All work is queued on `stream` and the call synchronises it before returning.
 * On error *ctx is NULL. */
op_status op_init(op_ctx **ctx, const op_problem *pb, const double *V, const double *U0,
                  void *stream);

/* As op_init, with the raw initial block drawn on the device from `seed` instead of read
 * from the caller (§5 starts from random data): U0[i][j] is standard normal number
 * k = i p + j of the SplitMix64 counter stream key = seed ^ 0xD1B54A32D192ED03 (output m of
 * the stream is mix64(key + (m + 1) 0x9E3779B97F4A7C15); uniform m is ((output m >> 11) +
 * 0.5) 2^-53; normal k is sqrt(-2 ln u_2k) cos(2 pi u_2k+1), Box-Muller).  V is n FP64
 * values in host memory.  Allocates and frees a temporary n x p FP64 block. */
op_status op_init_seeded(op_ctx **ctx, const op_problem *pb, const double *V,
                         unsigned long long seed, void *stream);

/* The raw initial block of op_init_seeded, drawn into caller-owned device memory U0
 * (n x p FP64, ld = p) on `stream` (enqueue only). */
op_status op_gaussian_block(unsigned long long seed, long long n, int p, double *U0,
                            void *stream);

/* As op_init, but V (n FP64) and U0 (n x p FP64, ld = p) are device pointers. */
op_status op_init_device(op_ctx **ctx, const op_problem *pb, const double *V_dev,
                         const double *U0_dev, void *stream);

/* Advance `nsteps` time steps (Steps 1-4 each, §4.1), updating the energy every step.
 * Synchronises the stream at least once per step (Step-1 CG convergence checks).
 * `st` may be NULL. */
op_status op_step(op_ctx *ctx, int nsteps, op_stats *st);

/* Algorithm 1: step until the stop rule `stop` (op_stop) holds for `tol`, or
 * `max_steps` steps.  The residual is evaluated every pb->check_every steps and at
 * the end.  Returns OP_OK when the rule holds (or after max_steps for OP_STOP_STEPS),
 * OP_ERR_STATE if max_steps ran out first.  `st` may be NULL. */
op_status op_solve(op_ctx *ctx, double tol, int max_steps, int stop, op_stats *st);

/* Communication of row-sharded steps (op_step_sharded), counted over the call. */
typedef struct {
  int slabs;                 /* slabs the grid was split into                          */
  long long halo_copies;     /* plane copies into a neighbour's halo                   */
  long long halo_bytes;      /* bytes of those copies (n_plane x ld FP64 values each)   */
  long long reductions;      /* sums over the slabs (the all-reduces of a multi-GPU run) */
  long long reduction_bytes; /* FP64 bytes one slab contributes to them, summed         */
} op_shard_stats;

/* Advance `nsteps` time steps of an OP_FP64 context (G flow) with the grid split into
 * `nslab` slabs of whole planes along its slowest axis (z in 3-D, y in 2-D; sizes differ
 * by at most one plane), the row sharding a multi-GPU run would use.  The scheme needs no
 * orthogonalisation (§1, Theorem 4.1), so the slabs exchange only
 *   - one halo plane per face before each stencil apply: once per Step-1 CG iteration
 *     (the direction block), once at the CG start (W) and once for the energy (U+), and
 *   - sums over the slabs: three p-vectors at the CG start, two reductions of p and of
 *     2p values per CG iteration, the three p x p inner matrices <W,U>, <W,W>, <U,U> per
 *     step (Steps 2-3 of §4.1 are then computed once) and p values for the energy.
 * Step 4 is local to each slab.  Step 1 is the FP64 block CG of the context's
 * cg_precond (whatever `step1` selects), each column stopping at ||r_j|| <= rtol ||u_j||
 * with the context's tolerance rule; the Gram and update use the context's fp64_gemm.
 * The results equal op_step's up to the order of the sums.
 * On this single-device library the slabs are buffers of their own on the context's
 * device (allocated by the call: about 6 (n/nslab + 2 n_plane) x ld FP64 values per slab
 * beside the context, freed on return), processed one after another on the context's
 * stream; U and W are copied into the slabs at the start and back at the end, so the
 * context continues with op_step or any other call.  `comm` (may be NULL) receives the
 * exchanges the steps made.  OP_ERR_ARG for other precisions, the L2 flow, nslab outside
 * 1 .. planes or nsteps < 0.  Synchronises once per CG iteration.  `st` may be NULL. */
op_status op_step_sharded(op_ctx *ctx, int nslab, int nsteps, op_stats *st,
                          op_shard_stats *comm);

/* E(U) = 1/2 tr(U^T H U) (§2.2) of the current U, unshifted H. Synchronises. */
op_status op_energy(op_ctx *ctx, double *E);

/* r of the current U (see OP_STOP_RESIDUAL); also sets stats.residual. Synchronises. */
op_status op_residual(op_ctx *ctx, double *r);

/* Copy the current U (n x p, FP64, ld = p) into caller-owned host memory. Synchronises. */
op_status op_get_U(op_ctx *ctx, double *U_host);

/* Copy the current U into caller-owned device memory as an n x p block (ld = p) of
 * FP64 (prec = OP_FP64) or FP32 (prec = OP_FP32).  Synchronises. */
op_status op_get_U_device(op_ctx *ctx, void *U_dev, int prec);

/* p eigenvalue estimates, ascending, into caller-owned host memory (kind: op_eig_kind).
 * OP_EIG_PAPER runs one extra Step-1 solve for the current U. Synchronises. */
op_status op_eigenvalues(op_ctx *ctx, double *lam, int kind);

/* Current statistics (no device work). */
op_status op_get_stats(op_ctx *ctx, op_stats *st);

/* Per-kernel timing with CUDA events recorded on the context's stream around each
 * launch group of a step (kinds: op_profile_name(0 .. op_profile_kinds()-1)).
 * Enabling (or disabling) synchronises the stream and resets the totals. */
op_status op_profile_enable(op_ctx *ctx, int enable);
int op_profile_kinds(void);
const char *op_profile_name(int kind);  /* static storage; "" for an unknown kind */
/* Total device time (ms) and number of timed launch groups of `kind` since enabling. */
op_status op_profile_read(op_ctx *ctx, int kind, double *total_ms, long long *launches);

/* Checkpoint / resume.  The paper has no counterpart; the scheme is a one-step map,
 * so a context restored from a checkpoint continues bit-identically: the state is
 * U, the Step-1 warm start W, sigma, tau and the step statistics, and for FP64 contexts
 * with the mixed-precision Step 1 also the block before the last update (the next
 * Step 1 starts from that block's residual carried over the update, which restore
 * rebuilds).
 * op_checkpoint_size: bytes of a checkpoint of ctx (0 for NULL).
 * op_checkpoint: writes the state into caller-owned host memory buf (len >= size).
 * op_restore: loads a state written by op_checkpoint into a context of the same
 *   problem size (n, p, ld) and precision (OP_ERR_ARG otherwise, or for a buffer
 *   that is not a checkpoint).  Both synchronise the context's stream. */
size_t op_checkpoint_size(const op_ctx *ctx);
op_status op_checkpoint(op_ctx *ctx, void *buf, size_t len);
op_status op_restore(op_ctx *ctx, const void *buf, size_t len);

/* Self-test of failure detection (the paper has no counterpart).  Every wait inside
 * this library's kernels is bounded: on expiry the kernel sets an error word and
 * the call returns OP_ERR_TIMEOUT instead of hanging.  This call makes one wait of
 * each kind (the TMA ring's clock-bounded wait with a 0.2 s limit and the tensor-core
 * kernels' iteration-bounded wait) run out on an mbarrier that nothing completes;
 * it returns OP_OK when both gave up, and their durations in seconds[0..1] (may be
 * NULL).  Allocates 32 bytes of device memory; synchronises `stream`; takes about
 * a second. */
op_status op_selftest_bounded_waits(double *seconds, void *stream);

/* Peak-rate microbenchmarks (the paper has no counterpart): the roofline denominators of
 * the units the kernels are bound by, measured by this library on the current device
 * without reading or changing any GPU setting.  OP_PEAK_FP64_FMA: FP64 FMA on the CUDA
 * cores (independent chains, 2 flops per FMA); OP_PEAK_TF32_MMA / OP_PEAK_BF16_MMA:
 * tcgen05.mma kind::tf32 / kind::f16 (BF16) at M = 128, N = 256 from operands resident in
 * shared memory, one CTA per SM.  *tflops receives flops / s / 1e12 of the third of three
 * launches timed with CUDA events on `stream`.  Allocates and frees a few KB; synchronises. */
typedef enum {
  OP_PEAK_FP64_FMA = 0,
  OP_PEAK_TF32_MMA = 1,
  OP_PEAK_BF16_MMA = 2,
  OP_PEAK_BF16_MMA_N64 = 3,  /* BF16 at N = 64 (the FP64 digit products' MMA shape), a new
                                A tile every MMA */
  OP_PEAK_BF16_MMA_N64_AREUSE = 4  /* the same, each A tile kept in the tensor core's
                                      collector buffer over four MMAs with different B
                                      (the digit products' issue pattern) */
} op_peak_kind;
op_status op_peak_rate(int kind, double *tflops, void *stream);

/* Free the context's device memory. NULL is allowed. */
void op_destroy(op_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Batches: many independent problems (uneven n and p) advanced together.
 * A time step of every problem is one replay of a CUDA graph of batched kernels
 * (work lists over (problem, grid-point range), (problem, Gram chunk),
 * (problem, update tile), one CTA per problem for the FP64 core); Step 1 runs a
 * fixed number `cg_iters` of CG iterations per step whose kernels return at once
 * for problems whose CG has converged.  The CG tolerance (a context's cg_rtol when it
 * is positive, else the adaptive rule of op_problem.cg_rtol with the FP32 floor), the
 * energy, err_E and the freeze of converged problems are computed on the device.
 * ------------------------------------------------------------------------- */
typedef struct op_batch op_batch;

/* Group `count` contexts (each OP_FP32 of the G flow, p <= 128, plain or Jacobi CG;
 * not copied, still owned by the caller) into a batch.  The batch captures and
 * replays its graphs on a stream of its own; `stream` and the contexts' streams are
 * synchronised at creation, and every batch call that returns results synchronises
 * the batch stream.  While the batch exists the contexts must not be stepped on
 * their own (they may be read: op_get_U, op_eigenvalues, op_residual,
 * op_get_stats).  Destroy the batch before the contexts. */
op_status op_batch_create(op_batch **b, op_ctx *const *ctxs, int count, int cg_iters,
                          void *stream);   /* 1 <= cg_iters <= 200 */
/* Work-list granularity: grid points per stencil/CG/energy item (>= 32) and per Gram
 * chunk (>= 256, multiple of 32).  Rebuilds the graphs.  Synchronises. */
op_status op_batch_set_tiles(op_batch *b, int rows_per_item, int gram_rows);
op_status op_batch_get_tiles(op_batch *b, int *rows_per_item, int *gram_rows);
/* Autotuner: time `steps_per_trial` steps for each candidate granularity (the steps
 * advance the problems), keep the fastest and append it to the JSON-lines file
 * `cache_path` (may be NULL) keyed by the batch's shape; a cached entry for the same
 * shape is reused without trials.  *best_ms (may be NULL): ms per step. */
op_status op_batch_autotune(op_batch *b, const char *cache_path, int steps_per_trial,
                            double *best_ms);
/* Advance every unfrozen problem by `nsteps` steps; synchronises at the end and
 * updates each context's statistics. */
op_status op_batch_step(op_batch *b, int nsteps);
/* Step until every problem meets the stop rule (OP_STOP_ERR_E, evaluated on the device
 * every step, or OP_STOP_RESIDUAL, evaluated every check_every steps) or max_steps;
 * converged problems are frozen.  *nconverged (may be NULL) receives the count.
 * OP_ERR_STATE if some problem did not converge. */
op_status op_batch_solve(op_batch *b, double tol, int max_steps, int stop, int check_every,
                         int *nconverged);
/* Clear the freeze of every problem (e.g. to continue past a looser rule). */
op_status op_batch_unfreeze(op_batch *b);
/* Statistics of problem i and its freeze state (0 active, 1 converged, 2 diverged). */
op_status op_batch_stats(op_batch *b, int i, op_stats *st, int *frozen);
void op_batch_destroy(op_batch *b);

/* ---------------------------------------------------------------------------
 * Kernel-level API: single steps of the path on caller-owned device buffers.
 * `prec` selects the element type T of the blocks: double (OP_FP64) or float
 * (OP_FP32).  Blocks are n x ld, ld >= p, ld a multiple of 8.
 * ------------------------------------------------------------------------- */

/* Y = (H + sigma) X: the 5-point (2D) / 7-point (3D) stencil of -1/2 Delta_h plus
 * diag(V + sigma) (the operator of the source problems of Step 1).
 * Geometry, p and T (pb->prec) come from pb; V_t: n values of V in T (device);
 * X, Y: n x ld blocks of T (device, must not alias). */
op_status op_apply_H(const op_problem *pb, int ld, const void *V_t, double sigma,
                     const void *X, void *Y, void *stream);

/* Step 1: W = (H + sigma)^-1 U by p independent conjugate-gradient solves, warm-started
 * from the W passed in, each column to ||u - (H+sigma) w|| <= rtol ||u||, at most
 * max_iter iterations.  V_t as in op_apply_H; U, W: n x ld blocks of T.  Scratch: ws
 * (device) of at least op_cg_workspace() bytes.  *iters (host) receives the iteration
 * count.  Synchronises `stream` once per iteration (convergence checks). */
op_status op_cg_solve(const op_problem *pb, int ld, const void *V_t, double sigma,
                      const void *U, void *W, double rtol, int max_iter, void *ws,
                      size_t ws_bytes, int *iters, void *stream);
size_t op_cg_workspace(const op_problem *pb, int ld);

/* Inner matrices of [U W] (§2.1): C = <W,U> (C_ij = w_i . u_j), S = <W,W>, D = <U,U>,
 * each ld x ld FP64 row-major on the device (entries with i or j >= p are zero).
 * Any of C, S, D may be NULL to skip it.  OP_FP64: FP64 FMA, chunk partials in FP64.
 * OP_FP32: tcgen05 tensor-core MMAs (TF32 inputs split hi + lo, four MMAs per
 * product, FP32 accumulation per chunk of grid points, chunk partials summed in FP64).
 * OP_MIX_BF16X3: FP32 blocks, BF16 inputs split in three, six kind::f16 MMAs per product.
 * ws: device scratch of at least op_gram_workspace() bytes; its first int is set when a
 * bounded device wait gave up (check with op_ws_status). */
op_status op_gram(int prec, long long n, int p, int ld, const void *U, const void *W,
                  double *C, double *S, double *D, void *ws, size_t ws_bytes, void *stream);
size_t op_gram_workspace(int prec, long long n, int ld);

/* op_gram without any device allocation (no counterpart in the paper: a service for
 * callers that cannot allocate device memory or hand over a workspace, e.g. because
 * another allocator with a hard budget owns all device memory, or because the calling
 * loop may not enter the driver's allocator).  Arguments and results as op_gram minus the
 * workspace, for prec OP_FP64 or OP_FP32 only (OP_MIX_BF16X3 returns OP_ERR_ARG).  The
 * reduction partials live in one library-owned device array of 16 MiB.
 * - Memory: the array belongs to the library's module; with CUDA's default lazy module
 *   loading the driver reserves it on the first call on each device (16 MiB inside the
 *   caller's device-memory budget, held until the process exits), so a caller with a fixed
 *   budget should make that first call during its set-up.
 * - Limit: one 128 x 128 (OP_FP32) or 64 x 64 (OP_FP64) FP64 tile per output tile must
 *   fit, i.e. with all three products ld <= 896 (OP_FP32) or ld <= 960 (OP_FP64); larger
 *   sizes return OP_ERR_ARG with a message.
 * - Accuracy: OP_FP32 splits the grid points into the same chunks as op_gram and adds the
 *   FP64 chunk partials into one tile per output tile with atomics (so the FP64 chunk sums
 *   are taken in a run-dependent order; the FP32 rounding bound is op_gram's).  OP_FP64
 *   uses fewer, longer chunks than op_gram when the array is small (FP64 register sums).
 * - The first call on a device looks up the array's device address (with that device
 *   current) and keeps it; make that first call before any stream capture, and do not
 *   call this after cudaDeviceReset() on that device (the module and the address go away).
 * - Every call uses the same array: calls that overlap on the GPU (other streams,
 *   other host threads) race and corrupt each other's results.
 * - Synchronises `stream` before returning (it reads back the bounded-wait flag:
 *   OP_ERR_TIMEOUT if set).  Calls no cudaMalloc / cudaFree. */
op_status op_gram_noalloc(int prec, long long n, int p, int ld, const void *U, const void *W,
                          double *C, double *S, double *D, void *stream);

/* Synchronises `stream`; OP_ERR_TIMEOUT if the last op_gram / op_update on ws reported a
 * bounded device wait that gave up, else OP_OK. */
op_status op_ws_status(void *ws, void *stream);

/* FP64-accurate Gram and update on the tensor cores (the OP_GEMM_TC arithmetic of
 * op_fp64_gemm) on caller-owned FP64 blocks (n x ld, ld a multiple of 8, 16-byte aligned).
 * ws: device scratch of at least op_fp64tc_workspace(n, ld) bytes (about 14 bytes per
 * element of [U W] for up to 8 GiB of digit planes, plus 2 ld x 2 ld FP64); its first int
 * is set when a bounded device wait gave up (op_ws_status).  Enqueue only.
 * op_gram_fp64tc: C = <W,U>, S = <W,W>, D = <U,U> as op_gram (ld x ld FP64, zero outside
 *   p x p; any may be NULL; W may be NULL when only D is wanted).
 * op_update_fp64tc: Unew = U KU + W KW (computed as U + [U W][KU - I; KW]; W and KW may
 *   be NULL for Unew = U KU); KU, KW: ld x ld FP64; Unew must not alias U or W. */
size_t op_fp64tc_workspace(long long n, int ld);
op_status op_gram_fp64tc(long long n, int p, int ld, const double *U, const double *W,
                         double *C, double *S, double *D, void *ws, size_t ws_bytes,
                         void *stream);
op_status op_update_fp64tc(long long n, int p, int ld, const double *U, const double *W,
                           const double *KU, const double *KW, double *Unew, void *ws,
                           size_t ws_bytes, void *stream);

/* Steps 2-3 of §4.1 in FP64: from C = <W,U>, S = <W,W> (ld x ld device, FP64) form
 * M = I + tau/2 (C - C^T) + tau^2/4 (S - C C^T), B = M^-1 (p <= 128: FP32 Gauss-Jordan
 * refined by FP64 Newton-Schulz steps, two for OP_FP64 and one for OP_FP32; larger p:
 * FP64 LU; no pivoting is needed because the symmetric part of M is >= I by
 * Lemma 3.1), tau/2 A = I - B + tau/2 C^T B, and the
 * Step-4 coefficients KU = I - tau A = 2B - I - tau C^T B, KW = tau B (ld x ld FP64
 * device, zero outside p x p).  For the exact W = GU (C symmetric) these are the
 * paper's Steps 2-3; for any other W they solve the midpoint scheme (4.1) exactly
 * for the operator built from W, so Step 4 keeps <U,U>.  KU_t / KW_t (may be NULL)
 * receive the same matrices in the block type of `prec`.  ws: at least
 * op_core_workspace() bytes.  A zero or non-finite pivot is reported by
 * op_core_status() on the same workspace (the coefficients are then KU = I, KW = 0). */
op_status op_core(int prec, int p, int ld, double tau, const double *C, const double *S,
                  double *KU, double *KW, void *KU_t, void *KW_t, void *ws, size_t ws_bytes,
                  void *stream);
size_t op_core_workspace(int p, int ld);
/* Synchronises `stream`; returns OP_ERR_NOTSPD if the last op_core on ws broke down. */
op_status op_core_status(void *ws, void *stream);

/* Step 4: Unew = U KU + W KW (KU, KW: ld x ld in the block type T, device).
 * OP_FP64: FP64 FMA.  OP_FP32: tcgen05 tensor-core MMAs with the 3xTF32 split
 * (hi*hi + hi*lo + lo*hi).  OP_MIX_BF16X3: FP32 blocks and KU, KW, BF16 x 3 pieces and
 * six kind::f16 MMAs per product.  Unew must not alias U or W.  ws: device scratch of at least
 * op_update_workspace() bytes (first int: timeout flag, see op_ws_status). */
op_status op_update(int prec, long long n, int p, int ld, const void *U, const void *W,
                    const void *KU_t, const void *KW_t, void *Unew, void *ws, size_t ws_bytes,
                    void *stream);
size_t op_update_workspace(int prec, int ld);

#ifdef __cplusplus
}
#endif
#endif /* OPEVO_H */
