// Internal launchers of the opevo kernels.  Every launcher only enqueues work
// on `st` and returns OP_OK or the launch error; buffers are device pointers.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace opevo {

// ---- optional per-kernel timing with CUDA events on the launching stream ----------
enum ProfKind {
  PK_CG_INIT = 0,
  PK_CG_APPLY,
  PK_CG_AXPY,
  PK_CG_DIR,
  PK_CG_FIN,
  PK_GRAM,
  PK_CORE,
  PK_UPDATE,
  PK_ENERGY,
  PK_RESIDUAL,
  PK_REFINE,   // FP64 residual, scaling and correction of the mixed-precision Step 1
  PK_COUNT
};
struct Prof {
  static constexpr int kMax = 64;
  bool on = false;
  bool created = false;
  cudaEvent_t ev[2 * kMax];
  int kind[kMax];
  int n = 0;
  double ms[PK_COUNT];
  long long cnt[PK_COUNT];
};
const char *prof_name(int kind);
op_status prof_enable(Prof *p, bool on);
void prof_destroy(Prof *p);
// begin/end bracket one launch (or a group of launches) of `kind`; no-ops when off
void prof_begin(Prof *p, int kind, cudaStream_t st);
void prof_end(Prof *p, cudaStream_t st);
// accumulate the recorded pairs; the stream must have been synchronised
void prof_harvest(Prof *p);

// ---- batches of independent problems (FP32 blocks) ------------------------
// One problem of a batch: device pointers into the problem's own context.  The
// batched kernels read these descriptors from device memory; a work list maps
// each CTA to (problem, piece of work).
struct BatchProb {
  Geom g;
  int p, ld;
  float shift;             // cdiag + sigma in FP32 (the CG operator's diagonal offset)
  double tau;
  const float *Vt;
  float *U[2];             // U and U+ (roles alternate with the step parity)
  float *W, *R, *P, *Q;    // Step-1 solution and CG buffers (P, Q: direction buffers)
  double *part;            // row-kernel CTA partials [items][<= 3][ld] + column sums [2][ld]
  int jacobi;              // Step-1 CG preconditioned with diag(H + sigma); R holds r / d
  double *state;           // CG state [6][ld]
  int *active, *ctl;       // CG control (ctl[0..1] active counts, ctl[2] iterations)
  double *cg_rtol2;        // squared relative CG tolerance of the current step
  double fixed_rtol;       // the context's cg_rtol when positive (else the adaptive rule)
  double *C, *S, *D, *KU, *KW;
  float *KT_hi, *KT_lo;
  int *core_status;
  double *core_M, *core_X, *core_B, *core_R;  // ld x ld each
  double *gram_part;       // Gram chunk partials [splits][jobs][128 x 128]
  int *err;
  double *dsc;             // scalars: 0..2 core stats, 4..5 energy
  int *frozen;             // non-zero: converged, every batched kernel skips it
  int n_row_items;         // row items of this problem (CG partial rows)
  int n_gram_splits;
  int gram_jobs;
};
struct RowItem {
  int prob, local;         // problem, index of this item among the problem's items
  long long r0, r1;        // grid points [r0, r1)
};
struct GramItem {
  int prob, job, split;
  long long r0, r1;
};
struct TileItem {
  int prob;
  long long m0;            // first grid point of a 128-point tile
  int n0;                  // first output column
};

// Batched launchers (grid = item count; problems by blockIdx where noted).
op_status launch_b_cg_init(const BatchProb *B, const RowItem *items, int nitems, int parity,
                           cudaStream_t st);
op_status launch_b_fin_init(const BatchProb *B, int nprob, int max_ld, cudaStream_t st);
op_status launch_b_cg_iter(const BatchProb *B, const RowItem *items, int nitems, int nprob,
                           int max_ld, int k, cudaStream_t st);
op_status launch_b_energy(const BatchProb *B, const RowItem *items, int nitems, int nprob,
                          int max_ld, int parity, cudaStream_t st);
op_status launch_b_gram(const BatchProb *B, const GramItem *items, int nitems, int nprob,
                        int parity, cudaStream_t st);
size_t gram_tc_tile_bytes();      // bytes of one 128 x 128 FP64 partial tile
int gram_tc_jobs_all(int ld);     // tensor-core Gram jobs for C, S and D
op_status launch_b_core(const BatchProb *B, int nprob, int max_ld, cudaStream_t st);
op_status launch_b_update(const BatchProb *B, const TileItem *items, int nitems, int nprob,
                          int max_ld, int parity, cudaStream_t st);

// ---- stencil and Step-1 CG (stencil_cg.cu) --------------------------------
// Vt: n values of V in T; the diagonal of H + sigma is Vt_i + cdiag + sigma.
// Y = scale (H + sigma) X.
template <typename T>
op_status launch_apply(const Geom &g, const T *Vt, double sigma, const T *X, T *Y, int ld,
                       cudaStream_t st, double scale = 1.0);

// out[0] = sum X .* ((H + sigma) X), out[1] = sum X .* X (FP64, device); part is
// scratch of [max_blocks][2][ld] doubles.  With err (device int, set when a bounded
// wait gave up), FP32 blocks on 3-D grids use the TMA plane-marching kernel.
template <typename T>
op_status launch_quad(const Geom &g, const T *Vt, double sigma, const T *X, int ld, double *part,
                      double *out, cudaStream_t st, int *err = nullptr);

// out[0] = sum X .* X; part as above.
template <typename T>
op_status launch_sumsq(long long n, int ld, const T *X, double *part, double *out,
                       cudaStream_t st);


// CG workspace layout and the solver loop.
struct CGWork {
  void *R, *P, *Q;       // n x ld blocks of T (FP32 path: P, Q are the two direction buffers)
  double *part;          // CTA partials [max_blocks][2][ld] + per-column sums [2][ld]
  double *state;         // [6][ld]: rr, target, alpha, beta, bnorm2, scratch
  int *active;           // [ld]
  int *ctl;              // [4] device: active counts (two parities), iterations done,
                         // error flag (a bounded wait of a TMA kernel gave up)
  int *host_ctl;         // >= 4 ints of host memory (pinned for the context)
  int max_blocks;
  int expect_iters = 0;  // iterations of the previous solve (first chunk length)
  bool jacobi = false;   // CG preconditioned with diag(H + sigma)
  Prof *prof = nullptr;  // optional timing
};
// bytes of the CTA-partials scratch used by the reductions of a row width ld
size_t part_bytes(int ld);
size_t cg_workspace_bytes(long long n, int ld, int elem);
void cg_carve(void *ws, long long n, int ld, int elem, CGWork *w);

template <typename T>
op_status cg_solve(const Geom &g, const T *Vt, double sigma, const T *U, T *W, int p, int ld,
                   double rtol, int max_iter, CGWork &w, int *iters, cudaStream_t st);

// Step 1 in FP64 by iterative refinement around an FP32 CG: each cycle forms the FP64
// residual R = U - (H + sigma) W and its column norms (w64: FP64 scratch, its R block and
// reductions), stops when every column meets ||r_j|| <= rtol ||u_j||, else solves
// (H + sigma) d = r_j / ||r_j|| by the FP32 CG of w32 (V in FP32: Vt32; rhs r32, solution
// d32: n x ld FP32 blocks) to a relative tolerance that the cycle needs, and adds
// ||r_j|| d_j to W in FP64.  scale: ld doubles plus ld floats of device scratch (16-byte
// aligned).  *iters: FP32 CG iterations of all cycles; *cycles: FP64 residual evaluations.
// Uprev (may be null): the block U was before the last update while w64's R block still
// holds Uprev - (H + sigma) W for the current W and sigma; the first residual is then
// R + U - Uprev, one pass over three blocks instead of a stencil apply.  *fresh (may be
// null): whether the residual left in w64's R was formed by the stencil.
op_status cg_refine(const Geom &g, const double *Vt, const float *Vt32, double sigma,
                    const double *U, double *W, int p, int ld, double rtol, int max_iter,
                    CGWork &w64, CGWork &w32, float *r32, float *d32, double *scale, int *iters,
                    int *cycles, cudaStream_t st, const double *Uprev = nullptr,
                    bool *fresh = nullptr);

// w64's R block = U - (H + sigma) W, element by element as the refinement forms it (the
// same values whatever the launch shape); used to rebuild a carried residual on restore.
op_status refine_residual(const Geom &g, const double *Vt, double sigma, const double *U,
                          const double *W, int ld, CGWork &w64, cudaStream_t st);

// Forward convolution of the learned warm start on the tensor cores (conv_tc.cu): X
// [N^3][cin] FP32, W [taps * cin][cout] FP32 (taps 27: the 3x3x3 cross-correlation, zero
// padded; taps 1: pointwise), BF16 operands with FP32 accumulation; Z = conv + bias and
// A = silu(Z) ([N^3][cout] FP32, either may be null).  cout <= 128.  scratch: device memory
// of conv_tc_scratch_bytes (the BF16 weights, K-major), 16-byte aligned; *err is set when a
// bounded wait of the kernel gives up.
size_t conv_tc_scratch_bytes(int taps, int cin, int cout);
op_status conv_bf16_tc(const float *X, int N, int taps, int cin, int cout, const float *W,
                       const float *bias, float *Z, float *A, void *scratch, size_t scratch_bytes,
                       int *err, cudaStream_t st);

// FP32 CG direction kernel on 3-D grids with TMA-staged stencil planes (stencil_tma.cu).
struct CgTmaGeom {
  int nx, ny, nz, ld;
  int ntx, nty, nch;   // 8 x 8 tiles in x and y; 32-column chunks
  int slabs;           // z slabs per column (columns = nch * ntx * nty)
  long long items;     // slabs * columns
  float shift;         // cdiag + sigma
  float cx, cy, cz;    // off-diagonal stencil weights
};
struct CgTmaPlan {
  CgTmaGeom tg;
  CUtensorMap halo[3];  // 10 x 10 x 32 boxes of R, P, Q
  int grid;             // persistent CTAs (rows of the partials buffer)
};
// Grids and blocks the TMA kernel handles (3-D, >= 32 columns, 16-byte aligned blocks).
bool cg_tma_eligible(const Geom &g, int ld, const void *R, const void *P, const void *Q);
op_status cg_tma_prepare(const Geom &g, double sigma, int ld, const float *R, const float *P,
                         const float *Q, CgTmaPlan *plan);
// part[grid][2][ld] = (X . (H + sigma) X, X . X) for FP32 blocks on 3-D grids; *grid
// receives the number of partial rows.
op_status tma_quad(const Geom &g, double sigma, int ld, const float *Vt, const float *X,
                   double *part, int *err, int *grid, cudaStream_t st);
// Pn = R (first) or R + beta Po, Po = P (po 0) or Q (po 1); part[grid][ld] = Pn . A Pn.
op_status cg_tma_p(const CgTmaPlan &plan, bool first, int po, float *Pn, const float *Vt,
                   const double *beta, const int *nact_prev, double *part, int *err,
                   cudaStream_t st);

// Copy the first p columns of an n x ld block (elements of src_size bytes: 4 or 8)
// into an n x p block of dst_size-byte elements (opnet.cu).
op_status launch_unpad_to(long long n, int p, int ld, const void *src, int src_size, void *dst,
                          int dst_size, cudaStream_t st);

// Copy an n x p FP64 block into an n x ld block of T (zero padding).
template <typename T>
op_status launch_pad_copy(long long n, int p, int ld, const double *src, T *dst, cudaStream_t st);
// Copy an n x ld block of T into an n x p FP64 block (drop padding).
template <typename T>
op_status launch_unpad_copy(long long n, int p, int ld, const T *src, double *dst,
                            cudaStream_t st);

// ---- Gram matrices (gram.cu) -------------------------------------------------
size_t gram_workspace_bytes(long long n, int ld, int elem);
template <typename T>
op_status gram(long long n, int p, int ld, const T *U, const T *W, double *C, double *S,
               double *D, void *ws, size_t ws_bytes, cudaStream_t st);

// FP32 blocks on the tensor cores (gram_tc.cu): same outputs as gram<float>; *err is set
// (device int) when a bounded wait inside the kernel gave up.
size_t gram_tc_workspace_bytes(long long n, int ld);
// split = 1: four-term TF32 split (FP32-class accuracy); 0: one TF32 MMA per product.
op_status gram_tc(long long n, int p, int ld, const float *U, const float *W, double *C, double *S,
                  double *D, void *ws, size_t ws_bytes, int *err, cudaStream_t st, int split = 1);

// Same outputs with the chunk split limited by a fixed scratch of part_bytes.
template <typename T>
op_status gram_fixed_scratch(long long n, int p, int ld, const T *U, const T *W, double *C,
                             double *S, double *D, void *part, size_t part_bytes, cudaStream_t st);
op_status gram_tc_fixed_scratch(long long n, int p, int ld, const float *U, const float *W,
                                double *C, double *S, double *D, void *part, size_t part_bytes,
                                int *err, cudaStream_t st);

// ---- dense FP64 p x p algebra (dense.cu) --------------------------------------
size_t core_workspace_bytes(int p, int ld);
// ws layout begins with an int status word (0 ok, 1 not SPD).
// tcws (may be null): an fp64tc scratch of fp64tc_workspace_bytes(p, ld) or more; with it,
// p > 128 inverts the Step-2 matrix by Newton-Schulz on the tensor-core FP64 products
// (host-checked convergence, FP64 LU when it does not converge), else by FP64 LU.
template <typename T>
op_status core(int p, int ld, double tau, const double *C, const double *S, double *KU,
               double *KW, T *KU_t, T *KW_t, void *ws, cudaStream_t st, void *tcws = nullptr,
               size_t tcb = 0, int *err = nullptr);
// The midpoint step as an exact Cayley transform for any <U, U> (2p x 2p solve with the
// joint Gram of [U W], Gauss-Jordan with partial pivoting): KU, KW (FP64 and T copies)
// with U+ = U KU + W KW.  aug: cayley_workspace_bytes(p) of device scratch; status word
// at ws as in core().  p <= 256.
size_t cayley_workspace_bytes(int p);
template <typename T>
op_status core_cayley(int p, int ld, double tau, const double *C, const double *S,
                      const double *D, double *KU, double *KW, T *KU_t, T *KW_t, void *aug,
                      void *ws, cudaStream_t st);
// Cholesky-QR coefficients: from D = U0^T U0, KU = R^-1 with R = chol(D)^T, written
// as an ld x ld FP64 matrix (zero outside p x p). Status word as in core().
// FP64-accurate Gram and update on the tensor cores (exact BF16 digit products, fp64tc.cu).
// gram_fp64tc: C = <W,U>, S = <W,W>, D = <U,U> (W may be null when only D is wanted).
// update_fp64tc: Unew = U + [U W][KU - I; KW] (delta) or [U W][KU; KW]; W, KW may be null.
// ws: fp64tc_workspace_bytes(n, ld) bytes; err: set when a bounded wait gave up.
size_t fp64tc_workspace_bytes(long long n, int ld);
op_status gram_fp64tc(long long n, int p, int ld, const double *U, const double *W, double *C,
                      double *S, double *D, void *ws, size_t ws_bytes, int *err, cudaStream_t st);
op_status update_fp64tc(long long n, int ld, const double *U, const double *W, const double *KU,
                        const double *KW, bool delta, double *Unew, void *ws, size_t ws_bytes,
                        int *err, cudaStream_t st);

op_status cholqr_coeff(int p, int ld, const double *D, double *KU, void *ws, cudaStream_t st);
// Eigenvalues (ascending) of the symmetric part of the p x p matrix A (stride ld)
// by cyclic Jacobi on the device; `work` holds 2 p*p doubles; lam receives p values.
op_status sym_eigvals(int p, int ld, const double *A, double *work, double *lam,
                      cudaStream_t st);
// Scalars of the last step from C, S, D: g2 = tr S - ||C||_F^2, orth = ||D - I||_F,
// trS = tr S; written to out[0..2].
op_status launch_core_stats(int p, int ld, const double *C, const double *S, const double *D,
                            double *out, cudaStream_t st);
// Convert an ld x ld FP64 matrix to T.
template <typename T>
op_status launch_convert(int count, const double *src, T *dst, cudaStream_t st);

// T copies of -Theta and I (p x p inside ld x ld) for R = H U - U Theta.
template <typename T>
op_status launch_resid_coeff(int p, int ld, const double *Th, T *negTh, T *Id, cudaStream_t st);
// lam (ascending) = 1/mu - sigma for mu ascending.
op_status launch_paper_lams(int p, const double *mu, double sigma, double *lam, cudaStream_t st);

// ---- Step 4 (update.cu, update_tc.cu) -------------------------------------------------
// Unew = U KU + W KW; W and KW may be nullptr (then Unew = U KU).
template <typename T>
op_status update(long long n, int ld, const T *U, const T *W, const T *KU, const T *KW, T *Unew,
                 cudaStream_t st);
// KT = [KU - I; KW]^T split into TF32 hi / lo parts (ld x 2 ld each) from FP64 or FP32
// KU, KW (update_tc adds U back, so it computes U KU + W KW).
op_status launch_make_kt(int ld, const double *KU, const double *KW, float *KT_hi, float *KT_lo,
                         cudaStream_t st);
op_status launch_make_kt_f32(int ld, const float *KU, const float *KW, float *KT_hi,
                             float *KT_lo, cudaStream_t st);
// Unew = [U W] [KU; KW] on the tensor cores (FP32 blocks); *err as for gram_tc.
op_status update_tc(long long n, int ld, const float *U, const float *W, const float *KT_hi,
                    const float *KT_lo, float *Unew, int *err, cudaStream_t st, int split = 1);
// BF16 x 3 form: KT = the three BF16 pieces of [KU - I; KW]^T (3 x ld x 2 ld values,
// kt_bf16_bytes(ld)), then Unew = U + [U W] KT^T with six MMAs per product.
size_t kt_bf16_bytes(int ld);
op_status launch_make_kt_bf16(int ld, const double *KU, const double *KW, uint16_t *KT,
                              cudaStream_t st);
op_status launch_make_kt_bf16_f32(int ld, const float *KU, const float *KW, uint16_t *KT,
                                  cudaStream_t st);
op_status update_bf16(long long n, int ld, const float *U, const float *W, const uint16_t *KT,
                      float *Unew, int *err, cudaStream_t st, bool three = true);

}  // namespace opevo
