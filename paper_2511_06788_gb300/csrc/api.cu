// C ABI of the library (include/opevo.h): validation, the per-context device
// state and the host loop of Algorithm 1 (§4.1) over the device kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace opevo {

static thread_local char g_err[1024] = "";
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(); }

int num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();
    v = 152;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

op_status cuda_status(cudaError_t e, const char *what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return e == cudaErrorMemoryAllocation ? OP_ERR_OOM : OP_ERR_CUDA;
}

op_status make_geom(const op_problem *pb, Geom *g) {
  if (!pb) {
    set_error("null problem");
    return OP_ERR_ARG;
  }
  if (pb->dim != 2 && pb->dim != 3) {
    set_error("dim must be 2 or 3 (got %d)", pb->dim);
    return OP_ERR_ARG;
  }
  g->dim = pb->dim;
  g->nx = pb->shape[0];
  g->ny = pb->shape[1];
  g->nz = pb->dim == 3 ? pb->shape[2] : 1;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) {
    set_error("grid shape must be positive");
    return OP_ERR_ARG;
  }
  g->n = (long long)g->nx * g->ny * g->nz;
  g->cdiag = 0.0;
  g->c[0] = g->c[1] = g->c[2] = 0.0;
  for (int d = 0; d < pb->dim; ++d) {
    const double len = pb->hi[d] - pb->lo[d];
    if (!(len > 0.0)) {
      set_error("box must satisfy hi > lo on every axis");
      return OP_ERR_ARG;
    }
    const double h = len / (pb->shape[d] + 1);
    g->cdiag += 1.0 / (h * h);
    g->c[d] = 0.5 / (h * h);
  }
  return OP_OK;
}

// Lower bound of spec(H): sum_d (2/h_d^2) sin^2(pi / (2 (n_d + 1))) + min V.
static double spectrum_lower_bound(const op_problem *pb, double vmin) {
  double lap = 0.0;
  for (int d = 0; d < pb->dim; ++d) {
    const double h = (pb->hi[d] - pb->lo[d]) / (pb->shape[d] + 1);
    const double s = sin(M_PI / (2.0 * (pb->shape[d] + 1)));
    lap += 2.0 / (h * h) * s * s;
  }
  return lap + vmin;
}

}  // namespace opevo

using namespace opevo;

#include "ctx.cuh"

namespace {

op_status dev_alloc(op_ctx *c, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_status(e, "cudaMalloc");
  }
  c->allocs.push_back(*p);
  return OP_OK;
}

void free_all(op_ctx *c) {
  prof_destroy(&c->prof);
  for (void *p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->hsc) cudaFreeHost(c->hsc);
  if (c->hpin_int) cudaFreeHost(c->hpin_int);
  c->hsc = nullptr;
  c->hpin_int = nullptr;
}

op_status check_problem(const op_problem *pb) {
  if (!pb) {
    set_error("null problem");
    return OP_ERR_ARG;
  }
  if (pb->p < 1) {
    set_error("p must be >= 1 (got %d)", pb->p);
    return OP_ERR_ARG;
  }
  if (pb->prec != OP_FP64 && pb->prec != OP_FP32 && pb->prec != OP_MIX_TF32 &&
      pb->prec != OP_MIX_BF16X3 && pb->prec != OP_MIX_BF16) {
    set_error("unsupported precision mode %d", pb->prec);
    return OP_ERR_ARG;
  }
  if (pb->cg_precond != OP_PRECOND_NONE && pb->cg_precond != OP_PRECOND_JACOBI) {
    set_error("unsupported CG preconditioner %d", pb->cg_precond);
    return OP_ERR_ARG;
  }
  if (pb->flow != OP_FLOW_G && pb->flow != OP_FLOW_L2) {
    set_error("unsupported flow %d", pb->flow);
    return OP_ERR_ARG;
  }
  if (pb->step1 != OP_STEP1_AUTO && pb->step1 != OP_STEP1_CG && pb->step1 != OP_STEP1_REFINE) {
    set_error("unsupported step1 solver %d", pb->step1);
    return OP_ERR_ARG;
  }
  if (pb->step1 == OP_STEP1_REFINE && pb->prec != OP_FP64) {
    set_error("the mixed-precision Step 1 refines FP64 blocks (prec %d)", pb->prec);
    return OP_ERR_ARG;
  }
  if (pb->fp64_gemm != OP_GEMM_TC && pb->fp64_gemm != OP_GEMM_FMA) {
    set_error("unsupported fp64_gemm %d", pb->fp64_gemm);
    return OP_ERR_ARG;
  }
  if (pb->flow == OP_FLOW_L2 && pb->adapt_every > 0) {
    set_error("the adaptive shift re-tunes the step of the G flow only (flow %d)", pb->flow);
    return OP_ERR_ARG;
  }
  if (pb->flow == OP_FLOW_L2 && pb->p > 256) {
    set_error("the L2 flow's exact Cayley step takes p <= 256 (got %d)", pb->p);
    return OP_ERR_ARG;
  }
  Geom g;
  OP_TRY(make_geom(pb, &g));
  if (pb->p > g.n) {
    set_error("p (%d) exceeds the number of grid points (%lld)", pb->p, g.n);
    return OP_ERR_ARG;
  }
  if (round_up(pb->p, 8) > 4096) {
    set_error("p too large (max 4096)");
    return OP_ERR_ARG;
  }
  return OP_OK;
}

template <typename T> op_status energy_impl(op_ctx *c) {
  OP_TRY(launch_quad<T>(c->g, (const T *)c->Vt, 0.0, (const T *)c->U, c->ld, c->part, c->dsc + 4,
                        c->st, c->dev_err));
  OP_CUDA(cudaMemcpyAsync(c->hsc + 4, c->dsc + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                          c->st));
  OP_CUDA(cudaMemcpyAsync(c->hpin_int + 1, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost,
                          c->st));
  OP_CUDA(cudaStreamSynchronize(c->st));
  if (c->hpin_int[1]) {
    set_error("a kernel gave up a bounded device wait");
    return OP_ERR_TIMEOUT;
  }
  c->E = 0.5 * c->hsc[4];
  c->stats.energy = c->E;
  return OP_OK;
}

// Inner matrices: FP32 blocks on the tensor cores, FP64 blocks on the FP64 pipe.
template <typename T>
op_status gram_any(op_ctx *c, const T *U, const T *W, double *C, double *S, double *D) {
  if constexpr (std::is_same<T, float>::value)
    return gram_tc(c->n, c->p, c->ld, U, W, C, S, D, c->gram_ws, c->gram_bytes, c->dev_err,
                   c->st,
                   c->prec == OP_MIX_TF32     ? 0
                   : c->prec == OP_MIX_BF16X3 ? 2
                   : c->prec == OP_MIX_BF16   ? 3
                                              : 1);
  else if (c->tc_ws)
    return gram_fp64tc(c->n, c->p, c->ld, U, W, C, S, D, c->tc_ws, c->tc_bytes, c->dev_err,
                       c->st);
  else
    return gram<T>(c->n, c->p, c->ld, U, W, C, S, D, c->gram_ws, c->gram_bytes, c->st);
}

// Step 4 of an FP64 context: U+ = U + [U W][KU - I; KW] on the tensor cores, or
// [U W][KU; KW] by FP64 FMA.
op_status update_fp64(op_ctx *c, const double *U, const double *W, const double *KU,
                      const double *KW, double *Unew) {
  if (c->tc_ws)
    return update_fp64tc(c->n, c->ld, U, W, KU, KW, true, Unew, c->tc_ws, c->tc_bytes, c->dev_err,
                         c->st);
  return update<double>(c->n, c->ld, U, W, KU, KW, Unew, c->st);
}

// Step 1 for the context: CG in the block precision, or (FP64 contexts) iterative
// refinement around an FP32 CG.
// recycle (step_impl): the first residual may be carried over from the last step;
// *fresh: the refinement's R block now holds U - (H + sigma) W formed by the stencil.
template <typename T>
op_status solve_step1(op_ctx *c, const T *U, T *W, double rtol, int max_iter, int *iters,
                      bool recycle = false, bool *fresh = nullptr) {
  const bool carry = recycle && c->rec_ok;
  c->rec_ok = false;
  if (fresh) *fresh = false;
  if constexpr (std::is_same<T, double>::value) {
    if (c->refine) {
      c->cgw32.Q = c->U2;  // the update's output block is free during Step 1
      int cycles = 0;
      return cg_refine(c->g, (const double *)c->Vt, c->Vt32, c->sigma, U, W, c->p, c->ld, rtol,
                       max_iter, c->cgw, c->cgw32, (float *)c->cgw.P,
                       (float *)c->cgw.P + (size_t)c->n * c->ld, c->ref_scale, iters, &cycles,
                       c->st, carry ? (const double *)c->U2 : nullptr, fresh);
    }
  }
  return cg_solve<T>(c->g, (const T *)c->Vt, c->sigma, U, W, c->p, c->ld, rtol, max_iter, c->cgw,
                     iters, c->st);
}

template <typename T> op_status step_impl(op_ctx *c) {
  NvtxRange step_range("opevo step");
  int iters = 0;
  bool fresh = false;  // Step 1 left a stencil-formed residual for the next step
  if (c->pb.flow == OP_FLOW_L2) {
    // the L2 gradient flow: W = -(H + sigma) U
    NvtxRange r("step 1: W = -(H + sigma) U");
    prof_begin(&c->prof, PK_CG_APPLY, c->st);
    OP_TRY(launch_apply<T>(c->g, (const T *)c->Vt, c->sigma, (const T *)c->U, (T *)c->W, c->ld,
                           c->st, -1.0));
    prof_end(&c->prof, c->st);
  } else {
    // Step 1: W = (H + sigma)^-1 U, warm-started from the previous W
    NvtxRange r("step 1: CG");
    OP_TRY(solve_step1<T>(c, (const T *)c->U, (T *)c->W, cg_rtol_for(c), cg_max_iter(c),
                          &iters, true, &fresh));
  }
  NvtxRange r_rest("Grams, core, update, energy");
  // inner matrices <W,U>, <W,W>, <U,U>
  prof_begin(&c->prof, PK_GRAM, c->st);
  OP_TRY(gram_any<T>(c, (const T *)c->U, (const T *)c->W, c->C, c->S, c->D));
  prof_end(&c->prof, c->st);
  // Steps 2-3 (FP64) and the Step-4 coefficients
  prof_begin(&c->prof, PK_CORE, c->st);
  OP_TRY(launch_core_stats(c->p, c->ld, c->C, c->S, c->D, c->dsc, c->st));
  if (c->pb.flow == OP_FLOW_L2)
    // the L2 flow's large W amplifies any drift of <U, U> through the p x p Steps 2-3
    // (they assume <U, U> = I); the exact Cayley form keeps <U, U> instead
    OP_TRY(core_cayley<T>(c->p, c->ld, c->tau, c->C, c->S, c->D, c->KU, c->KW, (T *)c->KU_t,
                          (T *)c->KW_t, c->cayley_ws, c->core_ws, c->st));
  else
    OP_TRY(core<T>(c->p, c->ld, c->tau, c->C, c->S, c->KU, c->KW, (T *)c->KU_t, (T *)c->KW_t,
                   c->core_ws, c->st, c->tc_ws ? c->tc_ws : c->core_tc_ws,
                   c->tc_ws ? c->tc_bytes : c->core_tc_bytes, c->dev_err));
  prof_end(&c->prof, c->st);
  // Step 4
  prof_begin(&c->prof, PK_UPDATE, c->st);
  if constexpr (std::is_same<T, float>::value) {
    if (c->prec == OP_MIX_BF16X3 || c->prec == OP_MIX_BF16) {
      // the three BF16 pieces of [KU - I; KW]^T take 12 ld^2 bytes of the 16 ld^2 of KT_hi|lo
      OP_TRY(launch_make_kt_bf16(c->ld, c->KU, c->KW, (uint16_t *)c->KT_hi, c->st));
      OP_TRY(update_bf16(c->n, c->ld, (const float *)c->U, (const float *)c->W,
                         (const uint16_t *)c->KT_hi, (float *)c->U2, c->dev_err, c->st,
                         c->prec == OP_MIX_BF16X3));
    } else {
      OP_TRY(launch_make_kt(c->ld, c->KU, c->KW, c->KT_hi, c->KT_lo, c->st));
      OP_TRY(update_tc(c->n, c->ld, (const float *)c->U, (const float *)c->W, c->KT_hi,
                       c->KT_lo, (float *)c->U2, c->dev_err, c->st,
                       c->prec == OP_MIX_TF32 ? 0 : 1));
    }
  } else {
    OP_TRY(update_fp64(c, (const double *)c->U, (const double *)c->W, c->KU, c->KW,
                       (double *)c->U2));
  }
  prof_end(&c->prof, c->st);
  void *tmp = c->U;
  c->U = c->U2;
  c->U2 = tmp;
  // E(U^{n+1}) for Algorithm 1's err_E
  prof_begin(&c->prof, PK_ENERGY, c->st);
  OP_TRY(launch_quad<T>(c->g, (const T *)c->Vt, 0.0, (const T *)c->U, c->ld, c->part, c->dsc + 4,
                        c->st, c->dev_err));
  prof_end(&c->prof, c->st);
  OP_CUDA(cudaMemcpyAsync(c->hsc, c->dsc, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaMemcpyAsync(c->hpin_int, c->core_ws, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaMemcpyAsync(c->hpin_int + 1, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaStreamSynchronize(c->st));
  prof_harvest(&c->prof);
  if (c->hpin_int[1]) {
    set_error("a kernel gave up a bounded device wait (tensor-core MMAs or TMA copies)");
    return OP_ERR_TIMEOUT;
  }
  if (*c->hpin_int) {
    set_error("Step 2 factorisation broke down (zero or non-finite pivot)");
    return OP_ERR_NOTSPD;
  }
  const double Enew = 0.5 * c->hsc[4];
  if (!isfinite(Enew)) {
    set_error("non-finite energy after step %d", c->stats.steps + 1);
    return OP_ERR_DIVERGED;
  }
  c->stats.err_E = fabs(Enew - c->E) / fabs(c->E);
  c->E = Enew;
  c->stats.energy = Enew;
  c->stats.g_residual = c->hsc[0];
  c->stats.orth = c->hsc[1];
  c->g_rel = (c->hsc[2] > 0.0 && c->hsc[0] > 0.0) ? sqrt(c->hsc[0] / c->hsc[2]) : 0.0;
  c->stats.steps += 1;
  c->stats.last_cg_iters = iters;
  c->stats.cg_iters += iters;
  // the step is complete: U2 holds the block before the update, R its residual with W
  c->rec_ok = fresh;
  return OP_OK;
}

// r = ||H U - U Theta||_F / (||H + sigma||_G sqrt(p)), Theta = U^T H U.
template <typename T> op_status residual_impl(op_ctx *c, double *r) {
  if (c) c->rec_ok = false;  // its scratch or its result replaces a carried residual
  T *Y = (T *)c->cgw.Q, *Z = (T *)c->cgw.R;
  prof_begin(&c->prof, PK_RESIDUAL, c->st);
  OP_TRY(launch_apply<T>(c->g, (const T *)c->Vt, 0.0, (const T *)c->U, Y, c->ld, c->st));
  OP_TRY(gram_any<T>(c, (const T *)c->U, Y, c->Th, nullptr, nullptr));
  OP_TRY(launch_resid_coeff<T>(c->p, c->ld, c->Th, (T *)c->KU_t, (T *)c->KW_t, c->st));
  bool done = false;
  if constexpr (std::is_same<T, double>::value) {
    if (c->tc_ws) {
      // R = [U HU][-Theta; I] (no delta form: the coefficients are not near the identity)
      OP_TRY(update_fp64tc(c->n, c->ld, (const double *)c->U, Y, (const double *)c->KU_t,
                           (const double *)c->KW_t, false, Z, c->tc_ws, c->tc_bytes, c->dev_err,
                           c->st));
      done = true;
    }
  }
  if (!done)
    OP_TRY(update<T>(c->n, c->ld, (const T *)c->U, Y, (const T *)c->KU_t, (const T *)c->KW_t, Z,
                     c->st));
  OP_TRY(launch_sumsq<T>(c->n, c->ld, Z, c->part, c->dsc + 6, c->st));
  prof_end(&c->prof, c->st);
  OP_CUDA(cudaMemcpyAsync(c->hsc + 6, c->dsc + 6, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaStreamSynchronize(c->st));
  prof_harvest(&c->prof);
  *r = sqrt(c->hsc[6]) / (c->hnorm * sqrt((double)c->p));
  c->stats.residual = *r;
  return OP_OK;
}

template <typename T> op_status eig_impl(op_ctx *c, double *lam, int kind) {
  if (c) c->rec_ok = false;  // its scratch or its result replaces a carried residual
  if (kind == OP_EIG_RITZ) {
    T *Y = (T *)c->cgw.Q;
    OP_TRY(launch_apply<T>(c->g, (const T *)c->Vt, 0.0, (const T *)c->U, Y, c->ld, c->st));
    OP_TRY(gram_any<T>(c, (const T *)c->U, Y, c->Th, nullptr, nullptr));
    OP_TRY(sym_eigvals(c->p, c->ld, c->Th, c->eig_work, c->lam_d, c->st));
  } else {
    int iters = 0;
    const double tight = c->prec == OP_FP64 ? 1e-13 : 1e-6;
    OP_TRY(solve_step1<T>(c, (const T *)c->U, (T *)c->W, tight, 20000, &iters));
    OP_TRY(gram_any<T>(c, (const T *)c->U, (const T *)c->W, c->Th, nullptr, nullptr));
    OP_TRY(sym_eigvals(c->p, c->ld, c->Th, c->eig_work, c->eig_work + (size_t)c->p * c->p,
                       c->st));
    OP_TRY(launch_paper_lams(c->p, c->eig_work + (size_t)c->p * c->p, c->sigma, c->lam_d, c->st));
  }
  OP_CUDA(cudaMemcpyAsync(lam, c->lam_d, c->p * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaStreamSynchronize(c->st));
  return OP_OK;
}

// Status of the set-up's Cholesky-QR: synchronises; OP_ERR_NOTSPD when U0^T U0 was
// not positive definite.
op_status cholqr_check(op_ctx *c) {
  OP_CUDA(cudaMemcpyAsync(c->hpin_int, c->core_ws, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaMemcpyAsync(c->hpin_int + 1, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost,
                          c->st));
  OP_CUDA(cudaStreamSynchronize(c->st));
  if (c->hpin_int[1]) {
    set_error("a kernel of the set-up gave up a bounded device wait");
    return OP_ERR_TIMEOUT;
  }
  if (c->hpin_int[0]) {
    set_error("Cholesky-QR of U0 failed: U0^T U0 is not positive definite");
    return OP_ERR_NOTSPD;
  }
  return OP_OK;
}

// Cholesky-QR (FP64) of the raw n x p block at U0 (device, FP64) into c->U: with
// D = U0^T U0 and R = chol(D)^T, U = U0 R^-1 (R's diagonal positive, so U is the Q of
// the Householder QR with a positive diagonal of R).  The set-up stays FP64 in every
// mode: the midpoint scheme preserves U^T U, so the orthogonality error U0 starts
// with stays for the whole run (an FP32 Cholesky-QR gave 1e-5 at p = 1024).
template <typename T> op_status orthonormalise_impl(op_ctx *c, const double *U0_dev) {
  if (c) c->rec_ok = false;  // its scratch or its result replaces a carried residual
  const size_t blk = (size_t)c->n * c->ld * sizeof(double);
  const size_t gbytes = gram_workspace_bytes(c->n, c->ld, 8);
  void *A64 = nullptr, *Q64 = nullptr, *gws = nullptr, *tc_tmp = nullptr;
  auto release = [&]() {
    for (void *p : {A64, Q64, gws, tc_tmp}) {
      if (!p) continue;
      cudaFree(p);
      for (auto it = c->allocs.begin(); it != c->allocs.end(); ++it)
        if (*it == p) {
          c->allocs.erase(it);
          break;
        }
    }
  };
  double *A, *Q;
  void *ws = c->gram_ws;
  size_t wsb = c->gram_bytes;
  op_status s = OP_OK;
  // the FP64 products of the set-up: on the tensor cores (digit products) unless the
  // problem asks for FP64 FMA; FP32 contexts borrow a scratch for it during the set-up
  const bool use_tc = c->pb.fp64_gemm == OP_GEMM_TC;
  void *tcw = c->tc_ws;
  size_t tcb = c->tc_bytes;
  if constexpr (std::is_same<T, double>::value) {
    A = (double *)c->U2;  // FP64 contexts: the context's own blocks are the scratch
    Q = (double *)c->U;
  } else {
    if ((s = dev_alloc(c, &A64, blk)) || (s = dev_alloc(c, &Q64, blk))) {
      release();
      return s;
    }
    A = (double *)A64;
    Q = (double *)Q64;
  }
  if (use_tc && !tcw) {
    tcb = fp64tc_workspace_bytes(c->n, c->ld);
    if ((s = dev_alloc(c, &tc_tmp, tcb))) {
      release();
      return s;
    }
    tcw = tc_tmp;
  }
  if (!use_tc && wsb < gbytes) {
    if ((s = dev_alloc(c, &gws, gbytes))) {
      release();
      return s;
    }
    ws = gws;
    wsb = gbytes;
  }
  if ((s = launch_pad_copy<double>(c->n, c->p, c->ld, U0_dev, A, c->st)) ||
      (s = use_tc ? gram_fp64tc(c->n, c->p, c->ld, A, nullptr, nullptr, nullptr, c->D, tcw, tcb,
                                c->dev_err, c->st)
                  : gram<double>(c->n, c->p, c->ld, A, A, nullptr, nullptr, c->D, ws, wsb,
                                 c->st)) ||
      (s = cholqr_coeff(c->p, c->ld, c->D, c->KU, c->core_ws, c->st)) ||
      (s = use_tc ? update_fp64tc(c->n, c->ld, A, nullptr, c->KU, nullptr, false, Q, tcw, tcb,
                                  c->dev_err, c->st)
                  : update<double>(c->n, c->ld, A, nullptr, c->KU, nullptr, Q, c->st))) {
    release();
    return s;
  }
  if constexpr (!std::is_same<T, double>::value) {
    // convert in chunks of at most 2^30 elements
    const long long total = c->n * c->ld;
    for (long long o = 0; o < total && !s; o += (1ll << 30)) {
      const long long cnt = (total - o) < (1ll << 30) ? (total - o) : (1ll << 30);
      s = launch_convert<T>((int)cnt, Q + o, (T *)c->U + o, c->st);
    }
  }
  if (s == OP_OK) s = cholqr_check(c);
  else cudaStreamSynchronize(c->st);
  release();
  return s;
}

template <typename T>
op_status init_impl(op_ctx *c, const double *V, const double *U0, bool device) {
  if (c) c->rec_ok = false;  // its scratch or its result replaces a carried residual
  const long long n = c->n;
  const int ld = c->ld;
  const size_t blk = (size_t)n * ld * sizeof(T);
  // potential: min / max for the default shift and the residual normalisation
  std::vector<double> Vh(n);
  if (device) {
    OP_CUDA(cudaMemcpy(Vh.data(), V, n * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    memcpy(Vh.data(), V, n * sizeof(double));
  }
  double vmin = Vh[0], vmax = Vh[0];
  for (long long i = 0; i < n; ++i) {
    if (!isfinite(Vh[i])) {
      set_error("V has a non-finite value at %lld", i);
      return OP_ERR_ARG;
    }
    vmin = Vh[i] < vmin ? Vh[i] : vmin;
    vmax = Vh[i] > vmax ? Vh[i] : vmax;
  }
  const double L = spectrum_lower_bound(&c->pb, vmin);
  c->sigma = isnan(c->pb.sigma) ? (1.0 - L > 0.0 ? 1.0 - L : 0.0) : c->pb.sigma;
  c->hnorm = 2.0 * c->g.cdiag +
             (fabs(vmax + c->sigma) > fabs(vmin + c->sigma) ? fabs(vmax + c->sigma)
                                                            : fabs(vmin + c->sigma));
  // default step: 1.5 (L + sigma) for the G flow; the explicit scale 1 / ||H + sigma||
  // for the L2 flow
  if (isnan(c->pb.tau))
    c->tau = c->pb.flow == OP_FLOW_L2 ? 1.0 / c->hnorm : 1.5 * (L + c->sigma);
  else
    c->tau = c->pb.tau;
  if (!(c->tau > 0.0) || !isfinite(c->sigma)) {
    set_error("tau must be positive (got %g) and sigma finite", c->tau);
    return OP_ERR_ARG;
  }
  c->Lb = L;
  c->sigma0 = c->sigma;
  c->adapt_off = 0;
  // device buffers
  void *p;
  OP_TRY(dev_alloc(c, &c->U, blk));
  OP_TRY(dev_alloc(c, &c->U2, blk));
  OP_TRY(dev_alloc(c, &c->W, blk));
  OP_TRY(dev_alloc(c, &c->Vt, (size_t)n * sizeof(T)));
  const size_t mat = (size_t)ld * ld * sizeof(double);
  OP_TRY(dev_alloc(c, &p, 6 * mat));
  c->C = (double *)p;
  c->S = c->C + (size_t)ld * ld;
  c->D = c->S + (size_t)ld * ld;
  c->KU = c->D + (size_t)ld * ld;
  c->KW = c->KU + (size_t)ld * ld;
  c->Th = c->KW + (size_t)ld * ld;
  OP_TRY(dev_alloc(c, &p, (2 * (size_t)c->p * c->p + c->p) * sizeof(double)));
  c->eig_work = (double *)p;
  c->lam_d = c->eig_work + 2 * (size_t)c->p * c->p;
  OP_TRY(dev_alloc(c, &c->KU_t, (size_t)ld * ld * sizeof(T)));
  OP_TRY(dev_alloc(c, &c->KW_t, (size_t)ld * ld * sizeof(T)));
  OP_TRY(dev_alloc(c, &c->cg_ws, cg_workspace_bytes(n, ld, sizeof(T))));
  cg_carve(c->cg_ws, n, ld, sizeof(T), &c->cgw);
  c->cgw.prof = &c->prof;
  c->cgw.jacobi = c->pb.cg_precond == OP_PRECOND_JACOBI;
  c->refine = sizeof(T) == 8 && c->pb.flow == OP_FLOW_G &&
              (c->pb.step1 == OP_STEP1_REFINE ||
               (c->pb.step1 == OP_STEP1_AUTO && c->pb.fp64_gemm == OP_GEMM_TC));
  c->Vt32 = nullptr;
  c->ref_scale = nullptr;
  if (c->refine) {
    // the FP32 CG's blocks: R, P in the FP64 block Q, its direction buffer Q in U2 (set per
    // call); the rhs and solution in the FP64 block P; its reductions of its own
    const size_t b32 = (size_t)n * ld * sizeof(float);
    memset(&c->cgw32, 0, sizeof(c->cgw32));
    c->cgw32.R = c->cgw.Q;
    c->cgw32.P = (char *)c->cgw.Q + b32;
    c->cgw32.Q = nullptr;
    c->cgw32.max_blocks = c->cgw.max_blocks;
    const size_t pb = (part_bytes(ld) + 255) / 256 * 256;
    const size_t sb = ((size_t)6 * ld * sizeof(double) + 255) / 256 * 256;
    const size_t ab = ((size_t)ld * sizeof(int) + 255) / 256 * 256;
    OP_TRY(dev_alloc(c, &p, pb + sb + ab + 256 + (size_t)ld * (sizeof(double) + sizeof(float))));
    c->cgw32.part = (double *)p;
    c->cgw32.state = (double *)((char *)p + pb);
    c->cgw32.active = (int *)((char *)p + pb + sb);
    c->cgw32.ctl = (int *)((char *)p + pb + sb + ab);
    c->ref_scale = (double *)((char *)p + pb + sb + ab + 256);
    c->cgw32.jacobi = c->cgw.jacobi;
    c->cgw32.prof = &c->prof;
    c->cgw32.expect_iters = 0;
    OP_TRY(dev_alloc(c, &p, (size_t)n * sizeof(float)));
    c->Vt32 = (float *)p;
  }
  c->gram_bytes = gram_workspace_bytes(n, ld, sizeof(T));
  if (sizeof(T) == 4) {
    const size_t tcb = gram_tc_workspace_bytes(n, ld);
    if (tcb > c->gram_bytes) c->gram_bytes = tcb;
    OP_TRY(dev_alloc(c, &p, 2 * (size_t)ld * 2 * ld * sizeof(float)));
    c->KT_hi = (float *)p;
    c->KT_lo = c->KT_hi + (size_t)ld * 2 * ld;
  }
  OP_TRY(dev_alloc(c, &c->gram_ws, c->gram_bytes));
  c->tc_ws = nullptr;
  c->tc_bytes = 0;
  if (sizeof(T) == 8 && c->pb.fp64_gemm == OP_GEMM_TC) {
    c->tc_bytes = fp64tc_workspace_bytes(n, ld);
    OP_TRY(dev_alloc(c, &c->tc_ws, c->tc_bytes));
  }
  c->core_tc_ws = nullptr;
  c->core_tc_bytes = 0;
  if (!c->tc_ws && c->p > 128 && c->pb.fp64_gemm == OP_GEMM_TC) {
    c->core_tc_bytes = fp64tc_workspace_bytes(c->p, ld);
    OP_TRY(dev_alloc(c, &c->core_tc_ws, c->core_tc_bytes));
  }
  OP_TRY(dev_alloc(c, &p, 256));
  c->dev_err = (int *)p;
  OP_CUDA(cudaMemsetAsync(c->dev_err, 0, 256, c->st));
  OP_TRY(dev_alloc(c, &c->core_ws, core_workspace_bytes(c->p, ld)));
  c->cayley_ws = nullptr;
  if (c->pb.flow == OP_FLOW_L2) OP_TRY(dev_alloc(c, &c->cayley_ws, cayley_workspace_bytes(c->p)));
  OP_TRY(dev_alloc(c, &p, part_bytes(ld)));
  c->part = (double *)p;
  OP_TRY(dev_alloc(c, &p, 64 * sizeof(double)));
  c->dsc = (double *)p;
  OP_CUDA(cudaMallocHost((void **)&c->hsc, 64 * sizeof(double)));
  OP_CUDA(cudaMallocHost((void **)&c->hpin_int, 16 * sizeof(int)));
  c->cgw.host_ctl = c->hpin_int + 4;
  c->cgw32.host_ctl = c->hpin_int + 8;
  OP_CUDA(cudaMemsetAsync(c->W, 0, blk, c->st));
  OP_CUDA(cudaMemsetAsync(c->U2, 0, blk, c->st));

  // V in T
  void *V64 = nullptr;
  OP_TRY(dev_alloc(c, &V64, n * sizeof(double)));
  OP_CUDA(cudaMemcpyAsync(V64, device ? (const void *)V : (const void *)Vh.data(),
                          n * sizeof(double),
                          device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
  OP_TRY(launch_convert<T>((int)n, (const double *)V64, (T *)c->Vt, c->st));
  if (c->Vt32) OP_TRY(launch_convert<float>((int)n, (const double *)V64, c->Vt32, c->st));
  // raw U0 (n x p FP64) on the device (a device U0 is read in place)
  void *U0d = nullptr;
  if (!device) {
    OP_TRY(dev_alloc(c, &U0d, (size_t)n * c->p * sizeof(double)));
    OP_CUDA(cudaMemcpyAsync(U0d, U0, (size_t)n * c->p * sizeof(double), cudaMemcpyHostToDevice,
                            c->st));
  }
  op_status s = orthonormalise_impl<T>(c, device ? U0 : (const double *)U0d);
  OP_CUDA(cudaStreamSynchronize(c->st));
  for (void *q : {V64, U0d}) {
    if (!q) continue;
    cudaFree(q);
    for (auto it = c->allocs.begin(); it != c->allocs.end(); ++it)
      if (*it == q) {
        c->allocs.erase(it);
        break;
      }
  }
  if (s) return s;
  c->g_rel = 1.0;
  c->stats.sigma = c->sigma;
  c->stats.tau = c->tau;
  c->stats.residual = NAN;
  OP_TRY(energy_impl<T>(c));
  c->stats.err_E = fabs(c->E);  // err_E^0 = |E(U^0)| (Algorithm 1)
  return OP_OK;
}

op_status init_common(op_ctx **out, const op_problem *pb, const double *V, const double *U0,
                      void *stream, bool device) {
  if (!out) {
    set_error("null ctx pointer");
    return OP_ERR_ARG;
  }
  *out = nullptr;
  OP_TRY(check_problem(pb));
  if (!V || !U0) {
    set_error("V and U0 must be non-null");
    return OP_ERR_ARG;
  }
  op_ctx *c = new op_ctx();
  memset(&c->stats, 0, sizeof(c->stats));
  c->pb = *pb;
  make_geom(pb, &c->g);
  c->n = c->g.n;
  c->p = pb->p;
  c->ld = round_up(pb->p, 8);
  c->prec = pb->prec;
  c->elem = pb->prec == OP_FP64 ? 8 : 4;  // OP_FP32 and OP_MIX_TF32 store FP32 blocks
  c->st = (cudaStream_t)stream;
  op_status s = c->prec == OP_FP64 ? init_impl<double>(c, V, U0, device)
                                   : init_impl<float>(c, V, U0, device);
  if (s != OP_OK) {
    cudaStreamSynchronize(c->st);
    free_all(c);
    delete c;
    return s;
  }
  *out = c;
  return OP_OK;
}

// Raw initial block from a seed: normal k of the SplitMix64 counter stream
// key = seed ^ (1 * 0xD1B54A32D192ED03) (stream tag 1), drawn by the Box-Muller transform
// from uniforms 2k and 2k+1 (output j of the stream is mix64(key + (j + 1) * golden
// gamma); a uniform is ((z >> 11) + 0.5) 2^-53).  SplitMix64: Steele, Lea and Flood,
// "Fast splittable pseudorandom number generators" (OOPSLA 2014).
__device__ __forceinline__ unsigned long long splitmix_mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_gaussian_block(long long count, unsigned long long key, double *__restrict__ out) {
  const unsigned long long gamma = 0x9E3779B97F4A7C15ull;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x) {
    const unsigned long long z1 = splitmix_mix(key + (unsigned long long)(2 * k + 1) * gamma);
    const unsigned long long z2 = splitmix_mix(key + (unsigned long long)(2 * k + 2) * gamma);
    const double u1 = ((double)(z1 >> 11) + 0.5) * 0x1p-53;
    const double u2 = ((double)(z2 >> 11) + 0.5) * 0x1p-53;
    out[k] = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
  }
}

op_status launch_gaussian_block(unsigned long long seed, long long count, double *out,
                                cudaStream_t st) {
  const unsigned long long key = seed ^ (1ull * 0xD1B54A32D192ED03ull);
  k_gaussian_block<<<num_sms() * 8, 256, 0, st>>>(count, key, out);
  count_launch();
  OP_LAUNCH("k_gaussian_block");
  return OP_OK;
}

op_status init_seeded(op_ctx **out, const op_problem *pb, const double *V,
                      unsigned long long seed, void *stream) {
  if (!out) {
    set_error("null ctx pointer");
    return OP_ERR_ARG;
  }
  *out = nullptr;
  OP_TRY(check_problem(pb));
  if (!V) {
    set_error("V must be non-null");
    return OP_ERR_ARG;
  }
  Geom g;
  OP_TRY(make_geom(pb, &g));
  cudaStream_t st = (cudaStream_t)stream;
  double *Vd = nullptr, *U0d = nullptr;
  const size_t ubytes = (size_t)g.n * pb->p * sizeof(double);
  cudaError_t e = cudaMalloc((void **)&Vd, g.n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void **)&U0d, ubytes);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Vd, V, g.n * sizeof(double), cudaMemcpyHostToDevice, st);
  op_status s = OP_OK;
  if (e == cudaSuccess) {
    const op_status gs = launch_gaussian_block(seed, g.n * pb->p, U0d, st);
    if (gs != OP_OK) {
      cudaStreamSynchronize(st);
      cudaFree(Vd);
      cudaFree(U0d);
      return gs;
    }
  }
  if (e != cudaSuccess)
    s = cuda_status(e, "op_init_seeded");
  else
    s = init_common(out, pb, Vd, U0d, stream, true);
  cudaStreamSynchronize(st);
  if (Vd) cudaFree(Vd);
  if (U0d) cudaFree(U0d);
  return s;
}

}  // namespace

// Adaptive shift (op_problem.adapt_every): from the Ritz values lambda_1 <= .. <=
// lambda_p of the current U, sigma = max(sigma_0, lambda_p - 2 lambda_1) and
// tau = 1.5 (L + sigma).  With G = (H + sigma)^-1 and tau ~ 1/mu_1, the slowest
// directions contract per step in proportion to (lambda_1 + sigma) (lambda_{p+1} -
// lambda_p) / ((lambda_p + sigma) (lambda_{p+1} + sigma)), which is largest at
// sigma ~ lambda_p - 2 lambda_1.  Changes below 10 % are skipped.  The previous
// sigma and tau are returned for the energy guard.  Synchronises the context's stream.
double opevo::cg_rtol_for(op_ctx *c) {
  if (c->pb.cg_rtol > 0.0) return c->pb.cg_rtol;
  const double floor = c->prec == OP_FP64 ? 1e-13 : 1e-6;
  double r = 0.1 * c->g_rel;
  if (!(r < 1e-2)) r = 1e-2;
  if (c->cg_cap > 0.0 && r > c->cg_cap) r = c->cg_cap;
  if (r < floor) r = floor;
  return r;
}

int opevo::cg_max_iter(op_ctx *c) { return c->pb.cg_max_iter > 0 ? c->pb.cg_max_iter : 2000; }

op_status opevo::retune_shift(op_ctx *c, double *prev_sigma, double *prev_tau) {
  if (c) c->rec_ok = false;  // its scratch or its result replaces a carried residual
  std::vector<double> lam(c->p);
  OP_TRY(c->prec == OP_FP64 ? eig_impl<double>(c, lam.data(), OP_EIG_RITZ)
                            : eig_impl<float>(c, lam.data(), OP_EIG_RITZ));
  *prev_sigma = c->sigma;
  *prev_tau = c->tau;
  double s = lam[c->p - 1] - 2.0 * lam[0];
  if (!(s > c->sigma0)) s = c->sigma0;
  if (!isfinite(s) || fabs(s - c->sigma) <= 0.1 * fabs(c->sigma + c->Lb)) return OP_OK;
  c->sigma = s;
  c->tau = 1.5 * (c->Lb + s);
  c->stats.sigma = c->sigma;
  c->stats.tau = c->tau;
  return OP_OK;
}

extern "C" {

const char *op_version(void) { return "opevo 0.1 (sm_103a)"; }

const char *op_last_error(void) { return g_err; }

long long op_kernel_launches(void) { return g_launches.load(); }

op_status op_init(op_ctx **ctx, const op_problem *pb, const double *V, const double *U0,
                  void *stream) {
  g_err[0] = 0;
  return init_common(ctx, pb, V, U0, stream, false);
}

op_status op_init_seeded(op_ctx **ctx, const op_problem *pb, const double *V,
                         unsigned long long seed, void *stream) {
  g_err[0] = 0;
  return init_seeded(ctx, pb, V, seed, stream);
}

op_status op_init_device(op_ctx **ctx, const op_problem *pb, const double *V_dev,
                         const double *U0_dev, void *stream) {
  g_err[0] = 0;
  return init_common(ctx, pb, V_dev, U0_dev, stream, true);
}

op_status op_step(op_ctx *c, int nsteps, op_stats *st) {
  if (!c || nsteps < 0) {
    set_error("op_step: null context or negative step count");
    return OP_ERR_ARG;
  }
  auto t0 = std::chrono::steady_clock::now();
  for (int k = 0; k < nsteps; ++k) {
    op_status s = c->prec == OP_FP64 ? step_impl<double>(c) : step_impl<float>(c);
    if (s != OP_OK) return s;
  }
  c->stats.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                    .count();
  if (st) *st = c->stats;
  return OP_OK;
}

op_status op_residual(op_ctx *c, double *r) {
  if (!c || !r) {
    set_error("op_residual: null argument");
    return OP_ERR_ARG;
  }
  return c->prec == OP_FP64 ? residual_impl<double>(c, r) : residual_impl<float>(c, r);
}

op_status op_solve(op_ctx *c, double tol, int max_steps, int stop, op_stats *st) {
  if (!c || max_steps < 0 || (stop != OP_STOP_RESIDUAL && stop != OP_STOP_ERR_E &&
                              stop != OP_STOP_STEPS)) {
    set_error("op_solve: bad arguments");
    return OP_ERR_ARG;
  }
  auto t0 = std::chrono::steady_clock::now();
  const int every = c->pb.check_every > 0 ? c->pb.check_every : 10;
  // the inner solves must be more accurate than the outer target: r ~ rtol for the
  // residual rule, err_E ~ r^2 for Algorithm 1's rule
  c->cg_cap = stop == OP_STOP_RESIDUAL ? 0.1 * tol : (stop == OP_STOP_ERR_E ? 0.1 * sqrt(tol) : 0.0);
  bool done = false;
  double r = NAN;
  const int adapt = c->pb.adapt_every;
  double prev_sigma = c->sigma, prev_tau = c->tau, E_before = 0.0;
  bool probation = false;  // the step after a re-tune: undo it if the energy rises
  for (int k = 0; k <= max_steps; ++k) {
    if (stop == OP_STOP_ERR_E && c->stats.err_E <= tol) {
      done = true;
      break;
    }
    if (stop == OP_STOP_RESIDUAL && k % every == 0) {
      OP_TRY(op_residual(c, &r));
      if (r <= tol) {
        done = true;
        break;
      }
    }
    if (k == max_steps) break;
    if (adapt > 0 && !c->adapt_off && c->stats.steps > 0 && c->stats.steps % adapt == 0) {
      OP_TRY(retune_shift(c, &prev_sigma, &prev_tau));
      probation = c->sigma != prev_sigma;
      E_before = c->E;
    }
    op_status s = c->prec == OP_FP64 ? step_impl<double>(c) : step_impl<float>(c);
    if (s != OP_OK) return s;
    if (probation) {
      probation = false;
      if (c->E > E_before + 1e-12 * fabs(E_before)) {  // energy rose: undo, stop adapting
        c->sigma = prev_sigma;
        c->tau = prev_tau;
        c->stats.sigma = c->sigma;
        c->stats.tau = c->tau;
        c->adapt_off = 1;
      }
    }
  }
  c->cg_cap = 0.0;
  if (stop == OP_STOP_STEPS) done = true;
  if (stop != OP_STOP_RESIDUAL || !done) OP_TRY(op_residual(c, &r));
  c->stats.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                    .count();
  if (st) *st = c->stats;
  if (!done) {
    set_error("op_solve: stop rule not met after %d steps", max_steps);
    return OP_ERR_STATE;
  }
  return OP_OK;
}

namespace {
struct CkptHeader {
  char magic[8];  // "OPEVOCK2"
  long long n;
  int p, ld, prec, elem;
  double sigma, tau, sigma0, Lb, E, g_rel;
  int adapt_off, expect_iters;
  int carried;  // the block before the last update follows W (the carried residual's U)
  op_stats stats;
};
const char kCkptMagic[8] = {'O', 'P', 'E', 'V', 'O', 'C', 'K', '2'};
// blocks of a checkpoint: U, W, and with the mixed-precision Step 1 the block before the
// last update, from which restore rebuilds the residual the next Step 1 starts from
int ckpt_blocks(const op_ctx *c) { return c->refine ? 3 : 2; }
}  // namespace

size_t op_checkpoint_size(const op_ctx *c) {
  if (!c) return 0;
  return sizeof(CkptHeader) + ckpt_blocks(c) * (size_t)c->n * c->ld * c->elem;
}

op_status op_checkpoint(op_ctx *c, void *buf, size_t len) {
  if (!c || !buf || len < op_checkpoint_size(c)) {
    set_error("op_checkpoint: null argument or buffer smaller than op_checkpoint_size");
    return OP_ERR_ARG;
  }
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kCkptMagic, 8);
  h.n = c->n;
  h.p = c->p;
  h.ld = c->ld;
  h.prec = c->prec;
  h.elem = c->elem;
  h.sigma = c->sigma;
  h.tau = c->tau;
  h.sigma0 = c->sigma0;
  h.Lb = c->Lb;
  h.E = c->E;
  h.g_rel = c->g_rel;
  h.adapt_off = c->adapt_off;
  h.expect_iters = c->cgw.expect_iters;
  h.carried = c->rec_ok ? 1 : 0;
  h.stats = c->stats;
  const size_t blk = (size_t)c->n * c->ld * c->elem;
  char *out = (char *)buf;
  memcpy(out, &h, sizeof(h));
  OP_CUDA(cudaMemcpyAsync(out + sizeof(h), c->U, blk, cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaMemcpyAsync(out + sizeof(h) + blk, c->W, blk, cudaMemcpyDeviceToHost, c->st));
  if (ckpt_blocks(c) > 2)
    OP_CUDA(cudaMemcpyAsync(out + sizeof(h) + 2 * blk, c->U2, blk, cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaStreamSynchronize(c->st));
  return OP_OK;
}

op_status op_restore(op_ctx *c, const void *buf, size_t len) {
  if (!c || !buf || len < sizeof(CkptHeader)) {
    set_error("op_restore: null argument or buffer too small");
    return OP_ERR_ARG;
  }
  CkptHeader h;
  memcpy(&h, buf, sizeof(h));
  if (memcmp(h.magic, kCkptMagic, 8) != 0 || h.n != c->n || h.p != c->p || h.ld != c->ld ||
      h.prec != c->prec || h.elem != c->elem || len < op_checkpoint_size(c)) {
    set_error("op_restore: not a checkpoint of a context with this size and precision");
    return OP_ERR_ARG;
  }
  const size_t blk = (size_t)c->n * c->ld * c->elem;
  const char *in = (const char *)buf;
  OP_CUDA(cudaMemcpyAsync(c->U, in + sizeof(h), blk, cudaMemcpyHostToDevice, c->st));
  OP_CUDA(cudaMemcpyAsync(c->W, in + sizeof(h) + blk, blk, cudaMemcpyHostToDevice, c->st));
  c->rec_ok = false;
  if (ckpt_blocks(c) > 2 && h.carried) {
    // the carried residual: the same values the checkpointed context held
    OP_CUDA(cudaMemcpyAsync(c->U2, in + sizeof(h) + 2 * blk, blk, cudaMemcpyHostToDevice, c->st));
    OP_TRY(refine_residual(c->g, (const double *)c->Vt, h.sigma, (const double *)c->U2,
                           (const double *)c->W, c->ld, c->cgw, c->st));
    c->rec_ok = true;
  }
  OP_CUDA(cudaStreamSynchronize(c->st));
  c->sigma = h.sigma;
  c->tau = h.tau;
  c->sigma0 = h.sigma0;
  c->Lb = h.Lb;
  c->E = h.E;
  c->g_rel = h.g_rel;
  c->adapt_off = h.adapt_off;
  c->cgw.expect_iters = h.expect_iters;
  c->stats = h.stats;
  return OP_OK;
}

op_status op_energy(op_ctx *c, double *E) {
  if (!c || !E) {
    set_error("op_energy: null argument");
    return OP_ERR_ARG;
  }
  op_status s = c->prec == OP_FP64 ? energy_impl<double>(c) : energy_impl<float>(c);
  if (s == OP_OK) *E = c->E;
  return s;
}

op_status op_get_U(op_ctx *c, double *U_host) {
  if (c) c->rec_ok = false;  // its scratch or its result replaces a carried residual
  if (!c || !U_host) {
    set_error("op_get_U: null argument");
    return OP_ERR_ARG;
  }
  // stage through the CG scratch (3 blocks of T >= n x p doubles for ld <= 1.5 p... ) in
  // row chunks that fit one scratch block of T
  const size_t cap_rows = ((size_t)c->n * c->ld * c->elem) / ((size_t)c->p * sizeof(double));
  const long long rows = cap_rows > 0 ? (long long)cap_rows : 1;
  double *stage = (double *)c->cgw.R;
  for (long long r0 = 0; r0 < c->n; r0 += rows) {
    const long long cnt = (c->n - r0) < rows ? (c->n - r0) : rows;
    op_status s;
    if (c->prec == OP_FP64)
      s = launch_unpad_copy<double>(cnt, c->p, c->ld, (const double *)c->U + r0 * c->ld, stage,
                                    c->st);
    else
      s = launch_unpad_copy<float>(cnt, c->p, c->ld, (const float *)c->U + r0 * c->ld, stage,
                                   c->st);
    if (s) return s;
    OP_CUDA(cudaMemcpyAsync(U_host + r0 * c->p, stage, (size_t)cnt * c->p * sizeof(double),
                            cudaMemcpyDeviceToHost, c->st));
    OP_CUDA(cudaStreamSynchronize(c->st));
  }
  return OP_OK;
}

op_status op_get_U_device(op_ctx *c, void *U_dev, int prec) {
  if (!c || !U_dev || (prec != OP_FP64 && prec != OP_FP32) || ((uintptr_t)U_dev & 15)) {
    set_error("op_get_U_device: null or unaligned pointer, or prec not OP_FP64 / OP_FP32");
    return OP_ERR_ARG;
  }
  OP_TRY(launch_unpad_to(c->n, c->p, c->ld, c->U, c->prec == OP_FP64 ? 8 : 4, U_dev,
                         prec == OP_FP64 ? 8 : 4, c->st));
  OP_CUDA(cudaStreamSynchronize(c->st));
  return OP_OK;
}

op_status op_eigenvalues(op_ctx *c, double *lam, int kind) {
  if (!c || !lam || (kind != OP_EIG_RITZ && kind != OP_EIG_PAPER)) {
    set_error("op_eigenvalues: bad arguments");
    return OP_ERR_ARG;
  }
  return c->prec == OP_FP64 ? eig_impl<double>(c, lam, kind) : eig_impl<float>(c, lam, kind);
}

op_status op_profile_enable(op_ctx *c, int enable) {
  if (!c) {
    set_error("op_profile_enable: null context");
    return OP_ERR_ARG;
  }
  OP_CUDA(cudaStreamSynchronize(c->st));
  return prof_enable(&c->prof, enable != 0);
}

int op_profile_kinds(void) { return PK_COUNT; }

const char *op_profile_name(int kind) { return prof_name(kind); }

op_status op_profile_read(op_ctx *c, int kind, double *total_ms, long long *launches) {
  if (!c || kind < 0 || kind >= PK_COUNT || !total_ms || !launches) {
    set_error("op_profile_read: bad arguments");
    return OP_ERR_ARG;
  }
  *total_ms = c->prof.ms[kind];
  *launches = c->prof.cnt[kind];
  return OP_OK;
}

op_status op_get_stats(op_ctx *c, op_stats *st) {
  if (!c || !st) {
    set_error("op_get_stats: null argument");
    return OP_ERR_ARG;
  }
  *st = c->stats;
  return OP_OK;
}

void op_destroy(op_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  free_all(c);
  delete c;
}

// ---------------------------------------------------------------------------
// Kernel-level entry points
// ---------------------------------------------------------------------------
static op_status check_blocks(int prec, int p, int ld, const void *a, const void *b) {
  if (prec != OP_FP64 && prec != OP_FP32 && prec != OP_MIX_BF16X3) {
    set_error("unsupported precision mode %d", prec);
    return OP_ERR_ARG;
  }
  if (p < 1 || ld < p || ld % 8 != 0) {
    set_error("need 1 <= p <= ld and ld %% 8 == 0 (p=%d ld=%d)", p, ld);
    return OP_ERR_ARG;
  }
  if (!a || !b || ((uintptr_t)a & 15) || ((uintptr_t)b & 15)) {
    set_error("block pointers must be non-null and 16-byte aligned");
    return OP_ERR_ARG;
  }
  return OP_OK;
}

op_status op_apply_H(const op_problem *pb, int ld, const void *V_t, double sigma, const void *X,
                     void *Y, void *stream) {
  Geom g;
  OP_TRY(make_geom(pb, &g));
  OP_TRY(check_blocks(pb->prec, pb->p, ld, X, Y));
  if (!V_t) {
    set_error("null V");
    return OP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (pb->prec == OP_FP64)
    return launch_apply<double>(g, (const double *)V_t, sigma, (const double *)X, (double *)Y, ld,
                                st);
  return launch_apply<float>(g, (const float *)V_t, sigma, (const float *)X, (float *)Y, ld, st);
}

size_t op_cg_workspace(const op_problem *pb, int ld) {
  Geom g;
  if (!pb || make_geom(pb, &g) != OP_OK || ld < 8) return 0;
  const int elem = pb->prec == OP_FP64 ? 8 : 4;
  return cg_workspace_bytes(g.n, ld, elem) + 64;
}

op_status op_cg_solve(const op_problem *pb, int ld, const void *V_t, double sigma, const void *U,
                      void *W, double rtol, int max_iter, void *ws, size_t ws_bytes, int *iters,
                      void *stream) {
  Geom g;
  OP_TRY(make_geom(pb, &g));
  OP_TRY(check_blocks(pb->prec, pb->p, ld, U, W));
  if (!V_t || !ws || !iters || ws_bytes < op_cg_workspace(pb, ld) || max_iter < 0) {
    set_error("op_cg_solve: bad V, workspace (%zu < %zu), iters or max_iter", ws_bytes,
              op_cg_workspace(pb, ld));
    return OP_ERR_ARG;
  }
  const int elem = pb->prec == OP_FP64 ? 8 : 4;
  if (pb->cg_precond != OP_PRECOND_NONE && pb->cg_precond != OP_PRECOND_JACOBI) {
    set_error("op_cg_solve: unsupported CG preconditioner %d", pb->cg_precond);
    return OP_ERR_ARG;
  }
  CGWork w;
  cg_carve(ws, g.n, ld, elem, &w);
  w.jacobi = pb->cg_precond == OP_PRECOND_JACOBI;
  int host_ctl[4] = {0, 0, 0, 0};
  w.host_ctl = host_ctl;
  cudaStream_t st = (cudaStream_t)stream;
  op_status s;
  if (pb->prec == OP_FP64)
    s = cg_solve<double>(g, (const double *)V_t, sigma, (const double *)U, (double *)W, pb->p, ld,
                         rtol, max_iter, w, iters, st);
  else
    s = cg_solve<float>(g, (const float *)V_t, sigma, (const float *)U, (float *)W, pb->p, ld,
                        rtol, max_iter, w, iters, st);
  return s;
}

// Kernel-level scratch of op_gram / op_update starts with a 256-byte header whose first
// int is the "bounded device wait gave up" flag (read back by op_ws_status).
static const size_t kWsHeader = 256;

size_t op_gram_workspace(int prec, long long n, int ld) {
  if (prec == OP_FP32 || prec == OP_MIX_BF16X3) return kWsHeader + gram_tc_workspace_bytes(n, ld);
  return kWsHeader + gram_workspace_bytes(n, ld, 8);
}

op_status op_gram(int prec, long long n, int p, int ld, const void *U, const void *W, double *C,
                  double *S, double *D, void *ws, size_t ws_bytes, void *stream) {
  OP_TRY(check_blocks(prec, p, ld, U, W));
  if (n < 1 || !ws || ws_bytes < kWsHeader) {
    set_error("op_gram: n must be positive and ws hold at least op_gram_workspace() bytes");
    return OP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  OP_CUDA(cudaMemsetAsync(ws, 0, sizeof(int), st));
  void *part = (char *)ws + kWsHeader;
  const size_t pbytes = ws_bytes - kWsHeader;
  if (prec == OP_FP64)
    return gram<double>(n, p, ld, (const double *)U, (const double *)W, C, S, D, part, pbytes, st);
  return gram_tc(n, p, ld, (const float *)U, (const float *)W, C, S, D, part, pbytes, (int *)ws,
                 st, prec == OP_MIX_BF16X3 ? 2 : 1);
}

op_status op_ws_status(void *ws, void *stream) {
  if (!ws) {
    set_error("null workspace");
    return OP_ERR_ARG;
  }
  int h = 0;
  OP_CUDA(cudaMemcpyAsync(&h, ws, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  OP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (h) {
    set_error("a bounded device wait gave up (tensor-core pipeline did not complete)");
    return OP_ERR_TIMEOUT;
  }
  return OP_OK;
}

size_t op_core_workspace(int p, int ld) { return core_workspace_bytes(p, ld); }

op_status op_core(int prec, int p, int ld, double tau, const double *C, const double *S,
                  double *KU, double *KW, void *KU_t, void *KW_t, void *ws, size_t ws_bytes,
                  void *stream) {
  if (prec != OP_FP64 && prec != OP_FP32) {
    set_error("unsupported precision mode %d", prec);
    return OP_ERR_ARG;
  }
  if (p < 1 || ld < p || ld % 8 || !C || !S || !KU || !KW || !ws ||
      ws_bytes < core_workspace_bytes(p, ld) || !(tau > 0.0)) {
    set_error("op_core: bad arguments");
    return OP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == OP_FP64)
    return core<double>(p, ld, tau, C, S, KU, KW, (double *)KU_t, (double *)KW_t, ws, st);
  return core<float>(p, ld, tau, C, S, KU, KW, (float *)KU_t, (float *)KW_t, ws, st);
}

op_status op_core_status(void *ws, void *stream) {
  if (!ws) {
    set_error("null workspace");
    return OP_ERR_ARG;
  }
  int h = 0;
  OP_CUDA(cudaMemcpyAsync(&h, ws, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  OP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (h) {
    set_error("Cholesky pivot not positive");
    return OP_ERR_NOTSPD;
  }
  return OP_OK;
}

size_t op_update_workspace(int prec, int ld) {
  return kWsHeader +
         (prec == OP_FP32 || prec == OP_MIX_BF16X3 ? 2 * (size_t)ld * 2 * ld * sizeof(float) : 0);
}

op_status op_update(int prec, long long n, int p, int ld, const void *U, const void *W,
                    const void *KU_t, const void *KW_t, void *Unew, void *ws, size_t ws_bytes,
                    void *stream) {
  OP_TRY(check_blocks(prec, p, ld, U, W));
  if (!KU_t || !KW_t || !Unew || n < 1 || Unew == U || Unew == W || !ws ||
      ws_bytes < op_update_workspace(prec, ld)) {
    set_error("op_update: bad arguments (outputs must not alias inputs; ws >= "
              "op_update_workspace())");
    return OP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  OP_CUDA(cudaMemsetAsync(ws, 0, sizeof(int), st));
  if (prec == OP_FP64)
    return update<double>(n, ld, (const double *)U, (const double *)W, (const double *)KU_t,
                          (const double *)KW_t, (double *)Unew, st);
  float *KT_hi = (float *)((char *)ws + kWsHeader);
  float *KT_lo = KT_hi + (size_t)ld * 2 * ld;
  if (prec == OP_MIX_BF16X3) {
    OP_TRY(launch_make_kt_bf16_f32(ld, (const float *)KU_t, (const float *)KW_t,
                                   (uint16_t *)KT_hi, st));
    return update_bf16(n, ld, (const float *)U, (const float *)W, (const uint16_t *)KT_hi,
                       (float *)Unew, (int *)ws, st);
  }
  OP_TRY(launch_make_kt_f32(ld, (const float *)KU_t, (const float *)KW_t, KT_hi, KT_lo, st));
  return update_tc(n, ld, (const float *)U, (const float *)W, KT_hi, KT_lo, (float *)Unew,
                   (int *)ws, st);
}

op_status op_gaussian_block(unsigned long long seed, long long n, int p, double *U0,
                            void *stream) {
  if (n < 1 || p < 1 || !U0) {
    set_error("op_gaussian_block: need n >= 1, p >= 1 and an output block");
    return OP_ERR_ARG;
  }
  return launch_gaussian_block(seed, n * p, U0, (cudaStream_t)stream);
}

size_t op_fp64tc_workspace(long long n, int ld) {
  if (n < 1 || ld < 8) return 0;
  return kWsHeader + fp64tc_workspace_bytes(n, ld);
}

op_status op_gram_fp64tc(long long n, int p, int ld, const double *U, const double *W, double *C,
                         double *S, double *D, void *ws, size_t ws_bytes, void *stream) {
  if (n < 1 || p < 1 || ld < p || ld % 8 || !U || ((uintptr_t)U & 15) ||
      (W && ((uintptr_t)W & 15)) || (!W && (C || S)) || !ws ||
      ws_bytes < op_fp64tc_workspace(n, ld)) {
    set_error("op_gram_fp64tc: bad arguments (n=%lld p=%d ld=%d; C and S need W; ws >= "
              "op_fp64tc_workspace())", n, p, ld);
    return OP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  OP_CUDA(cudaMemsetAsync(ws, 0, sizeof(int), st));
  return gram_fp64tc(n, p, ld, U, W, C, S, D, (char *)ws + kWsHeader, ws_bytes - kWsHeader,
                     (int *)ws, st);
}

op_status op_update_fp64tc(long long n, int p, int ld, const double *U, const double *W,
                           const double *KU, const double *KW, double *Unew, void *ws,
                           size_t ws_bytes, void *stream) {
  if (n < 1 || p < 1 || ld < p || ld % 8 || !U || !KU || !Unew || (W && !KW) ||
      ((uintptr_t)U & 15) || (W && ((uintptr_t)W & 15)) || ((uintptr_t)Unew & 15) ||
      Unew == U || Unew == W || !ws || ws_bytes < op_fp64tc_workspace(n, ld)) {
    set_error("op_update_fp64tc: bad arguments (n=%lld p=%d ld=%d; outputs must not alias "
              "inputs; ws >= op_fp64tc_workspace())", n, p, ld);
    return OP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  OP_CUDA(cudaMemsetAsync(ws, 0, sizeof(int), st));
  return update_fp64tc(n, ld, U, W, KU, W ? KW : nullptr, true, Unew, (char *)ws + kWsHeader,
                       ws_bytes - kWsHeader, (int *)ws, st);
}

}  // extern "C"
