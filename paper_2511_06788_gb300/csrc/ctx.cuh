// Private definition of a solver context (shared by api.cu and batch.cu).
#pragma once

#include <vector>

#include "common.cuh"
#include "kernels.cuh"

using namespace opevo;

struct op_ctx {
  op_problem pb;
  Geom g;
  long long n;
  int p, ld, prec, elem;
  double sigma, tau, hnorm;
  double Lb, sigma0;     // spectrum lower bound L and the initial sigma (adaptive shift)
  int adapt_off;         // adaptation stopped (a re-tune raised the energy)
  cudaStream_t st;
  // blocks (element type T)
  void *U, *U2, *W, *Vt;
  // p x p (ld x ld) FP64 matrices
  double *C, *S, *D, *KU, *KW, *Th, *eig_work, *lam_d;
  void *KU_t, *KW_t;
  float *KT_hi, *KT_lo;  // FP32 blocks: [KU; KW]^T split for the tensor-core update
  int *dev_err;          // set by a tensor-core kernel whose bounded wait gave up
  void *cg_ws, *gram_ws, *core_ws;
  void *cayley_ws;       // OP_FLOW_L2: the 2p x 3p system of the exact Cayley step
  void *tc_ws;           // FP64 contexts with fp64_gemm = OP_GEMM_TC: digit planes etc.
  size_t tc_bytes;
  void *core_tc_ws;      // p > 128 with OP_GEMM_TC: the core's Newton-Schulz products (the
  size_t core_tc_bytes;  // FP64 contexts use tc_ws)
  // FP64 contexts with the mixed-precision Step 1: V in FP32, the FP32 CG's scratch (its
  // blocks alias the FP64 CG blocks Q and U2, its rhs and solution the FP64 block P)
  bool refine;
  // the refinement's R block holds U2 - (H + sigma) W, formed by the stencil at the end of
  // the last step (U2: the block before that step's update): the next Step 1 may start
  // from R + U - U2.  Cleared by every call that writes R, U2, W or sigma otherwise.
  bool rec_ok;
  float *Vt32;
  CGWork cgw32;
  double *ref_scale;
  size_t gram_bytes;
  CGWork cgw;
  Prof prof;
  double *part;  // [max_blocks][2][ld] for quad / sumsq
  double *dsc;   // device scalars: 0..2 core stats, 4..5 quad, 6 sumsq
  double *hsc;   // pinned mirror
  int *hpin_int;
  op_stats stats;
  double E;
  double g_rel;  // last relative G-residual sqrt(g2 / trS)
  double cg_cap; // op_solve: upper bound of the adaptive CG tolerance (from its stop rule)
  std::vector<void *> allocs;
};

namespace opevo {
// Adaptive shift (op_problem.adapt_every): re-tune c->sigma and c->tau from the Ritz
// values of the current U; the previous values are returned (api.cu).
op_status retune_shift(op_ctx *c, double *prev_sigma, double *prev_tau);
// Step-1 CG tolerance and iteration cap of the context's next step (api.cu).
double cg_rtol_for(op_ctx *c);
int cg_max_iter(op_ctx *c);
}  // namespace opevo
