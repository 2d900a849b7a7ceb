// Batches of independent eigenproblems (uneven n and p) advanced together.
//
// Every problem keeps its own context (buffers, scalars); a batch only adds
// descriptors of those buffers and work lists that map each CTA of a batched
// kernel to (problem, piece of work): grid-point ranges for the stencil / CG /
// energy kernels, (job, chunk) for the tensor-core Gram, 128-point tiles for
// the tensor-core update, and one CTA per problem for the core solve.  One time
// step of all problems is a fixed sequence of these launches (Step 1 with a
// fixed number of CG iterations whose kernels return at once for problems whose
// CG has converged), captured once as a CUDA graph per step parity (U and U+
// swap roles) and replayed.  The adaptive CG tolerance, the energy, err_E and
// the freeze of problems whose Algorithm-1 stop rule holds are computed on the
// device, so a run of steps needs no host synchronisation.
//
// The work-list granularity (grid points per row item, per Gram chunk) is
// chosen by timed trials on the batch itself (op_batch_autotune) and kept in a
// JSON cache keyed by the batch's shape.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "ctx.cuh"
#include "kernels.cuh"

// Per-problem step record on the device (doubles).
enum { BS_E = 0, BS_ERR = 1, BS_G2 = 2, BS_ORTH = 3, BS_TRS = 4, BS_STEPS = 5, BS_ITERS = 6,
       BS_LAST_ITERS = 7, BS_FIELDS = 8 };

namespace opevo {
namespace {

struct BatchCtl {
  int stop;       // OP_STOP_* of the current op_batch_solve (-1: none)
  double tol;
  double cg_cap;  // upper bound of the adaptive CG tolerance
};

// CG tolerance of each problem for the coming step (device side): the context's cg_rtol
// when positive, else the adaptive rule rtol = max(1e-6, min(1e-2, 0.1 g, cap)),
// g = relative G-residual of the last step.
__global__ void k_b_set_tol(const BatchProb *__restrict__ B, const double *__restrict__ stats,
                            const BatchCtl *__restrict__ ctl, int nprob) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nprob) return;
  if (B[b].fixed_rtol > 0.0) {
    *B[b].cg_rtol2 = B[b].fixed_rtol * B[b].fixed_rtol;
    return;
  }
  const double *s = stats + (long long)b * BS_FIELDS;
  double g = (s[BS_TRS] > 0.0 && s[BS_G2] > 0.0) ? sqrt(s[BS_G2] / s[BS_TRS]) : 1.0;
  double r = 0.1 * g;
  if (!(r < 1e-2)) r = 1e-2;
  if (ctl->cg_cap > 0.0 && r > ctl->cg_cap) r = ctl->cg_cap;
  if (r < 1e-6) r = 1e-6;
  *B[b].cg_rtol2 = r * r;
}

// After the step: energy, err_E, statistics; freeze when Algorithm 1's rule holds.
__global__ void k_b_step_end(const BatchProb *__restrict__ B, double *__restrict__ stats,
                             const BatchCtl *__restrict__ ctl, int nprob) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nprob) return;
  const BatchProb &pb = B[b];
  if (*pb.frozen) return;
  double *s = stats + (long long)b * BS_FIELDS;
  const double E = 0.5 * pb.dsc[4];
  const double err = fabs(E - s[BS_E]) / fabs(s[BS_E]);
  s[BS_ERR] = err;
  s[BS_E] = E;
  s[BS_G2] = pb.dsc[0];
  s[BS_ORTH] = pb.dsc[1];
  s[BS_TRS] = pb.dsc[2];
  s[BS_STEPS] += 1.0;
  s[BS_ITERS] += (double)pb.ctl[2];
  s[BS_LAST_ITERS] = (double)pb.ctl[2];
  if (ctl->stop == OP_STOP_ERR_E && err <= ctl->tol) *pb.frozen = 1;
  if (!isfinite(E)) *pb.frozen = 2;  // diverged: stop touching it, report on the host
}

}  // namespace
}  // namespace opevo

struct op_batch {
  std::vector<op_ctx *> ctx;
  int count = 0, max_ld = 0;
  cudaStream_t st = nullptr;
  int cg_iters = 12;
  int rows_per_item = 256;
  int gram_rows = 2048;
  int parity = 0;
  std::vector<void *> slot0, slot1;  // the two U buffers of each problem (U[0], U[1])
  // device
  BatchProb *d_prob = nullptr;
  RowItem *d_rows = nullptr;
  GramItem *d_gram = nullptr;
  TileItem *d_tiles = nullptr;
  int n_rows = 0, n_gram = 0, n_tiles = 0;
  double *d_rtol2 = nullptr, *d_stats = nullptr;
  int *d_frozen = nullptr;
  BatchCtl *d_ctl = nullptr;
  // host mirrors
  std::vector<double> h_stats;
  std::vector<int> h_frozen;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  size_t nodes[2] = {0, 0};  // kernels per graph (for the launch counter)
};

namespace {

void free_graphs(op_batch *b) {
  for (auto &e : b->exec)
    if (e) {
      cudaGraphExecDestroy(e);
      e = nullptr;
    }
}

void free_lists(op_batch *b) {
  for (void *p : {(void *)b->d_rows, (void *)b->d_gram, (void *)b->d_tiles})
    if (p) cudaFree(p);
  b->d_rows = nullptr;
  b->d_gram = nullptr;
  b->d_tiles = nullptr;
}

template <typename X> op_status upload(X **dst, const std::vector<X> &v, cudaStream_t st) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  OP_CUDA(cudaMalloc((void **)dst, std::max<size_t>(1, v.size()) * sizeof(X)));
  if (!v.empty())
    OP_CUDA(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, st));
  return OP_OK;
}

// Work lists and the per-problem item counts for the current granularity.
op_status build_lists(op_batch *b) {
  std::vector<RowItem> rows;
  std::vector<GramItem> gram;
  std::vector<TileItem> tiles;
  std::vector<BatchProb> probs(b->count);
  const size_t tile_bytes = gram_tc_tile_bytes();
  for (int i = 0; i < b->count; ++i) {
    op_ctx *c = b->ctx[i];
    BatchProb &pb = probs[i];
    memset(&pb, 0, sizeof(pb));
    pb.g = c->g;
    pb.p = c->p;
    pb.ld = c->ld;
    pb.shift = (float)(c->g.cdiag + c->sigma);
    pb.tau = c->tau;
    pb.Vt = (const float *)c->Vt;
    pb.U[0] = (float *)b->slot0[i];
    pb.U[1] = (float *)b->slot1[i];
    pb.W = (float *)c->W;
    pb.R = (float *)c->cgw.R;
    pb.P = (float *)c->cgw.P;
    pb.Q = (float *)c->cgw.Q;
    pb.part = c->cgw.part;
    pb.jacobi = c->cgw.jacobi ? 1 : 0;
    pb.state = c->cgw.state;
    pb.active = c->cgw.active;
    pb.ctl = c->cgw.ctl;
    pb.cg_rtol2 = b->d_rtol2 + i;
    pb.fixed_rtol = c->pb.cg_rtol > 0.0 ? c->pb.cg_rtol : 0.0;
    pb.C = c->C;
    pb.S = c->S;
    pb.D = c->D;
    pb.KU = c->KU;
    pb.KW = c->KW;
    pb.KT_hi = c->KT_hi;
    pb.KT_lo = c->KT_lo;
    pb.core_status = (int *)c->core_ws;
    double *M = (double *)((char *)c->core_ws + 256);
    const size_t m2 = (size_t)c->ld * c->ld;
    pb.core_M = M;
    pb.core_X = M + m2;
    pb.core_B = M + 2 * m2;
    pb.core_R = M + 3 * m2;
    pb.gram_part = (double *)c->gram_ws;
    pb.err = c->dev_err;
    pb.dsc = c->dsc;
    pb.frozen = b->d_frozen + i;
    // row items
    const long long n = c->n;
    const long long rpi = b->rows_per_item;
    int local = 0;
    for (long long r0 = 0; r0 < n; r0 += rpi, ++local) rows.push_back({i, local, r0, std::min(n, r0 + rpi)});
    // the CG partials of a row item take up to 3 ld doubles (the context's buffer
    // holds max_blocks x 2 ld)
    if (3 * local > 2 * c->cgw.max_blocks) {
      set_error("op_batch: problem %d needs %d row items (max %d): raise rows_per_item", i, local,
                2 * c->cgw.max_blocks / 3);
      return OP_ERR_ARG;
    }
    pb.n_row_items = local;
    // Gram chunks (all three products)
    const int nj = gram_tc_jobs_all(c->ld);
    long long gr = b->gram_rows;
    int ns = (int)((n + gr - 1) / gr);
    if ((size_t)ns * nj * tile_bytes > c->gram_bytes) {
      ns = (int)(c->gram_bytes / ((size_t)nj * tile_bytes));
      if (ns < 1) {
        set_error("op_batch: Gram scratch too small for problem %d", i);
        return OP_ERR_ARG;
      }
      gr = (n + ns - 1) / ns;
      gr = (gr + 31) / 32 * 32;
      ns = (int)((n + gr - 1) / gr);
    }
    pb.n_gram_splits = ns;
    pb.gram_jobs = nj;
    for (int sp = 0; sp < ns; ++sp)
      for (int j = 0; j < nj; ++j) gram.push_back({i, j, sp, sp * gr, std::min(n, (sp + 1) * gr)});
    // update tiles
    for (long long m0 = 0; m0 < n; m0 += 128)
      for (int n0 = 0; n0 < c->ld; n0 += 128) tiles.push_back({i, m0, n0});
  }
  free_lists(b);
  OP_TRY(upload(&b->d_prob, probs, b->st));
  OP_TRY(upload(&b->d_rows, rows, b->st));
  OP_TRY(upload(&b->d_gram, gram, b->st));
  OP_TRY(upload(&b->d_tiles, tiles, b->st));
  b->n_rows = (int)rows.size();
  b->n_gram = (int)gram.size();
  b->n_tiles = (int)tiles.size();
  OP_CUDA(cudaStreamSynchronize(b->st));
  return OP_OK;
}

// Enqueue one time step of every problem with U[parity] as the current block.
op_status enqueue_step(op_batch *b, int parity) {
  const int np = b->count, ml = b->max_ld;
  cudaStream_t st = b->st;
  opevo::k_b_set_tol<<<(np + 127) / 128, 128, 0, st>>>(b->d_prob, b->d_stats, b->d_ctl, np);
  count_launch();
  OP_TRY(launch_b_cg_init(b->d_prob, b->d_rows, b->n_rows, parity, st));
  OP_TRY(launch_b_fin_init(b->d_prob, np, ml, st));
  for (int k = 0; k < b->cg_iters; ++k)
    OP_TRY(launch_b_cg_iter(b->d_prob, b->d_rows, b->n_rows, np, ml, k, st));
  OP_TRY(launch_b_gram(b->d_prob, b->d_gram, b->n_gram, np, parity, st));
  OP_TRY(launch_b_core(b->d_prob, np, ml, st));
  OP_TRY(launch_b_update(b->d_prob, b->d_tiles, b->n_tiles, np, ml, parity, st));
  OP_TRY(launch_b_energy(b->d_prob, b->d_rows, b->n_rows, np, ml, parity ^ 1, st));
  opevo::k_b_step_end<<<(np + 127) / 128, 128, 0, st>>>(b->d_prob, b->d_stats, b->d_ctl, np);
  count_launch();
  OP_LAUNCH("batched step");
  return OP_OK;
}

op_status build_graphs(op_batch *b) {
  free_graphs(b);
  const long long before = launches_so_far();
  for (int q = 0; q < 2; ++q) {
    cudaGraph_t g = nullptr;
    OP_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    const op_status s = enqueue_step(b, q);
    const cudaError_t e = cudaStreamEndCapture(b->st, &g);
    if (s != OP_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    b->nodes[q] = nn;
    const cudaError_t e2 = cudaGraphInstantiate(&b->exec[q], g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return cuda_status(e2, "cudaGraphInstantiate");
  }
  // captured launches run only when a graph is replayed (counted there)
  count_launches(before - launches_so_far());
  return OP_OK;
}

// Copy the device records back and mirror them into the contexts.
op_status sync_back(op_batch *b) {
  OP_CUDA(cudaMemcpyAsync(b->h_stats.data(), b->d_stats, b->h_stats.size() * sizeof(double),
                          cudaMemcpyDeviceToHost, b->st));
  OP_CUDA(cudaMemcpyAsync(b->h_frozen.data(), b->d_frozen, b->count * sizeof(int),
                          cudaMemcpyDeviceToHost, b->st));
  int errs[1] = {0};
  OP_CUDA(cudaStreamSynchronize(b->st));
  for (int i = 0; i < b->count; ++i) {
    op_ctx *c = b->ctx[i];
    const double *s = &b->h_stats[(size_t)i * BS_FIELDS];
    c->stats.energy = s[BS_E];
    c->E = s[BS_E];
    c->stats.err_E = s[BS_ERR];
    c->stats.g_residual = s[BS_G2];
    c->stats.orth = s[BS_ORTH];
    c->stats.steps = (int)s[BS_STEPS];
    c->stats.cg_iters = (long long)s[BS_ITERS];
    c->stats.last_cg_iters = (int)s[BS_LAST_ITERS];
    c->g_rel = (s[BS_TRS] > 0 && s[BS_G2] > 0) ? sqrt(s[BS_G2] / s[BS_TRS]) : 0.0;
    int derr = 0;
    OP_CUDA(cudaMemcpy(&derr, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    errs[0] |= derr;
  }
  if (errs[0]) {
    set_error("op_batch: a tensor-core kernel timed out waiting for its MMAs");
    return OP_ERR_TIMEOUT;
  }
  for (int i = 0; i < b->count; ++i)
    if (b->h_frozen[i] == 2) {
      set_error("op_batch: problem %d diverged (non-finite energy)", i);
      return OP_ERR_DIVERGED;
    }
  return OP_OK;
}

// The contexts' U / U2 pointers follow the batch parity (U[parity] is current).
void point_contexts(op_batch *b) {
  for (int i = 0; i < b->count; ++i) {
    b->ctx[i]->U = b->parity ? b->slot1[i] : b->slot0[i];
    b->ctx[i]->U2 = b->parity ? b->slot0[i] : b->slot1[i];
  }
}

std::string signature(op_batch *b) {
  char buf[128];
  long long sn = 0, snp = 0;
  for (op_ctx *c : b->ctx) {
    sn += c->n;
    snp += c->n * c->ld;
  }
  snprintf(buf, sizeof(buf), "count=%d,sum_n=%lld,sum_nld=%lld,max_ld=%d,cg=%d", b->count, sn, snp,
           b->max_ld, b->cg_iters);
  return buf;
}

}  // namespace

extern "C" {

op_status op_batch_create(op_batch **out, op_ctx *const *ctxs, int count, int cg_iters,
                          void *stream) {
  if (!out || !ctxs || count < 1 || cg_iters < 1 || cg_iters > 200) {
    set_error("op_batch_create: bad arguments (need contexts, count >= 1 and 1 <= cg_iters <= "
              "200; got count=%d cg_iters=%d)", count, cg_iters);
    return OP_ERR_ARG;
  }
  *out = nullptr;
  op_batch *b = new op_batch();
  b->count = count;
  b->cg_iters = cg_iters;
  // the graphs are captured and replayed on a stream of the batch's own (capture is
  // not possible on the legacy default stream); pending work of the caller's stream
  // and of the contexts is finished first
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    set_error("op_batch_create: could not create the batch stream");
    return OP_ERR_CUDA;
  }
  for (int i = 0; i < count; ++i) {
    op_ctx *c = ctxs[i];
    if (!c || (c->prec != OP_FP32) || c->p > 128 || c->pb.flow != OP_FLOW_G) {
      set_error("op_batch_create: context %d must be an OP_FP32 context of the G flow with "
                "p <= 128", i);
      cudaStreamDestroy(b->st);
      delete b;
      return OP_ERR_ARG;
    }
    cudaStreamSynchronize(c->st);
    b->ctx.push_back(c);
    b->slot0.push_back(c->U);
    b->slot1.push_back(c->U2);
    b->max_ld = std::max(b->max_ld, c->ld);
  }
  b->h_stats.assign((size_t)count * BS_FIELDS, 0.0);
  b->h_frozen.assign(count, 0);
  op_status s = OP_OK;
  auto fail = [&](op_status e) {
    op_batch_destroy(b);
    return e;
  };
  if (cudaMalloc((void **)&b->d_rtol2, count * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void **)&b->d_stats, (size_t)count * BS_FIELDS * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void **)&b->d_frozen, count * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void **)&b->d_ctl, sizeof(BatchCtl)) != cudaSuccess) {
    set_error("op_batch_create: device allocation failed");
    return fail(OP_ERR_OOM);
  }
  // initial records: energy of U0, relative G-residual 1 (loose first CG tolerance)
  for (int i = 0; i < count; ++i) {
    double *s0 = &b->h_stats[(size_t)i * BS_FIELDS];
    s0[BS_E] = ctxs[i]->E;
    s0[BS_ERR] = fabs(ctxs[i]->E);
    s0[BS_G2] = 1.0;
    s0[BS_TRS] = 1.0;
    s0[BS_STEPS] = ctxs[i]->stats.steps;
    s0[BS_ITERS] = (double)ctxs[i]->stats.cg_iters;
  }
  BatchCtl ctl{-1, 0.0, 0.0};
  if (cudaMemcpy(b->d_stats, b->h_stats.data(), b->h_stats.size() * sizeof(double),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->d_frozen, 0, count * sizeof(int)) != cudaSuccess ||
      cudaMemcpy(b->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("op_batch_create: initial copies failed");
    return fail(OP_ERR_CUDA);
  }
  // the batch steps from U (slot 0, parity 0)
  if ((s = build_lists(b)) != OP_OK || (s = build_graphs(b)) != OP_OK) return fail(s);
  *out = b;
  return OP_OK;
}

op_status op_batch_set_tiles(op_batch *b, int rows_per_item, int gram_rows) {
  if (!b || rows_per_item < 32 || gram_rows < 256 || (gram_rows % 32)) {
    set_error("op_batch_set_tiles: rows_per_item >= 32, gram_rows >= 256 and a multiple of 32");
    return OP_ERR_ARG;
  }
  OP_CUDA(cudaStreamSynchronize(b->st));
  b->rows_per_item = rows_per_item;
  b->gram_rows = gram_rows;
  OP_TRY(build_lists(b));
  return build_graphs(b);
}

op_status op_batch_get_tiles(op_batch *b, int *rows_per_item, int *gram_rows) {
  if (!b || !rows_per_item || !gram_rows) {
    set_error("op_batch_get_tiles: null argument");
    return OP_ERR_ARG;
  }
  *rows_per_item = b->rows_per_item;
  *gram_rows = b->gram_rows;
  return OP_OK;
}

op_status op_batch_step(op_batch *b, int nsteps) {
  NvtxRange range("opevo batch step");
  if (!b || nsteps < 0) {
    set_error("op_batch_step: bad arguments");
    return OP_ERR_ARG;
  }
  for (int k = 0; k < nsteps; ++k) {
    OP_CUDA(cudaGraphLaunch(b->exec[b->parity], b->st));
    count_launches((long long)b->nodes[b->parity]);
    b->parity ^= 1;
  }
  point_contexts(b);
  return sync_back(b);
}

op_status op_batch_solve(op_batch *b, double tol, int max_steps, int stop, int check_every,
                         int *nconverged) {
  if (!b || max_steps < 0 || !(tol > 0.0) || (stop != OP_STOP_ERR_E && stop != OP_STOP_RESIDUAL)) {
    set_error("op_batch_solve: bad arguments");
    return OP_ERR_ARG;
  }
  if (check_every < 1) check_every = 10;
  BatchCtl ctl{stop, tol, stop == OP_STOP_RESIDUAL ? 0.1 * tol : 0.1 * sqrt(tol)};
  OP_CUDA(cudaMemcpyAsync(b->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, b->st));
  int done_steps = 0, conv = 0;
  // adaptive shift per problem (op_problem.adapt_every of its context): re-tuned at the
  // first check at or after each multiple of adapt_every steps; the descriptors the
  // replayed kernels read are updated in place.  A re-tune after which the energy has
  // risen by the next check is undone and adaptation stops for that problem.
  struct Guard {
    bool pending = false;
    double E = 0.0, sigma = 0.0, tau = 0.0;
    int next = 0;
  };
  std::vector<Guard> guard(b->count);
  for (int i = 0; i < b->count; ++i) {
    const int a = b->ctx[i]->pb.adapt_every;
    if (a > 0) guard[i].next = (b->ctx[i]->stats.steps / a + 1) * a;
  }
  auto push_shift = [&](int i) -> op_status {
    op_ctx *c = b->ctx[i];
    const float shift = (float)(c->g.cdiag + c->sigma);
    const double tau = c->tau;
    OP_CUDA(cudaMemcpyAsync(&b->d_prob[i].shift, &shift, sizeof(float), cudaMemcpyHostToDevice,
                            b->st));
    OP_CUDA(cudaMemcpyAsync(&b->d_prob[i].tau, &tau, sizeof(double), cudaMemcpyHostToDevice,
                            b->st));
    return OP_OK;
  };
  while (true) {
    for (int i = 0; i < b->count; ++i) {
      op_ctx *c = b->ctx[i];
      Guard &gd = guard[i];
      if (b->h_frozen[i] == 1 || c->pb.adapt_every <= 0) continue;
      if (gd.pending) {
        gd.pending = false;
        if (c->E > gd.E + 1e-12 * fabs(gd.E)) {
          c->sigma = gd.sigma;
          c->tau = gd.tau;
          c->stats.sigma = c->sigma;
          c->stats.tau = c->tau;
          c->adapt_off = 1;
          OP_TRY(push_shift(i));
        }
      }
      if (!c->adapt_off && c->stats.steps >= gd.next) {
        gd.next = c->stats.steps + c->pb.adapt_every;
        double ps = 0.0, pt = 0.0;
        OP_TRY(retune_shift(c, &ps, &pt));
        if (c->sigma != ps) {
          gd.pending = true;
          gd.E = c->E;
          gd.sigma = ps;
          gd.tau = pt;
          OP_TRY(push_shift(i));
        }
      }
    }
    // residual rule: evaluate the residual of every active problem on the host side
    conv = 0;
    for (int i = 0; i < b->count; ++i) {
      if (b->h_frozen[i] == 1) {
        ++conv;
        continue;
      }
      if (stop == OP_STOP_RESIDUAL) {
        double r = 0.0;
        OP_TRY(op_residual(b->ctx[i], &r));
        if (r <= tol) {
          b->h_frozen[i] = 1;
          ++conv;
        }
      }
    }
    if (stop == OP_STOP_RESIDUAL)
      OP_CUDA(cudaMemcpyAsync(b->d_frozen, b->h_frozen.data(), b->count * sizeof(int),
                              cudaMemcpyHostToDevice, b->st));
    if (conv == b->count || done_steps >= max_steps) break;
    const int n = std::min(check_every, max_steps - done_steps);
    OP_TRY(op_batch_step(b, n));
    done_steps += n;
  }
  BatchCtl off{-1, 0.0, 0.0};
  OP_CUDA(cudaMemcpyAsync(b->d_ctl, &off, sizeof(off), cudaMemcpyHostToDevice, b->st));
  OP_CUDA(cudaStreamSynchronize(b->st));
  if (nconverged) *nconverged = conv;
  if (conv < b->count) {
    set_error("op_batch_solve: %d of %d problems met the stop rule in %d steps", conv, b->count,
              max_steps);
    return OP_ERR_STATE;
  }
  return OP_OK;
}

op_status op_batch_unfreeze(op_batch *b) {
  if (!b) {
    set_error("null batch");
    return OP_ERR_ARG;
  }
  std::fill(b->h_frozen.begin(), b->h_frozen.end(), 0);
  OP_CUDA(cudaMemcpyAsync(b->d_frozen, b->h_frozen.data(), b->count * sizeof(int),
                          cudaMemcpyHostToDevice, b->st));
  OP_CUDA(cudaStreamSynchronize(b->st));
  return OP_OK;
}

op_status op_batch_autotune(op_batch *b, const char *cache_path, int steps_per_trial,
                            double *best_ms) {
  if (!b || steps_per_trial < 1) {
    set_error("op_batch_autotune: bad arguments");
    return OP_ERR_ARG;
  }
  const std::string sig = signature(b);
  // cached result for this batch shape?
  if (cache_path) {
    FILE *f = fopen(cache_path, "r");
    if (f) {
      char line[512];
      while (fgets(line, sizeof(line), f)) {
        char s[256];
        int r = 0, g = 0;
        double ms = 0.0;
        if (sscanf(line, " {\"signature\": \"%255[^\"]\", \"rows_per_item\": %d, \"gram_rows\": %d, "
                         "\"ms_per_step\": %lf}",
                   s, &r, &g, &ms) == 4 &&
            sig == s) {
          fclose(f);
          if (best_ms) *best_ms = ms;
          return op_batch_set_tiles(b, r, g);
        }
      }
      fclose(f);
    }
  }
  const int rows_c[] = {128, 256, 512, 1024};
  const int gram_c[] = {1024, 2048, 4096};
  double best = 1e300;
  int br = b->rows_per_item, bg = b->gram_rows;
  cudaEvent_t e0, e1;
  OP_CUDA(cudaEventCreate(&e0));
  OP_CUDA(cudaEventCreate(&e1));
  for (int r : rows_c)
    for (int g : gram_c) {
      if (op_batch_set_tiles(b, r, g) != OP_OK) continue;  // a granularity the scratch rejects
      OP_TRY(op_batch_step(b, 1));                       // warm
      OP_CUDA(cudaEventRecord(e0, b->st));
      for (int k = 0; k < steps_per_trial; ++k) {
        OP_CUDA(cudaGraphLaunch(b->exec[b->parity], b->st));
        count_launches((long long)b->nodes[b->parity]);
        b->parity ^= 1;
      }
      OP_CUDA(cudaEventRecord(e1, b->st));
      OP_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      OP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      point_contexts(b);
      OP_TRY(sync_back(b));
      const double per = ms / steps_per_trial;
      if (per < best) {
        best = per;
        br = r;
        bg = g;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  OP_TRY(op_batch_set_tiles(b, br, bg));
  if (best_ms) *best_ms = best;
  if (cache_path) {
    FILE *f = fopen(cache_path, "a");
    if (f) {
      fprintf(f, "{\"signature\": \"%s\", \"rows_per_item\": %d, \"gram_rows\": %d, "
                 "\"ms_per_step\": %.6f}\n",
              sig.c_str(), br, bg, best);
      fclose(f);
    }
  }
  return OP_OK;
}

op_status op_batch_stats(op_batch *b, int i, op_stats *st, int *frozen) {
  if (!b || i < 0 || i >= b->count || !st) {
    set_error("op_batch_stats: bad arguments");
    return OP_ERR_ARG;
  }
  *st = b->ctx[i]->stats;
  if (frozen) *frozen = b->h_frozen[i];
  return OP_OK;
}

void op_batch_destroy(op_batch *b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  free_graphs(b);
  free_lists(b);
  for (void *p : {(void *)b->d_prob, (void *)b->d_rtol2, (void *)b->d_stats, (void *)b->d_frozen,
                  (void *)b->d_ctl})
    if (p) cudaFree(p);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

}  // extern "C"
