// Row-sharded time steps: the grid split into slabs along its slowest axis (z in 3-D,
// y in 2-D), each slab in buffers of its own, the way each rank of a multi-GPU run
// would hold it.  The scheme needs no orthogonalisation of the block (§1, Theorem 4.1),
// so a step of a row-sharded run exchanges only
//   - one halo plane per slab face before every stencil apply (Step 1 is p independent
//     source problems on the stencil, §4.1; the energy needs one apply of U+), and
//   - sums over the slabs: the CG's per-column dot products (p values each) and, once
//     per step, the three p x p inner matrices <W,U>, <W,W>, <U,U> of Steps 2-3.
// Steps 2-3 (p x p) are computed once from the summed matrices (every rank would
// compute the same), and Step 4 is local to each slab.
//
// On one device the slabs are processed one after another on the context's stream:
// a halo exchange is a pair of device copies between neighbouring slabs' buffers, and
// a sum over slabs adds each slab's own total in slab order.  The per-slab work reuses
// the library's kernels (the stencil apply on the slab's local grid, the FP64 Gram and
// update on the slab's own rows); the CG's fused vector updates and their dot products
// are the small kernels below.
#include <math.h>

#include <chrono>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "ctx.cuh"

namespace opevo {
namespace {

constexpr int kShCols = 32;    // columns per CTA (a warp reads 256 contiguous bytes of a row)
constexpr int kShRows = 8;     // rows per CTA pass
constexpr int kShMaxBlk = 256; // row blocks per slab (partials per slab and column)

enum { SH_INIT = 0, SH_ALPHA = 1, SH_BETA = 2, SH_SUM = 3 };

// Column sums over the CTA's rows of acc[NC] into part[blockIdx.x][NC][ld].
template <int NC>
__device__ __forceinline__ void sh_block_sums(const double (&acc)[NC], int col, int ld,
                                              double *__restrict__ part) {
  __shared__ double sh[NC][kShRows][kShCols];
#pragma unroll
  for (int k = 0; k < NC; ++k) sh[k][threadIdx.y][threadIdx.x] = acc[k];
  __syncthreads();
  if (threadIdx.y == 0 && col < ld) {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < kShRows; ++r) s += sh[k][r][threadIdx.x];
      part[((size_t)blockIdx.x * NC + k) * ld + col] = s;
    }
  }
}

// CG start on one slab's own rows (pointers at the first own row; Q = (H + sigma) W):
// R = U - Q, Z = R / d (Jacobi, d = V + shift) or R, P = Z; partials R.Z, R.R, U.U.
__global__ void __launch_bounds__(kShCols *kShRows)
    k_sh_init(long long m, int ld, const double *__restrict__ U, const double *__restrict__ Q,
              const double *__restrict__ V, double shift, int jacobi, double *__restrict__ R,
              double *__restrict__ P, double *__restrict__ part) {
  const int col = blockIdx.y * kShCols + threadIdx.x;
  double acc[3] = {0.0, 0.0, 0.0};
  if (col < ld)
    for (long long i = (long long)blockIdx.x * kShRows + threadIdx.y; i < m;
         i += (long long)gridDim.x * kShRows) {
      const long long e = i * ld + col;
      const double u = U[e], r = u - Q[e];
      const double z = jacobi ? r / (V[i] + shift) : r;
      R[e] = r;
      P[e] = z;
      acc[0] += r * z;
      acc[1] += r * r;
      acc[2] += u * u;
    }
  sh_block_sums<3>(acc, col, ld, part);
}

// Partials of X.Y per column over one slab's own rows.
__global__ void __launch_bounds__(kShCols *kShRows)
    k_sh_dot(long long m, int ld, const double *__restrict__ X, const double *__restrict__ Y,
             double *__restrict__ part) {
  const int col = blockIdx.y * kShCols + threadIdx.x;
  double acc[1] = {0.0};
  if (col < ld)
    for (long long i = (long long)blockIdx.x * kShRows + threadIdx.y; i < m;
         i += (long long)gridDim.x * kShRows) {
      const long long e = i * ld + col;
      acc[0] += X[e] * Y[e];
    }
  sh_block_sums<1>(acc, col, ld, part);
}

// W += alpha P, R -= alpha Q (columns with alpha != 0), Z = R / d or R (Z stored in Q
// for Jacobi); partials R.Z, R.R of the new residual.
__global__ void __launch_bounds__(kShCols *kShRows)
    k_sh_axpy(long long m, int ld, const double *__restrict__ V, double shift, int jacobi,
              const double *__restrict__ alpha, const double *__restrict__ P,
              double *__restrict__ Q, double *__restrict__ W, double *__restrict__ R,
              double *__restrict__ part) {
  const int col = blockIdx.y * kShCols + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (col < ld) {
    const double a = alpha[col];
    for (long long i = (long long)blockIdx.x * kShRows + threadIdx.y; i < m;
         i += (long long)gridDim.x * kShRows) {
      const long long e = i * ld + col;
      double r = R[e];
      if (a != 0.0) {
        W[e] += a * P[e];
        r -= a * Q[e];
        R[e] = r;
      }
      const double z = jacobi ? r / (V[i] + shift) : r;
      if (jacobi) Q[e] = z;
      acc[0] += r * z;
      acc[1] += r * r;
    }
  }
  sh_block_sums<2>(acc, col, ld, part);
}

// P = Z + beta P on one slab's own rows.
__global__ void __launch_bounds__(kShCols *kShRows)
    k_sh_dir(long long m, int ld, const double *__restrict__ beta, const double *__restrict__ Z,
             double *__restrict__ P) {
  const int col = blockIdx.y * kShCols + threadIdx.x;
  if (col >= ld) return;
  const double b = beta[col];
  for (long long i = (long long)blockIdx.x * kShRows + threadIdx.y; i < m;
       i += (long long)gridDim.x * kShRows) {
    const long long e = i * ld + col;
    P[e] = Z[e] + b * P[e];
  }
}

// The sum over slabs of part[slab][blk][nc][ld] (each slab's total first, then the slab
// totals in slab order) and the CG's per-column scalars from it.  state: [5][ld] = rho,
// target, alpha, beta, rr.  *ctl counts the columns left active (INIT, BETA).
__global__ void k_sh_reduce(int mode, int nslab, int nblk, int nc, int ld,
                            const double *__restrict__ part, double rtol2,
                            double *__restrict__ state, int *__restrict__ active,
                            int *__restrict__ ctl, double *__restrict__ out) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ld) return;
  double tot[3] = {0.0, 0.0, 0.0};
  for (int s = 0; s < nslab; ++s) {
    double ss[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < nblk; ++b)
      for (int k = 0; k < nc; ++k) ss[k] += part[(((size_t)s * nblk + b) * nc + k) * ld + col];
    for (int k = 0; k < nc; ++k) tot[k] += ss[k];
  }
  double *rho = state, *target = state + ld, *alpha = state + 2 * ld, *beta = state + 3 * ld,
         *rr = state + 4 * ld;
  if (mode == SH_INIT) {
    rho[col] = tot[0];
    rr[col] = tot[1];
    target[col] = rtol2 * tot[2];
    const int act = tot[1] > target[col];
    active[col] = act;
    if (act) atomicAdd(ctl, 1);
  } else if (mode == SH_ALPHA) {
    const double pq = tot[0];
    alpha[col] = (active[col] && pq > 0.0) ? rho[col] / pq : 0.0;
  } else if (mode == SH_BETA) {
    const double rn = tot[0];
    beta[col] = (active[col] && rho[col] > 0.0) ? rn / rho[col] : 0.0;
    rho[col] = rn;
    rr[col] = tot[1];
    const int act = tot[1] > target[col];
    active[col] = act;
    if (act) atomicAdd(ctl, 1);
  } else {
    out[col] = tot[0];
  }
}

// out[e] = sum over slabs of in[slab][e], e < count, for the three matrices C, S, D
// (in: [nslab][3][count]).
__global__ void k_sh_sum_mats(int nslab, long long count, const double *__restrict__ in,
                              double *__restrict__ C, double *__restrict__ S,
                              double *__restrict__ D) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (e >= count) return;
  double s = 0.0;
  for (int q = 0; q < nslab; ++q) s += in[((size_t)q * 3 + k) * count + e];
  (k == 0 ? C : k == 1 ? S : D)[e] = s;
}

// *dst = sum of v[0 .. ld) in order.
__global__ void k_sh_total(int ld, const double *__restrict__ v, double *__restrict__ dst) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int j = 0; j < ld; ++j) s += v[j];
  *dst = s;
}

struct Slab {
  long long z0, own;  // first owned plane along the slowest axis, owned planes
  int lo, hi;         // halo planes below / above (a neighbour slab exists)
  Geom g;             // local grid: lo + own + hi planes
  long long off;      // first owned row of the local buffers
  long long rows;     // owned rows
  double *V = nullptr, *U = nullptr, *U2 = nullptr, *W = nullptr, *R = nullptr,
         *P = nullptr, *Q = nullptr;
};

struct Shard {
  op_ctx *c = nullptr;
  int ns = 0, nblk = 0, ld = 0;
  long long plane = 0;
  std::vector<Slab> s;
  double *part = nullptr, *state = nullptr, *mats = nullptr, *esum = nullptr, *edev = nullptr;
  int *active = nullptr, *ctl = nullptr;
  void *gws = nullptr;
  size_t gws_bytes = 0;
  int *hctl = nullptr;
  double *hsc = nullptr;
  std::vector<void *> allocs;
  op_shard_stats comm{};

  ~Shard() {
    if (c) cudaStreamSynchronize(c->st);
    for (void *p : allocs) cudaFree(p);
    if (hctl) cudaFreeHost(hctl);
    if (hsc) cudaFreeHost(hsc);
  }
  op_status alloc(void **p, size_t bytes) {
    *p = nullptr;
    const cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      *p = nullptr;
      return cuda_status(e, "cudaMalloc (sharded step)");
    }
    allocs.push_back(*p);
    return OP_OK;
  }
};

dim3 sh_grid(const Shard &h, long long rows) {
  long long nb = (rows + kShRows - 1) / kShRows;
  if (nb > h.nblk) nb = h.nblk;
  if (nb < 1) nb = 1;
  return dim3((unsigned)nb, (unsigned)((h.ld + kShCols - 1) / kShCols));
}

// Zero the partial rows a slab's launch does not write (slabs with fewer row blocks).
op_status sh_clear_part(Shard &h, int nc) {
  OP_CUDA(cudaMemsetAsync(h.part, 0, (size_t)h.ns * h.nblk * nc * h.ld * sizeof(double), h.c->st));
  return OP_OK;
}

double *slab_part(Shard &h, int s, int nc) { return h.part + (size_t)s * h.nblk * nc * h.ld; }

op_status sh_reduce(Shard &h, int mode, int nc, double rtol2, double *out = nullptr) {
  k_sh_reduce<<<(h.ld + 127) / 128, 128, 0, h.c->st>>>(mode, h.ns, h.nblk, nc, h.ld, h.part,
                                                        rtol2, h.state, h.active, h.ctl, out);
  count_launch();
  OP_LAUNCH("k_sh_reduce");
  h.comm.reductions += 1;
  h.comm.reduction_bytes += (long long)nc * h.ld * (long long)sizeof(double);
  return OP_OK;
}

// Halo exchange of block X (member pointer of Slab): each slab's boundary planes are
// copied into its neighbours' halo planes.
op_status sh_exchange(Shard &h, double *Slab::*X) {
  const size_t bytes = (size_t)h.plane * h.ld * sizeof(double);
  for (int q = 0; q + 1 < h.ns; ++q) {
    Slab &a = h.s[q], &b = h.s[q + 1];
    // a's upper halo <- b's first own plane; b's lower halo <- a's last own plane
    OP_CUDA(cudaMemcpyAsync(a.*X + (size_t)(a.lo + a.own) * h.plane * h.ld,
                            b.*X + (size_t)b.lo * h.plane * h.ld, bytes, cudaMemcpyDeviceToDevice,
                            h.c->st));
    OP_CUDA(cudaMemcpyAsync(b.*X, a.*X + (size_t)(a.lo + a.own - 1) * h.plane * h.ld, bytes,
                            cudaMemcpyDeviceToDevice, h.c->st));
    h.comm.halo_copies += 2;
    h.comm.halo_bytes += 2 * (long long)bytes;
  }
  return OP_OK;
}

op_status sh_setup(Shard &h, op_ctx *c, int nslab) {
  h.c = c;
  h.ns = nslab;
  h.ld = c->ld;
  const Geom &G = c->g;
  const bool d3 = G.dim == 3;
  const long long nslow = d3 ? G.nz : G.ny;
  h.plane = d3 ? (long long)G.nx * G.ny : (long long)G.nx;
  h.comm.slabs = nslab;
  h.s.resize(nslab);
  long long z = 0, max_rows = 0;
  for (int q = 0; q < nslab; ++q) {
    Slab &S = h.s[q];
    S.z0 = z;
    S.own = nslow / nslab + (q < nslow % nslab ? 1 : 0);
    z += S.own;
    S.lo = q > 0;
    S.hi = q + 1 < nslab;
    S.g = G;
    const long long planes = S.lo + S.own + S.hi;
    if (d3)
      S.g.nz = (int)planes;
    else
      S.g.ny = (int)planes;
    S.g.n = planes * h.plane;
    S.off = S.lo * h.plane;
    S.rows = S.own * h.plane;
    if (S.rows > max_rows) max_rows = S.rows;
  }
  const long long mb = (max_rows + kShRows - 1) / kShRows;
  h.nblk = (int)(mb < kShMaxBlk ? mb : kShMaxBlk);
  const size_t ld = (size_t)h.ld;
  for (Slab &S : h.s) {
    const size_t blk = (size_t)S.g.n * ld * sizeof(double);
    OP_TRY(h.alloc((void **)&S.V, (size_t)S.g.n * sizeof(double)));
    double **bufs[6] = {&S.U, &S.U2, &S.W, &S.R, &S.P, &S.Q};
    for (double **b : bufs) {
      OP_TRY(h.alloc((void **)b, blk));
      OP_CUDA(cudaMemsetAsync(*b, 0, blk, c->st));
    }
    // V, U and W of the slab's planes, halos included (rows are contiguous per plane)
    const size_t first = (size_t)(S.z0 - S.lo) * h.plane;
    OP_CUDA(cudaMemcpyAsync(S.V, (const double *)c->Vt + first, (size_t)S.g.n * sizeof(double),
                            cudaMemcpyDeviceToDevice, c->st));
    OP_CUDA(cudaMemcpyAsync(S.U, (const double *)c->U + first * ld, blk, cudaMemcpyDeviceToDevice,
                            c->st));
    OP_CUDA(cudaMemcpyAsync(S.W, (const double *)c->W + first * ld, blk, cudaMemcpyDeviceToDevice,
                            c->st));
  }
  OP_TRY(h.alloc((void **)&h.part, (size_t)nslab * h.nblk * 3 * ld * sizeof(double)));
  OP_TRY(h.alloc((void **)&h.state, 5 * ld * sizeof(double)));
  OP_TRY(h.alloc((void **)&h.mats, (size_t)nslab * 3 * ld * ld * sizeof(double)));
  OP_TRY(h.alloc((void **)&h.esum, ld * sizeof(double)));
  OP_TRY(h.alloc((void **)&h.edev, sizeof(double)));
  OP_TRY(h.alloc((void **)&h.active, ld * sizeof(int)));
  OP_TRY(h.alloc((void **)&h.ctl, sizeof(int)));
  for (const Slab &S : h.s) {
    const size_t b = c->tc_ws ? fp64tc_workspace_bytes(S.rows, h.ld)
                              : gram_workspace_bytes(S.rows, h.ld, (int)sizeof(double));
    if (b > h.gws_bytes) h.gws_bytes = b;
  }
  OP_TRY(h.alloc(&h.gws, h.gws_bytes));
  OP_CUDA(cudaMallocHost((void **)&h.hctl, 4 * sizeof(int)));
  OP_CUDA(cudaMallocHost((void **)&h.hsc, 8 * sizeof(double)));
  return OP_OK;
}

// Step 1 on the slabs: block CG (Jacobi-preconditioned when the context asks for it),
// warm-started from W, each column stopping when ||r_j|| <= rtol ||u_j||.
op_status sh_step1(Shard &h, double rtol, int max_iter, int *iters) {
  op_ctx *c = h.c;
  const int jac = c->pb.cg_precond == OP_PRECOND_JACOBI;
  const double shift = c->g.cdiag + c->sigma;
  const double rtol2 = rtol * rtol;
  OP_TRY(sh_exchange(h, &Slab::W));
  OP_TRY(sh_clear_part(h, 3));
  for (int q = 0; q < h.ns; ++q) {
    Slab &S = h.s[q];
    OP_TRY(launch_apply<double>(S.g, S.V, c->sigma, S.W, S.Q, h.ld, c->st));
    const size_t o = (size_t)S.off * h.ld;
    k_sh_init<<<sh_grid(h, S.rows), dim3(kShCols, kShRows), 0, c->st>>>(
        S.rows, h.ld, S.U + o, S.Q + o, S.V + S.off, shift, jac, S.R + o, S.P + o,
        slab_part(h, q, 3));
    count_launch();
    OP_LAUNCH("k_sh_init");
  }
  OP_CUDA(cudaMemsetAsync(h.ctl, 0, sizeof(int), c->st));
  OP_TRY(sh_reduce(h, SH_INIT, 3, rtol2));
  int k = 0;
  for (;;) {
    OP_CUDA(cudaMemcpyAsync(h.hctl, h.ctl, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    OP_CUDA(cudaStreamSynchronize(c->st));
    if (h.hctl[0] == 0 || k >= max_iter) break;
    // Q = (H + sigma) P with P's halo planes from the neighbours; alpha = rho / P.Q
    OP_TRY(sh_exchange(h, &Slab::P));
    OP_TRY(sh_clear_part(h, 1));
    for (int q = 0; q < h.ns; ++q) {
      Slab &S = h.s[q];
      OP_TRY(launch_apply<double>(S.g, S.V, c->sigma, S.P, S.Q, h.ld, c->st));
      const size_t o = (size_t)S.off * h.ld;
      k_sh_dot<<<sh_grid(h, S.rows), dim3(kShCols, kShRows), 0, c->st>>>(
          S.rows, h.ld, S.P + o, S.Q + o, slab_part(h, q, 1));
      count_launch();
      OP_LAUNCH("k_sh_dot");
    }
    OP_TRY(sh_reduce(h, SH_ALPHA, 1, rtol2));
    OP_TRY(sh_clear_part(h, 2));
    for (int q = 0; q < h.ns; ++q) {
      Slab &S = h.s[q];
      const size_t o = (size_t)S.off * h.ld;
      k_sh_axpy<<<sh_grid(h, S.rows), dim3(kShCols, kShRows), 0, c->st>>>(
          S.rows, h.ld, S.V + S.off, shift, jac, h.state + 2 * h.ld, S.P + o, S.Q + o, S.W + o,
          S.R + o, slab_part(h, q, 2));
      count_launch();
      OP_LAUNCH("k_sh_axpy");
    }
    OP_CUDA(cudaMemsetAsync(h.ctl, 0, sizeof(int), c->st));
    OP_TRY(sh_reduce(h, SH_BETA, 2, rtol2));
    for (int q = 0; q < h.ns; ++q) {
      Slab &S = h.s[q];
      const size_t o = (size_t)S.off * h.ld;
      k_sh_dir<<<sh_grid(h, S.rows), dim3(kShCols, kShRows), 0, c->st>>>(
          S.rows, h.ld, h.state + 3 * h.ld, (jac ? S.Q : S.R) + o, S.P + o);
      count_launch();
      OP_LAUNCH("k_sh_dir");
    }
    ++k;
  }
  *iters = k;
  return OP_OK;
}

op_status sh_step(Shard &h) {
  op_ctx *c = h.c;
  const int ld = h.ld;
  int iters = 0;
  OP_TRY(sh_step1(h, cg_rtol_for(c), cg_max_iter(c), &iters));
  // Steps 2-3: each slab's inner matrices over its own rows, summed over the slabs
  const size_t mat = (size_t)ld * ld;
  for (int q = 0; q < h.ns; ++q) {
    Slab &S = h.s[q];
    const size_t o = (size_t)S.off * ld;
    double *Cq = h.mats + (size_t)q * 3 * mat;
    if (c->tc_ws)
      OP_TRY(gram_fp64tc(S.rows, c->p, ld, S.U + o, S.W + o, Cq, Cq + mat, Cq + 2 * mat, h.gws,
                         h.gws_bytes, c->dev_err, c->st));
    else
      OP_TRY(gram<double>(S.rows, c->p, ld, S.U + o, S.W + o, Cq, Cq + mat, Cq + 2 * mat, h.gws,
                          h.gws_bytes, c->st));
  }
  k_sh_sum_mats<<<dim3((unsigned)((mat + 255) / 256), 3), 256, 0, c->st>>>(
      h.ns, (long long)mat, h.mats, c->C, c->S, c->D);
  count_launch();
  OP_LAUNCH("k_sh_sum_mats");
  h.comm.reductions += 1;
  h.comm.reduction_bytes += 3 * (long long)mat * (long long)sizeof(double);
  OP_TRY(launch_core_stats(c->p, ld, c->C, c->S, c->D, c->dsc, c->st));
  OP_TRY(core<double>(c->p, ld, c->tau, c->C, c->S, c->KU, c->KW, (double *)c->KU_t,
                      (double *)c->KW_t, c->core_ws, c->st, c->tc_ws ? c->tc_ws : c->core_tc_ws,
                      c->tc_ws ? c->tc_bytes : c->core_tc_bytes, c->dev_err));
  // Step 4 on each slab's own rows
  for (Slab &S : h.s) {
    const size_t o = (size_t)S.off * ld;
    if (c->tc_ws)
      OP_TRY(update_fp64tc(S.rows, ld, S.U + o, S.W + o, c->KU, c->KW, true, S.U2 + o, h.gws,
                           h.gws_bytes, c->dev_err, c->st));
    else
      OP_TRY(update<double>(S.rows, ld, S.U + o, S.W + o, c->KU, c->KW, S.U2 + o, c->st));
    double *t = S.U;
    S.U = S.U2;
    S.U2 = t;
  }
  // E(U+) = 1/2 sum_j u_j . H u_j with U+'s halo planes from the neighbours
  OP_TRY(sh_exchange(h, &Slab::U));
  OP_TRY(sh_clear_part(h, 1));
  for (int q = 0; q < h.ns; ++q) {
    Slab &S = h.s[q];
    OP_TRY(launch_apply<double>(S.g, S.V, 0.0, S.U, S.Q, ld, c->st));
    const size_t o = (size_t)S.off * ld;
    k_sh_dot<<<sh_grid(h, S.rows), dim3(kShCols, kShRows), 0, c->st>>>(S.rows, ld, S.U + o,
                                                                         S.Q + o,
                                                                         slab_part(h, q, 1));
    count_launch();
    OP_LAUNCH("k_sh_dot");
  }
  OP_TRY(sh_reduce(h, SH_SUM, 1, 0.0, h.esum));
  k_sh_total<<<1, 32, 0, c->st>>>(ld, h.esum, h.edev);
  count_launch();
  OP_LAUNCH("k_sh_total");
  OP_CUDA(cudaMemcpyAsync(h.hsc, c->dsc, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaMemcpyAsync(h.hsc + 4, h.edev, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaMemcpyAsync(h.hctl + 1, c->core_ws, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaMemcpyAsync(h.hctl + 2, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  OP_CUDA(cudaStreamSynchronize(c->st));
  if (h.hctl[2]) {
    set_error("a kernel gave up a bounded device wait (tensor-core MMAs or TMA copies)");
    return OP_ERR_TIMEOUT;
  }
  if (h.hctl[1]) {
    set_error("Step 2 factorisation broke down (zero or non-finite pivot)");
    return OP_ERR_NOTSPD;
  }
  const double Enew = 0.5 * h.hsc[4];
  if (!isfinite(Enew)) {
    set_error("non-finite energy after step %d", c->stats.steps + 1);
    return OP_ERR_DIVERGED;
  }
  c->stats.err_E = fabs(Enew - c->E) / fabs(c->E);
  c->E = Enew;
  c->stats.energy = Enew;
  c->stats.g_residual = h.hsc[0];
  c->stats.orth = h.hsc[1];
  c->g_rel = (h.hsc[2] > 0.0 && h.hsc[0] > 0.0) ? sqrt(h.hsc[0] / h.hsc[2]) : 0.0;
  c->stats.steps += 1;
  c->stats.last_cg_iters = iters;
  c->stats.cg_iters += iters;
  return OP_OK;
}

// The slabs' own rows of U and W back into the context's blocks.
op_status sh_gather(Shard &h) {
  op_ctx *c = h.c;
  const size_t ld = (size_t)h.ld;
  for (Slab &S : h.s) {
    const size_t bytes = (size_t)S.rows * ld * sizeof(double);
    const size_t dst = (size_t)S.z0 * h.plane * ld, src = (size_t)S.off * ld;
    OP_CUDA(cudaMemcpyAsync((double *)c->U + dst, S.U + src, bytes, cudaMemcpyDeviceToDevice,
                            c->st));
    OP_CUDA(cudaMemcpyAsync((double *)c->W + dst, S.W + src, bytes, cudaMemcpyDeviceToDevice,
                            c->st));
  }
  OP_CUDA(cudaStreamSynchronize(c->st));
  return OP_OK;
}

}  // namespace
}  // namespace opevo

extern "C" op_status op_step_sharded(op_ctx *c, int nslab, int nsteps, op_stats *st,
                                     op_shard_stats *comm) {
  if (!c) {
    set_error("op_step_sharded: null context");
    return OP_ERR_ARG;
  }
  if (c->prec != OP_FP64 || c->pb.flow != OP_FLOW_G) {
    set_error("op_step_sharded: needs an OP_FP64 context of the G flow");
    return OP_ERR_ARG;
  }
  const long long nslow = c->g.dim == 3 ? c->g.nz : c->g.ny;
  if (nslab < 1 || nslab > nslow || nsteps < 0) {
    set_error("op_step_sharded: need 1 <= nslab <= %lld planes and nsteps >= 0 (nslab=%d "
              "nsteps=%d)", nslow, nslab, nsteps);
    return OP_ERR_ARG;
  }
  const auto t0 = std::chrono::steady_clock::now();
  // the carried Step-1 residual of op_step does not survive sharded steps
  c->rec_ok = false;
  {
    NvtxRange r("opevo sharded steps");
    Shard h;
    OP_TRY(sh_setup(h, c, nslab));
    // as with op_step, a step that fails after its update leaves the updated block
    op_status s = OP_OK;
    for (int k = 0; k < nsteps && s == OP_OK; ++k) s = sh_step(h);
    const op_status g = sh_gather(h);
    if (comm) *comm = h.comm;
    if (s != OP_OK) return s;
    OP_TRY(g);
  }
  c->stats.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                    .count();
  if (st) *st = c->stats;
  return OP_OK;
}
