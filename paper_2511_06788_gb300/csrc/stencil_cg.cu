// Step 1 of §4.1 (the p source problems (H + sigma) W = U) on the device:
// the 5/7-point stencil apply and the conjugate-gradient kernels.
//
// Layout: n x ld row-major blocks; one thread owns one 16-byte vector of one
// grid point's row (float4 / double2), so a warp reads whole rows with
// coalesced 16-byte loads; the six neighbours of a point are rows i +- 1,
// i +- nx, i +- nx*ny and are served by L1/L2 (the z-planes of a block of
// consecutive points stay resident in the 129 MB L2).
#include <stdio.h>

#include "common.cuh"
#include "kernels.cuh"

namespace opevo {

namespace {

template <typename T>
__device__ __forceinline__ void axpy_pack(Pack<T> &acc, const Pack<T> &x) {
#pragma unroll
  for (int k = 0; k < Pack<T>::N; ++k) acc.v[k] += x.v[k];
}

// (H + sigma) x at point i, columns col .. col+N-1.
// Vt: V in T; shift = cdiag + sigma in T, so the diagonal is Vt_i + shift.
template <typename T>
__device__ __forceinline__ Pack<T> stencil_at(const Geom &g, const T *__restrict__ Vt, T shift,
                                              const T *__restrict__ X, int ld, long long i,
                                              int col, Pack<T> *center) {
  const long long base = i * (long long)ld + col;
  Pack<T> xc = Pack<T>::load(X + base);
  const int ix = (int)(i % g.nx);
  const long long r = i / g.nx;
  const int iy = (int)(r % g.ny);
  const int iz = (int)(r / g.ny);
  Pack<T> sx = Pack<T>::zero(), sy = Pack<T>::zero(), sz = Pack<T>::zero();
  if (ix > 0) axpy_pack(sx, Pack<T>::load(X + base - ld));
  if (ix < g.nx - 1) axpy_pack(sx, Pack<T>::load(X + base + ld));
  const long long sty = (long long)g.nx * ld;
  if (iy > 0) axpy_pack(sy, Pack<T>::load(X + base - sty));
  if (iy < g.ny - 1) axpy_pack(sy, Pack<T>::load(X + base + sty));
  if (g.dim == 3) {
    const long long stz = (long long)g.nx * g.ny * ld;
    if (iz > 0) axpy_pack(sz, Pack<T>::load(X + base - stz));
    if (iz < g.nz - 1) axpy_pack(sz, Pack<T>::load(X + base + stz));
  }
  const T d = __ldg(Vt + i) + shift;
  const T cx = (T)g.c[0], cy = (T)g.c[1], cz = (T)g.c[2];
  Pack<T> y;
#pragma unroll
  for (int k = 0; k < Pack<T>::N; ++k)
    y.v[k] = d * xc.v[k] - cx * sx.v[k] - cy * sy.v[k] - cz * sz.v[k];
  if (center) *center = xc;
  return y;
}

// Column-wise block reduction of acc[ncomp][N] (per thread) into
// part[blockIdx.x][ncomp][ld]; the block covers vectors blockIdx.y*blockDim.x + tx.
template <typename T, int NCOMP>
__device__ __forceinline__ void block_colsum(double (&acc)[NCOMP][Pack<T>::N], int ld,
                                             double *__restrict__ part) {
  constexpr int N = Pack<T>::N;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int bx = blockDim.x;
  const int col0 = blockIdx.y * bx * N;
  double *dst = part + (long long)blockIdx.x * NCOMP * ld;
  if (blockDim.y == 1) {
#pragma unroll
    for (int c = 0; c < NCOMP; ++c)
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (col0 + tx * N + k < ld) dst[c * ld + col0 + tx * N + k] = acc[c][k];
    return;
  }
  // blockDim.x * blockDim.y <= 256 here, so the tile fits.
  __shared__ double red[256 * NCOMP * N];
  const int width = NCOMP * bx * N;
#pragma unroll
  for (int c = 0; c < NCOMP; ++c)
#pragma unroll
    for (int k = 0; k < N; ++k) red[ty * width + c * bx * N + tx * N + k] = acc[c][k];
  __syncthreads();
  const int t = ty * bx + tx;
  const int nthreads = bx * blockDim.y;
  for (int e = t; e < width; e += nthreads) {
    double s = 0.0;
    for (int y = 0; y < (int)blockDim.y; ++y) s += red[y * width + e];
    const int c = e / (bx * N), col = col0 + e % (bx * N);
    if (col < ld) dst[c * ld + col] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_apply(Geom g, const T *__restrict__ Vt, T shift,
                                               const T *__restrict__ X, T *__restrict__ Y, int ld) {
  const int col = (blockIdx.y * blockDim.x + threadIdx.x) * Pack<T>::N;
  if (col >= ld) return;
  for (long long i = blockIdx.x * (long long)blockDim.y + threadIdx.y; i < g.n;
       i += (long long)gridDim.x * blockDim.y) {
    Pack<T> y = stencil_at(g, Vt, shift, X, ld, i, col, (Pack<T> *)nullptr);
    y.store(Y + i * (long long)ld + col);
  }
}

// part[b][0][j] = sum x_j ((H+sigma) x)_j, part[b][1][j] = sum x_j^2.
template <typename T>
__global__ void __launch_bounds__(256) k_quad(Geom g, const T *__restrict__ Vt, T shift,
                                              const T *__restrict__ X, int ld,
                                              double *__restrict__ part) {
  constexpr int N = Pack<T>::N;
  const int col = (blockIdx.y * blockDim.x + threadIdx.x) * N;
  const long long i0 = (col < ld) ? blockIdx.x * (long long)blockDim.y + threadIdx.y : g.n;
  double acc[2][N] = {};
  for (long long i = i0; i < g.n;
       i += (long long)gridDim.x * blockDim.y) {
    Pack<T> xc;
    Pack<T> y = stencil_at(g, Vt, shift, X, ld, i, col, &xc);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      acc[0][k] += (double)xc.v[k] * (double)y.v[k];
      acc[1][k] += (double)xc.v[k] * (double)xc.v[k];
    }
  }
  block_colsum<T, 2>(acc, ld, part);
}

// R = U - (H+sigma) W; P = R; part[b][0] = ||R_j||^2, part[b][1] = ||U_j||^2.
template <typename T>
__global__ void __launch_bounds__(256) k_cg_init(Geom g, const T *__restrict__ Vt, T shift,
                                                 const T *__restrict__ U, const T *__restrict__ W,
                                                 T *__restrict__ R, T *__restrict__ P, int ld,
                                                 double *__restrict__ part) {
  constexpr int N = Pack<T>::N;
  const int col = (blockIdx.y * blockDim.x + threadIdx.x) * N;
  const long long i0 = (col < ld) ? blockIdx.x * (long long)blockDim.y + threadIdx.y : g.n;
  double acc[2][N] = {};
  for (long long i = i0; i < g.n;
       i += (long long)gridDim.x * blockDim.y) {
    Pack<T> aw = stencil_at(g, Vt, shift, W, ld, i, col, (Pack<T> *)nullptr);
    const long long o = i * (long long)ld + col;
    Pack<T> u = Pack<T>::load(U + o);
    Pack<T> r;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      r.v[k] = u.v[k] - aw.v[k];
      acc[0][k] += (double)r.v[k] * (double)r.v[k];
      acc[1][k] += (double)u.v[k] * (double)u.v[k];
    }
    r.store(R + o);
    r.store(P + o);
  }
  block_colsum<T, 2>(acc, ld, part);
}

// Q = (H+sigma) P; part[b][0][j] = P_j . Q_j.
template <typename T>
__global__ void __launch_bounds__(256) k_cg_apply(Geom g, const T *__restrict__ Vt, T shift,
                                                  const T *__restrict__ P, T *__restrict__ Q,
                                                  int ld, double *__restrict__ part) {
  constexpr int N = Pack<T>::N;
  const int col = (blockIdx.y * blockDim.x + threadIdx.x) * N;
  const long long i0 = (col < ld) ? blockIdx.x * (long long)blockDim.y + threadIdx.y : g.n;
  double acc[1][N] = {};
  for (long long i = i0; i < g.n;
       i += (long long)gridDim.x * blockDim.y) {
    Pack<T> pc;
    Pack<T> q = stencil_at(g, Vt, shift, P, ld, i, col, &pc);
#pragma unroll
    for (int k = 0; k < N; ++k) acc[0][k] += (double)pc.v[k] * (double)q.v[k];
    q.store(Q + i * (long long)ld + col);
  }
  block_colsum<T, 1>(acc, ld, part);
}

// W += alpha P; R -= alpha Q; part[b][0][j] = ||R_j||^2.
template <typename T>
__global__ void __launch_bounds__(256) k_cg_axpy(long long n, int ld, T *__restrict__ W,
                                                 T *__restrict__ R, const T *__restrict__ P,
                                                 const T *__restrict__ Q,
                                                 const double *__restrict__ alpha,
                                                 double *__restrict__ part) {
  constexpr int N = Pack<T>::N;
  const int col = (blockIdx.y * blockDim.x + threadIdx.x) * N;
  const long long i0 = (col < ld) ? blockIdx.x * (long long)blockDim.y + threadIdx.y : n;
  T a[N];
#pragma unroll
  for (int k = 0; k < N; ++k) a[k] = (col < ld) ? (T)alpha[col + k] : T(0);
  double acc[1][N] = {};
  for (long long i = i0; i < n;
       i += (long long)gridDim.x * blockDim.y) {
    const long long o = i * (long long)ld + col;
    Pack<T> w = Pack<T>::load_rw(W + o), r = Pack<T>::load_rw(R + o);
    Pack<T> p = Pack<T>::load(P + o), q = Pack<T>::load(Q + o);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      w.v[k] += a[k] * p.v[k];
      r.v[k] -= a[k] * q.v[k];
      acc[0][k] += (double)r.v[k] * (double)r.v[k];
    }
    w.store(W + o);
    r.store(R + o);
  }
  block_colsum<T, 1>(acc, ld, part);
}

// P = R + beta P.
template <typename T>
__global__ void __launch_bounds__(256) k_cg_dir(long long n, int ld, const T *__restrict__ R,
                                                T *__restrict__ P,
                                                const double *__restrict__ beta) {
  constexpr int N = Pack<T>::N;
  const int col = (blockIdx.y * blockDim.x + threadIdx.x) * N;
  if (col >= ld) return;
  T b[N];
#pragma unroll
  for (int k = 0; k < N; ++k) b[k] = (T)beta[col + k];
  for (long long i = blockIdx.x * (long long)blockDim.y + threadIdx.y; i < n;
       i += (long long)gridDim.x * blockDim.y) {
    const long long o = i * (long long)ld + col;
    Pack<T> r = Pack<T>::load(R + o), pp = Pack<T>::load_rw(P + o);
#pragma unroll
    for (int k = 0; k < Pack<T>::N; ++k) pp.v[k] = r.v[k] + b[k] * pp.v[k];
    pp.store(P + o);
  }
}

// ---- single-block finalisers (deterministic reduction over blocks) -------------
__device__ __forceinline__ double sum_blocks(const double *part, int nblk, int stride, int e) {
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long long)b * stride + e];
  return s;
}

// state rows: 0 rr, 1 target, 2 alpha, 3 beta, 4 bnorm2
__global__ void k_cg_fin_init(const double *part, int nblk, int ld, int p, double rtol2,
                              double *state, int *active, int *nactive) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < ld; j += blockDim.x) {
    const double rr = sum_blocks(part, nblk, 2 * ld, j);
    const double bb = sum_blocks(part, nblk, 2 * ld, ld + j);
    state[0 * ld + j] = rr;
    state[1 * ld + j] = rtol2 * bb;
    state[2 * ld + j] = 0.0;
    state[3 * ld + j] = 0.0;
    state[4 * ld + j] = bb;
    const int a = (j < p) && (rr > rtol2 * bb) && (bb > 0.0);
    active[j] = a;
    if (a) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *nactive = cnt;
}

__global__ void k_cg_fin_alpha(const double *part, int nblk, int ld, double *state,
                               const int *active) {
  for (int j = threadIdx.x; j < ld; j += blockDim.x) {
    const double pq = sum_blocks(part, nblk, ld, j);
    const double rr = state[j];
    state[2 * ld + j] = (active[j] && pq > 0.0) ? rr / pq : 0.0;
  }
}

__global__ void k_cg_fin_beta(const double *part, int nblk, int ld, double *state, int *active,
                              int *nactive) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < ld; j += blockDim.x) {
    const double rrn = sum_blocks(part, nblk, ld, j);
    const double rr = state[j];
    int a = active[j];
    state[3 * ld + j] = (a && rr > 0.0) ? rrn / rr : 0.0;
    if (a) {
      state[j] = rrn;
      a = rrn > state[ld + j];
      active[j] = a;
    }
    if (a) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *nactive = cnt;
}

__global__ void k_colsum(const double *part, int nblk, int width, double *out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < width; e += gridDim.x * blockDim.x)
    out[e] = sum_blocks(part, nblk, width, e);
}

// part[b][0][j] = sum_i X_ij^2.
template <typename T>
__global__ void __launch_bounds__(256) k_sumsq(long long n, int ld, const T *__restrict__ X,
                                               double *__restrict__ part) {
  constexpr int N = Pack<T>::N;
  const int col = (blockIdx.y * blockDim.x + threadIdx.x) * N;
  const long long i0 = (col < ld) ? blockIdx.x * (long long)blockDim.y + threadIdx.y : n;
  double acc[1][N] = {};
  for (long long i = i0; i < n; i += (long long)gridDim.x * blockDim.y) {
    Pack<T> x = Pack<T>::load(X + i * (long long)ld + col);
#pragma unroll
    for (int k = 0; k < N; ++k) acc[0][k] += (double)x.v[k] * (double)x.v[k];
  }
  block_colsum<T, 1>(acc, ld, part);
}

// out[c] = sum_j sum_b part[b][c][j], c < ncomp (one CTA, fixed order).
__global__ void k_fin_total(const double *__restrict__ part, int nblk, int ncomp, int ld,
                            double *__restrict__ out) {
  __shared__ double sh[256];
  for (int c = 0; c < ncomp; ++c) {
    double s = 0.0;
    for (int j = threadIdx.x; j < ld; j += blockDim.x)
      for (int b = 0; b < nblk; ++b) s += part[((long long)b * ncomp + c) * ld + j];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0];
    __syncthreads();
  }
}

template <typename T>
__global__ void k_pad_copy(long long n, int p, int ld, const double *__restrict__ src,
                           T *__restrict__ dst) {
  const long long total = n * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / ld;
    const int j = (int)(e % ld);
    dst[e] = (j < p) ? (T)src[i * p + j] : T(0);
  }
}

template <typename T>
__global__ void k_unpad_copy(long long n, int p, int ld, const T *__restrict__ src,
                             double *__restrict__ dst) {
  const long long total = n * p;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / p;
    const int j = (int)(e % p);
    dst[e] = (double)src[i * ld + j];
  }
}

int grid_blocks(long long n, int rows) {
  long long want = (n + rows - 1) / rows;
  long long cap = (long long)kNumSMs * 8;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T>
op_status launch_apply(const Geom &g, const T *Vt, double sigma, const T *X, T *Y, int ld,
                       cudaStream_t st) {
  RowShape s = row_shape(ld, Pack<T>::N);
  k_apply<T><<<dim3(grid_blocks(g.n, s.rows), s.gy), s.block, 0, st>>>(
      g, Vt, (T)(g.cdiag + sigma), X, Y, ld); count_launch();
  OP_LAUNCH("k_apply");
  return OP_OK;
}

template <typename T>
op_status launch_quad(const Geom &g, const T *Vt, double sigma, const T *X, int ld, double *part,
                      double *out, cudaStream_t st) {
  RowShape s = row_shape(ld, Pack<T>::N);
  const int nb = grid_blocks(g.n, s.rows);
  k_quad<T><<<dim3(nb, s.gy), s.block, 0, st>>>(g, Vt, (T)(g.cdiag + sigma), X, ld, part); count_launch();
  k_fin_total<<<1, 256, 0, st>>>(part, nb, 2, ld, out); count_launch();
  OP_LAUNCH("k_quad");
  return OP_OK;
}

template <typename T>
op_status launch_sumsq(long long n, int ld, const T *X, double *part, double *out,
                       cudaStream_t st) {
  RowShape s = row_shape(ld, Pack<T>::N);
  const int nb = grid_blocks(n, s.rows);
  k_sumsq<T><<<dim3(nb, s.gy), s.block, 0, st>>>(n, ld, X, part); count_launch();
  k_fin_total<<<1, 256, 0, st>>>(part, nb, 1, ld, out); count_launch();
  OP_LAUNCH("k_sumsq");
  return OP_OK;
}

op_status launch_colsum(const double *part, int nblk, int ncomp, int ld, double *out,
                        cudaStream_t st) {
  const int width = ncomp * ld;
  k_colsum<<<(width + 255) / 256, 256, 0, st>>>(part, nblk, width, out); count_launch();
  OP_LAUNCH("k_colsum");
  return OP_OK;
}

size_t cg_workspace_bytes(long long n, int ld, int elem) {
  size_t blk = (size_t)n * ld * elem;
  blk = (blk + 255) / 256 * 256;
  size_t part = (size_t)kNumSMs * 8 * 2 * ld * sizeof(double);
  size_t state = (size_t)6 * ld * sizeof(double) + (size_t)ld * sizeof(int) + 256;
  return 3 * blk + part + state + 1024;
}

void cg_carve(void *ws, long long n, int ld, int elem, CGWork *w) {
  char *p = (char *)ws;
  size_t blk = (size_t)n * ld * elem;
  blk = (blk + 255) / 256 * 256;
  w->R = p;
  p += blk;
  w->P = p;
  p += blk;
  w->Q = p;
  p += blk;
  w->max_blocks = kNumSMs * 8;
  w->part = (double *)p;
  p += (size_t)w->max_blocks * 2 * ld * sizeof(double);
  w->state = (double *)p;
  p += (size_t)6 * ld * sizeof(double);
  w->active = (int *)p;
  p += ((size_t)ld * sizeof(int) + 255) / 256 * 256;
  w->nactive = (int *)p;
}

template <typename T>
op_status cg_solve(const Geom &g, const T *Vt, double sigma, const T *U, T *W, int p, int ld,
                   double rtol, int max_iter, CGWork &w, int *iters, cudaStream_t st) {
  RowShape s = row_shape(ld, Pack<T>::N);
  const int nb = grid_blocks(g.n, s.rows);
  const int fin_threads = ld < 1024 ? ld : 1024;
  T *R = (T *)w.R, *P = (T *)w.P, *Q = (T *)w.Q;
  double *alpha = w.state + 2 * ld, *beta = w.state + 3 * ld;
  const T sg = (T)(g.cdiag + sigma);

  prof_begin(w.prof, PK_CG_INIT, st);
  k_cg_init<T><<<dim3(nb, s.gy), s.block, 0, st>>>(g, Vt, sg, U, W, R, P, ld, w.part); count_launch();
  k_cg_fin_init<<<1, fin_threads, 0, st>>>(w.part, nb, ld, p, rtol * rtol, w.state, w.active,
                                           w.nactive); count_launch();
  prof_end(w.prof, st);
  OP_LAUNCH("k_cg_init");
  OP_CUDA(cudaMemcpyAsync(w.nactive_host, w.nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
  OP_CUDA(cudaStreamSynchronize(st));
  prof_harvest(w.prof);
  int it = 0;
  while (*w.nactive_host > 0 && it < max_iter) {
    prof_begin(w.prof, PK_CG_APPLY, st);
    k_cg_apply<T><<<dim3(nb, s.gy), s.block, 0, st>>>(g, Vt, sg, P, Q, ld, w.part); count_launch();
    prof_end(w.prof, st);
    prof_begin(w.prof, PK_CG_FIN, st);
    k_cg_fin_alpha<<<1, fin_threads, 0, st>>>(w.part, nb, ld, w.state, w.active); count_launch();
    prof_end(w.prof, st);
    prof_begin(w.prof, PK_CG_AXPY, st);
    k_cg_axpy<T><<<dim3(nb, s.gy), s.block, 0, st>>>(g.n, ld, W, R, P, Q, alpha, w.part); count_launch();
    prof_end(w.prof, st);
    prof_begin(w.prof, PK_CG_FIN, st);
    k_cg_fin_beta<<<1, fin_threads, 0, st>>>(w.part, nb, ld, w.state, w.active, w.nactive); count_launch();
    prof_end(w.prof, st);
    prof_begin(w.prof, PK_CG_DIR, st);
    k_cg_dir<T><<<dim3(nb, s.gy), s.block, 0, st>>>(g.n, ld, R, P, beta); count_launch();
    prof_end(w.prof, st);
    OP_LAUNCH("cg iteration");
    ++it;
    OP_CUDA(cudaMemcpyAsync(w.nactive_host, w.nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
    OP_CUDA(cudaStreamSynchronize(st));
    prof_harvest(w.prof);
  }
  *iters = it;
  return OP_OK;
}

template <typename T>
op_status launch_pad_copy(long long n, int p, int ld, const double *src, T *dst, cudaStream_t st) {
  k_pad_copy<T><<<kNumSMs * 8, 256, 0, st>>>(n, p, ld, src, dst); count_launch();
  OP_LAUNCH("k_pad_copy");
  return OP_OK;
}

template <typename T>
op_status launch_unpad_copy(long long n, int p, int ld, const T *src, double *dst,
                            cudaStream_t st) {
  k_unpad_copy<T><<<kNumSMs * 8, 256, 0, st>>>(n, p, ld, src, dst); count_launch();
  OP_LAUNCH("k_unpad_copy");
  return OP_OK;
}

// ---------------------------------------------------------------------------
// Event profiler
// ---------------------------------------------------------------------------
const char *prof_name(int kind) {
  static const char *names[PK_COUNT] = {"cg_init", "cg_apply", "cg_axpy", "cg_dir",
                                        "cg_finalize", "gram", "core", "update", "energy",
                                        "residual"};
  return (kind >= 0 && kind < PK_COUNT) ? names[kind] : "";
}

op_status prof_enable(Prof *p, bool on) {
  if (on && !p->created) {
    for (int i = 0; i < 2 * Prof::kMax; ++i) OP_CUDA(cudaEventCreate(&p->ev[i]));
    p->created = true;
  }
  p->on = on;
  p->n = 0;
  for (int k = 0; k < PK_COUNT; ++k) {
    p->ms[k] = 0.0;
    p->cnt[k] = 0;
  }
  return OP_OK;
}

void prof_destroy(Prof *p) {
  if (p->created)
    for (int i = 0; i < 2 * Prof::kMax; ++i) cudaEventDestroy(p->ev[i]);
  p->created = false;
  p->on = false;
}

void prof_begin(Prof *p, int kind, cudaStream_t st) {
  if (!p || !p->on || p->n >= Prof::kMax) return;
  p->kind[p->n] = kind;
  cudaEventRecord(p->ev[2 * p->n], st);
}

void prof_end(Prof *p, cudaStream_t st) {
  if (!p || !p->on || p->n >= Prof::kMax) return;
  cudaEventRecord(p->ev[2 * p->n + 1], st);
  p->n++;
}

void prof_harvest(Prof *p) {
  if (!p || !p->on) return;
  for (int i = 0; i < p->n; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev[2 * i], p->ev[2 * i + 1]) == cudaSuccess) {
      p->ms[p->kind[i]] += ms;
      p->cnt[p->kind[i]] += 1;
    }
  }
  p->n = 0;
}

#define OPEVO_INST(T)                                                                          \
  template op_status launch_sumsq<T>(long long, int, const T *, double *, double *,           \
                                     cudaStream_t);                                            \
  template op_status launch_apply<T>(const Geom &, const T *, double, const T *, T *, int,    \
                                     cudaStream_t);                                            \
  template op_status launch_quad<T>(const Geom &, const T *, double, const T *, int, double *, \
                                    double *, cudaStream_t);                                   \
  template op_status cg_solve<T>(const Geom &, const T *, double, const T *, T *, int, int,   \
                                 double, int, CGWork &, int *, cudaStream_t);                  \
  template op_status launch_pad_copy<T>(long long, int, int, const double *, T *,             \
                                        cudaStream_t);                                         \
  template op_status launch_unpad_copy<T>(long long, int, int, const T *, double *,           \
                                          cudaStream_t);
OPEVO_INST(float)
OPEVO_INST(double)
#undef OPEVO_INST

}  // namespace opevo
