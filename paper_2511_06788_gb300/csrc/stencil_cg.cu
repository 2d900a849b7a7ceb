// Step 1 of §4.1 (the p source problems (H + sigma) W = U) on the device:
// the 5/7-point stencil apply and the conjugate-gradient kernels.
//
// Layout: n x ld row-major blocks; one thread owns one 16-byte vector of one
// grid point's row (float4 / double2), so a warp reads whole rows with
// coalesced 16-byte loads; the six neighbours of a point are rows i +- 1,
// i +- nx, i +- nx*ny and are served by L1/L2 (the planes around the points a
// wave of CTAs works on stay resident in the 129 MB L2).
//
// Per-column dot products are accumulated per thread in the block type T and
// combined across threads and CTAs in FP64 (per-element FP64 work would make
// the FP32 kernels FP64-pipe bound on GB300).  Partial sums per CTA are
// reduced by one warp per column in a fixed order (deterministic).
//
// CG control lives on the device: the finalisers compute alpha, beta and the
// number of still-active columns; every kernel of an iteration returns at once
// when the previous iteration left no active column, so the host can queue
// several iterations between convergence checks.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace opevo {

namespace {

template <typename T>
__device__ __forceinline__ void add_pack(Pack<T> &acc, const Pack<T> &x) {
#pragma unroll
  for (int k = 0; k < Pack<T>::N; ++k) acc.v[k] += x.v[k];
}

// Grid coordinates of point i.
struct Coord {
  int ix, iy, iz;
};
__device__ __forceinline__ Coord coord_of(const Geom &g, long long i) {
  Coord c;
  const long long r = i / g.nx;
  c.ix = (int)(i - r * g.nx);
  c.iy = (int)(r % g.ny);
  c.iz = (int)(r / g.ny);
  return c;
}

// y = d x_c - cx sx - cy sy - cz sz for the neighbour sums s*.
template <typename T>
__device__ __forceinline__ Pack<T> combine(const Geom &g, T d, const Pack<T> &xc, const Pack<T> &sx,
                                           const Pack<T> &sy, const Pack<T> &sz) {
  const T cx = (T)g.c[0], cy = (T)g.c[1], cz = (T)g.c[2];
  Pack<T> y;
#pragma unroll
  for (int k = 0; k < Pack<T>::N; ++k)
    y.v[k] = d * xc.v[k] - cx * sx.v[k] - cy * sy.v[k] - cz * sz.v[k];
  return y;
}

// (H + sigma) x at point i, columns col .. col+N-1.  Vt: V in T; shift =
// cdiag + sigma in T, so the diagonal is Vt_i + shift.
template <typename T>
__device__ __forceinline__ Pack<T> stencil_at(const Geom &g, const T *__restrict__ Vt, T shift,
                                              const T *__restrict__ X, int ld, long long i,
                                              int col, Pack<T> *center) {
  const long long base = i * (long long)ld + col;
  const Coord c = coord_of(g, i);
  Pack<T> xc = Pack<T>::load(X + base);
  // each axis: one addition of the two neighbours (a missing neighbour reads as zero),
  // so the apply costs 3 additions and 4 multiply-adds per element
  const Pack<T> z = Pack<T>::zero();
  Pack<T> sx = c.ix > 0 ? Pack<T>::load(X + base - ld) : z;
  add_pack(sx, c.ix < g.nx - 1 ? Pack<T>::load(X + base + ld) : z);
  const long long sty = (long long)g.nx * ld;
  Pack<T> sy = c.iy > 0 ? Pack<T>::load(X + base - sty) : z;
  add_pack(sy, c.iy < g.ny - 1 ? Pack<T>::load(X + base + sty) : z);
  Pack<T> sz = z;
  if (g.dim == 3) {
    const long long stz = (long long)g.nx * g.ny * ld;
    sz = c.iz > 0 ? Pack<T>::load(X + base - stz) : z;
    add_pack(sz, c.iz < g.nz - 1 ? Pack<T>::load(X + base + stz) : z);
  }
  if (center) *center = xc;
  return combine(g, __ldg(Vt + i) + shift, xc, sx, sy, sz);
}

// Value of r + b p at a row offset (p omitted on the first CG iteration).
template <typename T, bool FIRST>
__device__ __forceinline__ Pack<T> dir_at(const T *__restrict__ R, const T *__restrict__ Po,
                                          const T (&b)[Pack<T>::N], long long off) {
  Pack<T> r = Pack<T>::load(R + off);
  if (!FIRST) {
    const Pack<T> q = Pack<T>::load(Po + off);
#pragma unroll
    for (int k = 0; k < Pack<T>::N; ++k) r.v[k] += b[k] * q.v[k];
  }
  return r;
}

// Column-wise block reduction of the per-thread partials acc[ncomp][N] (type T)
// into part[blockIdx.x][ncomp][ld] (FP64); the block covers the vectors
// blockIdx.y * blockDim.x + threadIdx.x of a row.
template <typename T, int NCOMP>
__device__ __forceinline__ void block_colsum(const T (&acc)[NCOMP][Pack<T>::N], int ld,
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
        if (col0 + tx * N + k < ld) dst[c * ld + col0 + tx * N + k] = (double)acc[c][k];
    return;
  }
  // blockDim.x * blockDim.y <= 256 here, so the tile fits.
  __shared__ double red[256 * NCOMP * N];
  const int width = NCOMP * bx * N;
#pragma unroll
  for (int c = 0; c < NCOMP; ++c)
#pragma unroll
    for (int k = 0; k < N; ++k) red[ty * width + c * bx * N + tx * N + k] = (double)acc[c][k];
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

#define ROW_PROLOGUE(NV)                                                            \
  constexpr int N = Pack<T>::N;                                                     \
  const int col = (blockIdx.y * blockDim.x + threadIdx.x) * N;                      \
  const long long i0 = (col < ld) ? blockIdx.x * (long long)blockDim.y + threadIdx.y : (NV); \
  const long long istep = (long long)gridDim.x * blockDim.y;

// ---------------------------------------------------------------------------
// Stencil kernels
// ---------------------------------------------------------------------------
// Y = scale (H + sigma) X (scale = 1 or -1).
template <typename T>
__global__ void __launch_bounds__(256) k_apply(Geom g, const T *__restrict__ Vt, T shift,
                                               const T *__restrict__ X, T *__restrict__ Y, int ld,
                                               T scale) {
  ROW_PROLOGUE(g.n)
  for (long long i = i0; i < g.n; i += istep) {
    Pack<T> y = stencil_at(g, Vt, shift, X, ld, i, col, (Pack<T> *)nullptr);
#pragma unroll
    for (int k = 0; k < N; ++k) y.v[k] *= scale;
    y.store(Y + i * (long long)ld + col);
  }
}

// part[b][0][j] = sum x_j ((H+sigma) x)_j, part[b][1][j] = sum x_j^2.
template <typename T>
__global__ void __launch_bounds__(256) k_quad(Geom g, const T *__restrict__ Vt, T shift,
                                              const T *__restrict__ X, int ld,
                                              double *__restrict__ part) {
  ROW_PROLOGUE(g.n)
  T acc[2][N] = {};
  for (long long i = i0; i < g.n; i += istep) {
    Pack<T> xc;
    Pack<T> y = stencil_at(g, Vt, shift, X, ld, i, col, &xc);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      acc[0][k] += xc.v[k] * y.v[k];
      acc[1][k] += xc.v[k] * xc.v[k];
    }
  }
  block_colsum<T, 2>(acc, ld, part);
}

// part[b][0][j] = sum_i X_ij^2.
template <typename T>
__global__ void __launch_bounds__(256) k_sumsq(long long n, int ld, const T *__restrict__ X,
                                               double *__restrict__ part) {
  ROW_PROLOGUE(n)
  T acc[1][N] = {};
  for (long long i = i0; i < n; i += istep) {
    Pack<T> x = Pack<T>::load(X + i * (long long)ld + col);
#pragma unroll
    for (int k = 0; k < N; ++k) acc[0][k] += x.v[k] * x.v[k];
  }
  block_colsum<T, 1>(acc, ld, part);
}

// ---------------------------------------------------------------------------
// CG kernels.  ctl[0], ctl[1]: active-column counts written by alternate
// iterations; ctl[2]: iterations done.  Iteration k reads nact_prev =
// ctl[(k+1)&1] (the count left by iteration k-1, or by the start-up for k = 0)
// and its beta finaliser accumulates into ctl[k&1].
// ---------------------------------------------------------------------------

// R = U - (H+sigma) W (and P = R when WRITE_P); part[b][0] = ||R_j||^2,
// part[b][1] = ||U_j||^2.  Resets the control words.
// R = U - (H+sigma) W (P = R as well when WRITE_P); part[b][.][j]: R_j.R_j, U_j.U_j.
// JACOBI (CG preconditioned with d = diag(H+sigma)): the residual buffer holds
// Z = R / d instead, and part[b][.][j] = R_j.Z_j, U_j.U_j, R_j.R_j.
template <typename T, bool WRITE_P, bool JACOBI>
__global__ void __launch_bounds__(256) k_cg_init(Geom g, const T *__restrict__ Vt, T shift,
                                                 const T *__restrict__ U, const T *__restrict__ W,
                                                 T *__restrict__ R, T *__restrict__ P, int ld,
                                                 double *__restrict__ part, int *ctl) {
  ROW_PROLOGUE(g.n)
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    ctl[1] = 0;
    ctl[2] = 0;
    ctl[3] = 0;
  }
  constexpr int NC = JACOBI ? 3 : 2;
  T acc[NC][N] = {};
  for (long long i = i0; i < g.n; i += istep) {
    Pack<T> aw = stencil_at(g, Vt, shift, W, ld, i, col, (Pack<T> *)nullptr);
    const long long o = i * (long long)ld + col;
    Pack<T> u = Pack<T>::load(U + o);
    Pack<T> r;
    if (JACOBI) {
      const T inv = T(1) / (__ldg(Vt + i) + shift);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T rk = u.v[k] - aw.v[k];
        r.v[k] = rk * inv;
        acc[0][k] += rk * r.v[k];
        acc[1][k] += u.v[k] * u.v[k];
        acc[NC - 1][k] += rk * rk;
      }
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        r.v[k] = u.v[k] - aw.v[k];
        acc[0][k] += r.v[k] * r.v[k];
        acc[1][k] += u.v[k] * u.v[k];
      }
    }
    r.store(R + o);
    if (WRITE_P) r.store(P + o);
  }
  block_colsum<T, NC>(acc, ld, part);
}

// R = R + U - Uprev (the residual of the block before an update, carried to the block
// after it with the same W: U - (H+sigma) W = (Uprev - (H+sigma) W) + (U - Uprev));
// part[b][.][j] = R_j.R_j, U_j.U_j.  Resets the control words as k_cg_init does.
template <typename T>
__global__ void __launch_bounds__(256) k_ref_recycle(long long n, const T *__restrict__ U,
                                                     const T *__restrict__ Uprev,
                                                     T *__restrict__ R, int ld,
                                                     double *__restrict__ part, int *ctl) {
  ROW_PROLOGUE(n)
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    ctl[1] = 0;
    ctl[2] = 0;
    ctl[3] = 0;
  }
  T acc[2][N] = {};
  for (long long i = i0; i < n; i += istep) {
    const long long o = i * (long long)ld + col;
    const Pack<T> u = Pack<T>::load(U + o), up = Pack<T>::load(Uprev + o);
    Pack<T> r = Pack<T>::load(R + o);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      r.v[k] += u.v[k] - up.v[k];
      acc[0][k] += r.v[k] * r.v[k];
      acc[1][k] += u.v[k] * u.v[k];
    }
    r.store(R + o);
  }
  block_colsum<T, 2>(acc, ld, part);
}

// ---- three-kernel iteration (FP64: no arithmetic is recomputed) -----------------
// Q = (H+sigma) P; part[b][0][j] = P_j . Q_j.
template <typename T>
__global__ void __launch_bounds__(256) k_cg_apply(Geom g, const T *__restrict__ Vt, T shift,
                                                  const T *__restrict__ P, T *__restrict__ Q,
                                                  int ld, const int *nact_prev,
                                                  double *__restrict__ part) {
  if (*nact_prev == 0) return;
  ROW_PROLOGUE(g.n)
  T acc[1][N] = {};
  for (long long i = i0; i < g.n; i += istep) {
    Pack<T> pc;
    Pack<T> q = stencil_at(g, Vt, shift, P, ld, i, col, &pc);
#pragma unroll
    for (int k = 0; k < N; ++k) acc[0][k] += pc.v[k] * q.v[k];
    q.store(Q + i * (long long)ld + col);
  }
  block_colsum<T, 1>(acc, ld, part);
}

// W += alpha P; R -= alpha Q; part[b][0][j] = ||R_j||^2.
// W += alpha P, R -= alpha Q; part[b][0][j] = R_j.R_j.  JACOBI: the residual buffer
// holds Z = R / d, Z -= alpha Q / d, part[b][.][j] = R_j.Z_j, R_j.R_j.
template <typename T, bool JACOBI>
__global__ void __launch_bounds__(256) k_cg_axpy(long long n, int ld, const T *__restrict__ Vt,
                                                 T shift, T *__restrict__ W, T *__restrict__ R,
                                                 const T *__restrict__ P, const T *__restrict__ Q,
                                                 const double *__restrict__ alpha,
                                                 const int *nact_prev, double *__restrict__ part) {
  if (*nact_prev == 0) return;
  ROW_PROLOGUE(n)
  T a[N];
#pragma unroll
  for (int k = 0; k < N; ++k) a[k] = (col < ld) ? (T)alpha[col + k] : T(0);
  constexpr int NC = JACOBI ? 2 : 1;
  T acc[NC][N] = {};
  for (long long i = i0; i < n; i += istep) {
    const long long o = i * (long long)ld + col;
    Pack<T> w = Pack<T>::load_rw(W + o), r = Pack<T>::load_rw(R + o);
    Pack<T> p = Pack<T>::load(P + o), q = Pack<T>::load(Q + o);
    if (JACOBI) {
      const T dg = __ldg(Vt + i) + shift, inv = T(1) / dg;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        w.v[k] += a[k] * p.v[k];
        r.v[k] -= a[k] * (q.v[k] * inv);
        const T rk = dg * r.v[k];
        acc[0][k] += rk * r.v[k];
        acc[1][k] += rk * rk;
      }
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        w.v[k] += a[k] * p.v[k];
        r.v[k] -= a[k] * q.v[k];
        acc[0][k] += r.v[k] * r.v[k];
      }
    }
    w.store(W + o);
    r.store(R + o);
  }
  block_colsum<T, NC>(acc, ld, part);
}

// P = R + beta P.
template <typename T>
__global__ void __launch_bounds__(256) k_cg_dir(long long n, int ld, const T *__restrict__ R,
                                                T *__restrict__ P, const double *__restrict__ beta,
                                                const int *nact_prev) {
  if (*nact_prev == 0) return;
  ROW_PROLOGUE(n)
  if (col >= ld) return;
  T b[N];
#pragma unroll
  for (int k = 0; k < N; ++k) b[k] = (T)beta[col + k];
  for (long long i = i0; i < n; i += istep) {
    const long long o = i * (long long)ld + col;
    Pack<T> r = Pack<T>::load(R + o), pp = Pack<T>::load_rw(P + o);
#pragma unroll
    for (int k = 0; k < N; ++k) pp.v[k] = r.v[k] + b[k] * pp.v[k];
    pp.store(P + o);
  }
}

// ---- two-kernel iteration (FP32: the stencil is recomputed instead of storing Q) ----
// Pn = R + beta Po (Pn = R on the first iteration); part[b][0][j] = Pn_j . (H+sigma) Pn_j.
// Reads R and Po (with the stencil halo), writes Pn.
template <typename T, bool FIRST>
__global__ void __launch_bounds__(256) k_cg_p(Geom g, const T *__restrict__ Vt, T shift,
                                              const T *__restrict__ R, const T *__restrict__ Po,
                                              T *__restrict__ Pn, int ld,
                                              const double *__restrict__ beta,
                                              const int *nact_prev, double *__restrict__ part) {
  if (*nact_prev == 0) return;
  ROW_PROLOGUE(g.n)
  T b[N];
#pragma unroll
  for (int k = 0; k < N; ++k) b[k] = (!FIRST && col < ld) ? (T)beta[col + k] : T(0);
  T acc[1][N] = {};
  const long long sty = (long long)g.nx * ld, stz = (long long)g.nx * g.ny * ld;
  for (long long i = i0; i < g.n; i += istep) {
    const long long base = i * (long long)ld + col;
    const Coord c = coord_of(g, i);
    const Pack<T> pc = dir_at<T, FIRST>(R, Po, b, base);
    Pack<T> sx = Pack<T>::zero(), sy = Pack<T>::zero(), sz = Pack<T>::zero();
    if (c.ix > 0) add_pack(sx, dir_at<T, FIRST>(R, Po, b, base - ld));
    if (c.ix < g.nx - 1) add_pack(sx, dir_at<T, FIRST>(R, Po, b, base + ld));
    if (c.iy > 0) add_pack(sy, dir_at<T, FIRST>(R, Po, b, base - sty));
    if (c.iy < g.ny - 1) add_pack(sy, dir_at<T, FIRST>(R, Po, b, base + sty));
    if (g.dim == 3) {
      if (c.iz > 0) add_pack(sz, dir_at<T, FIRST>(R, Po, b, base - stz));
      if (c.iz < g.nz - 1) add_pack(sz, dir_at<T, FIRST>(R, Po, b, base + stz));
    }
    const Pack<T> q = combine(g, __ldg(Vt + i) + shift, pc, sx, sy, sz);
#pragma unroll
    for (int k = 0; k < N; ++k) acc[0][k] += pc.v[k] * q.v[k];
    pc.store(Pn + base);
  }
  block_colsum<T, 1>(acc, ld, part);
}

// q = (H+sigma) Pn (recomputed); W += alpha Pn; R -= alpha q; part[b][0][j] = ||R_j||^2.
template <typename T, bool JACOBI>
__global__ void __launch_bounds__(256) k_cg_wr(Geom g, const T *__restrict__ Vt, T shift,
                                               T *__restrict__ W, T *__restrict__ R,
                                               const T *__restrict__ Pn, int ld,
                                               const double *__restrict__ alpha,
                                               const int *nact_prev, double *__restrict__ part) {
  if (*nact_prev == 0) return;
  ROW_PROLOGUE(g.n)
  T a[N];
#pragma unroll
  for (int k = 0; k < N; ++k) a[k] = (col < ld) ? (T)alpha[col + k] : T(0);
  constexpr int NC = JACOBI ? 2 : 1;
  T acc[NC][N] = {};
  for (long long i = i0; i < g.n; i += istep) {
    Pack<T> pc;
    const Pack<T> q = stencil_at(g, Vt, shift, Pn, ld, i, col, &pc);
    const long long o = i * (long long)ld + col;
    Pack<T> w = Pack<T>::load_rw(W + o), r = Pack<T>::load_rw(R + o);
    if (JACOBI) {  // r holds Z = R / d
      const T dg = __ldg(Vt + i) + shift, inv = T(1) / dg;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        w.v[k] += a[k] * pc.v[k];
        r.v[k] -= a[k] * (q.v[k] * inv);
        const T rk = dg * r.v[k];
        acc[0][k] += rk * r.v[k];
        acc[1][k] += rk * rk;
      }
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        w.v[k] += a[k] * pc.v[k];
        r.v[k] -= a[k] * q.v[k];
        acc[0][k] += r.v[k] * r.v[k];
      }
    }
    w.store(W + o);
    r.store(R + o);
  }
  block_colsum<T, NC>(acc, ld, part);
}

// ---- finalisers: one warp per column, lanes stride over the CTA partials ----------
__device__ __forceinline__ double warp_sum_blocks(const double *part, int nblk, int stride, int e) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(long long)b * stride + e];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// state rows: 0 rho (r.r, or r.z with the Jacobi preconditioner), 1 target, 2 alpha,
// 3 beta, 4 ||b||^2.  ncomp = 2: partials (r.r, b.b); 3: (r.z, b.b, r.r).  A column
// stays active while its unpreconditioned ||r||^2 is above rtol^2 ||b||^2.
__global__ void k_cg_fin_init(const double *part, int nblk, int ncomp, int ld, int p,
                              double rtol2, double *state, int *active, int *ctl) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= ld) return;
  const double rho = warp_sum_blocks(part, nblk, ncomp * ld, j);
  const double bb = warp_sum_blocks(part, nblk, ncomp * ld, ld + j);
  const double rr = ncomp == 3 ? warp_sum_blocks(part, nblk, ncomp * ld, 2 * ld + j) : rho;
  if ((threadIdx.x & 31) == 0) {
    state[0 * ld + j] = rho;
    state[1 * ld + j] = rtol2 * bb;
    state[2 * ld + j] = 0.0;
    state[3 * ld + j] = 0.0;
    state[4 * ld + j] = bb;
    const int a = (j < p) && (rr > rtol2 * bb) && (bb > 0.0);
    active[j] = a;
    if (a) atomicAdd(&ctl[1], 1);
  }
}

__global__ void k_cg_fin_alpha(const double *part, int nblk, int ld, double *state,
                               const int *active, const int *nact_prev, int *nact_next) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *nact_next = 0;
  if (*nact_prev == 0) return;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= ld) return;
  const double pq = warp_sum_blocks(part, nblk, ld, j);
  if ((threadIdx.x & 31) == 0) {
    const double rr = state[j];
    state[2 * ld + j] = (active[j] && pq > 0.0) ? rr / pq : 0.0;
  }
}

// ncomp = 1: partials (r.r); 2: (r.z, r.r) with the Jacobi preconditioner.
__global__ void k_cg_fin_beta(const double *part, int nblk, int ncomp, int ld, double *state,
                              int *active, const int *nact_prev, int *nact_next, int *iters) {
  if (*nact_prev == 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) *iters += 1;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= ld) return;
  const double rhon = warp_sum_blocks(part, nblk, ncomp * ld, j);
  const double rrn = ncomp == 2 ? warp_sum_blocks(part, nblk, ncomp * ld, ld + j) : rhon;
  if ((threadIdx.x & 31) == 0) {
    const double rho = state[j];
    int a = active[j];
    state[3 * ld + j] = (a && rho > 0.0) ? rhon / rho : 0.0;
    if (a) {
      state[j] = rhon;
      a = rrn > state[ld + j];
      active[j] = a;
    }
    if (a) atomicAdd(nact_next, 1);
  }
}

// colsum[e] = sum_b part[b][e] for e < ncomp*ld: one warp per entry, fixed order.
__global__ void k_fin_cols(const double *__restrict__ part, int nblk, int ncomp, int ld,
                           double *__restrict__ colsum) {
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= ncomp * ld) return;
  const double s = warp_sum_blocks(part, nblk, ncomp * ld, e);
  if ((threadIdx.x & 31) == 0) colsum[e] = s;
}

// out[c] = sum_j colsum[c][j], c < ncomp (one CTA, fixed order).
__global__ void k_fin_total(const double *__restrict__ colsum, int ncomp, int ld,
                            double *__restrict__ out) {
  __shared__ double sh[256];
  for (int c = 0; c < ncomp; ++c) {
    double s = 0.0;
    for (int j = threadIdx.x; j < ld; j += blockDim.x) s += colsum[c * ld + j];
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

// CTAs of a row kernel: four 256-thread CTAs per SM, fewer for small n.
int grid_blocks(long long n, int rows) {
  long long want = (n + rows - 1) / rows;
  long long cap = (long long)num_sms() * 4;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

int warp_blocks(int warps) { return (warps * 32 + 255) / 256; }

// The CTA partials buffer holds up to num_sms()*8 x 2 x ld doubles; per-column sums follow.
double *colsum_area(double *part, int ld) { return part + (size_t)num_sms() * 8 * 2 * ld; }

}  // namespace

size_t part_bytes(int ld) {
  return ((size_t)num_sms() * 8 * 2 * ld + 2 * (size_t)ld) * sizeof(double);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T>
op_status launch_apply(const Geom &g, const T *Vt, double sigma, const T *X, T *Y, int ld,
                       cudaStream_t st, double scale) {
  RowShape s = row_shape(ld, Pack<T>::N);
  k_apply<T><<<dim3(grid_blocks(g.n, s.rows), s.gy), s.block, 0, st>>>(
      g, Vt, (T)(g.cdiag + sigma), X, Y, ld, (T)scale);
  count_launch();
  OP_LAUNCH("k_apply");
  return OP_OK;
}

template <typename T>
op_status launch_quad(const Geom &g, const T *Vt, double sigma, const T *X, int ld, double *part,
                      double *out, cudaStream_t st, int *err) {
  int nb = 0;
  bool tma = false;
  if constexpr (std::is_same<T, float>::value)
    tma = err != nullptr && cg_tma_eligible(g, ld, X, X, X);
  if (tma) {
    if constexpr (std::is_same<T, float>::value)
      OP_TRY(tma_quad(g, sigma, ld, Vt, X, part, err, &nb, st));
  } else {
    RowShape s = row_shape(ld, Pack<T>::N);
    nb = grid_blocks(g.n, s.rows);
    k_quad<T><<<dim3(nb, s.gy), s.block, 0, st>>>(g, Vt, (T)(g.cdiag + sigma), X, ld, part);
    count_launch();
  }
  k_fin_cols<<<warp_blocks(2 * ld), 256, 0, st>>>(part, nb, 2, ld, colsum_area(part, ld));
  count_launch();
  k_fin_total<<<1, 256, 0, st>>>(colsum_area(part, ld), 2, ld, out);
  count_launch();
  OP_LAUNCH("k_quad");
  return OP_OK;
}

template <typename T>
op_status launch_sumsq(long long n, int ld, const T *X, double *part, double *out,
                       cudaStream_t st) {
  RowShape s = row_shape(ld, Pack<T>::N);
  const int nb = grid_blocks(n, s.rows);
  k_sumsq<T><<<dim3(nb, s.gy), s.block, 0, st>>>(n, ld, X, part);
  count_launch();
  k_fin_cols<<<warp_blocks(ld), 256, 0, st>>>(part, nb, 1, ld, colsum_area(part, ld));
  count_launch();
  k_fin_total<<<1, 256, 0, st>>>(colsum_area(part, ld), 1, ld, out);
  count_launch();
  OP_LAUNCH("k_sumsq");
  return OP_OK;
}

size_t cg_workspace_bytes(long long n, int ld, int elem) {
  size_t blk = (size_t)n * ld * elem;
  blk = (blk + 255) / 256 * 256;
  size_t state = (size_t)6 * ld * sizeof(double) + ((size_t)ld * sizeof(int) + 255) / 256 * 256;
  return 3 * blk + (part_bytes(ld) + 255) / 256 * 256 + state + 1024;
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
  w->max_blocks = num_sms() * 8;
  w->part = (double *)p;
  p += (part_bytes(ld) + 255) / 256 * 256;
  w->state = (double *)p;
  p += (size_t)6 * ld * sizeof(double);
  w->active = (int *)p;
  p += ((size_t)ld * sizeof(int) + 255) / 256 * 256;
  w->ctl = (int *)p;
}

template <typename T>
op_status cg_solve(const Geom &g, const T *Vt, double sigma, const T *U, T *W, int p, int ld,
                   double rtol, int max_iter, CGWork &w, int *iters, cudaStream_t st) {
  constexpr bool kFused = std::is_same<T, float>::value;
  RowShape s = row_shape(ld, Pack<T>::N);
  const int nb = grid_blocks(g.n, s.rows);
  const dim3 grid(nb, s.gy);
  const int fb = warp_blocks(ld);
  T *R = (T *)w.R, *P = (T *)w.P, *Q = (T *)w.Q;
  double *alpha = w.state + 2 * ld, *beta = w.state + 3 * ld;
  int *ctl = w.ctl;
  const T sg = (T)(g.cdiag + sigma);
  // FP32 on 3-D grids: the direction update and its stencil by the TMA plane-marching
  // kernel (its own persistent grid); the W/R update stays an L2-served row kernel,
  // which measured faster (its many independent loads hide latency better)
  CgTmaPlan plan;
  bool tma = false;
  int nb_p = nb;
  if constexpr (kFused) {
    tma = cg_tma_eligible(g, ld, R, P, Q);
    if (tma) {
      OP_TRY(cg_tma_prepare(g, sigma, ld, R, P, Q, &plan));
      nb_p = plan.grid;
    }
  }

  // Jacobi preconditioning: R holds Z = R / diag(H + sigma); the direction kernels
  // (P = Z + beta P and its stencil) are unchanged, the W/R kernels carry 1 / d
  const bool jac = w.jacobi;
  prof_begin(w.prof, PK_CG_INIT, st);
  // (a TMA plane-marching version of this pass measured slower than the row kernel)
  if (kFused) {
    if (jac)
      k_cg_init<T, false, true><<<grid, s.block, 0, st>>>(g, Vt, sg, U, W, R, P, ld, w.part, ctl);
    else
      k_cg_init<T, false, false><<<grid, s.block, 0, st>>>(g, Vt, sg, U, W, R, P, ld, w.part, ctl);
  } else {
    if (jac)
      k_cg_init<T, true, true><<<grid, s.block, 0, st>>>(g, Vt, sg, U, W, R, P, ld, w.part, ctl);
    else
      k_cg_init<T, true, false><<<grid, s.block, 0, st>>>(g, Vt, sg, U, W, R, P, ld, w.part, ctl);
  }
  count_launch();
  k_cg_fin_init<<<fb, 256, 0, st>>>(w.part, nb, jac ? 3 : 2, ld, p, rtol * rtol, w.state,
                                    w.active, ctl);
  count_launch();
  prof_end(w.prof, st);
  OP_LAUNCH("k_cg_init");

  // Queue iterations in chunks (the first one as long as the previous solve), then
  // read the active count back; kernels queued past convergence return at once.
  int launched = 0, done = 0;
  int chunk = w.expect_iters > 1 ? w.expect_iters : 2;
  while (launched < max_iter) {
    const int upto = (launched + chunk < max_iter) ? launched + chunk : max_iter;
    for (int k = launched; k < upto; ++k) {
      const int *nprev = ctl + ((k + 1) & 1);
      int *nnext = ctl + (k & 1);
      if (kFused) {
        T *Po = (k & 1) ? Q : P, *Pn = (k & 1) ? P : Q;
        prof_begin(w.prof, PK_CG_APPLY, st);
        if (tma) {
          if constexpr (kFused)
            OP_TRY(cg_tma_p(plan, k == 0, (k & 1) ? 1 : 0, Pn, Vt, beta, nprev, w.part, ctl + 3,
                            st));
        } else {
          if (k == 0)
            k_cg_p<T, true><<<grid, s.block, 0, st>>>(g, Vt, sg, R, Po, Pn, ld, beta, nprev,
                                                      w.part);
          else
            k_cg_p<T, false><<<grid, s.block, 0, st>>>(g, Vt, sg, R, Po, Pn, ld, beta, nprev,
                                                       w.part);
          count_launch();
        }
        prof_end(w.prof, st);
        prof_begin(w.prof, PK_CG_FIN, st);
        k_cg_fin_alpha<<<fb, 256, 0, st>>>(w.part, nb_p, ld, w.state, w.active, nprev, nnext);
        count_launch();
        prof_end(w.prof, st);
        prof_begin(w.prof, PK_CG_AXPY, st);
        if (jac)
          k_cg_wr<T, true><<<grid, s.block, 0, st>>>(g, Vt, sg, W, R, Pn, ld, alpha, nprev,
                                                      w.part);
        else
          k_cg_wr<T, false><<<grid, s.block, 0, st>>>(g, Vt, sg, W, R, Pn, ld, alpha, nprev,
                                                       w.part);
        count_launch();
        prof_end(w.prof, st);
        prof_begin(w.prof, PK_CG_FIN, st);
        k_cg_fin_beta<<<fb, 256, 0, st>>>(w.part, nb, jac ? 2 : 1, ld, w.state, w.active, nprev,
                                           nnext, ctl + 2);
        count_launch();
        prof_end(w.prof, st);
      } else {
        prof_begin(w.prof, PK_CG_APPLY, st);
        k_cg_apply<T><<<grid, s.block, 0, st>>>(g, Vt, sg, P, Q, ld, nprev, w.part);
        count_launch();
        prof_end(w.prof, st);
        prof_begin(w.prof, PK_CG_FIN, st);
        k_cg_fin_alpha<<<fb, 256, 0, st>>>(w.part, nb, ld, w.state, w.active, nprev, nnext);
        count_launch();
        prof_end(w.prof, st);
        prof_begin(w.prof, PK_CG_AXPY, st);
        if (jac)
          k_cg_axpy<T, true><<<grid, s.block, 0, st>>>(g.n, ld, Vt, sg, W, R, P, Q, alpha, nprev,
                                                        w.part);
        else
          k_cg_axpy<T, false><<<grid, s.block, 0, st>>>(g.n, ld, Vt, sg, W, R, P, Q, alpha,
                                                         nprev, w.part);
        count_launch();
        prof_end(w.prof, st);
        prof_begin(w.prof, PK_CG_FIN, st);
        k_cg_fin_beta<<<fb, 256, 0, st>>>(w.part, nb, jac ? 2 : 1, ld, w.state, w.active, nprev,
                                           nnext, ctl + 2);
        count_launch();
        prof_end(w.prof, st);
        prof_begin(w.prof, PK_CG_DIR, st);
        k_cg_dir<T><<<grid, s.block, 0, st>>>(g.n, ld, R, P, beta, nprev);
        count_launch();
        prof_end(w.prof, st);
      }
    }
    OP_LAUNCH("cg iteration");
    launched = upto;
    OP_CUDA(cudaMemcpyAsync(w.host_ctl, ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    OP_CUDA(cudaStreamSynchronize(st));
    prof_harvest(w.prof);
    if (w.host_ctl[3]) {
      set_error("a CG kernel gave up a bounded wait for its TMA copies");
      return OP_ERR_TIMEOUT;
    }
    done = w.host_ctl[2];
    // converged: no active column after the last queued iteration (or the solve
    // stopped inside the chunk)
    if (w.host_ctl[(upto - 1) & 1] == 0 || done < launched) break;
    chunk = 2;
  }
  *iters = done;
  w.expect_iters = done;
  return OP_OK;
}

// ---- mixed-precision Step 1 (FP64 iterative refinement around an FP32 CG) -------------
namespace {

// scale[j] = ||r_j|| for the active columns (0 otherwise), from the init finaliser's state;
// inv[j] = 1 / scale[j] in FP32 (0 for inactive columns).
__global__ void k_ref_scale(int ld, const double *__restrict__ state, const int *__restrict__ active,
                            double *__restrict__ scale, float *__restrict__ inv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ld) return;
  const double sc = active[j] ? sqrt(state[j]) : 0.0;
  scale[j] = sc;
  inv[j] = sc > 0.0 ? (float)(1.0 / sc) : 0.f;
}

// r32 = R / scale (column-wise; zero for inactive columns), four elements per thread.  The
// right-hand side of the FP32 solve only needs FP32 accuracy: an FP32 product with the
// reciprocal (no FP64 division per element).
__global__ void k_ref_rhs(long long total, int ld, const double *__restrict__ R,
                          const float *__restrict__ inv, float *__restrict__ r32) {
  for (long long e = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x); e < total;
       e += 4 * (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % ld);
    const double2 a = *reinterpret_cast<const double2 *>(R + e);
    const double2 b = *reinterpret_cast<const double2 *>(R + e + 2);
    const float4 w = *reinterpret_cast<const float4 *>(inv + j);
    *reinterpret_cast<float4 *>(r32 + e) =
        make_float4((float)a.x * w.x, (float)a.y * w.y, (float)b.x * w.z, (float)b.y * w.w);
  }
}

// W += scale_j d_j in FP64.
__global__ void k_ref_correct(long long total, int ld, const float *__restrict__ d32,
                              const double *__restrict__ scale, double *__restrict__ W) {
  for (long long e = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x); e < total;
       e += 4 * (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % ld);
    const float4 d = *reinterpret_cast<const float4 *>(d32 + e);
    double2 a = *reinterpret_cast<double2 *>(W + e);
    double2 b = *reinterpret_cast<double2 *>(W + e + 2);
    a.x += scale[j] * (double)d.x;
    a.y += scale[j + 1] * (double)d.y;
    b.x += scale[j + 2] * (double)d.z;
    b.y += scale[j + 3] * (double)d.w;
    *reinterpret_cast<double2 *>(W + e) = a;
    *reinterpret_cast<double2 *>(W + e + 2) = b;
  }
}

}  // namespace

op_status refine_residual(const Geom &g, const double *Vt, double sigma, const double *U,
                          const double *W, int ld, CGWork &w64, cudaStream_t st) {
  RowShape s = row_shape(ld, Pack<double>::N);
  const int nb = grid_blocks(g.n, s.rows);
  k_cg_init<double, false, false><<<dim3(nb, s.gy), s.block, 0, st>>>(
      g, Vt, g.cdiag + sigma, U, W, (double *)w64.R, nullptr, ld, w64.part, w64.ctl);
  count_launch();
  OP_LAUNCH("refine_residual");
  return OP_OK;
}

op_status cg_refine(const Geom &g, const double *Vt, const float *Vt32, double sigma,
                    const double *U, double *W, int p, int ld, double rtol, int max_iter,
                    CGWork &w64, CGWork &w32, float *r32, float *d32, double *scale, int *iters,
                    int *cycles, cudaStream_t st, const double *Uprev, bool *fresh) {
  RowShape s = row_shape(ld, Pack<double>::N);
  const int nb = grid_blocks(g.n, s.rows);
  const dim3 grid(nb, s.gy);
  const int fb = warp_blocks(ld);
  const double sg = g.cdiag + sigma;
  const long long total = g.n * ld;
  const int eb = (int)std::min<long long>((total / 4 + 255) / 256, (long long)num_sms() * 32);
  double *R = (double *)w64.R;
  std::vector<double> hs(2 * (size_t)ld);
  int inner = 0, cyc = 0;
  *iters = 0;
  *cycles = 0;
  for (; cyc < 12; ++cyc) {
    prof_begin(w64.prof, PK_REFINE, st);
    // R = U - (H + sigma) W and the column norms; active columns: ||r_j|| > rtol ||u_j||
    if (cyc == 0 && Uprev)
      k_ref_recycle<double><<<grid, s.block, 0, st>>>(g.n, U, Uprev, R, ld, w64.part, w64.ctl);
    else
      k_cg_init<double, false, false><<<grid, s.block, 0, st>>>(g, Vt, sg, U, W, R, nullptr, ld,
                                                               w64.part, w64.ctl);
    count_launch();
    k_cg_fin_init<<<fb, 256, 0, st>>>(w64.part, nb, 2, ld, p, rtol * rtol, w64.state, w64.active,
                                      w64.ctl);
    count_launch();
    prof_end(w64.prof, st);
    OP_LAUNCH("cg_refine residual");
    OP_CUDA(cudaMemcpyAsync(w64.host_ctl, w64.ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    OP_CUDA(cudaMemcpyAsync(hs.data(), w64.state, (size_t)ld * sizeof(double),
                            cudaMemcpyDeviceToHost, st));
    OP_CUDA(cudaMemcpyAsync(hs.data() + ld, w64.state + 4 * (size_t)ld, (size_t)ld * sizeof(double),
                            cudaMemcpyDeviceToHost, st));
    OP_CUDA(cudaStreamSynchronize(st));
    prof_harvest(w64.prof);
    if (w64.host_ctl[1] == 0 || inner >= max_iter) break;
    // the inner tolerance the worst active column needs, with a margin, not below what an
    // FP32 solve reaches
    double rho = 0.0;
    for (int j = 0; j < p; ++j)
      if (hs[ld + j] > 0.0 && hs[j] > rtol * rtol * hs[ld + j])
        rho = std::max(rho, sqrt(hs[j] / hs[ld + j]));
    double eta = rho > 0.0 ? 0.3 * rtol / rho : 0.5;
    eta = std::min(0.5, std::max(eta, 2e-6));
    prof_begin(w64.prof, PK_REFINE, st);
    float *inv = (float *)(scale + ld);
    k_ref_scale<<<(ld + 255) / 256, 256, 0, st>>>(ld, w64.state, w64.active, scale, inv);
    count_launch();
    k_ref_rhs<<<eb, 256, 0, st>>>(total, ld, R, inv, r32);
    count_launch();
    OP_CUDA(cudaMemsetAsync(d32, 0, (size_t)total * sizeof(float), st));
    prof_end(w64.prof, st);
    OP_LAUNCH("cg_refine rhs");
    int it = 0;
    OP_TRY(cg_solve<float>(g, Vt32, sigma, r32, d32, p, ld, eta, max_iter - inner, w32, &it, st));
    inner += it;
    prof_begin(w64.prof, PK_REFINE, st);
    k_ref_correct<<<eb, 256, 0, st>>>(total, ld, d32, scale, W);
    count_launch();
    prof_end(w64.prof, st);
    OP_LAUNCH("cg_refine correction");
  }
  *iters = inner;
  *cycles = cyc + 1;
  if (fresh) *fresh = cyc > 0 || !Uprev;
  return OP_OK;
}

template <typename T>
op_status launch_pad_copy(long long n, int p, int ld, const double *src, T *dst, cudaStream_t st) {
  k_pad_copy<T><<<num_sms() * 8, 256, 0, st>>>(n, p, ld, src, dst);
  count_launch();
  OP_LAUNCH("k_pad_copy");
  return OP_OK;
}

template <typename T>
op_status launch_unpad_copy(long long n, int p, int ld, const T *src, double *dst,
                            cudaStream_t st) {
  k_unpad_copy<T><<<num_sms() * 8, 256, 0, st>>>(n, p, ld, src, dst);
  count_launch();
  OP_LAUNCH("k_unpad_copy");
  return OP_OK;
}


// ---------------------------------------------------------------------------
// Batched kernels (FP32 blocks): one CTA per RowItem (problem, grid-point range).
// A CTA of 256 threads covers nv = ld/4 float4 vectors of 256/nv points per pass.
// ---------------------------------------------------------------------------
namespace {

struct FlatMap {
  int nv, rows, tx, ty;
  bool active;
};
__device__ __forceinline__ FlatMap flat_map(int ld) {
  FlatMap m;
  m.nv = ld >> 2;
  m.rows = 256 / m.nv;
  m.tx = threadIdx.x % m.nv;
  m.ty = threadIdx.x / m.nv;
  m.active = m.ty < m.rows;
  return m;
}

// Sum the per-thread partials acc[c][k] (column tx*4 + k) over the rows of the
// CTA into dst[c][ld] (FP64, fixed order).
template <int NCOMP>
__device__ __forceinline__ void flat_colsum(const float (&acc)[NCOMP][4], const FlatMap &m, int ld,
                                            double *__restrict__ dst) {
  __shared__ double red[256 * NCOMP * 4];
  const int width = NCOMP * ld;
  if (m.active) {
#pragma unroll
    for (int c = 0; c < NCOMP; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) red[m.ty * width + c * ld + m.tx * 4 + k] = (double)acc[c][k];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < width; e += blockDim.x) {
    double s = 0.0;
    for (int y = 0; y < m.rows; ++y) s += red[y * width + e];
    dst[e] = s;
  }
}

__global__ void __launch_bounds__(256) k_b_cg_init(const BatchProb *__restrict__ B,
                                                   const RowItem *__restrict__ items, int parity) {
  const RowItem it = items[blockIdx.x];
  const BatchProb &pb = B[it.prob];
  if (*pb.frozen) return;
  const int ld = pb.ld;
  const FlatMap m = flat_map(ld);
  if (it.local == 0 && threadIdx.x == 0) {
    pb.ctl[1] = 0;
    pb.ctl[2] = 0;
  }
  const float *U = pb.U[parity];
  // partials (r.z, u.u, r.r); without the Jacobi preconditioner z = r
  float acc[3][4] = {};
  if (m.active) {
    const int col = m.tx * 4;
    for (long long i = it.r0 + m.ty; i < it.r1; i += m.rows) {
      const Pack<float> aw = stencil_at(pb.g, pb.Vt, pb.shift, pb.W, ld, i, col, (Pack<float> *)nullptr);
      const long long o = i * (long long)ld + col;
      const Pack<float> u = Pack<float>::load(U + o);
      const float inv = pb.jacobi ? 1.f / (__ldg(pb.Vt + i) + pb.shift) : 1.f;
      Pack<float> r;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float rk = u.v[k] - aw.v[k];
        r.v[k] = pb.jacobi ? rk * inv : rk;
        acc[0][k] += rk * r.v[k];
        acc[1][k] += u.v[k] * u.v[k];
        acc[2][k] += rk * rk;
      }
      r.store(pb.R + o);
    }
  }
  flat_colsum<3>(acc, m, ld, pb.part + (long long)it.local * 3 * ld);
}

// Finalisers: grid (column warps, problems).
__global__ void k_b_fin_init(const BatchProb *__restrict__ B) {
  const BatchProb &pb = B[blockIdx.y];
  const int ld = pb.ld;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= ld || *pb.frozen) return;
  const double rho = warp_sum_blocks(pb.part, pb.n_row_items, 3 * ld, j);
  const double bb = warp_sum_blocks(pb.part, pb.n_row_items, 3 * ld, ld + j);
  const double rr = warp_sum_blocks(pb.part, pb.n_row_items, 3 * ld, 2 * ld + j);
  if ((threadIdx.x & 31) == 0) {
    const double rtol2 = *pb.cg_rtol2;
    double *state = pb.state;
    state[0 * ld + j] = rho;
    state[1 * ld + j] = rtol2 * bb;
    state[2 * ld + j] = 0.0;
    state[3 * ld + j] = 0.0;
    state[4 * ld + j] = bb;
    const int a = (j < pb.p) && (rr > rtol2 * bb) && (bb > 0.0);
    pb.active[j] = a;
    if (a) atomicAdd(&pb.ctl[1], 1);
  }
}

template <bool FIRST>
__global__ void __launch_bounds__(256) k_b_cg_p(const BatchProb *__restrict__ B,
                                                const RowItem *__restrict__ items, int k) {
  const RowItem it = items[blockIdx.x];
  const BatchProb &pb = B[it.prob];
  if (*pb.frozen || pb.ctl[(k + 1) & 1] == 0) return;
  const int ld = pb.ld;
  const FlatMap m = flat_map(ld);
  const float *R = pb.R;
  const float *Po = (k & 1) ? pb.Q : pb.P;
  float *Pn = (k & 1) ? pb.P : pb.Q;
  const Geom &g = pb.g;
  float acc[1][4] = {};
  if (m.active) {
    const int col = m.tx * 4;
    float b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = FIRST ? 0.f : (float)pb.state[3 * ld + col + q];
    const long long sty = (long long)g.nx * ld, stz = (long long)g.nx * g.ny * ld;
    for (long long i = it.r0 + m.ty; i < it.r1; i += m.rows) {
      const long long base = i * (long long)ld + col;
      const Coord c = coord_of(g, i);
      const Pack<float> pc = dir_at<float, FIRST>(R, Po, b, base);
      Pack<float> sx = Pack<float>::zero(), sy = Pack<float>::zero(), sz = Pack<float>::zero();
      if (c.ix > 0) add_pack(sx, dir_at<float, FIRST>(R, Po, b, base - ld));
      if (c.ix < g.nx - 1) add_pack(sx, dir_at<float, FIRST>(R, Po, b, base + ld));
      if (c.iy > 0) add_pack(sy, dir_at<float, FIRST>(R, Po, b, base - sty));
      if (c.iy < g.ny - 1) add_pack(sy, dir_at<float, FIRST>(R, Po, b, base + sty));
      if (g.dim == 3) {
        if (c.iz > 0) add_pack(sz, dir_at<float, FIRST>(R, Po, b, base - stz));
        if (c.iz < g.nz - 1) add_pack(sz, dir_at<float, FIRST>(R, Po, b, base + stz));
      }
      const Pack<float> q = combine(g, __ldg(pb.Vt + i) + pb.shift, pc, sx, sy, sz);
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[0][e] += pc.v[e] * q.v[e];
      pc.store(Pn + base);
    }
  }
  flat_colsum<1>(acc, m, ld, pb.part + (long long)it.local * ld);
}

__global__ void k_b_fin_alpha(const BatchProb *__restrict__ B, int k) {
  const BatchProb &pb = B[blockIdx.y];
  if (blockIdx.x == 0 && threadIdx.x == 0) pb.ctl[k & 1] = 0;
  if (*pb.frozen || pb.ctl[(k + 1) & 1] == 0) return;
  const int ld = pb.ld;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= ld) return;
  const double pq = warp_sum_blocks(pb.part, pb.n_row_items, ld, j);
  if ((threadIdx.x & 31) == 0) {
    const double rr = pb.state[j];
    pb.state[2 * ld + j] = (pb.active[j] && pq > 0.0) ? rr / pq : 0.0;
  }
}

__global__ void __launch_bounds__(256) k_b_cg_wr(const BatchProb *__restrict__ B,
                                                 const RowItem *__restrict__ items, int k) {
  const RowItem it = items[blockIdx.x];
  const BatchProb &pb = B[it.prob];
  if (*pb.frozen || pb.ctl[(k + 1) & 1] == 0) return;
  const int ld = pb.ld;
  const FlatMap m = flat_map(ld);
  const float *Pn = (k & 1) ? pb.P : pb.Q;
  // partials (r.z, r.r); with the Jacobi preconditioner R holds z = r / d
  float acc[2][4] = {};
  if (m.active) {
    const int col = m.tx * 4;
    float a[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = (float)pb.state[2 * ld + col + q];
    for (long long i = it.r0 + m.ty; i < it.r1; i += m.rows) {
      Pack<float> pc;
      const Pack<float> q = stencil_at(pb.g, pb.Vt, pb.shift, Pn, ld, i, col, &pc);
      const long long o = i * (long long)ld + col;
      Pack<float> w = Pack<float>::load_rw(pb.W + o), r = Pack<float>::load_rw(pb.R + o);
      if (pb.jacobi) {
        const float dg = __ldg(pb.Vt + i) + pb.shift, inv = 1.f / dg;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          w.v[e] += a[e] * pc.v[e];
          r.v[e] -= a[e] * (q.v[e] * inv);
          const float rk = dg * r.v[e];
          acc[0][e] += rk * r.v[e];
          acc[1][e] += rk * rk;
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          w.v[e] += a[e] * pc.v[e];
          r.v[e] -= a[e] * q.v[e];
          acc[0][e] += r.v[e] * r.v[e];
          acc[1][e] += r.v[e] * r.v[e];
        }
      }
      w.store(pb.W + o);
      r.store(pb.R + o);
    }
  }
  flat_colsum<2>(acc, m, ld, pb.part + (long long)it.local * 2 * ld);
}

__global__ void k_b_fin_beta(const BatchProb *__restrict__ B, int k) {
  const BatchProb &pb = B[blockIdx.y];
  if (*pb.frozen || pb.ctl[(k + 1) & 1] == 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) pb.ctl[2] += 1;
  const int ld = pb.ld;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= ld) return;
  const double rhon = warp_sum_blocks(pb.part, pb.n_row_items, 2 * ld, j);
  const double rrn = warp_sum_blocks(pb.part, pb.n_row_items, 2 * ld, ld + j);
  if ((threadIdx.x & 31) == 0) {
    double *state = pb.state;
    const double rho = state[j];
    int a = pb.active[j];
    state[3 * ld + j] = (a && rho > 0.0) ? rhon / rho : 0.0;
    if (a) {
      state[j] = rhon;
      a = rrn > state[ld + j];
      pb.active[j] = a;
    }
    if (a) atomicAdd(&pb.ctl[k & 1], 1);
  }
}

// Energy of the new U: part[item][0][j] = u_j . (H u)_j, part[item][1][j] = u_j . u_j.
__global__ void __launch_bounds__(256) k_b_quad(const BatchProb *__restrict__ B,
                                                const RowItem *__restrict__ items, int parity) {
  const RowItem it = items[blockIdx.x];
  const BatchProb &pb = B[it.prob];
  if (*pb.frozen) return;
  const int ld = pb.ld;
  const FlatMap m = flat_map(ld);
  const float *X = pb.U[parity];
  const float shift0 = (float)pb.g.cdiag;  // unshifted H
  float acc[2][4] = {};
  if (m.active) {
    const int col = m.tx * 4;
    for (long long i = it.r0 + m.ty; i < it.r1; i += m.rows) {
      Pack<float> xc;
      const Pack<float> y = stencil_at(pb.g, pb.Vt, shift0, X, ld, i, col, &xc);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc[0][e] += xc.v[e] * y.v[e];
        acc[1][e] += xc.v[e] * xc.v[e];
      }
    }
  }
  flat_colsum<2>(acc, m, ld, pb.part + (long long)it.local * 2 * ld);
}

// dsc[4] = sum_j sum_items part[.][0][j], dsc[5] likewise for component 1 (one CTA per problem).
__global__ void k_b_fin_energy(const BatchProb *__restrict__ B) {
  const BatchProb &pb = B[blockIdx.x];
  if (*pb.frozen) return;
  const int ld = pb.ld;
  __shared__ double sh[2][256];
  double s0 = 0.0, s1 = 0.0;
  for (int j = threadIdx.x; j < ld; j += blockDim.x)
    for (int b = 0; b < pb.n_row_items; ++b) {
      s0 += pb.part[((long long)b * 2 + 0) * ld + j];
      s1 += pb.part[((long long)b * 2 + 1) * ld + j];
    }
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pb.dsc[4] = sh[0][0];
    pb.dsc[5] = sh[1][0];
  }
}

}  // namespace

op_status launch_b_cg_init(const BatchProb *B, const RowItem *items, int nitems, int parity,
                           cudaStream_t st) {
  k_b_cg_init<<<nitems, 256, 0, st>>>(B, items, parity);
  count_launch();
  OP_LAUNCH("k_b_cg_init");
  return OP_OK;
}

op_status launch_b_fin_init(const BatchProb *B, int nprob, int max_ld, cudaStream_t st) {
  k_b_fin_init<<<dim3(warp_blocks(max_ld), nprob), 256, 0, st>>>(B);
  count_launch();
  OP_LAUNCH("k_b_fin_init");
  return OP_OK;
}

op_status launch_b_cg_iter(const BatchProb *B, const RowItem *items, int nitems, int nprob,
                           int max_ld, int k, cudaStream_t st) {
  const dim3 fg(warp_blocks(max_ld), nprob);
  if (k == 0)
    k_b_cg_p<true><<<nitems, 256, 0, st>>>(B, items, k);
  else
    k_b_cg_p<false><<<nitems, 256, 0, st>>>(B, items, k);
  count_launch();
  k_b_fin_alpha<<<fg, 256, 0, st>>>(B, k);
  count_launch();
  k_b_cg_wr<<<nitems, 256, 0, st>>>(B, items, k);
  count_launch();
  k_b_fin_beta<<<fg, 256, 0, st>>>(B, k);
  count_launch();
  OP_LAUNCH("batched cg iteration");
  return OP_OK;
}

op_status launch_b_energy(const BatchProb *B, const RowItem *items, int nitems, int nprob,
                          int max_ld, int parity, cudaStream_t st) {
  (void)max_ld;
  k_b_quad<<<nitems, 256, 0, st>>>(B, items, parity);
  count_launch();
  k_b_fin_energy<<<nprob, 256, 0, st>>>(B);
  count_launch();
  OP_LAUNCH("batched energy");
  return OP_OK;
}

// ---------------------------------------------------------------------------
// Event profiler
// ---------------------------------------------------------------------------
const char *prof_name(int kind) {
  static const char *names[PK_COUNT] = {"cg_init", "cg_apply", "cg_axpy", "cg_dir",
                                        "cg_finalize", "gram", "core", "update", "energy",
                                        "residual", "cg_refine"};
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
                                     cudaStream_t, double);                                    \
  template op_status launch_quad<T>(const Geom &, const T *, double, const T *, int, double *, \
                                    double *, cudaStream_t, int *);                            \
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
