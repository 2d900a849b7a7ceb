// Inner matrices of [U W] (§2.1; the matrices <GU,U>, <GU,GU> of Steps 2-3
// and <U,U> of Theorem 4.1): C = W^T U, S = W^T W, D = U^T U.
//
// Tall-skinny product: the n grid points are split into chunks; each CTA
// computes one 64 x 64 output tile of one product over one chunk, staging
// KC-row slabs of both operands in shared memory (16-byte vector loads,
// coalesced along the row), 16 x 16 threads with 4 x 4 outputs each.  FP32
// blocks accumulate a slab group of 256 rows in FP32 and flush into FP64
// registers; chunk partials are written in FP64 and summed over chunks in a
// fixed order by a second kernel (deterministic).
#include "common.cuh"
#include "kernels.cuh"

namespace opevo {

namespace {

constexpr int kTile = 64;

template <typename T> struct GramCfg;
template <> struct GramCfg<float> {
  static constexpr int KC = 32;
  static constexpr int FLUSH = 8;  // slabs between FP64 flushes (256 rows)
};
template <> struct GramCfg<double> {
  static constexpr int KC = 16;
  static constexpr int FLUSH = 1;
};

enum { PROD_C = 0, PROD_S = 1, PROD_D = 2 };

// Tile jobs are enumerated product by product (C: all nt x nt tiles; S and D:
// the tiles ti <= tj); `mask` selects the products that are computed.
__device__ __forceinline__ void decode_job(int idx, int mask, int nt, int *prod, int *ti,
                                           int *tj) {
  int pr = 0;
  for (; pr < 3; ++pr) {
    if (!((mask >> pr) & 1)) continue;
    const int cnt = pr == PROD_C ? nt * nt : nt * (nt + 1) / 2;
    if (idx < cnt) break;
    idx -= cnt;
  }
  *prod = pr;
  if (pr == PROD_C) {
    *ti = idx / nt;
    *tj = idx % nt;
  } else {
    int i = 0;
    while (idx >= nt - i) {
      idx -= nt - i;
      ++i;
    }
    *ti = i;
    *tj = i + idx;
  }
}

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) k_gram(long long n, int ld, const T *__restrict__ U,
                                              const T *__restrict__ W, int mask, int nt,
                                              int njobs, long long rows_per_split,
                                              double *__restrict__ part) {
  constexpr int KC = GramCfg<T>::KC;
  constexpr int N = Pack<T>::N;
  constexpr int PITCH = kTile + N;
  constexpr int VPR = kTile / N;  // vectors per tile row
  __shared__ __align__(16) T As[KC][PITCH];
  __shared__ __align__(16) T Bs[KC][PITCH];

  int prod, ti, tj;
  decode_job(blockIdx.x, mask, nt, &prod, &ti, &tj);
  const T *A = (prod == PROD_D) ? U : W;
  const T *B = (prod == PROD_S) ? W : U;
  const long long r0 = (long long)blockIdx.y * rows_per_split;
  long long r1 = r0 + rows_per_split;
  if (r1 > n) r1 = n;
  const int ca = ti * kTile, cb = tj * kTile;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int t = ty * 16 + tx;

  Acc acc[4][4];
  double accd[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[a][b] = Acc(0);
      accd[a][b] = 0.0;
    }

  int slab = 0;
  for (long long r = r0; r < r1; r += KC) {
#pragma unroll
    for (int q = 0; q < (KC * VPR) / 256; ++q) {
      const int v = t + 256 * q;
      const int rr = v / VPR, cv = v % VPR;
      const long long row = r + rr;
      Pack<T> xa = Pack<T>::zero(), xb = Pack<T>::zero();
      if (row < r1) {
        if (ca + cv * N < ld) xa = Pack<T>::load(A + row * ld + ca + cv * N);
        if (cb + cv * N < ld) xb = Pack<T>::load(B + row * ld + cb + cv * N);
      }
      xa.store(&As[rr][cv * N]);
      xb.store(&Bs[rr][cv * N]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      Acc av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = (Acc)As[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = (Acc)Bs[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
    if (++slab == GramCfg<T>::FLUSH) {
      slab = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          accd[a][b] += (double)acc[a][b];
          acc[a][b] = Acc(0);
        }
    }
  }
  double *dst = part + ((long long)blockIdx.y * njobs + blockIdx.x) * (kTile * kTile);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
      dst[(ty + 16 * a) * kTile + tx + 16 * b] = accd[a][b] + (double)acc[a][b];
}

__global__ void k_gram_reduce(int mask, int nt, int njobs, int nsplit,
                              const double *__restrict__ part, int p, int ld, double *C, double *S,
                              double *D) {
  int prod, ti, tj;
  decode_job(blockIdx.x, mask, nt, &prod, &ti, &tj);
  double *out = prod == PROD_C ? C : (prod == PROD_S ? S : D);
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < kTile * kTile;
       e += gridDim.y * blockDim.x) {
    const int i = ti * kTile + e / kTile, j = tj * kTile + e % kTile;
    if (i >= ld || j >= ld) continue;
    double s = 0.0;
#pragma unroll 8
    for (int sp = 0; sp < nsplit; ++sp)
      s += part[((long long)sp * njobs + blockIdx.x) * (kTile * kTile) + e];
    const double v = (i < p && j < p) ? s : 0.0;
    out[(long long)i * ld + j] = v;
    if (prod != PROD_C && ti != tj) out[(long long)j * ld + i] = v;
  }
}

struct GramPlan {
  int njobs;
  int nsplit;
  long long rows_per_split;
};

GramPlan plan_gram(long long n, int ld, int nprod, int kc) {
  const int nt = (ld + kTile - 1) / kTile;
  GramPlan g;
  g.njobs = nprod * nt * nt;  // upper bound (symmetric products use fewer)
  const int want = 4 * num_sms();
  long long ns = (want + g.njobs - 1) / g.njobs;
  long long maxs = (n + 255) / 256;
  if (ns > maxs) ns = maxs;
  if (ns < 1) ns = 1;
  long long rps = (n + ns - 1) / ns;
  rps = (rps + kc - 1) / kc * kc;
  g.nsplit = (int)((n + rps - 1) / rps);
  g.rows_per_split = rps;
  return g;
}

}  // namespace

size_t gram_workspace_bytes(long long n, int ld, int elem) {
  const int kc = elem == 4 ? GramCfg<float>::KC : GramCfg<double>::KC;
  GramPlan g = plan_gram(n, ld, 3, kc);
  return (size_t)g.njobs * g.nsplit * kTile * kTile * sizeof(double) + 512;
}

template <typename T>
op_status gram(long long n, int p, int ld, const T *U, const T *W, double *C, double *S,
               double *D, void *ws, size_t ws_bytes, cudaStream_t st) {
  if (ld % 8 != 0 || ld > 255 * kTile || p > ld || n < 1) {
    set_error("gram: bad sizes n=%lld p=%d ld=%d", n, p, ld);
    return OP_ERR_ARG;
  }
  const int nt = (ld + kTile - 1) / kTile;
  const int mask = (C ? 1 : 0) | (S ? 2 : 0) | (D ? 4 : 0);
  const int nj = (C ? nt * nt : 0) + (S ? nt * (nt + 1) / 2 : 0) + (D ? nt * (nt + 1) / 2 : 0);
  if (nj == 0) return OP_OK;
  GramPlan g = plan_gram(n, ld, 3, GramCfg<T>::KC);
  // recompute the split for the actual job count (more splits when fewer jobs)
  {
    const int want = 4 * num_sms();
    long long ns = (want + nj - 1) / nj;
    long long maxs = (n + 255) / 256;
    if (ns > maxs) ns = maxs;
    if (ns < 1) ns = 1;
    // never exceed the workspace sized for the 3-product plan
    const long long cap = ((long long)g.njobs * g.nsplit) / nj;
    if (ns > cap) ns = cap;
    long long rps = (n + ns - 1) / ns;
    rps = (rps + GramCfg<T>::KC - 1) / GramCfg<T>::KC * GramCfg<T>::KC;
    g.nsplit = (int)((n + rps - 1) / rps);
    g.rows_per_split = rps;
  }
  const size_t need = (size_t)nj * g.nsplit * kTile * kTile * sizeof(double);
  if (!ws || ws_bytes < need) {
    set_error("gram: workspace too small (%zu < %zu)", ws_bytes, need);
    return OP_ERR_ARG;
  }
  double *part = (double *)ws;
  k_gram<T, T><<<dim3(nj, g.nsplit), dim3(16, 16), 0, st>>>(n, ld, U, W, mask, nt, nj,
                                                           g.rows_per_split, part); count_launch();
  OP_LAUNCH("k_gram");
  k_gram_reduce<<<dim3(nj, kTile * kTile / 256), 256, 0, st>>>(mask, nt, nj, g.nsplit, part, p,
                                                                ld, C, S, D);
  count_launch();
  OP_LAUNCH("k_gram_reduce");
  return OP_OK;
}

// As gram(), but the chunk split is chosen so that the partials fit in part_bytes
// (fewer, longer chunks when the scratch is small).  OP_ERR_ARG if even one chunk
// per tile does not fit.
template <typename T>
op_status gram_fixed_scratch(long long n, int p, int ld, const T *U, const T *W, double *C,
                             double *S, double *D, void *part, size_t part_bytes, cudaStream_t st) {
  if (ld % 8 != 0 || ld > 255 * kTile || p > ld || n < 1) {
    set_error("gram: bad sizes n=%lld p=%d ld=%d", n, p, ld);
    return OP_ERR_ARG;
  }
  const int nt = (ld + kTile - 1) / kTile;
  const int mask = (C ? 1 : 0) | (S ? 2 : 0) | (D ? 4 : 0);
  const int nj = (C ? nt * nt : 0) + (S ? nt * (nt + 1) / 2 : 0) + (D ? nt * (nt + 1) / 2 : 0);
  if (nj == 0) return OP_OK;
  const size_t tile_bytes = (size_t)kTile * kTile * sizeof(double);
  const long long fit = (long long)(part_bytes / ((size_t)nj * tile_bytes));
  if (fit < 1) {
    set_error("gram: %d output tiles need %zu bytes of partials, the fixed scratch holds %zu",
              nj, (size_t)nj * tile_bytes, part_bytes);
    return OP_ERR_ARG;
  }
  long long ns = (4 * num_sms() + nj - 1) / nj;
  const long long maxs = (n + 255) / 256;
  if (ns > maxs) ns = maxs;
  if (ns > fit) ns = fit;
  if (ns < 1) ns = 1;
  long long rps = (n + ns - 1) / ns;
  rps = (rps + GramCfg<T>::KC - 1) / GramCfg<T>::KC * GramCfg<T>::KC;
  const int nsplit = (int)((n + rps - 1) / rps);
  k_gram<T, T><<<dim3(nj, nsplit), dim3(16, 16), 0, st>>>(n, ld, U, W, mask, nt, nj, rps,
                                                         (double *)part);
  count_launch();
  OP_LAUNCH("k_gram");
  k_gram_reduce<<<dim3(nj, kTile * kTile / 256), 256, 0, st>>>(mask, nt, nj, nsplit,
                                                                (const double *)part, p, ld, C,
                                                                S, D);
  count_launch();
  OP_LAUNCH("k_gram_reduce");
  return OP_OK;
}
template op_status gram_fixed_scratch<double>(long long, int, int, const double *, const double *,
                                              double *, double *, double *, void *, size_t,
                                              cudaStream_t);

template op_status gram<float>(long long, int, int, const float *, const float *, double *,
                               double *, double *, void *, size_t, cudaStream_t);
template op_status gram<double>(long long, int, int, const double *, const double *, double *,
                                double *, double *, void *, size_t, cudaStream_t);

}  // namespace opevo
