// Step 4 of §4.1, U^{n+1} = U^n - tau U^n A^n + tau W B^n, written as the
// rank-2p product Unew = [U W] [KU; KW] with KU = I - tau A, KW = tau B
// (with W = nullptr, the rank-p product Unew = U KU).
//
// Each CTA computes a 64-row x 64-column tile of Unew; KC-wide slabs of the
// n x 2p operand [U W] (16-byte loads along the row, stored k-major in shared
// memory) and of [KU; KW] are staged in shared memory; 16 x 16 threads with
// 4 x 4 outputs each.
#include "common.cuh"
#include "kernels.cuh"

namespace opevo {

namespace {

constexpr int kRows = 64, kCols = 64;

template <typename T> struct UpdCfg;
template <> struct UpdCfg<float> {
  static constexpr int KC = 32;
};
template <> struct UpdCfg<double> {
  static constexpr int KC = 16;
};

template <typename T>
__global__ void __launch_bounds__(256) k_update(long long n, int ld, const T *__restrict__ U,
                                                const T *__restrict__ W, const T *__restrict__ KU,
                                                const T *__restrict__ KW, T *__restrict__ Unew) {
  constexpr int KC = UpdCfg<T>::KC;
  constexpr int N = Pack<T>::N;
  constexpr int KV = KC / N;          // vectors per slab row of [U W]
  constexpr int CV = kCols / N;       // vectors per slab row of K
  __shared__ __align__(16) T As[KC][kRows + 1];
  __shared__ __align__(16) T Bs[KC][kCols + N];
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 16 + tx;
  // linear block index, column tiles fastest (the CTAs that share a row slab of [U W]
  // run together); grid.x is not limited to 65535 like grid.y
  const int nct = (ld + kCols - 1) / kCols;
  const long long r0 = (long long)(blockIdx.x / nct) * kRows;
  const int c0 = (int)(blockIdx.x % nct) * kCols;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);

  const int K = W ? 2 * ld : ld;  // W == nullptr: Unew = U KU (no W block)
  for (int k0 = 0; k0 < K; k0 += KC) {
#pragma unroll
    for (int q = 0; q < (kRows * KV) / 256; ++q) {
      const int v = t + 256 * q;
      const int r = v / KV, kv = v % KV;
      const int kk = k0 + kv * N;
      const long long row = r0 + r;
      Pack<T> x = Pack<T>::zero();
      if (row < n && kk < K)
        x = (kk < ld) ? Pack<T>::load(U + row * ld + kk) : Pack<T>::load(W + row * ld + kk - ld);
#pragma unroll
      for (int e = 0; e < N; ++e) As[kv * N + e][r] = x.v[e];
    }
#pragma unroll
    for (int q = 0; q < (KC * CV) / 256; ++q) {
      const int v = t + 256 * q;
      const int k = v / CV, cv = v % CV;
      const int kk = k0 + k, c = c0 + cv * N;
      Pack<T> x = Pack<T>::zero();
      if (kk < K && c < ld)
        x = (kk < ld) ? Pack<T>::load(KU + (long long)kk * ld + c)
                      : Pack<T>::load(KW + (long long)(kk - ld) * ld + c);
      x.store(&Bs[k][cv * N]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const long long row = r0 + ty + 16 * a;
    if (row >= n) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx + 16 * b;
      if (c < ld) Unew[row * ld + c] = acc[a][b];
    }
  }
}

}  // namespace

template <typename T>
op_status update(long long n, int ld, const T *U, const T *W, const T *KU, const T *KW, T *Unew,
                 cudaStream_t st) {
  const long long tiles = (long long)((ld + kCols - 1) / kCols) * ((n + kRows - 1) / kRows);
  if (tiles > 0x7fffffffll) {
    set_error("update: %lld tiles exceed the launch limit", tiles);
    return OP_ERR_ARG;
  }
  k_update<T><<<(unsigned)tiles, dim3(16, 16), 0, st>>>(n, ld, U, W, KU, KW, Unew);
  count_launch();
  OP_LAUNCH("k_update");
  return OP_OK;
}

template op_status update<float>(long long, int, const float *, const float *, const float *,
                                 const float *, float *, cudaStream_t);
template op_status update<double>(long long, int, const double *, const double *, const double *,
                                  const double *, double *, cudaStream_t);

}  // namespace opevo
