// Shared device/host helpers of the opevo CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "opevo.h"

namespace opevo {

// ---------------------------------------------------------------------------
// Error reporting (thread-local message returned by op_last_error()).
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
op_status cuda_status(cudaError_t e, const char *what);

#define OP_CUDA(call)                                                    \
  do {                                                                   \
    cudaError_t _e = (call);                                             \
    if (_e != cudaSuccess) return ::opevo::cuda_status(_e, #call);       \
  } while (0)

#define OP_LAUNCH(what)                                                  \
  do {                                                                   \
    cudaError_t _e = cudaGetLastError();                                 \
    if (_e != cudaSuccess) return ::opevo::cuda_status(_e, what);        \
  } while (0)

#define OP_TRY(expr)                                                     \
  do {                                                                   \
    op_status _s = (expr);                                               \
    if (_s != OP_OK) return _s;                                          \
  } while (0)

// ---------------------------------------------------------------------------
// Geometry of the finite-difference operator -1/2 Delta_h + diag(V).
// Row i of H + sigma:  (V_i + cdiag + sigma) x_i - sum_d c_d (x_{i-e_d} + x_{i+e_d}),
// cdiag = sum_d 1/h_d^2, c_d = 1/(2 h_d^2); neighbours outside the grid are zero.
// ---------------------------------------------------------------------------
struct Geom {
  int dim;
  int nx, ny, nz;
  long long n;
  double cdiag;
  double c[3];
};

op_status make_geom(const op_problem *pb, Geom *g);

// Number of kernels this library has launched (process-wide).
void count_launch();
void count_launches(long long k);
long long launches_so_far();

// 16-byte vector of T: float4 / double2.
template <typename T> struct V16;
template <> struct V16<float> {
  using type = float4;
  static constexpr int N = 4;
};
template <> struct V16<double> {
  using type = double2;
  static constexpr int N = 2;
};

template <typename T> struct Pack {
  static constexpr int N = V16<T>::N;
  T v[N];
  __device__ __forceinline__ static Pack load(const T *p) {
    Pack r;
    typename V16<T>::type x = __ldg(reinterpret_cast<const typename V16<T>::type *>(p));
    const T *s = reinterpret_cast<const T *>(&x);
#pragma unroll
    for (int k = 0; k < N; ++k) r.v[k] = s[k];
    return r;
  }
  __device__ __forceinline__ static Pack load_rw(const T *p) {
    Pack r;
    typename V16<T>::type x = *reinterpret_cast<const typename V16<T>::type *>(p);
    const T *s = reinterpret_cast<const T *>(&x);
#pragma unroll
    for (int k = 0; k < N; ++k) r.v[k] = s[k];
    return r;
  }
  __device__ __forceinline__ void store(T *p) const {
    typename V16<T>::type x;
    T *d = reinterpret_cast<T *>(&x);
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = v[k];
    *reinterpret_cast<typename V16<T>::type *>(p) = x;
  }
  __device__ __forceinline__ static Pack zero() {
    Pack r;
#pragma unroll
    for (int k = 0; k < N; ++k) r.v[k] = T(0);
    return r;
  }
};

// Launch-shape helper for "one thread per 16-byte vector of a grid point's row":
// block = (bx, rows), bx = min(nv, 256) vectors of a row; gridDim.y = gy column
// chunks when a row has more than 256 vectors.
struct RowShape {
  int nv;      // vectors per row (ld / N)
  dim3 block;  // (bx, rows per block)
  int rows;    // rows per block
  int gy;      // column chunks
};
// Blocks of the row kernels: up to kRowChunk vectors of a row (512 bytes) by as many rows
// as make 256 threads; wider blocks go as column chunks (grid.y), each chunk's CTAs
// resident together and sweeping the grid points in order, so that the rows a stencil
// reads one z plane away are still in L2 (a z plane of one chunk: nx ny 512 bytes).
constexpr int kRowChunk = 32;
inline RowShape row_shape(int ld, int vec) {
  RowShape s;
  s.nv = ld / vec;
  int bx = s.nv < kRowChunk ? s.nv : kRowChunk;
  int by = 256 / bx;
  if (by < 1) by = 1;
  s.block = dim3(bx, by, 1);
  s.rows = by;
  s.gy = (s.nv + bx - 1) / bx;
  return s;
}

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, looked
// up once per device; 152 on GB300, also the answer when no device can be queried).  Sizes
// grids and split counts, and with them the workspace sizes derived from it.
int num_sms();

// NVTX range over a host scope (the enqueue of one phase); profilers that record
// NVTX attribute the phase's kernels to it.  Costs a few ns when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

}  // namespace opevo
