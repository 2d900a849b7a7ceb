// Learned warm start: the 3-level convolutional U-Net of opnet.h, its subspace
// loss, hand-written backward pass and Adam, all on the device.
//
// Every convolution is an implicit GEMM, on the tensor cores (conv_tc.cu, BF16 operands,
// the default for the forward and for the data gradients of layers with at most 128
// input channels) or on FP32 CUDA cores (k_conv below):
//   forward  out[m][co] = b[co] + sum_k A[m][k] W[k][co],  A[m][t Cin + ci] = X[m + off_t][ci]
//   dgrad    the same kernel on dZ with the tap-reversed, transposed weights
//            (dX[m][ci] = sum_t sum_co dZ[m - off_t][co] W[t][ci][co]);
//   wgrad    (FP32 CUDA cores) dW[k][co] = sum_m A[m][k] dZ[m][co] (split over point chunks, partials
//            summed in a fixed order), with a row of ones appended to A so that
//            the same pass yields db = sum_m dZ[m] as row K of the (K + 1) x Cout
//            block that W and b form in the parameter vector.
// The loss reuses the library's Gram kernel (G = Y^T Y, P = U*^T Y) and its
// rank-2p update kernel (dL/dY = Y K_Y + U* K_U); the p x p algebra between them
// is FP64 in one CTA.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "opnet.h"

namespace opevo {
namespace {

constexpr int kLayers = 11;
enum { L_E0A, L_E0, L_E1A, L_E1, L_B2A, L_B2, L_D1A, L_D1, L_D0A, L_D0, L_OUT };
constexpr int kCin = 4;
constexpr float kVScale = 6.0f;

struct Layer {
  int taps, cin, cout, grid;
  long long woff;  // offset of W in the parameter vector; b follows at woff + taps*cin*cout
};

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
struct Box {
  double lo[3], h[3], len[3];
};

__global__ void k_features(int N, Box bx, const double *__restrict__ V, float *__restrict__ X) {
  const long long n = (long long)N * N * N;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n;
       m += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(m % N), iy = (int)((m / N) % N), iz = (int)(m / ((long long)N * N));
    const int id[3] = {ix, iy, iz};
    X[m * kCin] = (float)(V[m] / kVScale);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double x = bx.lo[d] + (id[d] + 1.0) * bx.h[d];
      X[m * kCin + 1 + d] = (float)(2.0 * (x - bx.lo[d]) / bx.len[d] - 1.0);
    }
  }
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// Implicit-GEMM convolution.  CTA tile: 64 points x 64 output channels, K steps
// of 16; 256 threads with 4 x 4 outputs each (points tm + 16 i, channels tn + 16 j).
struct ConvArgs {
  const float *X;      // [n][cin]
  const float *W;      // [taps * cin][cout]
  const float *bias;   // [cout] or null
  float *Z;            // pre-activation [n][cout] or null
  float *A;            // silu(Z) [n][cout] or null
  int N, taps, cin, cout;
};

constexpr int CM = 64, CN = 64, CK = 16;

__global__ void __launch_bounds__(256) k_conv(ConvArgs a) {
  __shared__ float As[CK][CM + 4];
  __shared__ float Bs[CK][CN + 4];
  __shared__ int pc[3][CM];
  const int tid = threadIdx.x;
  const int N = a.N;
  const long long n = (long long)N * N * N;
  const long long m0 = (long long)blockIdx.x * CM;
  const int n0 = blockIdx.y * CN;
  if (tid < CM) {
    const long long m = m0 + tid;
    if (m < n) {
      pc[0][tid] = (int)(m % N);
      pc[1][tid] = (int)((m / N) % N);
      pc[2][tid] = (int)(m / ((long long)N * N));
    } else {
      pc[0][tid] = -4;  // marks a point past the end
    }
  }
  __syncthreads();
  const int K = a.taps * a.cin;
  const int tm = tid & 15, tn = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < K; k0 += CK) {
    {  // A: element (kk, mm), kk = tid & 15 (consecutive channels), mm = tid / 16 + 16 r
      const int kk = tid & 15, k = k0 + kk;
      int ci = k, dx = 0, dy = 0, dz = 0;
      if (a.taps == 27) {
        const int t = k / a.cin;
        ci = k - t * a.cin;
        dx = t % 3 - 1;
        dy = (t / 3) % 3 - 1;
        dz = t / 9 - 1;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int mm = (tid >> 4) + 16 * r;
        float v = 0.f;
        const int x = pc[0][mm] + dx, y = pc[1][mm] + dy, z = pc[2][mm] + dz;
        if (k < K && pc[0][mm] >= 0 && x >= 0 && x < N && y >= 0 && y < N && z >= 0 && z < N)
          v = __ldg(a.X + (((long long)z * N + y) * N + x) * a.cin + ci);
        As[kk][mm] = v;
      }
    }
    {  // B: row kk = tid / 16, channels (tid & 15) * 4 .. + 3
      const int kk = tid >> 4, cc = (tid & 15) * 4, k = k0 + kk;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int co = n0 + cc + e;
        Bs[kk][cc + e] = (k < K && co < a.cout) ? __ldg(a.W + (long long)k * a.cout + co) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < CK; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][tm + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tn + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long m = m0 + tm + 16 * i;
    if (m >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int co = n0 + tn + 16 * j;
      if (co >= a.cout) continue;
      const float z = acc[i][j] + (a.bias ? a.bias[co] : 0.f);
      if (a.Z) a.Z[m * a.cout + co] = z;
      if (a.A) a.A[m * a.cout + co] = silu(z);
    }
  }
}

// Wf[(taps-1-t) * cout + co][ci] = W[t * cin + ci][co]: the dgrad weights.
__global__ void k_flip(const float *__restrict__ W, int taps, int cin, int cout,
                       float *__restrict__ Wf) {
  const int total = taps * cin * cout;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int co = e % cout, ci = (e / cout) % cin, t = e / (cout * cin);
    Wf[((long long)(taps - 1 - t) * cout + co) * cin + ci] = W[e];
  }
}

// Partial weight gradients over one chunk of points:
//   part[s][k][co] = sum_{m in chunk s} A[m][k] dZ[m][co], k <= K (A[m][K] = 1).
// CTA tile: 64 k x 64 co, 16 points per step; thread tile 4 x 4 (k tk + 16 i, co tc + 16 j).
struct WgradArgs {
  const float *X;   // [n][cin]
  const float *dZ;  // [n][cout]
  float *part;      // [splits][K + 1][cout]
  int N, taps, cin, cout;
  long long chunk;  // points per split (multiple of 16)
};

__global__ void __launch_bounds__(256) k_wgrad(WgradArgs a) {
  __shared__ float As[16][64 + 4];  // [m][k]
  __shared__ float Bs[16][64 + 4];  // [m][co]
  const int tid = threadIdx.x;
  const int N = a.N;
  const long long n = (long long)N * N * N;
  const int K = a.taps * a.cin;
  const int kb = blockIdx.x * 64, cb = blockIdx.y * 64;
  const long long ms = (long long)blockIdx.z * a.chunk;
  long long me = ms + a.chunk;
  if (me > n) me = n;
  // this thread's A column: k = kb + (tid & 63), fixed for the whole kernel
  const int kl = tid & 63, k = kb + kl;
  int ci = k, dx = 0, dy = 0, dz = 0;
  if (a.taps == 27 && k < K) {
    const int t = k / a.cin;
    ci = k - t * a.cin;
    dx = t % 3 - 1;
    dy = (t / 3) % 3 - 1;
    dz = t / 9 - 1;
  }
  const int tk = tid & 15, tc = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (long long m0 = ms; m0 < me; m0 += 16) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {  // A: 16 points x 64 k
      const int mm = (tid >> 6) + 4 * r;
      const long long m = m0 + mm;
      float v = 0.f;
      if (m < me) {
        if (k < K) {
          const int x = (int)(m % N) + dx, y = (int)((m / N) % N) + dy,
                    z = (int)(m / ((long long)N * N)) + dz;
          if (x >= 0 && x < N && y >= 0 && y < N && z >= 0 && z < N)
            v = __ldg(a.X + (((long long)z * N + y) * N + x) * a.cin + ci);
        } else if (k == K) {
          v = 1.f;
        }
      }
      As[mm][kl] = v;
    }
    {  // B: 16 points x 64 channels of dZ
      const int mm = tid >> 4, cc = (tid & 15) * 4;
      const long long m = m0 + mm;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int co = cb + cc + e;
        Bs[mm][cc + e] = (m < me && co < a.cout) ? __ldg(a.dZ + m * a.cout + co) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int mm = 0; mm < 16; ++mm) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[mm][tk + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[mm][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *dst = a.part + (long long)blockIdx.z * (K + 1) * a.cout;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int kk = kb + tk + 16 * i;
    if (kk > K) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int co = cb + tc + 16 * j;
      if (co < a.cout) dst[(long long)kk * a.cout + co] = acc[i][j];
    }
  }
}

// out[e] = sum_s part[s][e] (fixed order, FP32 partials summed in FP64).
__global__ void k_reduce_parts(const float *__restrict__ part, int splits, long long count,
                               float *__restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += part[(long long)k * count + e];
    out[e] = (float)s;
  }
}

// dZ = dA * silu'(Z)
__global__ void k_silu_back(long long count, const float *__restrict__ dA,
                            const float *__restrict__ Z, float *__restrict__ dZ) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    dZ[e] = dA[e] * silu_grad(Z[e]);
}

// Coarse point (kx, ky, kz) of an M^3 grid <-> fine points (2kx + a, 2ky + b, 2kz + c).
__device__ __forceinline__ long long fine_index(int M, long long mc, int a, int b, int c) {
  const int kx = (int)(mc % M), ky = (int)((mc / M) % M), kz = (int)(mc / ((long long)M * M));
  const long long Nf = 2LL * M;
  return ((long long)(2 * kz + c) * Nf + (2 * ky + b)) * Nf + (2 * kx + a);
}

// dst[mc][c] = mean of the 8 fine src[.][c]  (src rows of C channels; coarse M^3)
__global__ void k_pool(int M, int C, const float *__restrict__ src, float *__restrict__ dst) {
  const long long total = (long long)M * M * M * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long mc = e / C;
    const int c = (int)(e % C);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += src[fine_index(M, mc, q & 1, (q >> 1) & 1, q >> 2) * C + c];
    dst[e] = 0.125f * s;
  }
}

// dst_fine[m][c] += src_coarse[mc][c] / 8 for the 8 fine points of every coarse point
__global__ void k_pool_back_add(int M, int C, const float *__restrict__ src,
                                float *__restrict__ dst) {
  const long long total = (long long)M * M * M * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long mc = e / C;
    const int c = (int)(e % C);
    const float g = 0.125f * src[e];
#pragma unroll
    for (int q = 0; q < 8; ++q) dst[fine_index(M, mc, q & 1, (q >> 1) & 1, q >> 2) * C + c] += g;
  }
}

// dst_fine[m][off + c] = src_coarse[parent(m)][c]  (dst rows of ldd channels)
__global__ void k_up(int M, int C, const float *__restrict__ src, float *__restrict__ dst,
                     int ldd, int off) {
  const long long total = (long long)M * M * M * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long mc = e / C;
    const int c = (int)(e % C);
    const float v = src[e];
#pragma unroll
    for (int q = 0; q < 8; ++q) dst[fine_index(M, mc, q & 1, (q >> 1) & 1, q >> 2) * ldd + off + c] = v;
  }
}

// dst_coarse[mc][c] = sum of the 8 fine src[.][off + c]  (src rows of lds channels)
__global__ void k_up_back(int M, int C, const float *__restrict__ src, int lds, int off,
                          float *__restrict__ dst) {
  const long long total = (long long)M * M * M * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long mc = e / C;
    const int c = (int)(e % C);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += src[fine_index(M, mc, q & 1, (q >> 1) & 1, q >> 2) * lds + off + c];
    dst[e] = s;
  }
}

// dst[m][doff + c] = src[m][soff + c], c < C  (row strides lds, ldd)
__global__ void k_copy_cols(long long n, int C, const float *__restrict__ src, int lds, int soff,
                            float *__restrict__ dst, int ldd, int doff) {
  const long long total = n * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long m = e / C;
    const int c = (int)(e % C);
    dst[m * ldd + doff + c] = src[m * lds + soff + c];
  }
}

// Loss coefficients from G = Y^T Y (Gd) and P = U*^T Y (Pd), ld x ld FP64:
//   L = 1 - ||P||^2 / b + gamma ||Gh - I||^2 / p^2,  b = tr G, Gh = p G / b, E = Gh - I
//   K_Y = 2 ||P||^2 / b^2 I + gamma 4 / (p b) (E - tr(E G) / b I),  K_U = -2 / b P
// (dL/dY = Y K_Y + U* K_U).  One CTA; K_Y, K_U are written as p x p FP32 (ld = p).
__global__ void k_loss_coeff(int p, int ld, const double *__restrict__ Gd,
                             const double *__restrict__ Pd, double gamma, double *out,
                             float *__restrict__ KY, float *__restrict__ KU) {
  __shared__ double red[3][256];
  const int tid = threadIdx.x;
  double tr = 0.0, pp = 0.0, gg = 0.0;
  for (int e = tid; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e % p;
    const double g = Gd[(long long)i * ld + j], q = Pd[(long long)i * ld + j];
    if (i == j) tr += g;
    pp += q * q;
    gg += g * g;
  }
  red[0][tid] = tr;
  red[1][tid] = pp;
  red[2][tid] = gg;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (tid < o)
      for (int c = 0; c < 3; ++c) red[c][tid] += red[c][tid + o];
    __syncthreads();
  }
  const double b = red[0][0], ppt = red[1][0], ggt = red[2][0];
  // ||E||^2 = p^2 ||G||^2 / b^2 - 2 p tr G / b + p = p^2 ||G||^2 / b^2 - p
  // tr(E G) = p ||G||^2 / b - b
  const double e2 = (double)p * p * ggt / (b * b) - p;
  const double teg = p * ggt / b - b;
  const double L = 1.0 - ppt / b + gamma * e2 / ((double)p * p);
  const double cI = 2.0 * ppt / (b * b) - gamma * 4.0 / (p * b) * (1.0 + teg / b);
  const double cG = gamma * 4.0 / (p * b) * (p / b);
  for (int e = tid; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e % p;
    const double g = Gd[(long long)i * ld + j];
    KY[e] = (float)(cG * g + (i == j ? cI : 0.0));
    KU[e] = (float)(-2.0 / b * Pd[(long long)i * ld + j]);
  }
  if (tid == 0) out[0] = L;
}

// Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; theta -= lr (m c1) / (sqrt(v c2) + eps),
// c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t).
__global__ void k_adam(long long count, float *__restrict__ theta, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.0f - b1) * gi;
    const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    theta[e] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

template <typename S, typename D>
__global__ void k_unpad_to(long long n, int p, int ld, const S *__restrict__ src,
                           D *__restrict__ dst) {
  const long long total = n * p;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / p;
    const int j = (int)(e % p);
    dst[e] = (D)src[i * ld + j];
  }
}

int ew_blocks(long long count) {
  long long b = (count + 255) / 256;
  const long long cap = (long long)num_sms() * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

op_status launch_unpad_to(long long n, int p, int ld, const void *src, int src_size, void *dst,
                          int dst_size, cudaStream_t st) {
  const int nb = ew_blocks(n * p);
  if (src_size == 8 && dst_size == 8)
    k_unpad_to<double, double><<<nb, 256, 0, st>>>(n, p, ld, (const double *)src, (double *)dst);
  else if (src_size == 8 && dst_size == 4)
    k_unpad_to<double, float><<<nb, 256, 0, st>>>(n, p, ld, (const double *)src, (float *)dst);
  else if (src_size == 4 && dst_size == 8)
    k_unpad_to<float, double><<<nb, 256, 0, st>>>(n, p, ld, (const float *)src, (double *)dst);
  else
    k_unpad_to<float, float><<<nb, 256, 0, st>>>(n, p, ld, (const float *)src, (float *)dst);
  count_launch();
  OP_LAUNCH("k_unpad_to");
  return OP_OK;
}

}  // namespace opevo

// ---------------------------------------------------------------------------
// The network object
// ---------------------------------------------------------------------------
using namespace opevo;

struct opnet {
  opnet_config cfg;
  int N, p, c0, c1, c2;
  int conv_kind;         // OPNET_CONV_*: the forward convolutions' arithmetic
  void *conv_ws;         // BF16 weights of the tensor-core convolution (one layer at a time)
  size_t conv_ws_bytes;
  int *dev_err;          // set when a bounded wait of a tensor-core kernel gives up
  long long n0, n1, n2;  // points at the three levels
  Layer L[kLayers];
  long long nparam;
  cudaStream_t st;
  std::vector<void *> allocs;
  // parameters, gradient, Adam moments
  float *theta, *grad, *am, *av;
  long long adam_t;
  // forward tensors
  float *x0, *pool0, *pool1, *cat1, *cat0, *Y;
  float *Z[kLayers], *A[kLayers];
  // backward scratch
  float *dA, *dZ, *dX, *ge0, *ge1, *gsm, *Wf, *part, *dY;
  long long part_floats;
  // loss
  void *gram_ws;
  size_t gram_bytes;
  double *Gd, *Pd, *dsc;  // dsc[0]: loss
  float *KY, *KU;
  double *hsc;            // pinned: loss readback
};

namespace {

op_status net_alloc(opnet *net, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("opnet: cudaMalloc of %zu bytes failed (%s)", bytes, cudaGetErrorString(e));
    return OP_ERR_OOM;
  }
  net->allocs.push_back(*p);
  return OP_OK;
}

template <typename T>
op_status net_alloc_n(opnet *net, T **p, long long count) {
  return net_alloc(net, (void **)p, (size_t)count * sizeof(T));
}

op_status conv(const opnet *net, const float *X, int layer_grid, int taps, int cin, int cout,
               const float *W, const float *bias, float *Z, float *A) {
  ConvArgs a;
  a.X = X;
  a.W = W;
  a.bias = bias;
  a.Z = Z;
  a.A = A;
  a.N = layer_grid;
  a.taps = taps;
  a.cin = cin;
  a.cout = cout;
  const long long n = (long long)layer_grid * layer_grid * layer_grid;
  const dim3 grid((unsigned)((n + CM - 1) / CM), (unsigned)((cout + CN - 1) / CN));
  k_conv<<<grid, 256, 0, net->st>>>(a);
  count_launch();
  OP_LAUNCH("k_conv");
  return OP_OK;
}

op_status fwd_layer(opnet *net, int i, const float *X) {
  const Layer &l = net->L[i];
  const float *W = net->theta + l.woff;
  const float *b = W + (long long)l.taps * l.cin * l.cout;
  if (net->conv_kind == OPNET_CONV_BF16_TC)
    return conv_bf16_tc(X, l.grid, l.taps, l.cin, l.cout, W, b, net->Z[i],
                        i == L_OUT ? nullptr : net->A[i], net->conv_ws, net->conv_ws_bytes,
                        net->dev_err, net->st);
  return conv(net, X, l.grid, l.taps, l.cin, l.cout, W, b, net->Z[i],
              i == L_OUT ? nullptr : net->A[i]);
}

op_status forward(opnet *net, const double *V) {
  cudaStream_t st = net->st;
  Box bx;
  for (int d = 0; d < 3; ++d) {
    bx.lo[d] = net->cfg.lo[d];
    bx.len[d] = net->cfg.hi[d] - net->cfg.lo[d];
    bx.h[d] = bx.len[d] / (net->N + 1);
  }
  k_features<<<ew_blocks(net->n0), 256, 0, st>>>(net->N, bx, V, net->x0);
  count_launch();
  OP_LAUNCH("k_features");
  const int N = net->N, c0 = net->c0, c1 = net->c1, c2 = net->c2;
  OP_TRY(fwd_layer(net, L_E0A, net->x0));
  OP_TRY(fwd_layer(net, L_E0, net->A[L_E0A]));
  k_pool<<<ew_blocks(net->n1 * c0), 256, 0, st>>>(N / 2, c0, net->A[L_E0], net->pool0);
  count_launch();
  OP_TRY(fwd_layer(net, L_E1A, net->pool0));
  OP_TRY(fwd_layer(net, L_E1, net->A[L_E1A]));
  k_pool<<<ew_blocks(net->n2 * c1), 256, 0, st>>>(N / 4, c1, net->A[L_E1], net->pool1);
  count_launch();
  OP_TRY(fwd_layer(net, L_B2A, net->pool1));
  OP_TRY(fwd_layer(net, L_B2, net->A[L_B2A]));
  k_up<<<ew_blocks(net->n2 * c2), 256, 0, st>>>(N / 4, c2, net->A[L_B2], net->cat1, c2 + c1, 0);
  count_launch();
  k_copy_cols<<<ew_blocks(net->n1 * c1), 256, 0, st>>>(net->n1, c1, net->A[L_E1], c1, 0,
                                                        net->cat1, c2 + c1, c2);
  count_launch();
  OP_TRY(fwd_layer(net, L_D1A, net->cat1));
  OP_TRY(fwd_layer(net, L_D1, net->A[L_D1A]));
  k_up<<<ew_blocks(net->n1 * c1), 256, 0, st>>>(N / 2, c1, net->A[L_D1], net->cat0, c1 + c0, 0);
  count_launch();
  k_copy_cols<<<ew_blocks(net->n0 * c0), 256, 0, st>>>(net->n0, c0, net->A[L_E0], c0, 0,
                                                        net->cat0, c1 + c0, c1);
  count_launch();
  OP_TRY(fwd_layer(net, L_D0A, net->cat0));
  OP_TRY(fwd_layer(net, L_D0, net->A[L_D0A]));
  OP_TRY(fwd_layer(net, L_OUT, net->A[L_D0]));  // Z[L_OUT] = Y
  OP_LAUNCH("opnet forward");
  return OP_OK;
}

// Data gradient of a convolution layer, the adjoint of its correlation:
//   dX[m][ci] = sum_t sum_co dZ[m - off_t][co] W[t cin + ci][co],
// as the forward convolution kernel on dZ with the tap-reversed, transposed weights
// (k_flip into Wf, taps * cin * cout floats of scratch).  OPNET_CONV_BF16_TC runs it on the
// tensor cores when cin <= 128 (the kernel's output-channel limit; BF16 operands, FP32
// accumulation), otherwise it runs on the FP32 CUDA cores.  tc_ws: scratch of
// conv_tc_scratch_bytes(taps, cout, cin) bytes for the tensor-core form.
op_status conv_dgrad(int kind, const float *dZ, int N, int taps, int cin, int cout,
                     const float *W, float *Wf, float *dX, void *tc_ws, size_t tc_bytes, int *err,
                     cudaStream_t st) {
  const long long K = (long long)taps * cin;
  k_flip<<<ew_blocks(K * cout), 256, 0, st>>>(W, taps, cin, cout, Wf);
  count_launch();
  OP_LAUNCH("k_flip");
  if (kind == OPNET_CONV_BF16_TC && cin <= 128)
    return conv_bf16_tc(dZ, N, taps, cout, cin, Wf, nullptr, dX, nullptr, tc_ws, tc_bytes, err,
                        st);
  ConvArgs a;
  a.X = dZ;
  a.W = Wf;
  a.bias = nullptr;
  a.Z = dX;
  a.A = nullptr;
  a.N = N;
  a.taps = taps;
  a.cin = cout;
  a.cout = cin;
  const long long n = (long long)N * N * N;
  k_conv<<<dim3((unsigned)((n + CM - 1) / CM), (unsigned)((cin + CN - 1) / CN)), 256, 0, st>>>(a);
  count_launch();
  OP_LAUNCH("k_conv");
  return OP_OK;
}

// Gradient of layer i's parameters from its input X and dZ; dX (if not null) = d loss / d X.
op_status back_layer(opnet *net, int i, const float *X, const float *dZ, float *dX) {
  const Layer &l = net->L[i];
  cudaStream_t st = net->st;
  const long long n = (long long)l.grid * l.grid * l.grid;
  const int K = l.taps * l.cin;
  long long chunk = 2048;
  int splits = (int)((n + chunk - 1) / chunk);
  while ((long long)splits * (K + 1) * l.cout > net->part_floats) {  // cannot happen for the
    chunk *= 2;                                                        // sizes allocated
    splits = (int)((n + chunk - 1) / chunk);
  }
  WgradArgs w;
  w.X = X;
  w.dZ = dZ;
  w.part = net->part;
  w.N = l.grid;
  w.taps = l.taps;
  w.cin = l.cin;
  w.cout = l.cout;
  w.chunk = chunk;
  const dim3 grid((unsigned)((K + 1 + 63) / 64), (unsigned)((l.cout + 63) / 64), (unsigned)splits);
  k_wgrad<<<grid, 256, 0, st>>>(w);
  count_launch();
  const long long cnt = (long long)(K + 1) * l.cout;
  k_reduce_parts<<<ew_blocks(cnt), 256, 0, st>>>(net->part, splits, cnt, net->grad + l.woff);
  count_launch();
  OP_LAUNCH("k_wgrad");
  if (dX)
    OP_TRY(conv_dgrad(net->conv_kind, dZ, l.grid, l.taps, l.cin, l.cout, net->theta + l.woff,
                      net->Wf, dX, net->conv_ws, net->conv_ws_bytes, net->dev_err, st));
  return OP_OK;
}

// dA is the gradient of layer i's activation: dZ = dA silu'(Z), then back_layer.
op_status back_act_layer(opnet *net, int i, const float *dA, const float *X, float *dX) {
  const Layer &l = net->L[i];
  const long long cnt = (long long)l.grid * l.grid * l.grid * l.cout;
  k_silu_back<<<ew_blocks(cnt), 256, 0, net->st>>>(cnt, dA, net->Z[i], net->dZ);
  count_launch();
  return back_layer(net, i, X, net->dZ, dX);
}

op_status backward(opnet *net) {
  cudaStream_t st = net->st;
  const int N = net->N, c0 = net->c0, c1 = net->c1, c2 = net->c2;
  // output layer: dY -> grad_out, d(d0)
  OP_TRY(back_layer(net, L_OUT, net->A[L_D0], net->dY, net->dA));
  // d0: dA -> dX = d(d0a)
  OP_TRY(back_act_layer(net, L_D0, net->dA, net->A[L_D0A], net->dX));
  // d0a: input cat0 = [up(d1), e0]; d cat0 -> dA (n0 x (c1 + c0))
  OP_TRY(back_act_layer(net, L_D0A, net->dX, net->cat0, net->dA));
  k_up_back<<<ew_blocks(net->n1 * c1), 256, 0, st>>>(N / 2, c1, net->dA, c1 + c0, 0, net->gsm);
  count_launch();
  k_copy_cols<<<ew_blocks(net->n0 * c0), 256, 0, st>>>(net->n0, c0, net->dA, c1 + c0, c1,
                                                        net->ge0, c0, 0);
  count_launch();
  // d1 (gradient in gsm), d1a: input cat1 = [up(b2), e1]
  OP_TRY(back_act_layer(net, L_D1, net->gsm, net->A[L_D1A], net->dX));
  OP_TRY(back_act_layer(net, L_D1A, net->dX, net->cat1, net->dA));
  k_up_back<<<ew_blocks(net->n2 * c2), 256, 0, st>>>(N / 4, c2, net->dA, c2 + c1, 0, net->gsm);
  count_launch();
  k_copy_cols<<<ew_blocks(net->n1 * c1), 256, 0, st>>>(net->n1, c1, net->dA, c2 + c1, c2,
                                                        net->ge1, c1, 0);
  count_launch();
  // b2, b2a: input pool(e1)
  OP_TRY(back_act_layer(net, L_B2, net->gsm, net->A[L_B2A], net->dX));
  OP_TRY(back_act_layer(net, L_B2A, net->dX, net->pool1, net->dA));
  k_pool_back_add<<<ew_blocks(net->n2 * c1), 256, 0, st>>>(N / 4, c1, net->dA, net->ge1);
  count_launch();
  // e1, e1a: input pool(e0)
  OP_TRY(back_act_layer(net, L_E1, net->ge1, net->A[L_E1A], net->dX));
  OP_TRY(back_act_layer(net, L_E1A, net->dX, net->pool0, net->dA));
  k_pool_back_add<<<ew_blocks(net->n1 * c0), 256, 0, st>>>(N / 2, c0, net->dA, net->ge0);
  count_launch();
  // e0, e0a (the input features need no gradient)
  OP_TRY(back_act_layer(net, L_E0, net->ge0, net->A[L_E0A], net->dX));
  OP_TRY(back_act_layer(net, L_E0A, net->dX, net->x0, nullptr));
  OP_LAUNCH("opnet backward");
  return OP_OK;
}

// loss into net->dsc[0]; dY when want_grad
op_status loss(opnet *net, const float *Us, double gamma, bool want_grad) {
  const int p = net->p;
  const float *Y = net->Z[L_OUT];
  OP_TRY(gram<float>(net->n0, p, p, Y, Us, net->Pd, nullptr, net->Gd, net->gram_ws,
                     net->gram_bytes, net->st));
  k_loss_coeff<<<1, 256, 0, net->st>>>(p, p, net->Gd, net->Pd, gamma, net->dsc, net->KY, net->KU);
  count_launch();
  OP_LAUNCH("k_loss_coeff");
  if (want_grad) OP_TRY(update<float>(net->n0, p, Y, Us, net->KY, net->KU, net->dY, net->st));
  return OP_OK;
}

// After the stream has been synchronised: a tensor-core kernel that gave up a bounded wait.
op_status check_dev_err(opnet *net) {
  int h = 0;
  OP_CUDA(cudaMemcpy(&h, net->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    OP_CUDA(cudaMemset(net->dev_err, 0, sizeof(int)));
    set_error("opnet: a tensor-core convolution gave up a bounded device wait");
    return OP_ERR_TIMEOUT;
  }
  return OP_OK;
}

op_status read_loss(opnet *net, double *out) {
  OP_CUDA(cudaMemcpyAsync(net->hsc, net->dsc, sizeof(double), cudaMemcpyDeviceToHost, net->st));
  OP_CUDA(cudaStreamSynchronize(net->st));
  OP_TRY(check_dev_err(net));
  if (out) *out = net->hsc[0];
  if (!isfinite(net->hsc[0])) {
    set_error("opnet: non-finite loss");
    return OP_ERR_DIVERGED;
  }
  return OP_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

extern "C" {

op_status opnet_create(opnet **out, const opnet_config *cfg) {
  if (!out || !cfg) {
    set_error("opnet_create: null argument");
    return OP_ERR_ARG;
  }
  *out = nullptr;
  const int N = cfg->N, p = cfg->p;
  bool ok = N >= 4 && N <= 512 && N % 4 == 0 && p >= 8 && p <= 128 && p % 8 == 0;
  for (int d = 0; d < 3; ++d) {
    ok = ok && cfg->width[d] >= 1 && cfg->width[d] <= 128;
    ok = ok && isfinite(cfg->lo[d]) && isfinite(cfg->hi[d]) && cfg->hi[d] > cfg->lo[d];
  }
  if (!ok) {
    set_error("opnet_create: need N %% 4 == 0 in [4, 512], p %% 8 == 0 in [8, 128], widths "
              "in [1, 128], lo < hi");
    return OP_ERR_ARG;
  }
  opnet *net = new opnet();
  net->cfg = *cfg;
  net->N = N;
  net->p = p;
  net->c0 = cfg->width[0];
  net->c1 = cfg->width[1];
  net->c2 = cfg->width[2];
  net->st = (cudaStream_t)cfg->stream;
  net->n0 = (long long)N * N * N;
  net->n1 = net->n0 / 8;
  net->n2 = net->n1 / 8;
  const int c0 = net->c0, c1 = net->c1, c2 = net->c2;
  const int shapes[kLayers][4] = {
      {27, kCin, c0, N},         {27, c0, c0, N},     {27, c0, c1, N / 2}, {27, c1, c1, N / 2},
      {27, c1, c2, N / 4},       {27, c2, c2, N / 4}, {27, c2 + c1, c1, N / 2},
      {27, c1, c1, N / 2},       {27, c1 + c0, c1, N}, {27, c1, c1, N}, {1, c1, p, N}};
  long long off = 0, max_wf = 0, max_part = 0;
  for (int i = 0; i < kLayers; ++i) {
    Layer &l = net->L[i];
    l.taps = shapes[i][0];
    l.cin = shapes[i][1];
    l.cout = shapes[i][2];
    l.grid = shapes[i][3];
    l.woff = off;
    const long long K = (long long)l.taps * l.cin;
    off += K * l.cout + l.cout;
    if (K * l.cout > max_wf) max_wf = K * l.cout;
    const long long n = (long long)l.grid * l.grid * l.grid;
    const long long splits = (n + 2047) / 2048;
    if (splits * (K + 1) * l.cout > max_part) max_part = splits * (K + 1) * l.cout;
  }
  net->nparam = off;
  net->part_floats = max_part;
  const long long n0 = net->n0, n1 = net->n1, n2 = net->n2;
  int wide = c1 + c0;
  if (p > wide) wide = p;
  if (c2 + c1 > wide) wide = c2 + c1;  // coarser, but keep one size for the scratch
  op_status s = OP_OK;
#define NET_ALLOC(ptr, count) \
  if (s == OP_OK) s = net_alloc_n(net, &(ptr), (count))
  NET_ALLOC(net->theta, off);
  NET_ALLOC(net->grad, off);
  NET_ALLOC(net->am, off);
  NET_ALLOC(net->av, off);
  NET_ALLOC(net->x0, n0 * kCin);
  NET_ALLOC(net->pool0, n1 * c0);
  NET_ALLOC(net->pool1, n2 * c1);
  NET_ALLOC(net->cat1, n1 * (c2 + c1));
  NET_ALLOC(net->cat0, n0 * (c1 + c0));
  for (int i = 0; i < kLayers; ++i) {
    const Layer &l = net->L[i];
    const long long n = (long long)l.grid * l.grid * l.grid;
    NET_ALLOC(net->Z[i], n * l.cout);
    if (i != L_OUT) NET_ALLOC(net->A[i], n * l.cout);
    else net->A[i] = nullptr;
  }
  NET_ALLOC(net->dA, n0 * wide);
  NET_ALLOC(net->dZ, n0 * wide);
  NET_ALLOC(net->dX, n0 * wide);
  NET_ALLOC(net->ge0, n0 * c0);
  NET_ALLOC(net->ge1, n1 * c1);
  NET_ALLOC(net->gsm, n1 * (c1 > c2 ? c1 : c2));
  NET_ALLOC(net->Wf, max_wf);
  NET_ALLOC(net->part, max_part);
  NET_ALLOC(net->dY, n0 * p);
  NET_ALLOC(net->Gd, (long long)p * p);
  NET_ALLOC(net->Pd, (long long)p * p);
  NET_ALLOC(net->dsc, 8);
  NET_ALLOC(net->KY, (long long)p * p);
  NET_ALLOC(net->KU, (long long)p * p);
  NET_ALLOC(net->dev_err, 4);
#undef NET_ALLOC
  if (s == OP_OK) {
    net->gram_bytes = gram_workspace_bytes(n0, p, 4);
    s = net_alloc(net, &net->gram_ws, net->gram_bytes);
  }
  if (s == OP_OK) {
    // the tensor-core convolutions (the default): scratch for the widest layer's weights
    net->conv_kind = OPNET_CONV_BF16_TC;
    net->conv_ws_bytes = 0;
    for (int i = 0; i < kLayers; ++i) {
      const Layer &l = net->L[i];
      net->conv_ws_bytes =
          std::max(net->conv_ws_bytes, conv_tc_scratch_bytes(l.taps, l.cin, l.cout));
      // the tensor-core data gradient: the same kernel with cin and cout exchanged
      if (l.cin <= 128)
        net->conv_ws_bytes =
            std::max(net->conv_ws_bytes, conv_tc_scratch_bytes(l.taps, l.cout, l.cin));
    }
    s = net_alloc(net, &net->conv_ws, net->conv_ws_bytes);
  }
  if (s == OP_OK) {
    const cudaError_t e = cudaMemsetAsync(net->dev_err, 0, 4 * sizeof(int), net->st);
    if (e != cudaSuccess) s = cuda_status(e, "opnet_create: memset");
  }
  if (s == OP_OK && cudaMallocHost((void **)&net->hsc, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_error("opnet_create: pinned allocation failed");
    s = OP_ERR_OOM;
  }
  if (s == OP_OK) {
    const cudaError_t e = cudaMemsetAsync(net->theta, 0, (size_t)off * sizeof(float), net->st);
    if (e != cudaSuccess) s = cuda_status(e, "opnet_create: memset");
  }
  if (s == OP_OK) {
    cudaMemsetAsync(net->am, 0, (size_t)off * sizeof(float), net->st);
    cudaMemsetAsync(net->av, 0, (size_t)off * sizeof(float), net->st);
    const cudaError_t e = cudaStreamSynchronize(net->st);
    if (e != cudaSuccess) s = cuda_status(e, "opnet_create: synchronise");
  }
  if (s != OP_OK) {
    opnet_destroy(net);
    return s;
  }
  net->adam_t = 0;
  *out = net;
  return OP_OK;
}

long long opnet_param_count(const opnet *net) { return net ? net->nparam : -1; }

op_status opnet_layer(const opnet *net, int i, int *taps, int *cin, int *cout) {
  if (!net || i < 0 || i >= kLayers || !taps || !cin || !cout) {
    set_error("opnet_layer: null argument or layer index out of range");
    return OP_ERR_ARG;
  }
  *taps = net->L[i].taps;
  *cin = net->L[i].cin;
  *cout = net->L[i].cout;
  return OP_OK;
}

op_status opnet_set_params(opnet *net, const float *theta, long long count) {
  if (!net || !theta || count != net->nparam) {
    set_error("opnet_set_params: null argument or count != opnet_param_count");
    return OP_ERR_ARG;
  }
  OP_CUDA(cudaMemcpyAsync(net->theta, theta, (size_t)count * sizeof(float),
                          cudaMemcpyHostToDevice, net->st));
  OP_CUDA(cudaMemsetAsync(net->am, 0, (size_t)count * sizeof(float), net->st));
  OP_CUDA(cudaMemsetAsync(net->av, 0, (size_t)count * sizeof(float), net->st));
  OP_CUDA(cudaStreamSynchronize(net->st));
  net->adam_t = 0;
  return OP_OK;
}

op_status opnet_get_params(opnet *net, float *theta, long long count) {
  if (!net || !theta || count != net->nparam) {
    set_error("opnet_get_params: null argument or count != opnet_param_count");
    return OP_ERR_ARG;
  }
  OP_CUDA(cudaMemcpyAsync(theta, net->theta, (size_t)count * sizeof(float),
                          cudaMemcpyDeviceToHost, net->st));
  OP_CUDA(cudaStreamSynchronize(net->st));
  return OP_OK;
}

op_status opnet_forward(opnet *net, const double *V, float *Y) {
  if (!net || !V || !Y || !aligned16(Y)) {
    set_error("opnet_forward: null or unaligned pointer");
    return OP_ERR_ARG;
  }
  OP_TRY(forward(net, V));
  OP_CUDA(cudaMemcpyAsync(Y, net->Z[L_OUT], (size_t)net->n0 * net->p * sizeof(float),
                          cudaMemcpyDeviceToDevice, net->st));
  OP_CUDA(cudaStreamSynchronize(net->st));
  return check_dev_err(net);
}

op_status opnet_infer(opnet *net, const double *V, double *U0) {
  if (!net || !V || !U0 || !aligned16(U0)) {
    set_error("opnet_infer: null or unaligned pointer");
    return OP_ERR_ARG;
  }
  OP_TRY(forward(net, V));
  OP_TRY(launch_unpad_to(net->n0, net->p, net->p, net->Z[L_OUT], 4, U0, 8, net->st));
  OP_CUDA(cudaStreamSynchronize(net->st));
  return check_dev_err(net);
}

op_status opnet_conv(int kind, const float *X, int N, int taps, int cin, int cout,
                     const float *W, const float *bias, float *Z, float *A, void *stream) {
  if (!X || !W || (!Z && !A) || N < 1 || N > 512 || (taps != 1 && taps != 27) || cin < 1 ||
      cin > 512 || cout < 1 || cout > 128 ||
      (kind != OPNET_CONV_FP32 && kind != OPNET_CONV_BF16_TC)) {
    set_error("opnet_conv: bad arguments");
    return OP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (kind == OPNET_CONV_FP32) {
    ConvArgs a;
    a.X = X;
    a.W = W;
    a.bias = bias;
    a.Z = Z;
    a.A = A;
    a.N = N;
    a.taps = taps;
    a.cin = cin;
    a.cout = cout;
    const long long n = (long long)N * N * N;
    k_conv<<<dim3((unsigned)((n + CM - 1) / CM), (unsigned)((cout + CN - 1) / CN)), 256, 0, st>>>(a);
    count_launch();
    OP_LAUNCH("k_conv");
    OP_CUDA(cudaStreamSynchronize(st));
    return OP_OK;
  }
  const size_t wb = conv_tc_scratch_bytes(taps, cin, cout);
  void *ws = nullptr;
  OP_CUDA(cudaMalloc(&ws, wb + 256));
  int *err = (int *)((char *)ws + wb);
  auto ck = [](cudaError_t e, const char *what) {
    return e == cudaSuccess ? OP_OK : cuda_status(e, what);
  };
  op_status s = ck(cudaMemsetAsync(err, 0, sizeof(int), st), "opnet_conv: memset");
  if (s == OP_OK) s = conv_bf16_tc(X, N, taps, cin, cout, W, bias, Z, A, ws, wb, err, st);
  int h = 0;
  if (s == OP_OK) s = ck(cudaStreamSynchronize(st), "opnet_conv");
  if (s == OP_OK) s = ck(cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost), "opnet_conv");
  cudaFree(ws);
  if (s == OP_OK && h) {
    set_error("opnet_conv: a bounded device wait gave up");
    s = OP_ERR_TIMEOUT;
  }
  return s;
}

op_status opnet_conv_dgrad(int kind, const float *dZ, int N, int taps, int cin, int cout,
                           const float *W, float *dX, void *stream) {
  if (!dZ || !W || !dX || N < 1 || N > 512 || (taps != 1 && taps != 27) || cin < 1 ||
      cin > 512 || cout < 1 || cout > 512 ||
      (kind != OPNET_CONV_FP32 && kind != OPNET_CONV_BF16_TC) || ((uintptr_t)dZ & 15)) {
    set_error("opnet_conv_dgrad: bad arguments");
    return OP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t wf = ((size_t)taps * cin * cout * sizeof(float) + 255) / 256 * 256;
  const size_t wb = conv_tc_scratch_bytes(taps, cout, cin);
  void *ws = nullptr;
  OP_CUDA(cudaMalloc(&ws, wf + wb + 256));
  float *Wf = (float *)ws;
  void *tc = (char *)ws + wf;
  int *err = (int *)((char *)ws + wf + wb);
  auto ck = [](cudaError_t e, const char *what) {
    return e == cudaSuccess ? OP_OK : cuda_status(e, what);
  };
  op_status s = ck(cudaMemsetAsync(err, 0, sizeof(int), st), "opnet_conv_dgrad: memset");
  if (s == OP_OK) s = conv_dgrad(kind, dZ, N, taps, cin, cout, W, Wf, dX, tc, wb, err, st);
  int h = 0;
  if (s == OP_OK) s = ck(cudaStreamSynchronize(st), "opnet_conv_dgrad");
  if (s == OP_OK)
    s = ck(cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost), "opnet_conv_dgrad");
  cudaFree(ws);
  if (s == OP_OK && h) {
    set_error("opnet_conv_dgrad: a bounded device wait gave up");
    s = OP_ERR_TIMEOUT;
  }
  return s;
}

op_status opnet_set_conv(opnet *net, int kind) {
  if (!net || (kind != OPNET_CONV_FP32 && kind != OPNET_CONV_BF16_TC)) {
    set_error("opnet_set_conv: null net or unknown kind %d", kind);
    return OP_ERR_ARG;
  }
  net->conv_kind = kind;
  return OP_OK;
}

op_status opnet_loss_grad(opnet *net, const double *V, const float *Us, double gamma,
                          double *out, float *grad, long long count) {
  if (!net || !V || !Us || !out || !aligned16(Us) || !(gamma >= 0.0) ||
      (grad && count != net->nparam)) {
    set_error("opnet_loss_grad: bad arguments");
    return OP_ERR_ARG;
  }
  OP_TRY(forward(net, V));
  OP_TRY(loss(net, Us, gamma, grad != nullptr));
  if (grad) {
    OP_TRY(backward(net));
    OP_CUDA(cudaMemcpyAsync(grad, net->grad, (size_t)count * sizeof(float),
                            cudaMemcpyDeviceToHost, net->st));
  }
  return read_loss(net, out);
}

op_status opnet_train_step(opnet *net, const double *V, const float *Us, double gamma, double lr,
                           double beta1, double beta2, double eps, double *out) {
  if (!net || !V || !Us || !aligned16(Us) || !(gamma >= 0.0) || !(lr > 0.0) ||
      !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0)) {
    set_error("opnet_train_step: bad arguments");
    return OP_ERR_ARG;
  }
  OP_TRY(forward(net, V));
  OP_TRY(loss(net, Us, gamma, true));
  OP_TRY(backward(net));
  const long long t = ++net->adam_t;
  const double c1 = 1.0 / (1.0 - pow(beta1, (double)t)), c2 = 1.0 / (1.0 - pow(beta2, (double)t));
  k_adam<<<ew_blocks(net->nparam), 256, 0, net->st>>>(net->nparam, net->theta, net->grad, net->am,
                                                      net->av, (float)lr, (float)beta1,
                                                      (float)beta2, (float)eps, (float)c1,
                                                      (float)c2);
  count_launch();
  OP_LAUNCH("k_adam");
  return read_loss(net, out);
}

void opnet_destroy(opnet *net) {
  if (!net) return;
  if (net->st) cudaStreamSynchronize(net->st);
  else cudaDeviceSynchronize();
  for (void *p : net->allocs) cudaFree(p);
  if (net->hsc) cudaFreeHost(net->hsc);
  delete net;
}

}  // extern "C"
