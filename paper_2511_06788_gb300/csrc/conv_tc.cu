// Forward convolution of the learned warm start (opnet.h) on the tensor cores: an
// implicit GEMM with BF16 operands and FP32 accumulation in TMEM (tcgen05.mma
// kind::f16), bias and SiLU in the epilogue.
//
//   out[m][co] = b[co] + sum_k A[m][k] W[k][co],   A[m][t Cin + ci] = X[m + off_t][ci]
//
// with X channels-last [point][ci] on an N^3 grid, taps t = (dz+1) 9 + (dy+1) 3 + (dx+1)
// (27 taps, zero outside the grid) or the point itself (1 tap).
//
// Tiling: one CTA per 128 grid points (the MMA's M), all output channels at once
// (N = Cout rounded up to 16, at most 128), K in slabs of 64 (one 128-byte row of BF16
// per operand row, 128-byte swizzled K-major).  The 256 threads gather a slab of A
// (converting FP32 to BF16, round to nearest) and copy the slab of the weights, which a
// small kernel has laid out once per call as BF16 [Cout][K] (zero padded); one thread
// issues the four K = 16 MMAs of the slab.  Two slabs are staged in turn: the gather of
// slab s + 1 runs while the tensor core works on slab s.  Every wait is bounded; a wait
// that gives up sets the error word and the CTA writes nothing.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace opevo {
namespace {

constexpr int kCM = 128;                 // points per CTA (MMA M)
constexpr int kCK = 64;                  // K per slab (BF16: 128 bytes per operand row)
constexpr int kAPiece = kCM * 128;       // 16 KB
constexpr int kBMax = 128 * 128;         // up to 128 output channels x 128 bytes
constexpr int kCStage = kAPiece + kBMax;
constexpr int kCSmem = 2 * kCStage + 1024;

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Wt[co][k] = bf16(W[k][co]) for co < cout, k < K; zero in the padding (co < coutp, k < Kp).
__global__ void k_conv_wt(const float *__restrict__ W, int K, int cout, int Kp, int coutp,
                          uint16_t *__restrict__ Wt) {
  const long long total = (long long)coutp * Kp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int co = (int)(e / Kp), k = (int)(e % Kp);
    const float w = (co < cout && k < K) ? W[(long long)k * cout + co] : 0.f;
    Wt[e] = (uint16_t)bf16_bits(w);
  }
}

struct ConvTc {
  const float *X;       // [n][cin]
  const uint16_t *Wt;   // [coutp][Kp] BF16
  const float *bias;    // [cout] or null
  float *Z, *A;         // [n][cout] each, or null
  int N, taps, cin, cout, coutp, K, Kp;
  int *err;
};

// Eight consecutive K values k0 .. k0 + 7 of operand row (point) m, as four BF16 pairs.
__device__ __forceinline__ uint4 gather8(const ConvTc &a, int x, int y, int z, bool in, int k0) {
  float v[8];
  if (in && a.cin % 8 == 0 && k0 < a.K) {
    // one tap, eight consecutive channels (k0 and cin are multiples of 8)
    const int t = k0 / a.cin, ci = k0 - t * a.cin;
    int dx = 0, dy = 0, dz = 0;
    if (a.taps == 27) {
      dx = t % 3 - 1;
      dy = (t / 3) % 3 - 1;
      dz = t / 9 - 1;
    }
    const int xx = x + dx, yy = y + dy, zz = z + dz;
    if (xx >= 0 && xx < a.N && yy >= 0 && yy < a.N && zz >= 0 && zz < a.N) {
      const float4 *src = reinterpret_cast<const float4 *>(
          a.X + (((long long)zz * a.N + yy) * a.N + xx) * a.cin + ci);
      const float4 p = __ldg(src), q = __ldg(src + 1);
      v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
      v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = 0.f;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + e;
      float w = 0.f;
      if (in && k < a.K) {
        const int t = k / a.cin, ci = k - t * a.cin;
        int dx = 0, dy = 0, dz = 0;
        if (a.taps == 27) {
          dx = t % 3 - 1;
          dy = (t / 3) % 3 - 1;
          dz = t / 9 - 1;
        }
        const int xx = x + dx, yy = y + dy, zz = z + dz;
        if (xx >= 0 && xx < a.N && yy >= 0 && yy < a.N && zz >= 0 && zz < a.N)
          w = __ldg(a.X + (((long long)zz * a.N + yy) * a.N + xx) * a.cin + ci);
      }
      v[e] = w;
    }
  }
  return make_uint4(bf16_bits(v[0]) | (bf16_bits(v[1]) << 16), bf16_bits(v[2]) | (bf16_bits(v[3]) << 16),
                    bf16_bits(v[4]) | (bf16_bits(v[5]) << 16), bf16_bits(v[6]) | (bf16_bits(v[7]) << 16));
}

__global__ void __launch_bounds__(256) k_conv_tc(const ConvTc a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const long long n = (long long)a.N * a.N * a.N;
  const long long m0 = (long long)blockIdx.x * kCM;
  const uint32_t ncols = a.coutp <= 32 ? 32u : (a.coutp <= 64 ? 64u : 128u);

  if (warp == 0) tc::tmem_alloc(&tmem_sh, ncols);
  if (t == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
    abort_sh = 0;
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t idesc = tc::idesc_bf16(kCM, a.coutp);

  // this thread's four A chunks: rows r = (t + 256 i) / 8, 16-byte chunk kc = t % 8
  const int kc = t & 7;
  int px[4], py[4], pz[4];
  bool pin[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = (t >> 3) + 32 * i;
    const long long m = m0 + r;
    pin[i] = m < n;
    const long long mm = pin[i] ? m : 0;
    px[i] = (int)(mm % a.N);
    py[i] = (int)((mm / a.N) % a.N);
    pz[i] = (int)(mm / ((long long)a.N * a.N));
  }
  const int nslab = a.Kp / kCK;
  bool ok = true;
  for (int s = 0; s < nslab && ok; ++s) {
    const int b = s & 1;
    uint8_t *As = smem + b * kCStage, *Bs = As + kAPiece;
    if (s >= 2) {
      // the MMAs of slab s - 2 read this buffer
      if (t == 0 && !tc::mbar_wait(&mbar[b], (uint32_t)(((s - 2) >> 1) & 1))) abort_sh = 1;
      __syncthreads();
      if (abort_sh) {
        ok = false;
        break;
      }
    }
    const int k0 = s * kCK;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = (t >> 3) + 32 * i;
      const uint4 c = gather8(a, px[i], py[i], pz[i], pin[i], k0 + 8 * kc);
      *reinterpret_cast<uint4 *>(As + tc::sw128_offset(r, kc)) = c;
    }
    for (int c = t; c < a.coutp * 8; c += 256) {
      const int co = c >> 3, kk = c & 7;
      const uint4 w = __ldg(reinterpret_cast<const uint4 *>(a.Wt + (long long)co * a.Kp + k0 + 8 * kk));
      *reinterpret_cast<uint4 *>(Bs + tc::sw128_offset(co, kk)) = w;
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc::tc_fence_after();
      const uint32_t ab = tc::smem_u32(As), bb = tc::smem_u32(Bs);
#pragma unroll
      for (int ks = 0; ks < kCK / 16; ++ks)
        tc::mma_bf16(tmem, tc::desc_sw128(ab + ks * 32), tc::desc_sw128(bb + ks * 32), idesc,
                     (s > 0 || ks > 0) ? 1u : 0u);
      tc::mma_commit(&mbar[b]);
    }
  }
  // the last slab's MMAs complete after all the others
  if (ok && nslab > 0) {
    const int s = nslab - 1;
    if (t == 0 && !tc::mbar_wait(&mbar[s & 1], (uint32_t)((s >> 1) & 1))) abort_sh = 1;
  }
  __syncthreads();
  if (ok && !abort_sh) {
    tc::tc_fence_after();
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows), columns of its half
    const int q = warp & 3, h = warp >> 2, half = a.coutp / 2;
    const long long m = m0 + q * 32 + lane;
    for (int c0 = h * half; c0 < (h + 1) * half; c0 += 8) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
      if (m < n) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int co = c0 + j;
          if (co >= a.cout) continue;
          const float z = v[j] + (a.bias ? a.bias[co] : 0.f);
          if (a.Z) a.Z[m * a.cout + co] = z;
          if (a.A) a.A[m * a.cout + co] = z / (1.0f + expf(-z));
        }
      }
    }
  } else if (t == 0) {
    atomicExch(a.err, 1);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, ncols);
  }
}

}  // namespace

size_t conv_tc_scratch_bytes(int taps, int cin, int cout) {
  const long long Kp = ((long long)taps * cin + kCK - 1) / kCK * kCK;
  const long long coutp = (cout + 15) / 16 * 16;
  return (size_t)(Kp * coutp * 2 + 255) / 256 * 256;
}

op_status conv_bf16_tc(const float *X, int N, int taps, int cin, int cout, const float *W,
                       const float *bias, float *Z, float *A, void *scratch, size_t scratch_bytes,
                       int *err, cudaStream_t st) {
  if (!X || !W || !scratch || !err || N < 1 || (taps != 1 && taps != 27) || cin < 1 ||
      cout < 1 || cout > 128 || scratch_bytes < conv_tc_scratch_bytes(taps, cin, cout) ||
      ((uintptr_t)scratch & 15) != 0) {
    set_error("conv_bf16_tc: bad arguments (N=%d taps=%d cin=%d cout=%d)", N, taps, cin, cout);
    return OP_ERR_ARG;
  }
  if (cin % 8 == 0 && ((uintptr_t)X & 15) != 0) {
    set_error("conv_bf16_tc: X must be 16-byte aligned");
    return OP_ERR_ARG;
  }
  ConvTc a;
  a.X = X;
  a.Wt = (const uint16_t *)scratch;
  a.bias = bias;
  a.Z = Z;
  a.A = A;
  a.N = N;
  a.taps = taps;
  a.cin = cin;
  a.cout = cout;
  a.coutp = (cout + 15) / 16 * 16;
  a.K = taps * cin;
  a.Kp = (a.K + kCK - 1) / kCK * kCK;
  a.err = err;
  const long long wt = (long long)a.coutp * a.Kp;
  k_conv_wt<<<(unsigned)std::min<long long>((wt + 255) / 256, 4LL * num_sms()), 256, 0, st>>>(
      W, a.K, cout, a.Kp, a.coutp, (uint16_t *)scratch);
  count_launch();
  OP_LAUNCH("k_conv_wt");
  // per device, so set on every call (cheap)
  OP_CUDA(cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kCSmem));
  const long long n = (long long)N * N * N;
  k_conv_tc<<<(unsigned)((n + kCM - 1) / kCM), 256, kCSmem, st>>>(a);
  count_launch();
  OP_LAUNCH("k_conv_tc");
  return OP_OK;
}

}  // namespace opevo
