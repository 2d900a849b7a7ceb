// Step 4 of §4.1 for FP32 blocks on the 5th-generation tensor cores:
// Unew = [U W] [KU; KW] as tcgen05.mma kind::tf32 with FP32 accumulation in
// TMEM (split = 1: 3xTF32, hi*hi + hi*lo + lo*hi, FP32-class accuracy;
// split = 0, the TF32 mixed mode: one MMA on the TF32-rounded values).
//
// The tensor core adds into its FP32 accumulator with truncation, so the MMAs
// accumulate only the correction [U W] [KU - I; KW] (small once the iteration
// approaches the fixed point), each 32-wide K slab in a fresh accumulator (two
// TMEM accumulators alternate) that the 8 warps drain into FP32 registers while
// the next slab runs, and the epilogue adds U in one rounding.
//
// One CTA computes a 128-row x 128-column tile of Unew.  The contraction runs
// over the 2 ld columns of [U W] in slabs of 32: the A operand (128 grid points
// x 32) is read with 16-byte loads along the row, split and written into the
// 128B-swizzled K-major layout; the B operand is the transposed coefficient
// matrix [KU; KW]^T, split into TF32 hi/lo parts once per step (it is shared
// by all CTAs and read from L2).  Two shared-memory stages overlap the loads of
// slab s+1 with the MMAs of slab s.  The epilogue reads the accumulator with
// tcgen05.ld (one grid point per thread) and stores 128-byte rows.
#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace opevo {

namespace {

constexpr int kTM = 128;                        // grid points per tile
constexpr int kTN = 128;                        // output columns per tile
constexpr int kKS = 32;                         // K values per slab (128 bytes)
constexpr int kPieceA = kTM * 128;
constexpr int kPieceB = kTN * 128;
constexpr int kStage = 2 * kPieceA + 2 * kPieceB;
constexpr int kStages = 2;
constexpr int kSmem = kStages * kStage + 1024;
constexpr uint32_t kIdesc = tc::idesc_tf32(kTM, kTN);

// One CTA: output tile rows [m0, m0 + 128) x columns [n0, n0 + 128) of Unew.
__device__ __forceinline__ void update_tc_body(long long n, int ld, const float *__restrict__ U,
                                               const float *__restrict__ W,
                                               const float *__restrict__ KT_hi,
                                               const float *__restrict__ KT_lo,
                                               float *__restrict__ Unew, long long m0, int n0,
                                               int *err, int split) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar[2];  // one per TMEM accumulator
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

  const int K = 2 * ld;
  const int nslab = (K + kKS - 1) / kKS;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int kq = t & 7, rr = t >> 3;       // staging: K-chunk kq of rows rr + 32 j
  const int drow = (warp & 3) * 32 + lane;  // drain: tile row (TMEM lane)
  const int half = warp >> 2;               // drain: columns 64 half .. 64 half + 63

  if (warp == 0) tc::tmem_alloc(&tmem_base_sh, 2 * kTN);
  if (t == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
    abort_sh = 0;
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;

  float acc[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) acc[i] = 0.f;

  float4 va[4], vh[4], vl[4];
  auto load = [&](int s) {
    const int k = s * kKS + 4 * kq;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long row = m0 + rr + 32 * j;
      va[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < n && k < K) {
        const float *src = (k < ld) ? U + row * ld + k : W + row * ld + (k - ld);
        va[j] = __ldg(reinterpret_cast<const float4 *>(src));
      }
      const int col = n0 + rr + 32 * j;
      vh[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      vl[j] = vh[j];
      if (col < ld && k < K) {
        vh[j] = __ldg(reinterpret_cast<const float4 *>(KT_hi + (long long)col * K + k));
        vl[j] = __ldg(reinterpret_cast<const float4 *>(KT_lo + (long long)col * K + k));
      }
    }
  };
  auto drain = [&](int s) -> bool {
    const int a = s & 1;
    if (t == 0 && !tc::mbar_wait(&mbar[a], (uint32_t)((s >> 1) & 1))) abort_sh = 1;
    __syncthreads();
    if (abort_sh) return false;
    tc::tc_fence_after();
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float v[32];
      tc::tmem_ld32(tmem + lane_base + (uint32_t)(a * kTN + half * 64 + c * 32), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[c * 32 + i] += v[i];
    }
    tc::tc_fence_before();
    return true;
  };

  load(0);
  bool ok = true;
  for (int s = 0; s < nslab && ok; ++s) {
    const int st = s & 1;
    uint8_t *stage = smem + st * kStage;
    // stage st was read by the MMAs of slab s-2, which the drain of slab s-2 waited for
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = rr + 32 * j;
      float4 h, l;
      tc::split_tf32(va[j].x, h.x, l.x);
      tc::split_tf32(va[j].y, h.y, l.y);
      tc::split_tf32(va[j].z, h.z, l.z);
      tc::split_tf32(va[j].w, h.w, l.w);
      const uint32_t off = tc::sw128_offset(r, kq);
      *reinterpret_cast<float4 *>(stage + off) = h;
      *reinterpret_cast<float4 *>(stage + 2 * kPieceA + off) = vh[j];
      if (split) {
        *reinterpret_cast<float4 *>(stage + kPieceA + off) = l;
        *reinterpret_cast<float4 *>(stage + 2 * kPieceA + kPieceB + off) = vl[j];
      }
    }
    if (s + 1 < nslab) load(s + 1);
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc::tc_fence_after();
      const uint32_t base = tc::smem_u32(stage);
      const uint32_t d = tmem + (uint32_t)(st * kTN);
#pragma unroll
      for (int kk = 0; kk < kKS / 8; ++kk) {
        const uint64_t ah = tc::desc_sw128(base + kk * 32);
        const uint64_t al = tc::desc_sw128(base + kPieceA + kk * 32);
        const uint64_t bh = tc::desc_sw128(base + 2 * kPieceA + kk * 32);
        const uint64_t bl = tc::desc_sw128(base + 2 * kPieceA + kPieceB + kk * 32);
        tc::mma_tf32(d, ah, bh, kIdesc, kk > 0 ? 1u : 0u);
        if (split) {
          tc::mma_tf32(d, ah, bl, kIdesc, 1u);
          tc::mma_tf32(d, al, bh, kIdesc, 1u);
        }
      }
      tc::mma_commit(&mbar[st]);
    }
    if (s >= 1) ok = drain(s - 1);
  }
  if (ok) ok = drain(nslab - 1);
  __syncthreads();
  if (!ok || abort_sh) {
    if (t == 0) atomicExch(err, 1);
  } else {
    const long long row = m0 + drow;
    if (row < n) {
#pragma unroll
      for (int i = 0; i < 64; i += 4) {
        const int col = n0 + half * 64 + i;
        if (col < ld) {
          const float4 u = __ldg(reinterpret_cast<const float4 *>(U + row * ld + col));
          *reinterpret_cast<float4 *>(Unew + row * ld + col) =
              make_float4(u.x + acc[i], u.y + acc[i + 1], u.z + acc[i + 2], u.w + acc[i + 3]);
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * kTN);
}

__global__ void __launch_bounds__(256, 1)
    k_update_tc(long long n, int ld, const float *__restrict__ U, const float *__restrict__ W,
                const float *__restrict__ KT_hi, const float *__restrict__ KT_lo,
                float *__restrict__ Unew, int *err, int split) {
  update_tc_body(n, ld, U, W, KT_hi, KT_lo, Unew, (long long)blockIdx.x * kTM, blockIdx.y * kTN,
                 err, split);
}

// Batched: one CTA per TileItem (problem, 128-point tile, column tile); U -> U+.
__global__ void __launch_bounds__(256, 1)
    k_b_update_tc(const BatchProb *__restrict__ B, const TileItem *__restrict__ items, int parity) {
  const TileItem it = items[blockIdx.x];
  const BatchProb &pb = B[it.prob];
  if (*pb.frozen) return;
  update_tc_body(pb.g.n, pb.ld, pb.U[parity], pb.W, pb.KT_hi, pb.KT_lo, pb.U[parity ^ 1], it.m0,
                 it.n0, pb.err, 1);
}

// Batched KT = [KU - I; KW]^T split (grid: element blocks x problems).
__global__ void k_b_make_kt(const BatchProb *__restrict__ B) {
  const BatchProb &pb = B[blockIdx.y];
  if (*pb.frozen) return;
  const int ld = pb.ld, K = 2 * ld;
  const long long total = (long long)ld * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int nn = (int)(e / K), k = (int)(e % K);
    const double v = (k < ld) ? pb.KU[(long long)k * ld + nn] - (k == nn ? 1.0 : 0.0)
                              : pb.KW[(long long)(k - ld) * ld + nn];
    const float hi = tc::to_tf32((float)v);
    pb.KT_hi[e] = hi;
    pb.KT_lo[e] = tc::to_tf32((float)(v - (double)hi));
  }
}

// KT = [KU - I; KW]^T (ld x 2 ld, K-major rows) split into TF32 hi / lo parts
// (the identity is added back by the epilogue of k_update_tc).
template <typename S>
__global__ void k_make_kt(int ld, const S *__restrict__ KU, const S *__restrict__ KW,
                          float *__restrict__ KT_hi, float *__restrict__ KT_lo) {
  const int K = 2 * ld;
  const long long total = (long long)ld * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int nn = (int)(e / K), k = (int)(e % K);
    const double v = (k < ld) ? (double)KU[(long long)k * ld + nn] - (k == nn ? 1.0 : 0.0)
                              : (double)KW[(long long)(k - ld) * ld + nn];
    const float hi = tc::to_tf32((float)v);
    KT_hi[e] = hi;
    KT_lo[e] = tc::to_tf32((float)(v - (double)hi));
  }
}

}  // namespace

op_status launch_b_update(const BatchProb *B, const TileItem *items, int nitems, int nprob,
                          int max_ld, int parity, cudaStream_t st) {
  k_b_make_kt<<<dim3((2 * max_ld * max_ld + 255) / 256, nprob), 256, 0, st>>>(B);
  count_launch();
  OP_CUDA(cudaFuncSetAttribute(k_b_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  k_b_update_tc<<<nitems, 256, kSmem, st>>>(B, items, parity);
  count_launch();
  OP_LAUNCH("k_b_update_tc");
  return OP_OK;
}

op_status launch_make_kt(int ld, const double *KU, const double *KW, float *KT_hi, float *KT_lo,
                         cudaStream_t st) {
  k_make_kt<double><<<(2 * ld * ld + 255) / 256, 256, 0, st>>>(ld, KU, KW, KT_hi, KT_lo);
  count_launch();
  OP_LAUNCH("k_make_kt");
  return OP_OK;
}

op_status launch_make_kt_f32(int ld, const float *KU, const float *KW, float *KT_hi,
                             float *KT_lo, cudaStream_t st) {
  k_make_kt<float><<<(2 * ld * ld + 255) / 256, 256, 0, st>>>(ld, KU, KW, KT_hi, KT_lo);
  count_launch();
  OP_LAUNCH("k_make_kt");
  return OP_OK;
}

op_status update_tc(long long n, int ld, const float *U, const float *W, const float *KT_hi,
                    const float *KT_lo, float *Unew, int *err, cudaStream_t st, int split) {
  if (ld % 8 != 0 || n < 1) {
    set_error("update_tc: bad sizes n=%lld ld=%d", n, ld);
    return OP_ERR_ARG;
  }
  OP_CUDA(cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  const dim3 grid((unsigned)((n + kTM - 1) / kTM), (ld + kTN - 1) / kTN);
  k_update_tc<<<grid, 256, kSmem, st>>>(n, ld, U, W, KT_hi, KT_lo, Unew, err, split);
  count_launch();
  OP_LAUNCH("k_update_tc");
  return OP_OK;
}

}  // namespace opevo
