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
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"
#include "tma.cuh"

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

// ---- persistent, warp-specialised variant (ld a multiple of 32) ----------------------
// The same products, split and accumulation order as update_tc_body, so the result is
// bit-identical; only the staging and the division of labour differ.  One CTA per SM
// walks the output tiles blockIdx.x, blockIdx.x + gridDim.x, ... (consecutive tiles share
// their rows of [U W] through L2 when ld > 128), slab by slab, with four roles that
// meet only at mbarriers, so the tensor core is fed while earlier slabs drain:
//   warp 9, lane 0  TMA producer: the A slab (128 grid points x 32 K values of U or W)
//                   and the B slabs (128 columns of KT_hi / KT_lo) into a ring of kRing
//                   stages, each landing in the 128B-swizzled K-major layout;
//   warps 4..7      split the A slab into TF32 hi (in place) and lo;
//   warp 8, lane 0  issues the slab's MMAs into one of kAcc TMEM accumulators and
//                   commits them to that accumulator's "done" barrier and the stage's
//                   "empty" barrier;
//   warps 0..3      drain each accumulator into FP32 registers (one tile row per thread,
//                   all 128 columns), free it, and store U + acc when a tile ends.
// Every wait is bounded in time; a role that gives up raises a flag the others poll.
constexpr int kRing = 3;
constexpr int kAcc = 4;
constexpr int kStageR = 4 * kPieceA;  // A hi (TMA destination, split in place) | A lo | B hi | B lo
constexpr int kSmemR = kRing * kStageR + 1024;
constexpr uint64_t kWaitNs = 2000000000ull;  // every wait gives up after 2 s
constexpr int kWarpsWS = 10;

__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity,
                                              volatile int *abort) {
  return tc::wait_or_abort(bar, parity, abort, kWaitNs);
}

__global__ void __launch_bounds__(kWarpsWS * 32, 1)
    k_update_ws(const __grid_constant__ CUtensorMap mU, const __grid_constant__ CUtensorMap mW,
                const __grid_constant__ CUtensorMap mKh, const __grid_constant__ CUtensorMap mKl,
                long long n, int ld, const float *__restrict__ U, float *__restrict__ Unew,
                int *err, int split) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[kRing], empty[kRing], conv[kRing], done[kAcc], freed[kAcc];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nslab = 2 * ld / kKS;
  const int ntn = (ld + kTN - 1) / kTN;
  const long long ntiles = (n + kTM - 1) / kTM * ntn;
  const long long mine =
      ntiles > (long long)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long total = mine * nslab;

  if (warp == 0) tc::tmem_alloc(&tmem_base_sh, kAcc * kTN);
  if (t == 0) {
    for (int i = 0; i < kRing; ++i) {
      tma::bar_init(&full[i], 1);
      tma::bar_init(&empty[i], 1);
      tma::bar_init(&conv[i], 128);
    }
    for (int i = 0; i < kAcc; ++i) {
      tma::bar_init(&done[i], 1);
      tma::bar_init(&freed[i], 128);
    }
    tma::fence_bar_init();
    abort_sh = 0;
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  volatile int *abort = &abort_sh;

  if (warp == 9) {
    if (lane == 0) {  // ---- TMA producer
      long long g = 0;
      bool ok = true;
      for (long long i = 0; i < mine && ok; ++i) {
        const long long tile = blockIdx.x + i * gridDim.x;
        const int m0 = (int)(tile / ntn) * kTM, n0 = (int)(tile % ntn) * kTN;
        for (int s = 0; s < nslab; ++s, ++g) {
          const int st = (int)(g % kRing);
          // the stage's previous slab must have been read by its MMAs
          if (g >= kRing && !wait_or_abort(&empty[st], (uint32_t)((g / kRing - 1) & 1), abort)) {
            ok = false;
            break;
          }
          uint8_t *stage = smem + st * kStageR;
          const int k0 = s * kKS;
          tma::bar_expect(&full[st], (uint32_t)((split ? 3 : 2) * kPieceA));
          if (k0 < ld)
            tma::load_2d(stage, &mU, k0, m0, &full[st]);
          else
            tma::load_2d(stage, &mW, k0 - ld, m0, &full[st]);
          tma::load_2d(stage + 2 * kPieceA, &mKh, k0, n0, &full[st]);
          if (split) tma::load_2d(stage + 3 * kPieceA, &mKl, k0, n0, &full[st]);
        }
      }
      if (!ok) {
        atomicExch(err, 1);
        // copies still in flight land before the CTA may exit (only the last kRing can be)
        for (long long q = (g > kRing ? g - kRing : 0); q < g; ++q)
          (void)tma::bar_wait(&full[q % kRing], (uint32_t)((q / kRing) & 1), kWaitNs);
      }
    }
  } else if (warp == 8) {
    if (lane == 0) {  // ---- MMA issuer
      long long g = 0;
      for (; g < total; ++g) {
        const int st = (int)(g % kRing), a = (int)(g % kAcc);
        if (!wait_or_abort(&conv[st], (uint32_t)((g / kRing) & 1), abort)) break;
        if (g >= kAcc && !wait_or_abort(&freed[a], (uint32_t)((g / kAcc - 1) & 1), abort)) break;
        tc::tc_fence_after();
        const uint32_t base = tc::smem_u32(smem + st * kStageR);
        const uint32_t d = tmem + (uint32_t)(a * kTN);
#pragma unroll
        for (int kk = 0; kk < kKS / 8; ++kk) {
          const uint64_t ah = tc::desc_sw128(base + kk * 32);
          const uint64_t al = tc::desc_sw128(base + kPieceA + kk * 32);
          const uint64_t bh = tc::desc_sw128(base + 2 * kPieceA + kk * 32);
          const uint64_t bl = tc::desc_sw128(base + 3 * kPieceA + kk * 32);
          tc::mma_tf32(d, ah, bh, kIdesc, kk > 0 ? 1u : 0u);
          if (split) {
            tc::mma_tf32(d, ah, bl, kIdesc, 1u);
            tc::mma_tf32(d, al, bh, kIdesc, 1u);
          }
        }
        tc::mma_commit(&done[a]);
        tc::mma_commit(&empty[st]);
      }
      if (g < total) {
        atomicExch(err, 1);
        // MMAs issued but not drained: let them finish before the TMEM is freed
        if (g > 0) {
          const long long q = g - 1;
          (void)tc::mbar_wait(&done[q % kAcc], (uint32_t)((q / kAcc) & 1));
        }
      }
    }
  } else if (warp >= 4) {  // ---- splitters (warps 4..7)
    const int ct = t - 128;
    for (long long g = 0; g < total; ++g) {
      const int st = (int)(g % kRing);
      if (!wait_or_abort(&full[st], (uint32_t)((g / kRing) & 1), abort)) break;
      uint8_t *stage = smem + st * kStageR;
      // 1024 16-byte chunks of the A slab, 8 per thread (any bijection of chunks keeps
      // hi and lo in the same swizzled positions)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t off = (uint32_t)(ct + 128 * j) * 16u;
        float4 *pa = reinterpret_cast<float4 *>(stage + off);
        const float4 x = *pa;
        float4 h, l;
        tc::split_tf32(x.x, h.x, l.x);
        tc::split_tf32(x.y, h.y, l.y);
        tc::split_tf32(x.z, h.z, l.z);
        tc::split_tf32(x.w, h.w, l.w);
        *pa = h;
        if (split) *reinterpret_cast<float4 *>(stage + kPieceA + off) = l;
      }
      tc::fence_async_smem();
      tma::bar_arrive(&conv[st]);
    }
  } else {  // ---- drain and epilogue (warps 0..3: TMEM lanes 32 warp .. 32 warp + 31)
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const int trow = warp * 32 + lane;
    float acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0.f;
    long long g = 0;
    bool ok = true;
    for (long long i = 0; i < mine && ok; ++i) {
      for (int s = 0; s < nslab; ++s, ++g) {
        const int a = (int)(g % kAcc);
        if (!wait_or_abort(&done[a], (uint32_t)((g / kAcc) & 1), abort)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v[32];
          tc::tmem_ld32(tmem + lane_base + (uint32_t)(a * kTN + c * 32), v);
#pragma unroll
          for (int e = 0; e < 32; ++e) acc[c * 32 + e] += v[e];
        }
        tc::tc_fence_before();
        tma::bar_arrive(&freed[a]);
      }
      if (!ok) break;
      const long long tile = blockIdx.x + i * gridDim.x;
      const long long row = (tile / ntn) * kTM + trow;
      const int n0 = (int)(tile % ntn) * kTN;
      if (row < n) {
#pragma unroll
        for (int c = 0; c < 128; c += 4) {
          const int col = n0 + c;
          if (col < ld) {
            const float4 u = __ldg(reinterpret_cast<const float4 *>(U + row * ld + col));
            *reinterpret_cast<float4 *>(Unew + row * ld + col) =
                make_float4(u.x + acc[c], u.y + acc[c + 1], u.z + acc[c + 2], u.w + acc[c + 3]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 128; ++c) acc[c] = 0.f;
    }
    if (!ok && lane == 0) atomicExch(err, 1);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kAcc * kTN);
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

// ---- BF16 variants (register-staged, one output tile per CTA) -----------------------
// Operands split in three BF16 pieces; six kind::f16 MMAs per 16-value K step (piece
// index sum <= 2; the plain BF16 mode: the first piece and one MMA); a slab is 64 K
// values (one 128-byte row of BF16).  The B pieces
// KT0..KT2 of [KU - I; KW]^T are formed once per step (k_make_kt_bf16).  Accumulation,
// drain and epilogue are those of update_tc_body.
constexpr int kKSb = 64;
constexpr int kStageB16 = 6 * kPieceA;  // A0 A1 A2 B0 B1 B2
constexpr int kSmemB16 = 2 * kStageB16 + 1024;
constexpr uint32_t kIdescB16 = tc::idesc_bf16(kTM, kTN);

template <typename S>
__global__ void k_make_kt_bf16(int ld, const S *__restrict__ KU, const S *__restrict__ KW,
                               uint16_t *__restrict__ KT) {
  const int K = 2 * ld;
  const long long total = (long long)ld * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int nn = (int)(e / K), k = (int)(e % K);
    const double v = (k < ld) ? (double)KU[(long long)k * ld + nn] - (k == nn ? 1.0 : 0.0)
                              : (double)KW[(long long)(k - ld) * ld + nn];
    const __nv_bfloat16 b0 = __float2bfloat16_rn((float)v);
    const double r1 = v - (double)__bfloat162float(b0);
    const __nv_bfloat16 b1 = __float2bfloat16_rn((float)r1);
    const double r2 = r1 - (double)__bfloat162float(b1);
    KT[e] = __bfloat16_as_ushort(b0);
    KT[total + e] = __bfloat16_as_ushort(b1);
    KT[2 * total + e] = __bfloat16_as_ushort(__float2bfloat16_rn((float)r2));
  }
}

__global__ void __launch_bounds__(256, 1)
    k_update_bf16(long long n, int ld, const float *__restrict__ U, const float *__restrict__ W,
                  const uint16_t *__restrict__ KT, float *__restrict__ Unew, int *err,
                  int three) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

  const long long m0 = (long long)blockIdx.x * kTM;
  const int n0 = blockIdx.y * kTN;
  const int K = 2 * ld;
  const long long ktot = (long long)ld * K;
  const int nslab = (K + kKSb - 1) / kKSb;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int kq = t & 7, rr = t >> 3;        // staging: K-chunk kq (8 values) of rows rr + 32 j
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

  // one slab ahead in registers: 8 A values and 3 B chunks for each of 4 rows
  float va[4][8];
  uint4 vb[4][3];
  auto load = [&](int s) {
    const int k = s * kKSb + 8 * kq;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long row = m0 + rr + 32 * j;
      float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
      if (row < n && k < K) {
        const float *src = (k < ld) ? U + row * ld + k : W + row * ld + (k - ld);
        x0 = __ldg(reinterpret_cast<const float4 *>(src));
        x1 = __ldg(reinterpret_cast<const float4 *>(src + 4));
      }
      va[j][0] = x0.x; va[j][1] = x0.y; va[j][2] = x0.z; va[j][3] = x0.w;
      va[j][4] = x1.x; va[j][5] = x1.y; va[j][6] = x1.z; va[j][7] = x1.w;
      const int col = n0 + rr + 32 * j;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        vb[j][r] = make_uint4(0u, 0u, 0u, 0u);
        if (col < ld && k < K && (three || r == 0))
          vb[j][r] = __ldg(reinterpret_cast<const uint4 *>(KT + r * ktot + (long long)col * K + k));
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
    uint8_t *stage = smem + st * kStageB16;
    // stage st was read by the MMAs of slab s-2, which the drain of slab s-2 waited for
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t off = tc::sw128_offset(rr + 32 * j, kq);
      uint4 c0, c1, c2;
      tc::split8_bf16x3(va[j], c0, c1, c2);
      *reinterpret_cast<uint4 *>(stage + off) = c0;
      *reinterpret_cast<uint4 *>(stage + kPieceA + off) = c1;
      *reinterpret_cast<uint4 *>(stage + 2 * kPieceA + off) = c2;
#pragma unroll
      for (int r = 0; r < 3; ++r)
        *reinterpret_cast<uint4 *>(stage + (3 + r) * kPieceA + off) = vb[j][r];
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
      for (int kk = 0; kk < 4; ++kk) {
        uint64_t a[3], b[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          a[r] = tc::desc_sw128(base + r * kPieceA + kk * 32);
          b[r] = tc::desc_sw128(base + (3 + r) * kPieceA + kk * 32);
        }
        tc::mma_bf16(d, a[0], b[0], kIdescB16, kk > 0 ? 1u : 0u);
        if (three) {
          tc::mma_bf16(d, a[0], b[1], kIdescB16, 1u);
          tc::mma_bf16(d, a[1], b[0], kIdescB16, 1u);
          tc::mma_bf16(d, a[0], b[2], kIdescB16, 1u);
          tc::mma_bf16(d, a[1], b[1], kIdescB16, 1u);
          tc::mma_bf16(d, a[2], b[0], kIdescB16, 1u);
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
  const uintptr_t a = (uintptr_t)U | (uintptr_t)W | (uintptr_t)KT_hi | (uintptr_t)KT_lo;
  if (ld % kKS == 0 && (a & 15) == 0 && n <= (long long)INT32_MAX - kTM) {
    CUtensorMap mU, mW, mKh, mKl;
    OP_TRY(tma_map_2d_f32_sw128(&mU, U, ld, n, kTM));
    OP_TRY(tma_map_2d_f32_sw128(&mW, W, ld, n, kTM));
    OP_TRY(tma_map_2d_f32_sw128(&mKh, KT_hi, 2 * ld, ld, kTN));
    OP_TRY(tma_map_2d_f32_sw128(&mKl, KT_lo, 2 * ld, ld, kTN));
    const long long ntiles = (n + kTM - 1) / kTM * ((ld + kTN - 1) / kTN);
    const int grid = (int)std::min<long long>(ntiles, num_sms());
    OP_CUDA(cudaFuncSetAttribute(k_update_ws, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemR));
    k_update_ws<<<grid, kWarpsWS * 32, kSmemR, st>>>(mU, mW, mKh, mKl, n, ld, U, Unew, err,
                                                     split);
    count_launch();
    OP_LAUNCH("k_update_ws");
    return OP_OK;
  }
  OP_CUDA(cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  const dim3 grid((unsigned)((n + kTM - 1) / kTM), (ld + kTN - 1) / kTN);
  k_update_tc<<<grid, 256, kSmem, st>>>(n, ld, U, W, KT_hi, KT_lo, Unew, err, split);
  count_launch();
  OP_LAUNCH("k_update_tc");
  return OP_OK;
}

size_t kt_bf16_bytes(int ld) { return (size_t)3 * ld * 2 * ld * sizeof(uint16_t); }

op_status launch_make_kt_bf16(int ld, const double *KU, const double *KW, uint16_t *KT,
                              cudaStream_t st) {
  k_make_kt_bf16<double><<<(2 * ld * ld + 255) / 256, 256, 0, st>>>(ld, KU, KW, KT);
  count_launch();
  OP_LAUNCH("k_make_kt_bf16");
  return OP_OK;
}

op_status launch_make_kt_bf16_f32(int ld, const float *KU, const float *KW, uint16_t *KT,
                                  cudaStream_t st) {
  k_make_kt_bf16<float><<<(2 * ld * ld + 255) / 256, 256, 0, st>>>(ld, KU, KW, KT);
  count_launch();
  OP_LAUNCH("k_make_kt_bf16");
  return OP_OK;
}

op_status update_bf16(long long n, int ld, const float *U, const float *W, const uint16_t *KT,
                      float *Unew, int *err, cudaStream_t st, bool three) {
  if (ld % 8 != 0 || n < 1) {
    set_error("update_bf16: bad sizes n=%lld ld=%d", n, ld);
    return OP_ERR_ARG;
  }
  OP_CUDA(cudaFuncSetAttribute(k_update_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSmemB16));
  const dim3 grid((unsigned)((n + kTM - 1) / kTM), (ld + kTN - 1) / kTN);
  k_update_bf16<<<grid, 256, kSmemB16, st>>>(n, ld, U, W, KT, Unew, err, three ? 1 : 0);
  count_launch();
  OP_LAUNCH("k_update_bf16");
  return OP_OK;
}

}  // namespace opevo
