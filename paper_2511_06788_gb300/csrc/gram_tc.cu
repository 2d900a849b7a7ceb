// Inner matrices of [U W] for FP32 blocks on the 5th-generation tensor cores:
// C = W^T U, S = W^T W, D = U^T U (§2.1; the matrices of Steps 2-3 and of
// Theorem 4.1) with tcgen05.mma kind::tf32 and FP32 accumulation in TMEM.
//
// FP32 accuracy from TF32 units (split = 1): every operand value x is split as
// x = hi + lo (hi = tf32(x), lo = tf32(x - hi)) and each product uses four
// MMAs, hi*hi + hi*lo + lo*hi + lo*lo (the lo*lo term would otherwise leave a
// one-signed error of ~2^-22 in the squared norms of <U,U> and <W,W>).  With
// split = 0 (the TF32 mixed mode) one MMA per product on tf32(x) is used.
//
// Work split: one CTA per (output tile of 128 x 128, chunk of grid points).
// The contraction index is the grid point (the row of the n x ld blocks), so
// the operand tiles are transposed while they are staged: each thread loads a
// 4 x 4 patch (4 grid points x 4 columns) with 16-byte loads, splits it, and
// writes 16-byte K-chunks into the 128B-swizzled K-major layout the MMA reads.
//
// Accumulation: the tensor core adds into its FP32 accumulator with
// truncation, so a long run of additions drifts by about (run length) x 2^-24
// of the accumulated value (for <U,U> = I that is a systematic error of the
// orthogonality).  Each 32-point slab therefore starts a fresh accumulator (two
// TMEM accumulators alternate) and, while the tensor core works on slab s, the
// 8 warps drain slab s-1 into FP32 registers (round-to-nearest additions).
// The loads run two slabs ahead of the shared-memory stores (one CTA per SM).
// Chunk partials are written in FP64 and summed over chunks in a fixed order.
#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace opevo {

namespace {

constexpr int kTM = 128;                      // output tile (rows and columns)
// reduce grid: one thread per output element of a tile (the split sums stay in order)
constexpr int kReduceSlices = kTM * kTM / 256;
constexpr int kKS = 32;                       // grid points per slab (one 128-byte K row)
constexpr int kPiece = kTM * 128;             // bytes of one operand piece (128 rows x 128 B)
constexpr int kStage = 4 * kPiece;            // A_hi, A_lo, B_hi, B_lo
constexpr int kStages = 2;
constexpr int kSmem = kStages * kStage + 1024;  // + alignment slack
constexpr uint32_t kIdesc = tc::idesc_tf32(kTM, kTM);

enum { PROD_C = 0, PROD_S = 1, PROD_D = 2 };

__device__ __forceinline__ void decode_job(int idx, int mask, int nt, int *prod, int *ti, int *tj) {
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

// 4 grid points x 4 columns of X starting at (row, col); zero outside [r1) x [ld).
__device__ __forceinline__ void load_patch(const float *__restrict__ X, long long row, long long r1,
                                           int col, int ld, float (&v)[4][4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row + r < r1 && col < ld) x = __ldg(reinterpret_cast<const float4 *>(X + (row + r) * ld + col));
    v[r][0] = x.x;
    v[r][1] = x.y;
    v[r][2] = x.z;
    v[r][3] = x.w;
  }
}

// Split the patch and store it transposed: operand row m = 4q + e gets the
// K-chunk kq = (v[0][e], .., v[3][e]).  Without `split` only tf32(x) is stored.
__device__ __forceinline__ void store_patch(uint8_t *hi, uint8_t *lo, int q, int kq,
                                            const float (&v)[4][4], bool split) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float4 h, l;
    tc::split_tf32(v[0][e], h.x, l.x);
    tc::split_tf32(v[1][e], h.y, l.y);
    tc::split_tf32(v[2][e], h.z, l.z);
    tc::split_tf32(v[3][e], h.w, l.w);
    const uint32_t off = tc::sw128_offset(4 * q + e, kq);
    *reinterpret_cast<float4 *>(hi + off) = h;
    if (split) *reinterpret_cast<float4 *>(lo + off) = l;
  }
}

// One CTA: output tile (ti, tj) of product `prod` over grid points [r0, r1) of the
// n x ld blocks U, W, written as a 128 x 128 FP64 partial tile at dst.
__device__ __forceinline__ void gram_tc_body(long long n, int ld, const float *__restrict__ U,
                                             const float *__restrict__ W, int prod, int ti,
                                             int tj, long long r0, long long r1,
                                             double *__restrict__ dst_tile, int *err, int split,
                                             bool atomic_out = false) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar[2];  // one per TMEM accumulator
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

  const float *A = (prod == PROD_D) ? U : W;
  const float *B = (prod == PROD_S) ? W : U;
  const int ca = ti * kTM, cb = tj * kTM;
  // diagonal tiles of S = W^T W and D = U^T U: A and B are the same data, staged once
  // (the B descriptors point at A's pieces; the MMAs and their order are unchanged)
  const bool same = (A == B) && (ca == cb);
  if (r1 > n) r1 = n;
  const int nslab = r1 > r0 ? (int)((r1 - r0 + kKS - 1) / kKS) : 0;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int kq = t & 7, q = t >> 3;        // staging patch: points 4kq.., columns 4q..
  const int row = (warp & 3) * 32 + lane;  // drain: accumulator row (TMEM lane)
  const int half = warp >> 2;              // drain: columns 64 half .. 64 half + 63

  if (warp == 0) tc::tmem_alloc(&tmem_base_sh, 2 * kTM);
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

  // drain the accumulator of slab s (called after the MMAs of slab s+1 were issued)
  auto drain = [&](int s) -> bool {
    const int a = s & 1;
    if (t == 0 && !tc::mbar_wait(&mbar[a], (uint32_t)((s >> 1) & 1))) abort_sh = 1;
    __syncthreads();
    if (abort_sh) return false;
    tc::tc_fence_after();
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float v[32];
      tc::tmem_ld32(tmem + lane_base + (uint32_t)(a * kTM + half * 64 + c * 32), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[c * 32 + i] += v[i];
    }
    tc::tc_fence_before();
    return true;
  };

  // stage slab s from the register buffer (va, vb), refill the buffer with slab s + 2,
  // issue the MMAs of slab s and drain slab s - 1
  auto step = [&](int s, float (&va)[4][4], float (&vb)[4][4]) -> bool {
    const int st = s & 1;
    uint8_t *stage = smem + st * kStage;
    // stage st was read by the MMAs of slab s-2, which the drain of slab s-2 waited for
    store_patch(stage, stage + kPiece, q, kq, va, split != 0);
    if (!same) store_patch(stage + 2 * kPiece, stage + 3 * kPiece, q, kq, vb, split != 0);
    if (s + 2 < nslab) {
      const long long r = r0 + (long long)(s + 2) * kKS + 4 * kq;
      load_patch(A, r, r1, ca + 4 * q, ld, va);
      if (!same) load_patch(B, r, r1, cb + 4 * q, ld, vb);
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc::tc_fence_after();
      const uint32_t base = tc::smem_u32(stage);
      const uint32_t bbase = same ? base : base + 2 * kPiece;
      const uint32_t d = tmem + (uint32_t)(st * kTM);
#pragma unroll
      for (int kk = 0; kk < kKS / 8; ++kk) {
        const uint64_t ah = tc::desc_sw128(base + kk * 32);
        const uint64_t al = tc::desc_sw128(base + kPiece + kk * 32);
        const uint64_t bh = tc::desc_sw128(bbase + kk * 32);
        const uint64_t bl = tc::desc_sw128(bbase + kPiece + kk * 32);
        tc::mma_tf32(d, ah, bh, kIdesc, kk > 0 ? 1u : 0u);
        if (split) {
          tc::mma_tf32(d, ah, bl, kIdesc, 1u);
          tc::mma_tf32(d, al, bh, kIdesc, 1u);
          tc::mma_tf32(d, al, bl, kIdesc, 1u);
        }
      }
      tc::mma_commit(&mbar[st]);
    }
    return s >= 1 ? drain(s - 1) : true;
  };

  float va0[4][4], vb0[4][4], va1[4][4], vb1[4][4];
  if (nslab > 0) {
    load_patch(A, r0 + 4 * kq, r1, ca + 4 * q, ld, va0);
    if (!same) load_patch(B, r0 + 4 * kq, r1, cb + 4 * q, ld, vb0);
  }
  if (nslab > 1) {
    load_patch(A, r0 + kKS + 4 * kq, r1, ca + 4 * q, ld, va1);
    if (!same) load_patch(B, r0 + kKS + 4 * kq, r1, cb + 4 * q, ld, vb1);
  }
  bool ok = true;
  for (int s = 0; s < nslab && ok; s += 2) {
    ok = step(s, va0, vb0);
    if (ok && s + 1 < nslab) ok = step(s + 1, va1, vb1);
  }
  if (ok && nslab > 0) ok = drain(nslab - 1);
  __syncthreads();
  if (!ok || abort_sh) {
    if (t == 0) atomicExch(err, 1);
  } else {
    double *dst = dst_tile + row * kTM + half * 64;
    if (atomic_out) {
      // the chunk partials of a tile meet in one FP64 tile (fixed-scratch entry point)
#pragma unroll
      for (int i = 0; i < 64; ++i) atomicAdd(dst + i, (double)acc[i]);
    } else {
#pragma unroll
      for (int i = 0; i < 64; ++i) dst[i] = (double)acc[i];
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * kTM);
}

// ---- BF16 variants -------------------------------------------------------------------
// The same tiling with BF16 operands: every value is split in three BF16 pieces
// (x = b0 + b1 + b2 to 2^-24), and each product takes the six MMAs (kind::f16) whose
// pieces have index sum <= 2 (one piece and one MMA in the plain BF16 mode); a slab is
// 64 grid points (one 128-byte row of BF16 K values).  The staging patch is 8 grid points x 4 columns; the register buffer runs
// one slab ahead.
constexpr int kKSb = 64;
constexpr int kStageB16 = 6 * kPiece;  // A0 A1 A2 B0 B1 B2
constexpr int kSmemB16 = 2 * kStageB16 + 1024;
constexpr uint32_t kIdescB16 = tc::idesc_bf16(kTM, kTM);

__device__ __forceinline__ void load_patch8(const float *__restrict__ X, long long row,
                                            long long r1, int col, int ld, float (&v)[8][4]) {
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row + r < r1 && col < ld) x = __ldg(reinterpret_cast<const float4 *>(X + (row + r) * ld + col));
    v[r][0] = x.x;
    v[r][1] = x.y;
    v[r][2] = x.z;
    v[r][3] = x.w;
  }
}

// operand row m = 4q + e gets the K-chunk kq (8 BF16 values) of each of the three pieces
// (of the first piece, bf16(x), only, when three == false)
__device__ __forceinline__ void store_patch8(uint8_t *piece0, int q, int kq, const float (&v)[8][4],
                                             bool three) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float col[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) col[r] = v[r][e];
    uint4 c0, c1, c2;
    tc::split8_bf16x3(col, c0, c1, c2);
    const uint32_t off = tc::sw128_offset(4 * q + e, kq);
    *reinterpret_cast<uint4 *>(piece0 + off) = c0;
    if (three) {
      *reinterpret_cast<uint4 *>(piece0 + kPiece + off) = c1;
      *reinterpret_cast<uint4 *>(piece0 + 2 * kPiece + off) = c2;
    }
  }
}

__device__ __forceinline__ void gram_bf16_body(long long n, int ld, const float *__restrict__ U,
                                               const float *__restrict__ W, int prod, int ti,
                                               int tj, long long r0, long long r1,
                                               double *__restrict__ dst_tile, int *err,
                                               bool three) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

  const float *A = (prod == PROD_D) ? U : W;
  const float *B = (prod == PROD_S) ? W : U;
  const int ca = ti * kTM, cb = tj * kTM;
  const bool same = (A == B) && (ca == cb);
  if (r1 > n) r1 = n;
  const int nslab = r1 > r0 ? (int)((r1 - r0 + kKSb - 1) / kKSb) : 0;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int kq = t & 7, q = t >> 3;
  const int row = (warp & 3) * 32 + lane;
  const int half = warp >> 2;

  if (warp == 0) tc::tmem_alloc(&tmem_base_sh, 2 * kTM);
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

  auto drain = [&](int s) -> bool {
    const int a = s & 1;
    if (t == 0 && !tc::mbar_wait(&mbar[a], (uint32_t)((s >> 1) & 1))) abort_sh = 1;
    __syncthreads();
    if (abort_sh) return false;
    tc::tc_fence_after();
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float v[32];
      tc::tmem_ld32(tmem + lane_base + (uint32_t)(a * kTM + half * 64 + c * 32), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[c * 32 + i] += v[i];
    }
    tc::tc_fence_before();
    return true;
  };

  float va[8][4], vb[8][4];
  if (nslab > 0) {
    load_patch8(A, r0 + 8 * kq, r1, ca + 4 * q, ld, va);
    if (!same) load_patch8(B, r0 + 8 * kq, r1, cb + 4 * q, ld, vb);
  }
  bool ok = true;
  for (int s = 0; s < nslab && ok; ++s) {
    const int st = s & 1;
    uint8_t *stage = smem + st * kStageB16;
    // stage st was read by the MMAs of slab s-2, which the drain of slab s-2 waited for
    store_patch8(stage, q, kq, va, three);
    if (!same) store_patch8(stage + 3 * kPiece, q, kq, vb, three);
    if (s + 1 < nslab) {
      const long long r = r0 + (long long)(s + 1) * kKSb + 8 * kq;
      load_patch8(A, r, r1, ca + 4 * q, ld, va);
      if (!same) load_patch8(B, r, r1, cb + 4 * q, ld, vb);
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc::tc_fence_after();
      const uint32_t base = tc::smem_u32(stage);
      const uint32_t bbase = same ? base : base + 3 * kPiece;
      const uint32_t d = tmem + (uint32_t)(st * kTM);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        uint64_t a[3], b[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          a[r] = tc::desc_sw128(base + r * kPiece + kk * 32);
          b[r] = tc::desc_sw128(bbase + r * kPiece + kk * 32);
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
  if (ok && nslab > 0) ok = drain(nslab - 1);
  __syncthreads();
  if (!ok || abort_sh) {
    if (t == 0) atomicExch(err, 1);
  } else {
    double *dst = dst_tile + row * kTM + half * 64;
#pragma unroll
    for (int i = 0; i < 64; ++i) dst[i] = (double)acc[i];
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * kTM);
}

__global__ void __launch_bounds__(256, 1)
    k_gram_bf16(long long n, int ld, const float *__restrict__ U, const float *__restrict__ W,
                int mask, int nt, int njobs, long long rows_per_split, double *__restrict__ part,
                int *err, int three) {
  int prod, ti, tj;
  decode_job(blockIdx.x, mask, nt, &prod, &ti, &tj);
  const long long r0 = (long long)blockIdx.y * rows_per_split;
  gram_bf16_body(n, ld, U, W, prod, ti, tj, r0, r0 + rows_per_split,
                 part + ((long long)blockIdx.y * njobs + blockIdx.x) * (kTM * kTM), err,
                 three != 0);
}

__global__ void __launch_bounds__(256, 1)
    k_gram_tc(long long n, int ld, const float *__restrict__ U, const float *__restrict__ W,
              int mask, int nt, int njobs, long long rows_per_split, double *__restrict__ part,
              int *err, int split, int atomic_out) {
  int prod, ti, tj;
  decode_job(blockIdx.x, mask, nt, &prod, &ti, &tj);
  const long long r0 = (long long)blockIdx.y * rows_per_split;
  const long long slot = atomic_out ? 0 : (long long)blockIdx.y;
  gram_tc_body(n, ld, U, W, prod, ti, tj, r0, r0 + rows_per_split,
               part + (slot * njobs + blockIdx.x) * (kTM * kTM), err, split, atomic_out != 0);
}

// Batched: one CTA per GramItem (problem, job, grid-point chunk); all three products.
__global__ void __launch_bounds__(256, 1)
    k_b_gram_tc(const BatchProb *__restrict__ Bp, const GramItem *__restrict__ items, int parity) {
  const GramItem it = items[blockIdx.x];
  const BatchProb &pb = Bp[it.prob];
  if (*pb.frozen) return;
  const int nt = (pb.ld + kTM - 1) / kTM;
  int prod, ti, tj;
  decode_job(it.job, 7, nt, &prod, &ti, &tj);
  gram_tc_body(pb.g.n, pb.ld, pb.U[parity], pb.W, prod, ti, tj, it.r0, it.r1,
               pb.gram_part + ((long long)it.split * pb.gram_jobs + it.job) * (kTM * kTM), pb.err,
               1);
}

// Batched reduce: grid (jobs, problems, element slices).
__global__ void k_b_gram_tc_reduce(const BatchProb *__restrict__ Bp) {
  const BatchProb &pb = Bp[blockIdx.y];
  if (*pb.frozen || (int)blockIdx.x >= pb.gram_jobs) return;
  const int ld = pb.ld, p = pb.p;
  const int nt = (ld + kTM - 1) / kTM;
  int prod, ti, tj;
  decode_job(blockIdx.x, 7, nt, &prod, &ti, &tj);
  double *out = prod == PROD_C ? pb.C : (prod == PROD_S ? pb.S : pb.D);
  for (int e = blockIdx.z * blockDim.x + threadIdx.x; e < kTM * kTM;
       e += gridDim.z * blockDim.x) {
    const int i = ti * kTM + e / kTM, j = tj * kTM + e % kTM;
    if (i >= ld || j >= ld) continue;
    double s = 0.0;
#pragma unroll 8
    for (int sp = 0; sp < pb.n_gram_splits; ++sp)
      s += pb.gram_part[((long long)sp * pb.gram_jobs + blockIdx.x) * (kTM * kTM) + e];
    const double v = (i < p && j < p) ? s : 0.0;
    out[(long long)i * ld + j] = v;
    if (prod != PROD_C && ti != tj) out[(long long)j * ld + i] = v;
  }
}

__global__ void k_gram_tc_reduce(int mask, int nt, int njobs, int nsplit,
                                 const double *__restrict__ part, int p, int ld, double *C,
                                 double *S, double *D) {
  int prod, ti, tj;
  decode_job(blockIdx.x, mask, nt, &prod, &ti, &tj);
  double *out = prod == PROD_C ? C : (prod == PROD_S ? S : D);
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < kTM * kTM; e += gridDim.y * blockDim.x) {
    const int i = ti * kTM + e / kTM, j = tj * kTM + e % kTM;
    if (i >= ld || j >= ld) continue;
    double s = 0.0;
#pragma unroll 8
    for (int sp = 0; sp < nsplit; ++sp)
      s += part[((long long)sp * njobs + blockIdx.x) * (kTM * kTM) + e];
    const double v = (i < p && j < p) ? s : 0.0;
    out[(long long)i * ld + j] = v;
    if (prod != PROD_C && ti != tj) out[(long long)j * ld + i] = v;
  }
}

int tc_jobs(int nt, int mask) {
  return ((mask & 1) ? nt * nt : 0) + ((mask & 2) ? nt * (nt + 1) / 2 : 0) +
         ((mask & 4) ? nt * (nt + 1) / 2 : 0);
}

}  // namespace

// Splits: about three CTAs per SM over all jobs, at least 512 grid points each.
static void plan_tc(long long n, int njobs, int *nsplit, long long *rps) {
  long long ns = (3 * num_sms() + njobs - 1) / njobs;
  const long long maxs = (n + 511) / 512;
  if (ns > maxs) ns = maxs;
  if (ns < 1) ns = 1;
  long long r = (n + ns - 1) / ns;
  r = (r + kKS - 1) / kKS * kKS;
  *rps = r;
  *nsplit = (int)((n + r - 1) / r);
}

size_t gram_tc_workspace_bytes(long long n, int ld) {
  (void)n;
  // plan_tc gives nj * nsplit <= 3 * num_sms() + nj for every subset of the products
  const int nt = (ld + kTM - 1) / kTM;
  return (size_t)(3 * num_sms() + tc_jobs(nt, 7)) * kTM * kTM * sizeof(double) + 256;
}

op_status gram_tc(long long n, int p, int ld, const float *U, const float *W, double *C, double *S,
                  double *D, void *ws, size_t ws_bytes, int *err, cudaStream_t st, int split) {
  if (ld % 8 != 0 || p > ld || n < 1) {
    set_error("gram_tc: bad sizes n=%lld p=%d ld=%d", n, p, ld);
    return OP_ERR_ARG;
  }
  const int nt = (ld + kTM - 1) / kTM;
  const int mask = (C ? 1 : 0) | (S ? 2 : 0) | (D ? 4 : 0);
  const int nj = tc_jobs(nt, mask);
  if (nj == 0) return OP_OK;
  int nsplit;
  long long rps;
  plan_tc(n, nj, &nsplit, &rps);
  const size_t need = (size_t)nj * nsplit * kTM * kTM * sizeof(double);
  if (!ws || ws_bytes < need) {
    set_error("gram_tc: workspace too small (%zu < %zu)", ws_bytes, need);
    return OP_ERR_ARG;
  }
  double *part = (double *)ws;
  if (split >= 2) {  // BF16: 2 three pieces, 3 one piece
    OP_CUDA(cudaFuncSetAttribute(k_gram_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemB16));
    k_gram_bf16<<<dim3(nj, nsplit), 256, kSmemB16, st>>>(n, ld, U, W, mask, nt, nj, rps, part,
                                                          err, split == 2 ? 1 : 0);
    count_launch();
    OP_LAUNCH("k_gram_bf16");
  } else {
    OP_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
    k_gram_tc<<<dim3(nj, nsplit), 256, kSmem, st>>>(n, ld, U, W, mask, nt, nj, rps, part, err,
                                                     split, 0);
    count_launch();
    OP_LAUNCH("k_gram_tc");
  }
  k_gram_tc_reduce<<<dim3(nj, kReduceSlices), 256, 0, st>>>(mask, nt, nj, nsplit, part, p, ld,
                                                             C, S, D);
  count_launch();
  OP_LAUNCH("k_gram_tc_reduce");
  return OP_OK;
}

// As gram_tc() (the same chunks of grid points, so the same FP32 runs and rounding
// bound), but the chunk partials of each output tile are added into one FP64 tile with
// atomics: part_bytes must hold one 128 x 128 FP64 tile per output tile.  The FP64
// chunk sums are taken in whatever order the CTAs finish.
op_status gram_tc_fixed_scratch(long long n, int p, int ld, const float *U, const float *W,
                                double *C, double *S, double *D, void *part, size_t part_bytes,
                                int *err, cudaStream_t st) {
  if (ld % 8 != 0 || p > ld || n < 1) {
    set_error("gram_tc: bad sizes n=%lld p=%d ld=%d", n, p, ld);
    return OP_ERR_ARG;
  }
  const int nt = (ld + kTM - 1) / kTM;
  const int mask = (C ? 1 : 0) | (S ? 2 : 0) | (D ? 4 : 0);
  const int nj = tc_jobs(nt, mask);
  if (nj == 0) return OP_OK;
  const size_t tile_bytes = (size_t)kTM * kTM * sizeof(double);
  if (part_bytes < (size_t)nj * tile_bytes) {
    set_error("gram_tc: %d output tiles need %zu bytes of partials, the fixed scratch holds %zu",
              nj, (size_t)nj * tile_bytes, part_bytes);
    return OP_ERR_ARG;
  }
  int nsplit;
  long long rps;
  plan_tc(n, nj, &nsplit, &rps);
  OP_CUDA(cudaMemsetAsync(part, 0, (size_t)nj * tile_bytes, st));
  OP_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  k_gram_tc<<<dim3(nj, nsplit), 256, kSmem, st>>>(n, ld, U, W, mask, nt, nj, rps, (double *)part,
                                                   err, 1, 1);
  count_launch();
  OP_LAUNCH("k_gram_tc");
  k_gram_tc_reduce<<<dim3(nj, kReduceSlices), 256, 0, st>>>(mask, nt, nj, 1, (const double *)part,
                                                             p, ld, C, S, D);
  count_launch();
  OP_LAUNCH("k_gram_tc_reduce");
  return OP_OK;
}

op_status launch_b_gram(const BatchProb *B, const GramItem *items, int nitems, int nprob,
                        int parity, cudaStream_t st) {
  OP_CUDA(cudaFuncSetAttribute(k_b_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  k_b_gram_tc<<<nitems, 256, kSmem, st>>>(B, items, parity);
  count_launch();
  OP_LAUNCH("k_b_gram_tc");
  // at most 3 * 8 * 8 + ... jobs for ld <= 1024: grid x covers the largest job count
  k_b_gram_tc_reduce<<<dim3(tc_jobs(8, 7), nprob, 4), 256, 0, st>>>(B);
  count_launch();
  OP_LAUNCH("k_b_gram_tc_reduce");
  return OP_OK;
}

size_t gram_tc_tile_bytes() { return (size_t)kTM * kTM * sizeof(double); }
int gram_tc_jobs_all(int ld) { return tc_jobs((ld + kTM - 1) / kTM, 7); }

}  // namespace opevo
