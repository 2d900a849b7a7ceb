// FP64-accurate products of FP64 blocks on the tensor cores: the inner matrices
// C = <W,U>, S = <W,W>, D = <U,U> (§2.1; Steps 2-3 of §4.1) and the rank-2p update
// U+ = U + [U W][KU - I; KW] (Step 4), for the FP64 mode of the scheme.
//
// GB300 runs FP64 FMA at about 2 per clock per SM, so an FP64 Gram or update of
// p ~ 10^3 orbitals takes seconds there.  Here every FP64 operand is written exactly as
// ND integer digits and the products of digits run on tcgen05 (kind::f16, BF16 operands,
// FP32 accumulation in TMEM), in exact integer arithmetic:
//
//   Digits.  A row r of an operand (the K-vector an output entry contracts over) gets an
//   exponent e_r with max_k |a_rk| < 2^e_r.  X = round(a 2^(B - e_r)), B = 8 ND - 1, is an
//   integer with |X| < 2^B, written in balanced base 256: X = sum_{s<ND} d_s 2^(8(ND-1-s)),
//   d_1.. in [-128, 127], d_0 in [-128, 128] (every digit is a BF16 value exactly).  The
//   digits keep all B bits of X; rounding a to X costs at most 2^-(B+1) max|a_r.|.
//   ND = 7 (B = 55) for the Gram, whose rows are orbitals over the grid (their maxima are
//   close to their typical values); ND = 8 (B = 63) for the update, whose rows are the 2p
//   values of [U W] at one grid point, where the largest can exceed the typical one by
//   orders of magnitude (localised orbitals): the eighth digit keeps the update's error
//   below that of FP64 FMA relative to the typical term.
//
//   Products.  sum_k X_ak X_bk = sum_{s,t} (sum_k d_s d'_t) 2^(8 (2 ND - 2 - s - t)); the
//   pairs with s + t <= ND - 1 (28 or 36 MMAs per K step) are kept, summed per level
//   l = s + t in one TMEM accumulator each (ND accumulators of 128 x 64).  The dropped
//   levels weigh at most about 2^-(B-1.6) of |X_a| |X_b| per term.
//
//   Exactness.  |d_s d'_t| <= 2^14, so over 256 K values a level-l sum is at most
//   (l + 1) 2^22: levels 0..3 stay within 2^24 and are exact FP32 integers whatever the
//   tensor core's rounding; higher levels can round by a few units of their own weight
//   (2^-32 and below of level 0).  Every 256 K values the accumulators are read out
//   (tcgen05.ld), converted to integers and added into two int64 registers per output,
//   hi = L0 2^24 + L1 2^16 + L2 2^8 + L3 and lo = sum_{l >= 4} L_l 2^(8 (ND - 1 - l))
//   (exact), and the TMEM accumulators start afresh.  At the end of a work item the output
//   is (2^(8 (ND - 4)) hi + lo) 2^(e_a + e_b - 2B + 8 (ND - 1)) in FP64.
//
// Data flow.  Split kernels write the digits as ND BF16 planes [digit][row][k]
// (k contiguous): the Gram contracts over grid points, so its split kernel transposes
// [U W] (tile transpose through shared memory) with one exponent per column and chunk of
// grid points; the update contracts over the 2p columns of [U W] (already contiguous) with
// one exponent per grid point.  The MMA kernel is warp specialised: one thread issues
// TMA loads of 32-wide K slabs of all 2 ND digit planes (64-byte swizzle) into a
// two-stage ring, two threads issue the digit-pair MMAs of each 16-wide K step (each for
// its own levels: the tensor core takes an MMA about every 45 clocks, and a single issuing
// thread loses hundreds of clocks at every barrier of the ring), and eight warps drain the
// accumulators.  CTAs run in clusters of two on two SMs; the pair computes
// two output tiles with the same 128 A rows and adjacent 64-row blocks of B, and each CTA
// loads one 64-row half of the A planes into both CTAs' shared memory (TMA multicast), so
// a stage moves 2/3 of its bytes from L2.  A slot of the ring is free when the MMAs of
// both CTAs have read it.  Every wait is bounded (2 s); a role that gives up sets the
// error word.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace opevo {

namespace {

// ND digits per value (7 for the Gram, 8 for the update: see the header); ND levels
constexpr int kMaxDigits = 8;
constexpr int kGramDigits = 7;    // the Gram: column exponents over grid points
constexpr int kUpdateDigits = 8;  // the update: row exponents over the 2p values of a point
constexpr int kBM = 128, kBN = 64;         // output tile: 128 A rows x 64 B rows
#ifndef FP64TC_KS
#define FP64TC_KS 32
#endif
#ifndef FP64TC_STAGES
#define FP64TC_STAGES 8
#endif
constexpr int kKS = FP64TC_KS;             // K per ring stage: 16 (32-byte rows) or 32 (64)
constexpr int kChunkStages = 256 / kKS;    // 256 K values between accumulator read-outs
constexpr int kAPlane = kBM * kKS * 2;     // 4 or 8 KB
constexpr int kBPlane = kBN * kKS * 2;     // 2 or 4 KB
template <int ND> constexpr int stage_bytes() { return ND * (kAPlane + kBPlane); }
// ring depth: as many stages as fit 226 KB, at most FP64TC_STAGES
template <int ND> constexpr int ring_stages() {
  return (226 * 1024) / stage_bytes<ND>() < FP64TC_STAGES ? (226 * 1024) / stage_bytes<ND>()
                                                          : FP64TC_STAGES;
}
static_assert(kKS == 16 || kKS == 32, "K slab of one or two MMA K steps");
static_assert(ring_stages<8>() >= 2, "ring of at least two stages");
template <int ND> constexpr int smem_bytes() { return ring_stages<ND>() * stage_bytes<ND>() + 1024; }
constexpr int kIssuers = 2;                // warps 1 .. kIssuers issue the MMAs
#ifndef FP64TC_DRAIN_WARPS
#define FP64TC_DRAIN_WARPS 8
#endif
constexpr int kDrainWarps = FP64TC_DRAIN_WARPS;   // 4 lane quarters x column groups
constexpr int kDrainCols = 4 * kBN / kDrainWarps;  // output columns per drain thread
static_assert(kDrainCols % 4 == 0 && kDrainCols >= 4, "drain column groups of four");
constexpr int kThreads = 32 * (1 + kIssuers + kDrainWarps);  // warp 0 TMA, then MMA, drain
constexpr uint32_t kTmemCols = 512;        // ND x 64 used
constexpr uint32_t kIdesc = tc::idesc_bf16(kBM, kBN);
constexpr uint64_t kWaitNs = 2000000000ull;

enum { MODE_GRAM = 0, MODE_UPDATE_DELTA = 1, MODE_UPDATE = 2 };

struct Job {
  int mode;
  long long npairs;      // work items in pairs that share their A rows (a cluster's CTAs)
  int npt;               // Gram: tile pairs per K range
  // Gram: upper-triangle tiles of Y^T Y (Y: nc columns), K ranges of krange grid points
  int nc, nI, nJ, ntiles;
  long long krange, kext;
  double *part;          // [item][128][64]
  // update: M tiles over the chunk's rows, N tiles over the ld output columns
  long long mrows;
  int ntn, kdim, ld;
  const double *base;    // U rows of the chunk (delta form) or nullptr
  double *out;           // U+ rows of the chunk
  const int *ea, *eb;    // exponents of the A rows and the B rows
  int *err;
};

// Upper-triangle tile t of an nI x nJ grid of 128 x 64 tiles: (I, J) with J >= 2 I.
__device__ __forceinline__ void tile_of(int t, int nJ, int *I, int *J) {
  int i = 0;
  for (;;) {
    const int cnt = nJ - 2 * i;
    if (t < cnt) break;
    t -= cnt;
    ++i;
  }
  *I = i;
  *J = 2 * i + t;
}

// Member r (0 or 1) of item pair `pair`: the two members share the A rows and the K range
// and take adjacent 64-row blocks of B.  A member past the last B block is a stand-in
// (valid = false): its B rows read as zeros and it writes nothing.  *item: the member's
// index among the unpaired items (the Gram's partial tile).
__device__ __forceinline__ void decode_pair(const Job &J, long long pair, int r, int *ra, int *rb,
                                            long long *k0, long long *klen, bool *valid,
                                            long long *item) {
  if (J.mode == MODE_GRAM) {
    const long long q = pair / J.npt;
    int tp = (int)(pair % J.npt), I = 0;
    for (;;) {
      const int cnt = (J.nJ - 2 * I + 1) / 2;
      if (tp < cnt) break;
      tp -= cnt;
      ++I;
    }
    const int Jt = 2 * I + 2 * tp + r;
    *valid = Jt < J.nJ;
    *ra = I * kBM;
    *rb = Jt * kBN;
    *k0 = q * J.krange;
    const long long e = (q + 1) * J.krange < J.kext ? (q + 1) * J.krange : J.kext;
    *klen = e > *k0 ? e - *k0 : 0;
    *item = q * J.ntiles + (long long)I * J.nJ - (long long)I * (I - 1) + (Jt - 2 * I);
  } else {
    const int npn = (J.ntn + 1) / 2;
    const int jn = (int)(pair % npn) * 2 + r;
    *valid = jn < J.ntn;
    *ra = (int)(pair / npn) * kBM;
    *rb = jn * kBN;
    *k0 = 0;
    *klen = J.kdim;
    *item = (pair / npn) * J.ntn + jn;
  }
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// TMA load of one box into the same shared-memory offset of both CTAs of the cluster, with
// completion counted in bytes on the barrier at the same offset of each.
__device__ __forceinline__ void load_3d_mc(void *dst, const CUtensorMap *map, int c0, int c1,
                                           int c2, uint64_t *bar) {
  const uint16_t mask = 0x3;
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".multicast::cluster [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(tma::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2),
      "r"(tma::smem_addr(bar)), "h"(mask)
      : "memory");
}
// One arrival on `bar` in both CTAs of the cluster when this thread's MMAs complete.
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar) {
  const uint16_t mask = 0x3;
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(tc::smem_u32(bar)), "h"(mask)
      : "memory");
}

// D[tmem] (+)= A B^T (BF16, K = 16) with the A operand kept in the tensor core's collector
// buffer across a run of MMAs that share it: C = 1 loads A and keeps it (fill), 2 reuses it
// (use), 3 reuses it for the last time (lastuse), 0 a lone MMA (A read and discarded).
template <int C>
__device__ __forceinline__ void mma_bf16_ca(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                            uint32_t idesc, uint32_t accumulate) {
  if constexpr (C == 1) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate) : "memory");
  } else if constexpr (C == 2) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate) : "memory");
  } else if constexpr (C == 3) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate) : "memory");
  } else {
    tc::mma_bf16(d_tmem, a_desc, b_desc, idesc, accumulate);
  }
}

// kIssuers threads issue the digit-pair MMAs, each for the levels in its mask: the pairs
// of one level (one accumulator) all come from one thread, in order, and while one thread
// waits at a barrier the others keep the tensor core busy.  The masks balance the pair
// counts l + 1 of the levels between the threads.
template <int ND> constexpr unsigned issuer_mask(int which) {
  constexpr unsigned all = (1u << ND) - 1u;
  if (kIssuers == 1) return all;
  if (kIssuers == 2) {
    constexpr unsigned a = ND == 7 ? 0x47u : 0x8Fu;  // {0,1,2,6} | {0,1,2,3,7}
    return which == 0 ? a : all & ~a;
  }
  // three: {0,1,6} {2,5} {3,4} (10 / 9 / 9 pairs) | {3,7} {4,6} {0,1,2,5} (12 each)
  constexpr unsigned m7[3] = {0x43u, 0x24u, 0x18u}, m8[3] = {0x88u, 0x50u, 0x27u};
  return ND == 7 ? m7[which] : m8[which];
}
// First and last t of A digit s's MMAs (t < ND - s) whose level s + t is in `mask`.
constexpr int run_first(int nd, unsigned mask, int s) {
  for (int t = 0; t < nd - s; ++t)
    if ((mask >> (s + t)) & 1u) return t;
  return -1;
}
constexpr int run_last(int nd, unsigned mask, int s) {
  for (int t = nd - s - 1; t >= 0; --t)
    if ((mask >> (s + t)) & 1u) return t;
  return -1;
}

// The MMAs of A digit S against B digits T.. (S + T in MASK); every level starts afresh at
// its first MMA, (0, l), when `first` is set.  With one issuer (REUSE) A is held in the
// collector buffer from the first MMA of the run to the last; two issuers interleave their
// MMAs on the one tensor core, so each MMA then reads its own A.
template <int ND, unsigned MASK, int S, int T>
__device__ __forceinline__ void mma_digit_run(uint32_t tmem, uint64_t ad, uint64_t bd0,
                                              uint32_t first) {
  if constexpr (T < ND - S) {
    if constexpr ((MASK >> (S + T)) & 1u) {
      constexpr int f = run_first(ND, MASK, S), l = run_last(ND, MASK, S);
      constexpr int C = kIssuers > 1 || f == l ? 0 : (T == f ? 1 : (T == l ? 3 : 2));
      mma_bf16_ca<C>(tmem + (uint32_t)((S + T) * kBN), ad,
                     bd0 + (uint64_t)((T * kBPlane) >> 4), kIdesc, S == 0 && first ? 0u : 1u);
    }
    mma_digit_run<ND, MASK, S, T + 1>(tmem, ad, bd0, first);
  }
}
template <int ND, unsigned MASK, int S>
__device__ __forceinline__ void mma_kstep(uint32_t tmem, uint64_t a0, uint64_t bd0,
                                          uint32_t first) {
  if constexpr (S < ND) {
    mma_digit_run<ND, MASK, S, 0>(tmem, a0 + (uint64_t)((S * kAPlane) >> 4), bd0, first);
    mma_kstep<ND, MASK, S + 1>(tmem, a0, bd0, first);
  }
}

// Shared-memory descriptor of a K-major operand tile in the layout swizzled over rows of
// 2 kKS bytes (64-byte swizzle for kKS = 32, 32-byte for 16; 8-row groups of 16 kKS
// bytes); `saddr` may be advanced by 32 bytes (one 16-wide BF16 K step) inside the row.
__device__ __forceinline__ uint64_t desc_sw(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);       // start address
  d |= (uint64_t)1 << 16;                         // leading byte offset (unused: K fits a row)
  d |= (uint64_t)((16 * kKS) >> 4) << 32;         // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                         // descriptor version
  d |= (uint64_t)(kKS == 32 ? 4 : 6) << 61;       // layout: 64- or 32-byte swizzle
  return d;
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Lane 0 waits (bounded, or until another role aborted); the result goes to the warp.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = tc::wait_or_abort(bar, parity, abort, kWaitNs) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <int ND>
__global__ void __launch_bounds__(kThreads, 1)
    k_fp64tc(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
             const Job J) {
  constexpr int kDigits = ND, kLevels = ND;
  constexpr int kStageBytes = stage_bytes<ND>();
  constexpr int kStages = ring_stages<ND>();
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[kStages], empty[kStages], accfull, accempty, fin;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const int rank = (int)cluster_rank();
  const long long cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;

  if (warp == 1) tc::tmem_alloc(&tmem_sh, kTmemCols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 2 * kIssuers);  // both issuers of both CTAs of the pair
    }
    tc::mbar_init(&accfull, kIssuers);
    tc::mbar_init(&accempty, kDrainWarps);
    tc::mbar_init(&fin, kIssuers);
    tc::fence_mbar_init();
    abort_sh = 0;
  }
  tc::tc_fence_before();
  __syncthreads();
  cluster_sync();  // the peer's copies and arrivals may target this CTA's barriers from here on
  tc::tc_fence_after();
  const uint32_t tmem = tmem_sh;
  volatile int *abort = &abort_sh;

  // ---- MMA issuers: the digit pairs of the levels in MASK ---------------------------------
  auto issue = [&](auto maskc) {
    constexpr unsigned MASK = decltype(maskc)::value;
    long long it = 0, chunk = 0;
    bool ok = true, issued = false;
    for (long long pr = cid; pr < J.npairs && ok; pr += ncl) {
      int ra, rb;
      long long k0, klen, item;
      bool valid;
      decode_pair(J, pr, rank, &ra, &rb, &k0, &klen, &valid, &item);
      const long long nst = (klen + kKS - 1) / kKS;
      for (long long st = 0; st < nst; ++st, ++it) {
        const bool cstart = (st % kChunkStages) == 0;
        if (cstart && chunk > 0) {
          // the accumulators start afresh once the drain warps have read them
          if (!tc::wait_or_abort(&accempty, (uint32_t)((chunk - 1) & 1), abort, kWaitNs)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
        }
        const int slot = (int)(it % kStages);
        if (!tc::wait_or_abort(&full[slot], (uint32_t)((it / kStages) & 1), abort, kWaitNs)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        // one descriptor per stage; an operand tile at byte offset o of the stage is the
        // descriptor plus o / 16 (the start-address field; offsets stay below 2^18)
        const uint64_t d0 = desc_sw(tc::smem_u32(smem + slot * kStageBytes));
#pragma unroll
        for (int ks = 0; ks < kKS / 16; ++ks)
          mma_kstep<ND, MASK, 0>(tmem, d0 + (uint64_t)((ks * 32) >> 4),
                                 d0 + (uint64_t)((kDigits * kAPlane + ks * 32) >> 4),
                                 (cstart && ks == 0) ? 1u : 0u);
        issued = true;
        mma_commit_mc(&empty[slot]);  // the slot is free in both CTAs once all have read it
        if ((st % kChunkStages) == kChunkStages - 1 || st == nst - 1) {
          tc::mma_commit(&accfull);
          ++chunk;
        }
      }
    }
    // every MMA has completed before TMEM is released
    if (issued) tc::mma_commit(&fin);
    else tc::mbar_arrive(&fin);
    tma::bar_wait(&fin, 0u, kWaitNs);
  };

  if (warp == 0) {
    // ---- TMA producer ----------------------------------------------------------------
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      for (long long pr = cid; pr < J.npairs && ok; pr += ncl) {
        int ra, rb;
        long long k0, klen, item;
        bool valid;
        decode_pair(J, pr, rank, &ra, &rb, &k0, &klen, &valid, &item);
        const long long nst = (klen + kKS - 1) / kKS;
        for (long long st = 0; st < nst; ++st, ++it) {
          const int slot = (int)(it % kStages);
          const long long use = it / kStages;
          if (use > 0 && !tc::wait_or_abort(&empty[slot], (uint32_t)((use - 1) & 1), abort,
                                            kWaitNs)) {
            ok = false;
            break;
          }
          // this CTA's bytes: its own B planes and both halves of the A planes
          tma::bar_expect(&full[slot], (uint32_t)kStageBytes);
          uint8_t *sb = smem + slot * kStageBytes;
          const int kc = (int)(k0 + st * kKS);
          const int half_off = rank * (kAPlane / 2);
#pragma unroll
          for (int s = 0; s < kDigits; ++s)
            load_3d_mc(sb + s * kAPlane + half_off, &mA, kc, ra + rank * (kBM / 2), s, &full[slot]);
#pragma unroll
          for (int t = 0; t < kDigits; ++t)
            tma::load_3d(sb + kDigits * kAPlane + t * kBPlane, &mB, kc, rb, t, &full[slot]);
        }
      }
      // the copies issued last must land, and both CTAs' MMAs release the slots, before the
      // CTA may exit (bounded)
      for (long long u = it - 1; u >= 0 && u >= it - kStages; --u) {
        tma::bar_wait(&full[u % kStages], (uint32_t)((u / kStages) & 1), kWaitNs);
        tma::bar_wait(&empty[u % kStages], (uint32_t)((u / kStages) & 1), kWaitNs);
      }
    }
  } else if (warp <= kIssuers) {
    if (lane == 0) {
      if (warp == 1)
        issue(std::integral_constant<unsigned, issuer_mask<ND>(0)>{});
      else if (warp == 2)
        issue(std::integral_constant<unsigned, issuer_mask<ND>(1)>{});
      else if constexpr (kIssuers > 2)
        issue(std::integral_constant<unsigned, issuer_mask<ND>(2)>{});
    }
  } else {
    // ---- drain warps ---------------------------------------------------------------------
    const int q = warp & 3;                         // TMEM lane quarter this warp may read
    const int half = (warp - kIssuers - 1) >> 2;    // output columns kDrainCols half + ...
    const int row = q * 32 + lane;                  // tile row
    const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * kDrainCols);
    long long chunk = 0;
    bool ok = true;
    for (long long pr = cid; pr < J.npairs && ok; pr += ncl) {
      int ra, rb;
      long long k0, klen, item;
      bool valid;
      decode_pair(J, pr, rank, &ra, &rb, &k0, &klen, &valid, &item);
      const long long nst = (klen + kKS - 1) / kKS;
      const long long nch = (nst + kChunkStages - 1) / kChunkStages;
      long long hi[kDrainCols], lo[kDrainCols];
#pragma unroll
      for (int j = 0; j < kDrainCols; ++j) hi[j] = lo[j] = 0;
      for (long long c = 0; c < nch; ++c, ++chunk) {
        if (!warp_wait(&accfull, (uint32_t)(chunk & 1), abort)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
#pragma unroll
        for (int g = 0; g < kDrainCols / 4; ++g) {
          uint32_t v[kLevels][4];
#pragma unroll
          for (int l = 0; l < kLevels; ++l) tmem_ld4(tbase + (uint32_t)(l * kBN + g * 4), v[l]);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            long long L[kLevels];
#pragma unroll
            for (int l = 0; l < kLevels; ++l) L[l] = (long long)__float2int_rz(__uint_as_float(v[l][e]));
            hi[g * 4 + e] += (L[0] << 24) + (L[1] << 16) + (L[2] << 8) + L[3];
            long long lv = 0;
#pragma unroll
            for (int l = 4; l < kLevels; ++l) lv += L[l] << (8 * (kLevels - 1 - l));
            lo[g * 4 + e] += lv;
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&accempty);
      }
      if (!ok) break;
      if (!valid) continue;  // a stand-in member: zeros in, nothing out
      // epilogue: (2^(8 (ND - 4)) hi + lo) 2^(e_a + e_b - 2 (8 ND - 1) + 8 (ND - 1))
      constexpr double kHiW = (double)(1ll << (8 * (ND - 4)));
      constexpr int kShift = -2 * (8 * ND - 1) + 8 * (ND - 1);
      if (J.mode == MODE_GRAM) {
        // rows and columns beyond nc hold zero digits (the loads past the planes read 0)
        const int ea = ra + row < J.nc ? J.ea[ra + row] : 0;
        double *dst = J.part + (item * kBM + row) * kBN + half * kDrainCols;
#pragma unroll
        for (int j = 0; j < kDrainCols; j += 2) {
          const int cb = rb + half * kDrainCols + j;
          const int eb0 = cb < J.nc ? J.eb[cb] : 0, eb1 = cb + 1 < J.nc ? J.eb[cb + 1] : 0;
          double2 o;
          o.x = ldexp(fma((double)hi[j], kHiW, (double)lo[j]), ea + eb0 + kShift);
          o.y = ldexp(fma((double)hi[j + 1], kHiW, (double)lo[j + 1]), ea + eb1 + kShift);
          *reinterpret_cast<double2 *>(dst + j) = o;
        }
      } else {
        const long long r = ra + row;
        if (r < J.mrows) {
          const int ea = J.ea[r];
#pragma unroll
          for (int j = 0; j < kDrainCols; j += 2) {
            const int col = rb + half * kDrainCols + j;
            if (col < J.ld) {
              double2 o;
              o.x = ldexp(fma((double)hi[j], kHiW, (double)lo[j]), ea + J.eb[col] + kShift);
              o.y = ldexp(fma((double)hi[j + 1], kHiW, (double)lo[j + 1]),
                          ea + J.eb[col + 1] + kShift);
              if (J.mode == MODE_UPDATE_DELTA) {
                const double2 b = *reinterpret_cast<const double2 *>(J.base + r * J.ld + col);
                o.x += b.x;
                o.y += b.y;
              }
              *reinterpret_cast<double2 *>(J.out + r * J.ld + col) = o;
            }
          }
        }
      }
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  cluster_sync();  // nothing of the peer's still targets this CTA's shared memory
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
  if (threadIdx.x == 0 && abort_sh) atomicExch(J.err, 1);
}

// ---- digits ----------------------------------------------------------------------------
// Exponent of the largest |value| of a row: max < 2^e (0 for an all-zero row).
__device__ __forceinline__ int exponent_of(double mx) {
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  return e;
}

// The ND balanced base-256 digits of X = round(a 2^(8 ND - 1 - e)) (|a| < 2^e), as BF16 bit
// patterns; integer arithmetic on the bits of a.  Subnormal a (below 2^-1022) count as 0.
template <int ND>
__device__ __forceinline__ void digits_of(double a, int e, uint16_t (&d)[ND]) {
  constexpr int kDigits = ND;
  const long long bits = __double_as_longlong(a);
  const int be = (int)((bits >> 52) & 0x7FF);
  long long X = 0;
  if (be != 0) {
    const long long mant = (bits & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll;
    // a 2^(8 ND - 1 - e) = mant 2^sh, sh <= 8 ND - 54 since |a| < 2^e
    const int sh = be - 1075 + 8 * ND - 1 - e;
    if (sh >= 0) {
      X = mant << sh;
    } else if (sh > -64) {
      const int r = -sh;
      X = (mant + (1ll << (r - 1))) >> r;
    }
    if (bits < 0) X = -X;
  }
#pragma unroll
  for (int s = kDigits - 1; s >= 1; --s) {
    const int lo8 = (int)(X & 0xFF);
    const int dd = lo8 - ((lo8 & 0x80) << 1);
    d[s] = (uint16_t)(__float_as_uint((float)dd) >> 16);
    X = (X - dd) >> 8;
  }
  d[0] = (uint16_t)(__float_as_uint((float)(int)X) >> 16);
}

// Column exponents of Y = [U W] (nc = ld or 2 ld columns) over grid points [x0, x0 + m),
// encoded as e + 4096 (0: all zero); grid (column blocks of 256, row splits).
__global__ void k_colexp(const double *__restrict__ U, const double *__restrict__ W, int ld,
                         int nc, long long x0, long long m, int *__restrict__ enc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double *X = c < ld ? U : W;
  const int cc = c < ld ? c : c - ld;
  const long long per = (m + gridDim.y - 1) / gridDim.y;
  const long long r0 = (long long)blockIdx.y * per;
  const long long r1 = r0 + per < m ? r0 + per : m;
  const double *col = X + x0 * ld + cc;
  double mx = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
  long long r = r0;
  for (; r + 4 <= r1; r += 4) {  // four independent loads in flight per thread
    mx = fmax(mx, fabs(col[r * ld]));
    m1 = fmax(m1, fabs(col[(r + 1) * ld]));
    m2 = fmax(m2, fabs(col[(r + 2) * ld]));
    m3 = fmax(m3, fabs(col[(r + 3) * ld]));
  }
  for (; r < r1; ++r) mx = fmax(mx, fabs(col[r * ld]));
  mx = fmax(fmax(mx, m1), fmax(m2, m3));
  if (mx > 0.0) atomicMax(enc + c, exponent_of(mx) + 4096);
}

__global__ void k_decode_exp(const int *__restrict__ enc, int *__restrict__ e, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) e[i] = enc[i] > 0 ? enc[i] - 4096 : 0;
}

// Digit planes P[s][c][x] (x contiguous, pitch xp) of the columns of Y over grid points
// [x0, x0 + m): 64 x 64 tiles transposed through shared memory; x in [m, xp) gets zeros.
template <int ND>
__global__ void __launch_bounds__(256)
    k_split_cols(const double *__restrict__ U, const double *__restrict__ W, int ld, int nc,
                 long long x0, long long m, long long xp, const int *__restrict__ ecol,
                 uint16_t *__restrict__ P) {
  __shared__ double tile[64][65];
  const long long xb = (long long)blockIdx.x * 64;
  const int cb = blockIdx.y * 64;
  for (int i = threadIdx.x; i < 64 * 64; i += 256) {
    const int r = i >> 6, cc = i & 63, c = cb + cc;
    const long long x = xb + r;
    double v = 0.0;
    if (x < m && c < nc) v = c < ld ? U[(x0 + x) * ld + c] : W[(x0 + x) * ld + (c - ld)];
    tile[r][cc] = v;
  }
  __syncthreads();
  const int cc = threadIdx.x >> 2, rq = (threadIdx.x & 3) * 16, c = cb + cc;
  if (c >= nc) return;
  constexpr int kDigits = ND;
  const int e = ecol[c];
  uint32_t w[kDigits][8];
#pragma unroll
  for (int r = 0; r < 16; r += 2) {
    uint16_t d0[kDigits], d1[kDigits];
    digits_of<ND>(tile[rq + r][cc], e, d0);
    digits_of<ND>(tile[rq + r + 1][cc], e, d1);
#pragma unroll
    for (int s = 0; s < kDigits; ++s) w[s][r >> 1] = (uint32_t)d0[s] | ((uint32_t)d1[s] << 16);
  }
  const long long off = (long long)c * xp + xb + rq;
#pragma unroll
  for (int s = 0; s < kDigits; ++s) {
    uint4 *dst = reinterpret_cast<uint4 *>(P + (long long)s * nc * xp + off);
    dst[0] = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    dst[1] = make_uint4(w[s][4], w[s][5], w[s][6], w[s][7]);
  }
}

// Digit planes Q[s][x][k] of the rows of [U W] (k < kdim = ld or 2 ld; W may be null when
// kdim = ld) over grid points [x0, x0 + m), one exponent per row; one warp per row.
template <int ND>
__global__ void __launch_bounds__(256)
    k_split_rows(const double *__restrict__ U, const double *__restrict__ W, int ld, int kdim,
                 long long x0, long long m, int *__restrict__ erow, uint16_t *__restrict__ Q) {
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= m) return;
  const double *ur = U + (x0 + r) * ld;
  const double *wr = W ? W + (x0 + r) * ld : nullptr;
  double mx = 0.0;
  for (int k = 2 * lane; k < kdim; k += 64) {
    const double2 v = *reinterpret_cast<const double2 *>(k < ld ? ur + k : wr + (k - ld));
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  constexpr int kDigits = ND;
  const int e = exponent_of(mx);
  if (lane == 0) erow[r] = e;
  for (int k = 8 * lane; k < kdim; k += 256) {
    const double *src = k < ld ? ur + k : wr + (k - ld);
    uint32_t w[kDigits][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 v = *reinterpret_cast<const double2 *>(src + 2 * i);
      uint16_t d0[kDigits], d1[kDigits];
      digits_of<ND>(v.x, e, d0);
      digits_of<ND>(v.y, e, d1);
#pragma unroll
      for (int s = 0; s < kDigits; ++s) w[s][i] = (uint32_t)d0[s] | ((uint32_t)d1[s] << 16);
    }
#pragma unroll
    for (int s = 0; s < kDigits; ++s)
      *reinterpret_cast<uint4 *>(Q + ((long long)s * m + r) * kdim + k) =
          make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  }
}

// Digit planes B[s][j][k] of the update's coefficient columns: column j of
// [KU - delta I; KW] (k < kdim; KW may be null when kdim = ld), one exponent per j;
// one warp per column.
template <int ND>
__global__ void __launch_bounds__(256)
    k_split_coef(const double *__restrict__ KU, const double *__restrict__ KW, int ld, int kdim,
                 int delta, int *__restrict__ ecol, uint16_t *__restrict__ B) {
  const int j = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= ld) return;
  auto val = [&](int k) -> double {
    if (k < ld) return KU[(long long)k * ld + j] - (delta && k == j ? 1.0 : 0.0);
    return KW[(long long)(k - ld) * ld + j];
  };
  double mx = 0.0;
  for (int k = lane; k < kdim; k += 32) mx = fmax(mx, fabs(val(k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  constexpr int kDigits = ND;
  const int e = exponent_of(mx);
  if (lane == 0) ecol[j] = e;
  for (int k = 8 * lane; k < kdim; k += 256) {
    uint32_t w[kDigits][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint16_t d0[kDigits], d1[kDigits];
      digits_of<ND>(val(k + 2 * i), e, d0);
      digits_of<ND>(val(k + 2 * i + 1), e, d1);
#pragma unroll
      for (int s = 0; s < kDigits; ++s) w[s][i] = (uint32_t)d0[s] | ((uint32_t)d1[s] << 16);
    }
#pragma unroll
    for (int s = 0; s < kDigits; ++s)
      *reinterpret_cast<uint4 *>(B + ((long long)s * ld + j) * kdim + k) =
          make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  }
}

// G[a][b] (upper triangle, b >= a) += sum over the K ranges of the tile partials, in the
// order of the K ranges; grid (tiles, element slices).
__global__ void k_gram_acc(const double *__restrict__ part, int ntiles, int nranges, int nJ,
                           int nc, double *__restrict__ G) {
  int I, Jt;
  tile_of(blockIdx.x, nJ, &I, &Jt);
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < kBM * kBN; e += gridDim.y * blockDim.x) {
    const int a = I * kBM + e / kBN, b = Jt * kBN + e % kBN;
    if (a >= nc || b >= nc || b < a) continue;
    double s = 0.0;
    for (int q = 0; q < nranges; ++q) s += part[((long long)q * ntiles + blockIdx.x) * (kBM * kBN) + e];
    G[(long long)a * nc + b] += s;
  }
}

// C = <W,U>, S = <W,W>, D = <U,U> from the upper triangle of G = [U W]^T [U W]
// (zero outside p x p); any output may be null.
__global__ void k_gram_scatter(const double *__restrict__ G, int nc, int ld, int p,
                               double *__restrict__ C, double *__restrict__ S,
                               double *__restrict__ D) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)ld * ld;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), j = (int)(e % ld);
    const bool in = i < p && j < p;
    const int a = i < j ? i : j, b = i < j ? j : i;
    if (D) D[e] = in ? G[(long long)a * nc + b] : 0.0;
    if (C) C[e] = in ? G[(long long)j * nc + ld + i] : 0.0;
    if (S) S[e] = in ? G[(long long)(ld + a) * nc + ld + b] : 0.0;
  }
}

// Clusters of two CTAs (one per SM) that can be resident at once, queried once per digit
// count on the current device.
template <int ND>
op_status resident_clusters(int *n) {
  static int dev_of = -1, cached = 0;
  int dev = 0;
  OP_CUDA(cudaGetDevice(&dev));
  if (dev_of != dev) {
    OP_CUDA(cudaFuncSetAttribute(k_fp64tc<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_bytes<ND>()));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * (unsigned)num_sms());
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem_bytes<ND>();
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int c = 0;
    OP_CUDA(cudaOccupancyMaxActiveClusters(&c, k_fp64tc<ND>, &cfg));
    if (c < 1) {
      set_error("k_fp64tc: no cluster of two CTAs fits an SM pair");
      return OP_ERR_CUDA;
    }
    cached = c;
    dev_of = dev;
  }
  *n = cached;
  return OP_OK;
}

template <int ND>
op_status launch_mma(const CUtensorMap &mA, const CUtensorMap &mB, const Job &J,
                     cudaStream_t st) {
  if (J.npairs <= 0) return OP_OK;
  int ncl = 0;
  OP_TRY(resident_clusters<ND>(&ncl));
  const long long clusters = std::min<long long>(J.npairs, ncl);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(2 * clusters));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem_bytes<ND>();
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  OP_CUDA(cudaLaunchKernelEx(&cfg, k_fp64tc<ND>, mA, mB, J));
  count_launch();
  OP_LAUNCH("k_fp64tc");
  return OP_OK;
}

long long chunk_rows(long long n, int ld) {
  // digit planes of one chunk: up to 8 x 2 ld x rows BF16 = 32 ld rows bytes, at most 8 GiB
  long long r = ((long long)8 << 30) / (32ll * ld);
  r = r / 256 * 256;
  if (r < 4096) r = 4096;
  const long long nr = (n + 63) / 64 * 64;
  return r < nr ? r : nr;
}

// Upper-triangle tiles of an nc x nc Gram in 128 x 64 tiles (every row of tiles I has
// nJ - 2 I >= 1 of them); *npt: the tile pairs (I, J), (I, J + 1) of the rows.
int gram_tiles(int nc, int *nI, int *nJ, int *npt = nullptr) {
  *nI = (nc + kBM - 1) / kBM;
  *nJ = (nc + kBN - 1) / kBN;
  int t = 0, pt = 0;
  for (int i = 0; i < *nI; ++i) {
    const int c = *nJ - 2 * i > 0 ? *nJ - 2 * i : 0;
    t += c;
    pt += (c + 1) / 2;
  }
  if (npt) *npt = pt;
  return t;
}

// K ranges per chunk: the fewest that make the tile pairs a near multiple of the clusters
// (two SMs each).
int gram_ranges(int npt, long long m) {
  const int slots = std::max(1, num_sms() / 2);
  const long long maxr = std::max<long long>(1, (m + 1023) / 1024);
  int best = 1;
  double best_eff = 0.0;
  for (int r = 1; r <= 64 && r <= maxr; ++r) {
    const long long items = (long long)npt * r;
    const long long waves = (items + slots - 1) / slots;
    const double eff = (double)items / (double)(waves * slots);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = r;
    }
    if (eff >= 0.95 && items >= slots) break;
  }
  return best;
}

// Scratch layout: digit planes of one chunk (7 x 2 ld x (rows + 64) BF16), row and column
// exponents, the Gram accumulator G (2 ld x 2 ld FP64), the coefficient planes
// (7 x ld x 2 ld BF16) and the Gram tile partials of one chunk.
struct Carve {
  uint16_t *planes;
  int *e1, *e2, *enc;
  double *part, *G;
  uint16_t *coef;
  size_t total;
};

long long gram_items(int ntiles, int npt, long long m) {
  const int nr = gram_ranges(npt, m);
  long long kr = (m + nr - 1) / nr;
  kr = (kr + kKS - 1) / kKS * kKS;
  return (long long)ntiles * ((m + kr - 1) / kr);
}

Carve carve(void *ws, long long n, int ld) {
  const long long rows = chunk_rows(n, ld);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t off = 0;
  Carve c;
  const uintptr_t p = (uintptr_t)ws;
  c.planes = (uint16_t *)(p + off);
  off += up((size_t)kMaxDigits * 2 * ld * (rows + 64) * 2);
  c.e1 = (int *)(p + off);
  off += up((size_t)(rows + 2 * ld) * 4);
  c.e2 = (int *)(p + off);
  off += up((size_t)2 * ld * 4);
  c.enc = (int *)(p + off);
  off += up((size_t)2 * ld * 4);
  c.G = (double *)(p + off);
  off += up((size_t)4 * ld * ld * 8);
  c.coef = (uint16_t *)(p + off);
  off += up((size_t)kMaxDigits * ld * 2 * ld * 2);
  c.part = (double *)(p + off);
  // the most items of any chunk, for [U W] (2 ld columns) and for U alone (ld)
  long long items = 0;
  for (int nc : {2 * ld, ld}) {
    int nI, nJ, npt;
    const int nt = gram_tiles(nc, &nI, &nJ, &npt);
    items = std::max(items, gram_items(nt, npt, std::min(rows, n)));
    if (n % rows) items = std::max(items, gram_items(nt, npt, n % rows));
  }
  off += up((size_t)items * kBM * kBN * 8);
  c.total = off;
  return c;
}

}  // namespace

size_t fp64tc_workspace_bytes(long long n, int ld) {
  if (n < 1 || ld < 8) return 0;
  return carve(nullptr, n, ld).total;
}

op_status gram_fp64tc(long long n, int p, int ld, const double *U, const double *W, double *C,
                      double *S, double *D, void *ws, size_t ws_bytes, int *err,
                      cudaStream_t st) {
  if (n < 1 || p < 1 || p > ld || ld % 8 != 0 || !U || (!W && (C || S))) {
    set_error("gram_fp64tc: bad sizes or missing W (n=%lld p=%d ld=%d)", n, p, ld);
    return OP_ERR_ARG;
  }
  if (!ws || ws_bytes < fp64tc_workspace_bytes(n, ld)) {
    set_error("gram_fp64tc: workspace too small (%zu < %zu)", ws_bytes,
              fp64tc_workspace_bytes(n, ld));
    return OP_ERR_ARG;
  }
  const Carve cv = carve(ws, n, ld);
  const int nc = W ? 2 * ld : ld;
  int nI, nJ, npt;
  const int ntiles = gram_tiles(nc, &nI, &nJ, &npt);
  const long long rows = chunk_rows(n, ld);
  OP_CUDA(cudaMemsetAsync(cv.G, 0, (size_t)nc * nc * sizeof(double), st));
  for (long long x0 = 0; x0 < n; x0 += rows) {
    const long long m = std::min(rows, n - x0);
    const long long xp = (m + 63) / 64 * 64;
    OP_CUDA(cudaMemsetAsync(cv.enc, 0, (size_t)nc * sizeof(int), st));
    const int ysplit = (int)std::min<long long>(std::max<long long>(1, m / 512),
                                                std::max(1, 4 * num_sms() / ((nc + 255) / 256)));
    k_colexp<<<dim3((nc + 255) / 256, ysplit), 256, 0, st>>>(U, W, ld, nc, x0, m, cv.enc);
    count_launch();
    k_decode_exp<<<(nc + 255) / 256, 256, 0, st>>>(cv.enc, cv.e2, nc);
    count_launch();
    k_split_cols<kGramDigits><<<dim3((unsigned)(xp / 64), (nc + 63) / 64), 256, 0, st>>>(
        U, W, ld, nc, x0, m, xp, cv.e2, cv.planes);
    count_launch();
    OP_LAUNCH("fp64tc split");
    CUtensorMap mA, mB;
    // A: each CTA of a pair loads (and multicasts) one 64-row half of the 128 A rows
    OP_TRY(tma_map_3d_bf16_sw(&mA, cv.planes, (uint64_t)xp, (uint64_t)nc, kGramDigits, kBM / 2, kKS));
    OP_TRY(tma_map_3d_bf16_sw(&mB, cv.planes, (uint64_t)xp, (uint64_t)nc, kGramDigits, kBN, kKS));
    const int nr = gram_ranges(npt, m);
    long long kr = (m + nr - 1) / nr;
    kr = (kr + kKS - 1) / kKS * kKS;
    const int nranges = (int)((m + kr - 1) / kr);
    Job J{};
    J.mode = MODE_GRAM;
    J.npairs = (long long)npt * nranges;
    J.npt = npt;
    J.nc = nc;
    J.nI = nI;
    J.nJ = nJ;
    J.ntiles = ntiles;
    J.krange = kr;
    J.kext = m;
    J.part = cv.part;
    J.ea = cv.e2;
    J.eb = cv.e2;
    J.err = err;
    OP_TRY(launch_mma<kGramDigits>(mA, mB, J, st));
    k_gram_acc<<<dim3(ntiles, 8), 256, 0, st>>>(cv.part, ntiles, nranges, nJ, nc, cv.G);
    count_launch();
    OP_LAUNCH("k_gram_acc");
  }
  k_gram_scatter<<<(ld * ld + 255) / 256, 256, 0, st>>>(cv.G, nc, ld, p, C, S, D);
  count_launch();
  OP_LAUNCH("k_gram_scatter");
  return OP_OK;
}

op_status update_fp64tc(long long n, int ld, const double *U, const double *W, const double *KU,
                        const double *KW, bool delta, double *Unew, void *ws, size_t ws_bytes,
                        int *err, cudaStream_t st) {
  if (n < 1 || ld % 8 != 0 || !U || !KU || (W && !KW) || !Unew) {
    set_error("update_fp64tc: bad arguments (n=%lld ld=%d)", n, ld);
    return OP_ERR_ARG;
  }
  if (!ws || ws_bytes < fp64tc_workspace_bytes(n, ld)) {
    set_error("update_fp64tc: workspace too small (%zu < %zu)", ws_bytes,
              fp64tc_workspace_bytes(n, ld));
    return OP_ERR_ARG;
  }
  const Carve cv = carve(ws, n, ld);
  const int kdim = W ? 2 * ld : ld;
  k_split_coef<kUpdateDigits><<<(ld * 32 + 255) / 256, 256, 0, st>>>(
      KU, W ? KW : nullptr, ld, kdim, delta ? 1 : 0, cv.e2, cv.coef);
  count_launch();
  OP_LAUNCH("k_split_coef");
  CUtensorMap mB;
  OP_TRY(tma_map_3d_bf16_sw(&mB, cv.coef, (uint64_t)kdim, (uint64_t)ld, kUpdateDigits, kBN, kKS));
  const long long rows = chunk_rows(n, ld);
  const int ntn = (ld + kBN - 1) / kBN;
  for (long long x0 = 0; x0 < n; x0 += rows) {
    const long long m = std::min(rows, n - x0);
    k_split_rows<kUpdateDigits><<<(unsigned)((m * 32 + 255) / 256), 256, 0, st>>>(
        U, W, ld, kdim, x0, m, cv.e1, cv.planes);
    count_launch();
    OP_LAUNCH("k_split_rows");
    CUtensorMap mA;
    OP_TRY(tma_map_3d_bf16_sw(&mA, cv.planes, (uint64_t)kdim, (uint64_t)m, kUpdateDigits, kBM / 2, kKS));
    Job J{};
    J.mode = delta ? MODE_UPDATE_DELTA : MODE_UPDATE;
    J.npairs = ((m + kBM - 1) / kBM) * ((ntn + 1) / 2);
    J.mrows = m;
    J.ntn = ntn;
    J.kdim = kdim;
    J.ld = ld;
    J.base = U + x0 * ld;
    J.out = Unew + x0 * ld;
    J.ea = cv.e1;
    J.eb = cv.e2;
    J.err = err;
    OP_TRY(launch_mma<kUpdateDigits>(mA, mB, J, st));
  }
  return OP_OK;
}

}  // namespace opevo
