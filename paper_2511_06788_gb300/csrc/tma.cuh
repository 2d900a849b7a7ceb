// Tensor Memory Accelerator (TMA) helpers for sm_103a: host-side encoding of
// tiled tensor maps (through the driver entry point, so the library needs no
// link against libcuda) and the device-side bulk-tensor load with mbarrier
// completion, written as inline PTX.
//
// Alignment rules honoured by every caller: the global base address is 16-byte
// aligned, every stride is a multiple of 16 bytes, the innermost box extent is a
// multiple of 16 bytes and every innermost load coordinate is a multiple of 4
// four-byte elements.  Loads may start at negative or out-of-range coordinates
// (the elements outside the tensor read as zero); this file issues no stores.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "common.cuh"

namespace opevo {

// 4-D FP32 tensor map over a row-major block laid out as [d3][d2][d1][d0]
// (d0 innermost, contiguous), box = (b0, b1, b2, b3) elements.
op_status tma_map_4d_f32(CUtensorMap *map, const void *base, const uint64_t dims[4],
                         const uint32_t box[4]);

// 2-D FP32 tensor map over a row-major [outer][inner] array with a box of 32 x
// box_outer elements landing in the 128-byte-swizzled layout (rows of 128 bytes,
// 16-byte chunk c of row r at chunk c ^ (r % 8) within each 1024-byte group of 8
// rows): the K-major operand layout of the tensor-core MMA.  The destination must
// be 1024-byte aligned and every inner coordinate a multiple of 4.
op_status tma_map_2d_f32_sw128(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer,
                               uint32_t box_outer);

// 3-D BF16 tensor map over [planes][rows][inner] (inner contiguous, a multiple of 8
// elements) with a box of box_k x box_rows x 1 elements, box_k = 32 or 16, landing in the
// K-major layout swizzled over rows of 2 box_k bytes (64- or 32-byte swizzle: 16-byte
// chunk c of row r at chunk c ^ ((r / 2) % 4), resp. c ^ ((r / 4) % 2), within each group
// of 8 rows).  Destinations must be 1024-byte aligned and every inner coordinate a
// multiple of 8.
op_status tma_map_3d_bf16_sw(CUtensorMap *map, const void *base, uint64_t inner,
                             uint64_t rows, uint64_t planes, uint32_t box_rows, uint32_t box_k);

namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_bar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of incoming bulk-copy data.
__device__ __forceinline__ void bar_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// One plain arrival (a phase with no data).
__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Wait until the phase of the given parity has completed; false once `limit_ns`
// nanoseconds have passed without that (the caller then reports an error).
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  const uint32_t a = smem_addr(bar);
  uint64_t t0 = 0;
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    const uint64_t now = global_ns();
    if (t0 == 0) {
      t0 = now;
    } else if (now - t0 > limit_ns) {
      return false;
    }
  }
}

// Generic-proxy shared-memory accesses of this thread become ordered before
// later async-proxy (TMA) accesses once a barrier orders the threads.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk tensor load of one box into shared memory; completion is counted in bytes
// on `bar`.
__device__ __forceinline__ void load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                        int c3, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                        uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void load_2d(void *dst, const CUtensorMap *map, int c0, int c1,
                                        uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace tma
}  // namespace opevo
