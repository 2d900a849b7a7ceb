// Peak-rate microbenchmarks of the units the scheme's kernels are bound by, for roofline
// denominators that the library measures itself (no GPU setting is read or changed):
//   OP_PEAK_FP64_FMA   FP64 FMA on the CUDA cores: 8 independent chains x = x a + b per
//                      thread, 2 flops each;
//   OP_PEAK_TF32_MMA   tcgen05.mma kind::tf32, M = 128, N = 256, K = 8 per instruction;
//   OP_PEAK_BF16_MMA   tcgen05.mma kind::f16 (BF16), M = 128, N = 256, K = 16;
//   OP_PEAK_BF16_MMA_N64  the same at N = 64, the shape of the FP64 digit products, on
//                      eight accumulators in turn, every MMA with a new A tile: reading
//                      A (128 x 16) from shared memory for each 128 x 64 x 16 product
//                      holds N = 64 to about half the N = 256 rate;
//   OP_PEAK_BF16_MMA_N64_AREUSE  N = 64 with each A tile held in the collector buffer over
//                      four MMAs against four different B tiles (fill, use, use, lastuse),
//                      the way the digit products issue them.
// The MMA kernels run one CTA per SM; one thread issues back-to-back MMAs on operand tiles
// resident in shared memory into two alternating TMEM accumulators (no memory traffic),
// then waits (bounded) for their completion.  Rates are flops over the CUDA-event time of
// the launch on `stream`.
#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace opevo {
namespace {

__global__ void __launch_bounds__(256) k_peak_dfma(int iters, double a, double b,
                                                   double *__restrict__ sink) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int kPM = 128, kPN = 256;

// BF16 MMA with the A operand's collector buffer: op 1 fill, 2 use, 3 lastuse.
__device__ __forceinline__ void mma_n64_areuse(uint32_t d, uint64_t ad, uint64_t bd, uint32_t id,
                                               uint32_t acc, int op) {
  if (op == 1)
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(d), "l"(ad), "l"(bd), "r"(id), "r"(acc) : "memory");
  else if (op == 2)
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(d), "l"(ad), "l"(bd), "r"(id), "r"(acc) : "memory");
  else
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(d), "l"(ad), "l"(bd), "r"(id), "r"(acc) : "memory");
}
constexpr int kPA = kPM * 128, kPB = kPN * 128;  // one 128-byte K row per operand row
constexpr int kPeakSmem = kPA + kPB + 1024;

// kind: 1 TF32 (K = 8 per MMA), 2 BF16 (K = 16), 3 BF16 at N = 64, 4 BF16 at N = 64 with A
// reuse; `mmas` instructions per CTA (a multiple of 4).
__global__ void __launch_bounds__(128, 1) k_peak_mma(int kind, int mmas, int *err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t done;
  __shared__ uint32_t tmem_sh;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // small non-zero operands (1/64 in both formats' bit patterns' range): no overflow
  for (int i = threadIdx.x; i < (kPA + kPB) / 4; i += blockDim.x) {
    const float v = 0.015625f * (float)((i % 7) - 3);
    if (kind == 1) {
      reinterpret_cast<float *>(smem)[i] = v;
    } else {
      const uint32_t h = __float_as_uint(v) >> 16;
      reinterpret_cast<uint32_t *>(smem)[i] = h | (h << 16);
    }
  }
  if (threadIdx.x < 32) tc::tmem_alloc(&tmem_sh, 512);
  if (threadIdx.x == 0) {
    tc::mbar_init(&done, 1);
    tc::fence_mbar_init();
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_sh;
  if (threadIdx.x == 0) {
    const uint32_t a = tc::smem_u32(smem), b = a + kPA;
    const int nn = kind >= 3 ? 64 : kPN;
    const uint32_t id = kind == 1 ? tc::idesc_tf32(kPM, kPN) : tc::idesc_bf16(kPM, nn);
    if (kind == 4) {
      // A fixed over four MMAs, B the four 64-row quarters of the B tile; K step per group
      for (int i = 0; i < mmas; i += 4) {
        const uint32_t k = (uint32_t)((i >> 2) & 3) * 32;
        const uint64_t ad = tc::desc_sw128(a + k);
        const uint32_t d = tmem + (uint32_t)(((i >> 2) & 1) * kPN);
        const uint32_t acc = i >= 8 ? 1u : 0u;
        mma_n64_areuse(d, ad, tc::desc_sw128(b + k), id, acc, 1);
        mma_n64_areuse(d + 64, ad, tc::desc_sw128(b + 8192 + k), id, acc, 2);
        mma_n64_areuse(d + 128, ad, tc::desc_sw128(b + 16384 + k), id, acc, 2);
        mma_n64_areuse(d + 192, ad, tc::desc_sw128(b + 24576 + k), id, acc, 3);
      }
    } else {
      // consecutive MMAs go to different accumulators (2 of 256 columns, or 8 of 64 at
      // N = 64), so no MMA waits for its predecessor's result
      const int nacc = kind == 3 ? 8 : 2;
      for (int i = 0; i < mmas; ++i) {
        const uint32_t k = (uint32_t)(i & 3) * 32;  // the four 32-byte K steps of the row
        const uint64_t ad = tc::desc_sw128(a + k), bd = tc::desc_sw128(b + k);
        const uint32_t d = tmem + (uint32_t)((i % nacc) * (512 / nacc));
        if (kind == 1)
          tc::mma_tf32(d, ad, bd, id, i >= nacc ? 1u : 0u);
        else
          tc::mma_bf16(d, ad, bd, id, i >= nacc ? 1u : 0u);
      }
    }
    tc::mma_commit(&done);
    if (!tc::mbar_wait(&done, 0)) atomicExch(err, 1);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

}  // namespace
}  // namespace opevo

using namespace opevo;

extern "C" op_status op_peak_rate(int kind, double *tflops, void *stream) {
  if (!tflops || kind < OP_PEAK_FP64_FMA || kind > OP_PEAK_BF16_MMA_N64_AREUSE) {
    set_error("op_peak_rate: bad kind %d or null output", kind);
    return OP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int sms = num_sms();
  void *buf = nullptr;
  OP_CUDA(cudaMalloc(&buf, (size_t)sms * 4 * 256 * sizeof(double) + 256));
  int *err = (int *)buf;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  op_status s = OP_OK;
  double flops = 0.0;
  float ms = 0.f;
  for (int rep = 0; rep < 3 && s == OP_OK; ++rep) {  // the last of three launches is timed
    cudaMemsetAsync(err, 0, sizeof(int), st);
    cudaEventRecord(e0, st);
    if (kind == OP_PEAK_FP64_FMA) {
      const int iters = 1 << 14, grid = sms * 4, block = 256;
      k_peak_dfma<<<grid, block, 0, st>>>(iters, 0.999999, 1e-7, (double *)((char *)buf + 256));
      flops = 2.0 * 8.0 * iters * (double)grid * block;
    } else {
      const int mmas = 1 << 15;
      cudaFuncSetAttribute(k_peak_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, kPeakSmem);
      k_peak_mma<<<sms, 128, kPeakSmem, st>>>(
          kind == OP_PEAK_TF32_MMA ? 1 : (kind == OP_PEAK_BF16_MMA ? 2 : kind), mmas, err);
      flops = 2.0 * kPM * (kind >= OP_PEAK_BF16_MMA_N64 ? 64 : kPN) *
              (kind == OP_PEAK_TF32_MMA ? 8 : 16) * (double)mmas * sms;
    }
    count_launch();
    cudaEventRecord(e1, st);
    const cudaError_t ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) s = cuda_status(ce, "op_peak_rate");
    else if (cudaGetLastError() != cudaSuccess) s = cuda_status(cudaErrorLaunchFailure, "op_peak_rate");
    cudaEventElapsedTime(&ms, e0, e1);
  }
  int h = 0;
  if (s == OP_OK) {
    cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (h) {
      set_error("op_peak_rate: a bounded wait gave up");
      s = OP_ERR_TIMEOUT;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (s == OP_OK) *tflops = flops / (ms * 1e-3) / 1e12;
  return s;
}
