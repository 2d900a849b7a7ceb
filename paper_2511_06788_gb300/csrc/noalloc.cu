// op_gram_noalloc: the inner matrices of [U W] computed without any device
// allocation by the library or the caller.
//
// Who needs it: a host program that cannot hand this library a workspace and
// must not let it call cudaMalloc, for example because all device memory is
// owned by another allocator with a hard budget (a framework's caching
// allocator or a fixed pool), or because the calling loop is latency critical
// and may not enter the driver's allocator.  The chunk partials of the Gram
// reduction then live in one fixed device array that this file defines; the
// caller still provides U, W and the output matrices.
//
// The array is a file-scope __device__ variable: it belongs to the library's
// module, so each GPU on which the module is loaded holds it (16 MiB) until the
// process exits; under CUDA's default lazy module loading that happens on the
// first call on the device.  Host code may not use its name as a device
// address, so the address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call, and kept
// (a cudaDeviceReset() unloads the module and invalidates it).
//
// FP32 blocks use the chunks of op_gram and add each chunk's FP64 partial tile
// into one tile per output tile with atomics, so one tile per output tile
// (not one per chunk) has to fit in the array.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace opevo {
namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr size_t kHeader = 256;                      // first int: bounded-wait flag
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_lock;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (set-up on first use).
op_status scratch_address(void **out) {
  int dev = 0;
  OP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("op_gram_noalloc: device ordinal %d out of range", dev);
    return OP_ERR_ARG;
  }
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(scratch)");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return OP_OK;
}

}  // namespace
}  // namespace opevo

using namespace opevo;

extern "C" op_status op_gram_noalloc(int prec, long long n, int p, int ld, const void *U,
                                     const void *W, double *C, double *S, double *D,
                                     void *stream) {
  if (prec != OP_FP64 && prec != OP_FP32) {
    set_error("op_gram_noalloc: unsupported precision mode %d", prec);
    return OP_ERR_ARG;
  }
  if (p < 1 || ld < p || ld % 8 != 0 || n < 1 || !U || !W || ((uintptr_t)U & 15) ||
      ((uintptr_t)W & 15)) {
    set_error("op_gram_noalloc: need n >= 1, 1 <= p <= ld, ld %% 8 == 0 and 16-byte aligned "
              "U, W (n=%lld p=%d ld=%d)", n, p, ld);
    return OP_ERR_ARG;
  }
  void *base = nullptr;
  OP_TRY(scratch_address(&base));
  cudaStream_t st = (cudaStream_t)stream;
  // the bounded-wait flag must start at zero; the partials are written before read
  OP_CUDA(cudaMemsetAsync(base, 0, sizeof(int), st));
  void *part = (char *)base + kHeader;
  const size_t part_bytes = kScratchBytes - kHeader;
  op_status s;
  if (prec == OP_FP64)
    s = gram_fixed_scratch<double>(n, p, ld, (const double *)U, (const double *)W, C, S, D, part,
                                   part_bytes, st);
  else
    s = gram_tc_fixed_scratch(n, p, ld, (const float *)U, (const float *)W, C, S, D, part,
                              part_bytes, (int *)base, st);
  if (s != OP_OK) return s;
  int flag = 0;
  OP_CUDA(cudaMemcpyAsync(&flag, base, sizeof(int), cudaMemcpyDeviceToHost, st));
  OP_CUDA(cudaStreamSynchronize(st));
  if (flag) {
    set_error("op_gram_noalloc: a bounded device wait gave up");
    return OP_ERR_TIMEOUT;
  }
  return OP_OK;
}
