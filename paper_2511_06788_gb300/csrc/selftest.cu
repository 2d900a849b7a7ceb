// Self-test of the library's failure detection on the device: every wait inside a
// kernel is bounded, and on expiry the kernel sets an error word that the host
// turns into OP_ERR_TIMEOUT.  The probes below wait on an mbarrier that nothing
// ever completes (a flag that no one sets), once with each kind of bounded wait the
// kernels use, and report that they gave up and how long that took.  Nothing is
// faulted or trapped; the GPU context stays usable.
#include "common.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace opevo {
namespace {

// mode 0: the %globaltimer-bounded wait of the TMA ring (limit_ns);
// mode 1: the iteration-bounded wait of the tensor-core kernels.
__global__ void k_wait_probe(int mode, unsigned long long limit_ns, int *gave_up,
                             unsigned long long *elapsed_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tma::bar_init(&bar, 1);
    tma::fence_bar_init();
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const unsigned long long t0 = tma::global_ns();
  const bool done = mode == 0 ? tma::bar_wait(&bar, 0, limit_ns) : tc::mbar_wait(&bar, 0);
  *elapsed_ns = tma::global_ns() - t0;
  *gave_up = done ? 0 : 1;
}

}  // namespace
}  // namespace opevo

using namespace opevo;

extern "C" op_status op_selftest_bounded_waits(double *seconds, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int *flags = nullptr;
  unsigned long long *el = nullptr;
  OP_CUDA(cudaMalloc(&flags, 2 * sizeof(int)));
  cudaError_t e = cudaMalloc(&el, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaFree(flags);
    return cuda_status(e, "cudaMalloc");
  }
  int hf[2] = {0, 0};
  unsigned long long he[2] = {0, 0};
  for (int mode = 0; mode < 2 && e == cudaSuccess; ++mode) {
    k_wait_probe<<<1, 32, 0, st>>>(mode, 200000000ull, flags + mode, el + mode);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(he, el, sizeof(he), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(flags);
  cudaFree(el);
  if (e != cudaSuccess) return cuda_status(e, "op_selftest_bounded_waits");
  if (seconds) {
    seconds[0] = 1e-9 * (double)he[0];
    seconds[1] = 1e-9 * (double)he[1];
  }
  if (!hf[0] || !hf[1]) {
    set_error("a bounded wait did not give up on an mbarrier that never completes");
    return OP_ERR_STATE;
  }
  return OP_OK;
}
