// Self-test of the bounded device waits.  Every wait in the library's kernels (on
// an mbarrier phase: TMA completions, MMA completions, accumulator hand-offs) gives
// up after a time limit, sets a flag in device memory and lets the kernel return,
// so that a stalled pipeline ends as a status (DPT_ERR_TIMEOUT) instead of a hung
// GPU.  This entry point exercises that path on purpose without any fault: one
// thread waits on a barrier phase that nothing completes, with a short limit.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/dpt.h"
#include "dpt_device.cuh"

namespace dpt {
namespace {

__global__ void k_wait_probe(unsigned* flag, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // phase 0 of a fresh barrier with one expected arrival that never comes
    if (mbar_wait_ns(&bar, 0, flag, limit_ns)) atomicExch(flag, 2u);
  }
}

}  // namespace
}  // namespace dpt

extern "C" dpt_status dpt_selftest_bounded_wait(double seconds, void* stream) {
  if (!(seconds > 0.0) || seconds > 5.0) return DPT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return DPT_ERR_NOMEM;
  }
  unsigned h = 0;
  dpt_status ret = DPT_ERR_CUDA;
  if (cudaMemsetAsync(flag, 0, sizeof(unsigned), s) == cudaSuccess) {
    dpt::k_wait_probe<<<1, 32, 0, s>>>(flag, (uint64_t)std::llround(seconds * 1e9));
    if (cudaGetLastError() == cudaSuccess &&
        cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess)
      ret = (h == 1u) ? DPT_ERR_TIMEOUT : DPT_ERR_CUDA;
  }
  cudaFree(flag);
  return ret;
}
