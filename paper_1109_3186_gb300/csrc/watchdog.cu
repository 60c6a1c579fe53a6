// watchdog.cu -- self-test of the device watchdog: the bounded mbarrier wait
// that every producer / consumer role of the tensor-core kernels uses,
// pointed at a barrier that nothing ever arrives at.  It must give up after
// its poll limit, raise the error word the host reads (the same path that
// turns a stuck pipeline into CHIRP_ETIMEOUT), and leave the context usable.
// No fault, trap or endless loop is involved.
#include <cuda_runtime.h>

#include <cstdio>

#include "internal.h"
#include "tc.cuh"

namespace {

thread_local char g_msg[200];

__global__ void k_watchdog(int* err, unsigned int polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    chirp::tc::mbar_init(&bar, 1);  // one arrival completes phase 0; none comes
    chirp::tc::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !chirp::tc::mbar_wait(&bar, 0, nullptr, polls)) atomicExch(err, 1);
}

}  // namespace

extern "C" int chirp_watchdog_selftest(unsigned int polls, double* waited_ms, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (polls == 0 || polls > (1u << 24))
    return chirp_report_error(CHIRP_EINVAL, "chirp_watchdog_selftest: polls must be in [1, 2^24]");
  int* d_err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int flag = 0;
  float ms = 0.f;
  cudaError_t e = cudaMalloc(&d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    k_watchdog<<<1, 32, 0, st>>>(d_err, polls);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_err) cudaFree(d_err);
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "chirp_watchdog_selftest: %s", cudaGetErrorString(e));
    return chirp_report_error(CHIRP_ECUDA, g_msg);
  }
  if (waited_ms) *waited_ms = ms;
  if (!flag)
    return chirp_report_error(CHIRP_ECUDA,
                              "chirp_watchdog_selftest: the wait on an unsignalled barrier "
                              "returned success");
  return chirp_report_error(CHIRP_ETIMEOUT,
                            "chirp_watchdog_selftest: the bounded wait gave up as designed");
}
