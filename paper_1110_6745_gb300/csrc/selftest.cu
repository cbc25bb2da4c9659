// selftest.cu -- a check of the bounded device-side wait (no counterpart in
// the paper). The streaming kernels wait on mbarriers for their TMA copies;
// every such wait gives up after kWaitLimitNs and reports OKZ_ETIMEOUT
// instead of spinning forever. This kernel makes that wait run out on
// purpose, in the same code path: it arms an mbarrier for a 16-byte
// transaction that is never issued, so the phase cannot complete; the wait
// returns false after the limit, the kernel records the timeout in its error
// word and exits normally (the context stays usable).
#include <cuda_runtime.h>

#include "okz_internal.h"
#include "okz_tma.cuh"

namespace okz {

__global__ void wait_timeout_kernel(unsigned int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  tma::mbar_init(&bar, 1);
  tma::mbar_init_fence();
  tma::mbar_expect_tx(&bar, 16);  // the one arrival, with 16 bytes that never come
  if (!tma::mbar_wait(&bar, 0u)) atomicOr(err, kErrWaitTimeout);
}

}  // namespace okz

using namespace okz;

okz_status okz_selftest_wait_timeout(void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int *err = nullptr;
  cudaError_t e = scratch_alloc((void **)&err, sizeof(unsigned int), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("okz_selftest_wait_timeout: device allocation failed");
    return OKZ_ENOMEM;
  }
  unsigned int h = 0;
  e = cudaMemsetAsync(err, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 32, 0, st>>>(err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h, err, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
  scratch_free(err, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "okz_selftest_wait_timeout");
  if (h & kErrWaitTimeout) {
    set_error("a bounded device-side wait timed out (as this self-test intends)");
    return OKZ_ETIMEOUT;
  }
  set_error("the wait completed although no transaction was issued");
  return OKZ_OK;
}
