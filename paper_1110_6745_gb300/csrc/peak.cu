// peak.cu -- measured INT32 ALU-pipe throughput of the current GPU (a
// diagnostic; the paper has no counterpart). The checkerboard sweep kernels
// are bound by three-input logic ops and funnel shifts, which issue to the
// ALU pipe; their roofline divides algorithmic ALU-pipe ops per second by the
// rate this kernel reaches with nothing but independent lop3.b32 chains:
// eight chains per thread, eight blocks of 256 threads per SM, no memory
// traffic inside the timed loop.
#include <cuda_runtime.h>

#include "okz_internal.h"

namespace okz {

namespace {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;

// Keeps the chains' results alive without a memory store per thread.
__device__ unsigned int g_peak_sink;

__global__ void __launch_bounds__(kPeakThreads)
alu_peak_kernel(int iters, uint32_t a, uint32_t b) {
  uint32_t x[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k)
    x[k] = threadIdx.x * 2654435761u + (uint32_t)k * 40503u + blockIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) x[k] = lop3<0x96>(x[k], a, b);
  }
  uint32_t r = 0;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) r ^= x[k];
  if (r == 0x9E3779B9u) g_peak_sink = r;  // practically never taken
}

}  // namespace

}  // namespace okz

using namespace okz;

okz_status okz_alu_peak(void *stream, int32_t iters, double *ops_per_s, double *best_ms) {
  if (iters < 1 || !ops_per_s) {
    set_error("okz_alu_peak: iters must be >= 1 and ops_per_s non-null");
    return OKZ_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "okz_alu_peak: device query");
  const int blocks = sms * kPeakBlocksPerSm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  if (e == cudaSuccess) {  // warm-up, then the best of three timed launches
    alu_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(iters / 8 + 1, 0x9E3779B9u, 0x7F4A7C15u);
    e = cudaGetLastError();
  }
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      alu_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(iters, 0x9E3779B9u, 0x7F4A7C15u);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (rep == 0 || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "okz_alu_peak");
  const double ops = (double)blocks * kPeakThreads * (double)iters * kPeakChains;
  *ops_per_s = ops / (best * 1e-3);
  if (best_ms) *best_ms = best;
  return OKZ_OK;
}
