// noalloc.cu -- okz_width2_noalloc: exact W^2 of caller-owned planes without
// allocating any memory.
//
// Who needs this: programs that cannot call cudaMalloc at the moment they
// want a measurement -- for example because a framework's caching allocator
// already owns all free device memory, because an allocation (and the device
// synchronisation it may bring) is not allowed on their latency-critical
// path, or because their policy forbids allocating after start-up. They keep
// their own lattice planes and only need the sums.
//
// The scratch this path needs (column heights, per-block partial sums and a
// result block) lives in one file-scope device array of fixed size, sized for
// the largest lattice the library streams (L = 131072). The array exists once
// per device that loads the library and stays allocated until the process
// exits. Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and keeps it.
#include <cuda_runtime.h>

#include <mutex>

#include "okz_internal.h"

namespace okz {

namespace {

constexpr int64_t kNoallocMaxL = 131072;
constexpr size_t kNoallocHcolBytes = (size_t)kNoallocMaxL * sizeof(int64_t);      // 1 MiB
constexpr size_t kNoallocPartialBytes = (size_t)kMaxReduceBlocks * 8 * sizeof(uint64_t);
constexpr size_t kNoallocBytes = kNoallocHcolBytes + kNoallocPartialBytes + sizeof(Ctrl);
// 1 MiB of column heights + 128 KiB of partial sums + the 256-byte result block
static_assert(kNoallocBytes == (1u << 20) + (128u << 10) + 256u, "documented scratch size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
okz_status scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range for the no-allocation scratch table");
    return OKZ_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the scratch array");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return OKZ_OK;
}

okz_i128 to_abi(__int128 v) {
  okz_i128 r;
  r.lo = (uint64_t)(unsigned __int128)v;
  r.hi = (int64_t)(uint64_t)((unsigned __int128)v >> 64);
  return r;
}

}  // namespace

}  // namespace okz

using namespace okz;

extern "C" okz_status okz_width2_noalloc(const uint32_t *planes, int64_t L, int64_t H0,
                                         void *stream, okz_i128 *S1, okz_i128 *S2,
                                         double *W2) {
  if (!planes || L < 32 || (L % 32) != 0) {
    set_error("okz_width2_noalloc: planes must be non-null and L a multiple of 32");
    return OKZ_EINVAL;
  }
  if (((uintptr_t)planes & 15u) != 0) {
    // the row kernels read the planes with 16-byte vector loads
    set_error("okz_width2_noalloc: planes must be 16-byte aligned");
    return OKZ_EINVAL;
  }
  if (L > kNoallocMaxL) {
    set_error("okz_width2_noalloc: L exceeds the fixed scratch size (L <= 131072)");
    return OKZ_EINVAL;
  }
  void *base = nullptr;
  okz_status st = scratch_address(&base);
  if (st != OKZ_OK) return st;
  int64_t *hcol = (int64_t *)base;
  unsigned long long *partials = (unsigned long long *)((char *)base + kNoallocHcolBytes);
  Ctrl *ctrl = (Ctrl *)((char *)base + kNoallocHcolBytes + kNoallocPartialBytes);
  cudaStream_t s = (cudaStream_t)stream;

  // the sums are overwritten by the kernels; clear the result block anyway so
  // that nothing from an earlier call can leak into this one
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s);
  if (e == cudaSuccess)
    e = launch_power_sums(planes, L, /*parity=*/false, 2, hcol, partials, ctrl, s);
  unsigned long long sums[4] = {0, 0, 0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sums, ctrl->sum, sizeof(sums), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "okz_width2_noalloc");

  const __int128 s1 = (__int128)(((unsigned __int128)sums[1] << 64) | sums[0]);  // about H0
  const __int128 s2 = (__int128)(((unsigned __int128)sums[3] << 64) | sums[2]);
  const __int128 N = (__int128)L * L;
  const __int128 h0 = H0;
  if (W2) *W2 = (double)(N * s2 - s1 * s1) / ((double)N * (double)N);
  if (S1) *S1 = to_abi(s1 + N * h0);
  if (S2) *S2 = to_abi(s2 + 2 * h0 * s1 + N * h0 * h0);
  return OKZ_OK;
}
