// convert.cu -- conversions between the height-parity plane and the slope
// planes of the C-ABI state format (Kelling & Odor, arXiv:1110.6745, Sec. II:
// two slope bits per site). With b = floor(h/2) mod 2 and p = (x+y) mod 2:
//   sigma_x(x,y) = +1 <=> b(x+1,y) ^ b(x,y) ^ p(x,y) == 0,
//   sigma_y(x,y) = +1 <=> b(x,y+1) ^ b(x,y) ^ p(x,y) == 0,
// and back, b(0,0) = (H0/2) mod 2, b along column 0 by a xor-scan of the Y
// bits, then along every row by a xor-scan of the X bits.
#include <cuda_runtime.h>

#include "okz_internal.h"
#include "okz_planes.cuh"

namespace okz {

__global__ void to_slopes_kernel(const uint32_t *__restrict__ B, int64_t L,
                                 uint32_t *__restrict__ out) {
  const int64_t W = L >> 5, words = L * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / W, w = i - y * W;
    const int64_t wr = (w == W - 1) ? 0 : w + 1, yu = (y == L - 1) ? 0 : y + 1;
    const uint32_t c = B[i];
    const uint32_t r = __funnelshift_r(c, B[y * W + wr], 1);
    const uint32_t P = odd_sites(y);
    out[i] = ~(c ^ r ^ P);                      // sigma_x = +1 where b(x+1) ^ b ^ p == 0
    out[words + i] = ~(c ^ B[yu * W + w] ^ P);  // sigma_y
  }
}

cudaError_t launch_to_slopes(const uint32_t *B, int64_t L, uint32_t *out, cudaStream_t st) {
  const int64_t words = L * (L >> 5);
  int64_t blocks = (words + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  to_slopes_kernel<<<(unsigned)blocks, 256, 0, st>>>(B, L, out);
  return cudaGetLastError();
}

// b(0,y): b(0,0) = (H0/2) mod 2, b(0,y+1) = b(0,y) ^ p(0,y) ^ !sigma_y-bit(0,y).
// One block: the column's Y bits are gathered 32 rows per word into shared
// memory (independent loads), then each thread xor-scans a run of words.
__global__ void __launch_bounds__(1024)
from_slopes_col_kernel(const uint32_t *__restrict__ slopes, int64_t L, long long H0,
                       int64_t *__restrict__ bcol) {
  extern __shared__ uint32_t dbits[];  // bit k of word j: b(0,32j+k+1) ^ b(0,32j+k)
  __shared__ uint32_t warp_x[32];
  const int64_t W = L >> 5, nw32 = L >> 5;
  const uint32_t *Yp = slopes + L * W;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t j = tid; j < nw32; j += blockDim.x) {
    uint32_t c[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) c[k] = Yp[(32 * j + k) * W];
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) m |= (((uint32_t)k & 1u) ^ (~c[k] & 1u)) << k;  // p(0,y) = y & 1
    dbits[j] = m;
  }
  __syncthreads();
  const int64_t R = (nw32 + blockDim.x - 1) / blockDim.x;
  const int64_t j0 = tid * R < nw32 ? tid * R : nw32;
  const int64_t j1 = j0 + R < nw32 ? j0 + R : nw32;
  uint32_t run = 0;
  for (int64_t j = j0; j < j1; ++j) run ^= __popc(dbits[j]) & 1u;
  uint32_t inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc ^= n;
  }
  if (lane == 31) warp_x[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t v = lane < nw ? warp_x[lane] : 0u, iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t n = __shfl_up_sync(0xFFFFFFFFu, iv, o);
      if (lane >= o) iv ^= n;
    }
    if (lane < nw) warp_x[lane] = iv ^ v;  // exclusive
  }
  __syncthreads();
  uint32_t b = (uint32_t)((H0 >> 1) & 1) ^ warp_x[warp] ^ inc ^ run;
  for (int64_t j = j0; j < j1; ++j) {
    const uint32_t m = dbits[j];
    for (int k = 0; k < 32; ++k) {
      bcol[32 * j + k] = b;
      b ^= (m >> k) & 1u;
    }
  }
}

// Rows: b(x+1,y) = b(x,y) ^ p(x,y) ^ !sigma_x-bit(x,y). A warp per row in
// chunks of 32 consecutive words (coalesced); in-word exclusive prefix xor,
// warp xor-scan of the words' parities, carry across chunks.
__global__ void __launch_bounds__(256)
from_slopes_row_kernel(const uint32_t *__restrict__ slopes, int64_t L,
                       const int64_t *__restrict__ bcol, uint32_t *__restrict__ B) {
  const int lane = threadIdx.x & 31;
  const int64_t W = L >> 5;
  const int64_t nch = (W + 31) >> 5;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t y = gwarp; y < L; y += nwarps) {
    const uint32_t P = odd_sites(y);
    uint32_t carry = (uint32_t)bcol[y];  // b at the first site of the chunk
    for (int64_t c = 0; c < nch; ++c) {
      const int64_t w = 32 * c + lane;
      const bool on = w < W;
      const uint32_t d = on ? P ^ ~slopes[y * W + w] : 0u;  // bit x: b(x+1) ^ b(x)
      const uint32_t par = __popc(d) & 1u;
      uint32_t inc = par;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc ^= n;
      }
      const uint32_t cin = carry ^ inc ^ par;  // b at my word's first site
      uint32_t e = d;                           // inclusive prefix xor
      e ^= e << 1;
      e ^= e << 2;
      e ^= e << 4;
      e ^= e << 8;
      e ^= e << 16;
      if (on) B[y * W + w] = (e ^ d) ^ (cin ? ~0u : 0u);  // exclusive prefix ^ carry
      carry ^= __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
  }
}

cudaError_t launch_from_slopes(const uint32_t *slopes, int64_t L, long long H0, int64_t *bcol,
                               uint32_t *B, cudaStream_t st) {
  const size_t smem = (size_t)(L >> 5) * sizeof(uint32_t);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(from_slopes_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  from_slopes_col_kernel<<<1, 1024, smem, st>>>(slopes, L, H0, bcol);
  int64_t nb = (L + 7) / 8;
  if (nb > 152 * 16) nb = 152 * 16;
  from_slopes_row_kernel<<<(unsigned)nb, 256, 0, st>>>(slopes, L, bcol, B);
  return cudaGetLastError();
}

}  // namespace okz
