// measure.cu -- height reconstruction and exact power sums (Kelling & Odor,
// arXiv:1110.6745, Sec. I, Eqs. (3) and (4)).
//
// Heights are anchored at H0 = h(0,0). By zero curl every path gives the
// same height; the kernels here go down column 0 first and then along each
// row:  h(x,y) - H0 = sum_{y'<y} sigma_y(0,y') + sum_{x'<x} sigma_x(x',y).
// Only the X plane and column 0 of the Y plane are read (0.125 B/site); on
// the height-parity plane (parity.cu) the slopes are formed on the fly.
//
// Power sums S_n = sum (h - H0)^n are exact: 64-bit per word and per thread,
// 128-bit per thread total, then per block, then a single-block final sum.
#include "okz_internal.h"
#include "okz_planes.cuh"

namespace okz {

namespace {

__device__ __forceinline__ int warp_exclusive_scan(int v, int lane) {
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += n;
  }
  return inc - v;
}

__device__ __forceinline__ long long warp_exclusive_scan64(long long v, int lane) {
  long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long n = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += n;
  }
  return inc - v;
}

}  // namespace

// hcol[y] = h(0,y) - H0 = sum_{y'<y} sigma_y(0,y'): one block, each thread a
// contiguous run of rows, block-wide exclusive scan of the run totals.
template <bool PAR>
__global__ void __launch_bounds__(1024)
colscan_kernel(const uint32_t *__restrict__ planes, int64_t L, int64_t *__restrict__ hcol) {
  __shared__ long long warp_tot[32];
  const int64_t W = L >> 5;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t R = (L + blockDim.x - 1) / blockDim.x;
  const int64_t y0 = tid * R < L ? tid * R : L;
  const int64_t y1 = y0 + R < L ? y0 + R : L;
  long long run = 0;
  for (int64_t y = y0; y < y1; ++y) run += 2 * (long long)col0_up<PAR>(planes, L, W, y) - 1;
  const long long pre = warp_exclusive_scan64(run, lane);
  if (lane == 31) warp_tot[warp] = pre + run;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    const long long v = lane < nw ? warp_tot[lane] : 0;
    const long long p = warp_exclusive_scan64(v, lane);
    if (lane < nw) warp_tot[lane] = p;
  }
  __syncthreads();
  long long h = warp_tot[warp] + pre;
  for (int64_t y = y0; y < y1; ++y) {
    hcol[y] = h;
    h += 2 * (long long)col0_up<PAR>(planes, L, W, y) - 1;
  }
}

// Byte table for the within-word sums: for byte value v and offsets
// e_0 = 0, e_{b+1} = e_b + 2 v_b - 1 (b = 0..7): cnt = popcount(v),
// A = sum e_b in [-28, 28], B = sum e_b^2 in [0, 140];
// packed as cnt | (A + 28) << 4 | B << 10.
__device__ __forceinline__ uint32_t byte_entry(uint32_t v) {
  int e = 0, A = 0, B = 0;
  for (int b = 0; b < 8; ++b) {
    A += e;
    B += e * e;
    e += 2 * (int)((v >> b) & 1u) - 1;
  }
  return (uint32_t)__popc(v) | ((uint32_t)(A + 28) << 4) | ((uint32_t)B << 10);
}

// Row sums. Each warp owns rows y = warp id, warp id + #warps, ...; lane l
// owns the contiguous words [l*wpl, (l+1)*wpl) of the row. NMOM = 2 gives
// S1, S2 with the byte table; NMOM = 4 gives S1..S4 with a bit loop.
template <int NMOM, bool PAR>
__global__ void __launch_bounds__(256)
rowsum_kernel(const uint32_t *__restrict__ Xp, int64_t L,
              const int64_t *__restrict__ hcol, unsigned long long *__restrict__ partials) {
  __shared__ uint32_t tab[256];
  __shared__ __int128 red[NMOM][256];
  const int tid = threadIdx.x, lane = tid & 31;
  tab[tid] = byte_entry(tid);
  __syncthreads();

  const int64_t W = L >> 5;
  const int64_t wpl = (W + 31) >> 5;
  const int64_t w0 = lane * wpl < W ? lane * wpl : W;
  const int64_t w1 = w0 + wpl < W ? w0 + wpl : W;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + tid) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;

  __int128 s[NMOM];
#pragma unroll
  for (int n = 0; n < NMOM; ++n) s[n] = 0;

  for (int64_t y = gwarp; y < L; y += nwarps) {
    const uint32_t *row = Xp + y * W;
    int c = 0;
    for (int64_t w = w0; w < w1; ++w) c += __popc(x_word<PAR>(row, W, w, y));
    const int d = 2 * c - 32 * (int)(w1 - w0);  // height change over my words
    long long a = hcol[y] + warp_exclusive_scan(d, lane);
    long long s1 = 0, s2 = 0;
    for (int64_t w = w0; w < w1; ++w) {
      const uint32_t v = x_word<PAR>(row, W, w, y);
      if (NMOM == 2) {
        long long es = 0, eq = 0;
        int o = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t T = tab[(v >> (8 * i)) & 0xFFu];
          const int A = (int)((T >> 4) & 63u) - 28;
          const int B = (int)(T >> 10);
          es += 8 * o + A;
          eq += 8 * o * o + 2 * o * A + B;
          o += 2 * (int)(T & 15u) - 8;
        }
        s1 += 32 * a + es;
        s2 += 32 * a * a + 2 * a * es + eq;
        a += 2 * __popc(v) - 32;
      } else {
        for (int b = 0; b < 32; ++b) {
          const __int128 h = a;
          s[0] += h;
          s[1] += h * h;
          s[2] += h * h * h;
          s[3] += h * h * h * h;
          a += 2 * (long long)((v >> b) & 1u) - 1;
        }
      }
    }
    if (NMOM == 2) {
      s[0] += s1;
      s[1] += s2;
    }
  }
#pragma unroll
  for (int n = 0; n < NMOM; ++n) red[n][tid] = s[n];
  __syncthreads();
  if (tid < NMOM) {
    __int128 tot = 0;
    for (int i = 0; i < 256; ++i) tot += red[tid][i];
    partials[blockIdx.x * 8 + 2 * tid] = (unsigned long long)tot;
    partials[blockIdx.x * 8 + 2 * tid + 1] = (unsigned long long)(tot >> 64);
  }
}

// Final exact sum of the per-block partials into ctrl->sum.
__global__ void __launch_bounds__(256)
partials_sum_kernel(const unsigned long long *__restrict__ partials, int nblocks, int nmom,
                    Ctrl *__restrict__ ctrl) {
  __shared__ __int128 red[4][256];
  const int tid = threadIdx.x;
  for (int n = 0; n < 4; ++n) {
    __int128 s = 0;
    if (n < nmom)
      for (int b = tid; b < nblocks; b += blockDim.x) {
        const unsigned __int128 lo = partials[b * 8 + 2 * n];
        const unsigned __int128 hi = partials[b * 8 + 2 * n + 1];
        s += (__int128)((hi << 64) | lo);
      }
    red[n][tid] = s;
  }
  __syncthreads();
  if (tid < 4) {
    __int128 tot = 0;
    for (int i = 0; i < 256; ++i) tot += red[tid][i];
    ctrl->sum[2 * tid] = (unsigned long long)tot;
    ctrl->sum[2 * tid + 1] = (unsigned long long)(tot >> 64);
  }
}

cudaError_t launch_colscan(const uint32_t *planes, int64_t L, bool parity, int64_t *hcol,
                           cudaStream_t st) {
  if (parity)
    colscan_kernel<true><<<1, 1024, 0, st>>>(planes, L, hcol);
  else
    colscan_kernel<false><<<1, 1024, 0, st>>>(planes, L, hcol);
  return cudaGetLastError();
}

static int reduce_blocks(int64_t L) {
  int64_t b = (L + 7) / 8;  // 8 warps per block, one row per warp
  if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
  return (int)b;
}

cudaError_t launch_power_sums(const uint32_t *planes, int64_t L, bool parity, int nmom,
                              int64_t *hcol, unsigned long long *partials, Ctrl *ctrl,
                              cudaStream_t st) {
  const int nb = reduce_blocks(L);
  if (parity) {
    colscan_kernel<true><<<1, 1024, 0, st>>>(planes, L, hcol);
    if (nmom == 2)
      rowsum_kernel<2, true><<<nb, 256, 0, st>>>(planes, L, hcol, partials);
    else
      rowsum_kernel<4, true><<<nb, 256, 0, st>>>(planes, L, hcol, partials);
  } else {
    colscan_kernel<false><<<1, 1024, 0, st>>>(planes, L, hcol);
    if (nmom == 2)
      rowsum_kernel<2, false><<<nb, 256, 0, st>>>(planes, L, hcol, partials);
    else
      rowsum_kernel<4, false><<<nb, 256, 0, st>>>(planes, L, hcol, partials);
  }
  partials_sum_kernel<<<1, 256, 0, st>>>(partials, nb, nmom, ctrl);
  return cudaGetLastError();
}

// h(x, y0 + r) for r < ny as int32, row-major; flags heights outside int32.
template <bool PAR>
__global__ void __launch_bounds__(256)
heights_kernel(const uint32_t *__restrict__ Xp, int64_t L, int64_t y0, int64_t ny,
               const int64_t *__restrict__ hcol, int32_t *__restrict__ out,
               Ctrl *__restrict__ ctrl) {
  const int lane = threadIdx.x & 31;
  const int64_t W = L >> 5;
  const int64_t wpl = (W + 31) >> 5;
  const int64_t w0 = lane * wpl < W ? lane * wpl : W;
  const int64_t w1 = w0 + wpl < W ? w0 + wpl : W;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const long long H0 = ctrl->H0;
  bool bad = false;
  for (int64_t r = gwarp; r < ny; r += nwarps) {
    const int64_t y = y0 + r;
    const uint32_t *row = Xp + y * W;
    int c = 0;
    for (int64_t w = w0; w < w1; ++w) c += __popc(x_word<PAR>(row, W, w, y));
    const int d = 2 * c - 32 * (int)(w1 - w0);
    long long h = H0 + hcol[y] + warp_exclusive_scan(d, lane);
    int32_t *o = out + r * L;
    for (int64_t w = w0; w < w1; ++w) {
      const uint32_t v = x_word<PAR>(row, W, w, y);
      for (int b = 0; b < 32; ++b) {
        bad |= (h < INT32_MIN) || (h > INT32_MAX);
        o[32 * w + b] = (int32_t)h;
        h += 2 * (long long)((v >> b) & 1u) - 1;
      }
    }
  }
  if (bad) atomicOr(&ctrl->err, kErrHeightRange);
}

cudaError_t launch_heights(const uint32_t *planes, int64_t L, bool parity, int64_t y0,
                           int64_t ny, int64_t *hcol, int32_t *out, Ctrl *ctrl,
                           cudaStream_t st) {
  int64_t nb = (ny + 7) / 8;
  if (nb > 152 * 16) nb = 152 * 16;
  if (nb < 1) nb = 1;
  if (parity) {
    colscan_kernel<true><<<1, 1024, 0, st>>>(planes, L, hcol);
    heights_kernel<true><<<(unsigned)nb, 256, 0, st>>>(planes, L, y0, ny, hcol, out, ctrl);
  } else {
    colscan_kernel<false><<<1, 1024, 0, st>>>(planes, L, hcol);
    heights_kernel<false><<<(unsigned)nb, 256, 0, st>>>(planes, L, y0, ny, hcol, out, ctrl);
  }
  return cudaGetLastError();
}

}  // namespace okz
