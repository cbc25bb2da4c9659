// measure.cu -- height reconstruction and exact power sums (Kelling & Odor,
// arXiv:1110.6745, Sec. I, Eqs. (3) and (4)).
//
// Heights are anchored at H0 = h(0,0). By zero curl every path gives the
// same height; the kernels here go down column 0 first and then along each
// row:  h(x,y) - H0 = sum_{y'<y} sigma_y(0,y') + sum_{x'<x} sigma_x(x',y).
// Only the X plane and column 0 of the Y plane are read (0.125 B/site); on
// the height-parity plane (parity.cu) the slopes are formed on the fly.
//
// A row is read by one warp in chunks of 32 consecutive words (lane l takes
// word 32c + l, so every load is coalesced); a warp scan of the words'
// height changes gives each lane the height at the start of its word.
// Power sums S_n = sum (h - H0)^n are exact: per word from byte tables of
// the in-byte offsets' powers, combined binomially with the word's start
// height, 128-bit per thread, then per block, then a single-block final sum.
#include "okz_internal.h"
#include "okz_planes.cuh"

namespace okz {

namespace {

__device__ __forceinline__ int warp_inclusive_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += n;
  }
  return v;
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

// Column-0 slope bits of rows 32j .. 32j+31 (bit k = [sigma_y(0, 32j+k) = +1]).
template <bool PAR>
__device__ __forceinline__ uint32_t col0_word(const uint32_t *__restrict__ P, int64_t L,
                                              int64_t W, int64_t j) {
  uint32_t c[33];
  const int64_t y0 = 32 * j;
  if (PAR) {
#pragma unroll
    for (int k = 0; k < 33; ++k) {
      int64_t y = y0 + k;
      if (y >= L) y -= L;
      c[k] = P[y * W];
    }
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) m |= (~(c[k] ^ c[k + 1] ^ (uint32_t)((y0 + k) & 1)) & 1u) << k;
    return m;
  }
  const uint32_t *Yp = P + L * W;
#pragma unroll
  for (int k = 0; k < 32; ++k) c[k] = Yp[(y0 + k) * W];
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < 32; ++k) m |= (c[k] & 1u) << k;
  return m;
}

}  // namespace

// hcol[y] = h(0,y) - H0 = sum_{y'<y} sigma_y(0,y'): one block. The column's
// slope bits are gathered into shared memory first (33 independent loads per
// 32 rows, so many are in flight), then each thread scans a contiguous run.
template <bool PAR>
__global__ void __launch_bounds__(1024)
colscan_kernel(const uint32_t *__restrict__ planes, int64_t L, int64_t *__restrict__ hcol) {
  extern __shared__ uint32_t col_bits[];  // L/32 words
  __shared__ long long warp_tot[32];
  const int64_t W = L >> 5;
  const int64_t nw32 = L >> 5;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t j = tid; j < nw32; j += blockDim.x) col_bits[j] = col0_word<PAR>(planes, L, W, j);
  __syncthreads();
  const int64_t R = (nw32 + blockDim.x - 1) / blockDim.x;  // words per thread
  const int64_t j0 = tid * R < nw32 ? tid * R : nw32;
  const int64_t j1 = j0 + R < nw32 ? j0 + R : nw32;
  long long run = 0;
  for (int64_t j = j0; j < j1; ++j) run += 2LL * __popc(col_bits[j]) - 32;
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
  for (int64_t j = j0; j < j1; ++j) {
    const uint32_t m = col_bits[j];
    for (int k = 0; k < 32; ++k) {
      hcol[32 * j + k] = h;
      h += 2 * (long long)((m >> k) & 1u) - 1;
    }
  }
}

// Byte tables for the within-word sums: for byte value v and in-byte offsets
// e_0 = 0, e_{b+1} = e_b + 2 v_b - 1 (b = 0..7), T_n = sum_b e_b^n:
//   A = popcount(v) | (T1 + 28) << 4 | T2 << 10        (T1 in [-28, 28], T2 <= 140)
//   B = (T3 + 784) | T4 << 11                          (|T3| <= 784, T4 <= 4676)
__device__ __forceinline__ void byte_entries(uint32_t v, uint32_t &A, uint32_t &B) {
  int e = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0;
  for (int b = 0; b < 8; ++b) {
    t1 += e;
    t2 += e * e;
    t3 += e * e * e;
    t4 += e * e * e * e;
    e += 2 * (int)((v >> b) & 1u) - 1;
  }
  A = (uint32_t)__popc(v) | ((uint32_t)(t1 + 28) << 4) | ((uint32_t)t2 << 10);
  B = (uint32_t)(t3 + 784) | ((uint32_t)t4 << 11);
}

// Row sums: each warp owns rows y = warp id, warp id + #warps, ... NMOM = 2
// gives S1, S2; NMOM = 4 gives S1..S4.
template <int NMOM, bool PAR>
__global__ void __launch_bounds__(256)
rowsum_kernel(const uint32_t *__restrict__ Xp, int64_t L,
              const int64_t *__restrict__ hcol, unsigned long long *__restrict__ partials) {
  __shared__ uint32_t tabA[256], tabB[256];
  __shared__ __int128 red[NMOM][256];
  const int tid = threadIdx.x, lane = tid & 31;
  {
    uint32_t A, B;
    byte_entries(tid, A, B);
    tabA[tid] = A;
    tabB[tid] = B;
  }
  __syncthreads();

  const int64_t W = L >> 5;
  const int64_t nch = (W + 31) >> 5;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + tid) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;

  __int128 s[NMOM];
#pragma unroll
  for (int n = 0; n < NMOM; ++n) s[n] = 0;

  for (int64_t y = gwarp; y < L; y += nwarps) {
    const uint32_t *row = Xp + y * W;
    long long carry = hcol[y];
    long long r1 = 0, r2 = 0;  // this row's S1, S2 (they fit 64 bits)
    for (int64_t c = 0; c < nch; ++c) {
      const int64_t w = 32 * c + lane;
      const bool on = w < W;
      const uint32_t v = on ? x_word<PAR>(row, W, w, y) : 0u;
      const int d = on ? 2 * __popc(v) - 32 : 0;
      const int incl = warp_inclusive_scan(d, lane);
      const long long a = carry + (incl - d);  // height at the start of word w
      carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
      if (!on) continue;
      int E1 = 0, E2 = 0, E3 = 0, E4 = 0, o = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t byte = (v >> (8 * i)) & 0xFFu;
        const uint32_t A = tabA[byte];
        const int T1 = (int)((A >> 4) & 63u) - 28, T2 = (int)(A >> 10);
        E1 += 8 * o + T1;
        E2 += 8 * o * o + 2 * o * T1 + T2;
        if (NMOM == 4) {
          const uint32_t B = tabB[byte];
          const int T3 = (int)(B & 2047u) - 784, T4 = (int)(B >> 11);
          E3 += 8 * o * o * o + 3 * o * o * T1 + 3 * o * T2 + T3;
          E4 += 8 * o * o * o * o + 4 * o * o * o * T1 + 6 * o * o * T2 + 4 * o * T3 + T4;
        }
        o += 2 * (int)(A & 15u) - 8;
      }
      // sum over the word of (a + e)^n, |a| <= L, binomially
      const long long a2 = a * a;
      r1 += 32 * a + E1;
      r2 += 32 * a2 + 2 * a * E1 + E2;
      if (NMOM == 4) {
        const long long a3 = a2 * a;  // |a|^3 <= 2^51 for L <= 2^17
        s[2] += (__int128)(32 * a3) + (__int128)(3 * a2) * E1 + (__int128)(3 * a) * E2 + E3;
        s[3] += (__int128)a2 * (32 * a2) + (__int128)(4 * a3) * E1 +
                (__int128)(6 * a2) * E2 + (__int128)(4 * a) * E3 + E4;
      }
    }
    s[0] += r1;
    s[1] += r2;
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

// S1, S2 for rows of a multiple of 128 words (L % 4096 == 0): lane l takes
// the four words 128c + 4l .. 128c + 4l + 3 of chunk c as one 16-byte load,
// so the warp scan runs once per four words, and the lane's sums are formed
// relative to its own start height (32-bit) and shifted once per chunk.
template <bool PAR>
__global__ void __launch_bounds__(256)
rowsum4_kernel(const uint32_t *__restrict__ Xp, int64_t L,
               const int64_t *__restrict__ hcol, unsigned long long *__restrict__ partials) {
  __shared__ uint32_t tabA[256];
  __shared__ __int128 red[2][256];
  const int tid = threadIdx.x, lane = tid & 31;
  {
    uint32_t A, B;
    byte_entries(tid, A, B);
    tabA[tid] = A;
  }
  __syncthreads();
  const int64_t W = L >> 5;
  const int64_t nch = W >> 7;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + tid) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  __int128 s1 = 0, s2 = 0;
  for (int64_t y = gwarp; y < L; y += nwarps) {
    const uint32_t *row = Xp + y * W;
    const uint32_t odd = odd_sites(y);
    long long carry = hcol[y];
    long long r1 = 0, r2 = 0;
    for (int64_t c = 0; c < nch; ++c) {
      const int64_t w0 = 128 * c + 4 * lane;
      const uint4 q = *reinterpret_cast<const uint4 *>(row + w0);
      uint32_t v[4] = {q.x, q.y, q.z, q.w};
      if (PAR) {  // X bits from the parity bits: ~(b ^ b(x+1) ^ p)
        uint32_t nxt = __shfl_down_sync(0xFFFFFFFFu, q.x, 1);
        if (lane == 31) nxt = row[(w0 + 4 == W) ? 0 : w0 + 4];
        const uint32_t n[4] = {q.y, q.z, q.w, nxt};
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = ~(v[j] ^ __funnelshift_r(v[j], n[j], 1) ^ odd);
      }
      int dj[4], dsum = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        dj[j] = 2 * __popc(v[j]) - 32;
        dsum += dj[j];
      }
      const int incl = warp_inclusive_scan(dsum, lane);
      const long long A0 = carry + (incl - dsum);  // height at the start of word w0
      carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
      int s1r = 0, s2r = 0, ap = 0;  // sums relative to A0; ap = offset of word j
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int E1 = 0, E2 = 0, o = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t A = tabA[(v[j] >> (8 * i)) & 0xFFu];
          const int T1 = (int)((A >> 4) & 63u) - 28, T2 = (int)(A >> 10);
          E1 += 8 * o + T1;
          E2 += 8 * o * o + 2 * o * T1 + T2;
          o += 2 * (int)(A & 15u) - 8;
        }
        s1r += 32 * ap + E1;
        s2r += 32 * ap * ap + 2 * ap * E1 + E2;
        ap += dj[j];
      }
      r1 += 128 * A0 + s1r;
      r2 += 128 * A0 * A0 + 2 * A0 * s1r + s2r;
    }
    s1 += r1;
    s2 += r2;
  }
  red[0][tid] = s1;
  red[1][tid] = s2;
  __syncthreads();
  if (tid < 2) {
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

static int reduce_blocks(int64_t L) {
  int64_t b = (L + 7) / 8;  // 8 warps per block, one row per warp
  if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
  return (int)b;
}

cudaError_t launch_colscan(const uint32_t *planes, int64_t L, bool parity, int64_t *hcol,
                           cudaStream_t st) {
  const size_t smem = (size_t)(L >> 5) * sizeof(uint32_t);
  if (parity) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(colscan_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    colscan_kernel<true><<<1, 1024, smem, st>>>(planes, L, hcol);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(colscan_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    colscan_kernel<false><<<1, 1024, smem, st>>>(planes, L, hcol);
  }
  return cudaGetLastError();
}

cudaError_t launch_power_sums(const uint32_t *planes, int64_t L, bool parity, int nmom,
                              int64_t *hcol, unsigned long long *partials, Ctrl *ctrl,
                              cudaStream_t st) {
  const int nb = reduce_blocks(L);
  cudaError_t e = launch_colscan(planes, L, parity, hcol, st);
  if (e != cudaSuccess) return e;
  if (nmom == 2 && L % 4096 == 0) {
    if (parity)
      rowsum4_kernel<true><<<nb, 256, 0, st>>>(planes, L, hcol, partials);
    else
      rowsum4_kernel<false><<<nb, 256, 0, st>>>(planes, L, hcol, partials);
  } else if (parity) {
    if (nmom == 2)
      rowsum_kernel<2, true><<<nb, 256, 0, st>>>(planes, L, hcol, partials);
    else
      rowsum_kernel<4, true><<<nb, 256, 0, st>>>(planes, L, hcol, partials);
  } else {
    if (nmom == 2)
      rowsum_kernel<2, false><<<nb, 256, 0, st>>>(planes, L, hcol, partials);
    else
      rowsum_kernel<4, false><<<nb, 256, 0, st>>>(planes, L, hcol, partials);
  }
  partials_sum_kernel<<<1, 256, 0, st>>>(partials, nb, nmom, ctrl);
  return cudaGetLastError();
}

// h(x, y0 + r) for r < ny as int32, row-major; flags heights outside int32.
// Each warp computes a chunk of 32 words (1024 heights) into shared memory
// and writes it out with coalesced stores.
template <bool PAR>
__global__ void __launch_bounds__(256)
heights_kernel(const uint32_t *__restrict__ Xp, int64_t L, int64_t y0, int64_t ny,
               const int64_t *__restrict__ hcol, int32_t *__restrict__ out,
               Ctrl *__restrict__ ctrl) {
  __shared__ int32_t stage[8][1024 + 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t *sm = stage[wib];
  const int64_t W = L >> 5;
  const int64_t nch = (W + 31) >> 5;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const long long H0 = ctrl->H0;
  bool bad = false;
  for (int64_t r = gwarp; r < ny; r += nwarps) {
    const int64_t y = y0 + r;
    const uint32_t *row = Xp + y * W;
    int32_t *o = out + r * L;
    long long carry = H0 + hcol[y];
    for (int64_t c = 0; c < nch; ++c) {
      const int64_t w = 32 * c + lane;
      const bool on = w < W;
      const uint32_t v = on ? x_word<PAR>(row, W, w, y) : 0u;
      const int d = on ? 2 * __popc(v) - 32 : 0;
      const int incl = warp_inclusive_scan(d, lane);
      long long h = carry + (incl - d);
      carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
      // lane's 32 heights at sm[33 * lane + b] (padded: conflict-free)
      for (int b = 0; b < 32; ++b) {
        bad |= on && ((h < INT32_MIN) || (h > INT32_MAX));
        sm[33 * lane + b] = (int32_t)h;
        h += 2 * (long long)((v >> b) & 1u) - 1;
      }
      __syncwarp();
      const int64_t nvalid = (W - 32 * c < 32 ? W - 32 * c : 32) * 32;  // heights in chunk
      for (int k = lane; k < nvalid; k += 32) o[1024 * c + k] = sm[33 * (k >> 5) + (k & 31)];
      __syncwarp();
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
  cudaError_t e = launch_colscan(planes, L, parity, hcol, st);
  if (e != cudaSuccess) return e;
  if (parity)
    heights_kernel<true><<<(unsigned)nb, 256, 0, st>>>(planes, L, y0, ny, hcol, out, ctrl);
  else
    heights_kernel<false><<<(unsigned)nb, 256, 0, st>>>(planes, L, y0, ny, hcol, out, ctrl);
  return cudaGetLastError();
}

}  // namespace okz
