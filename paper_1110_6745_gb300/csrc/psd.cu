// psd.cu -- interface profiles and the power spectrum on the k axes (Kelling &
// Odor, arXiv:1110.6745, Sec. III, Eqs. (15) and (16)).
//
// With the anchor c = H0: col[x] = sum_y (h(x,y) - c), row[y] = sum_x
// (h(x,y) - c). Zero curl makes every column of sigma_x sum the same way:
//   col[x+1] - col[x] = sum_y sigma_x(x,y) = 2 nX(x) - L,
//   row[y+1] - row[y] = sum_x sigma_y(x,y) = 2 nY(y) - L,
// nX(x) = up-bonds in column x of the X plane, nY(y) = up-bonds in row y of
// the Y plane; col[0] = sum_y (h(0,y) - c) (the column-0 scan) and
// row[0] = sum_x (L-1-x) sigma_x(x,0). A profile thus costs one pass of bit
// counting over the state (0.125 B/site on the parity plane).
//
// On the axes the transform of Eq. (16) (d = 2, mean removed) is
//   h(k,0) = (1/L) sum_x col[x] e^{-2 pi i k x / L} (k != 0),
// likewise h(0,k) with row, and the spectrum averaged over the two
// directions is S[k] = (|h(k,0)|^2 + |h(0,k)|^2) / 2, S[0] = 0 (the mean is
// removed). The transforms are radix-2 FFTs in fp64 on the exact sums.
#include "okz_internal.h"
#include "okz_planes.cuh"

namespace okz {

namespace {

constexpr int kBandMax = 2048;  // rows per band (shared row counters)
constexpr int kCountThreads = 256;

struct BandPlan {
  int64_t R, nb, cb;  // rows per band, bands, column blocks
};

// About four blocks per SM of a 152-SM part; bands of 16 .. 2048 rows.
BandPlan band_plan(int64_t L) {
  const int64_t W = L >> 5;
  const int64_t cb = (W + kCountThreads - 1) / kCountThreads;
  const int64_t nbt = (4 * 152 + cb - 1) / cb;
  int64_t R = (L + nbt - 1) / nbt;
  if (R < 16) R = 16;
  if (R > kBandMax) R = kBandMax;
  return {R, (L + R - 1) / R, cb};
}

struct PsdLayout {
  size_t cntX, cntY, a, tw, total;
};

size_t take(size_t &off, size_t n) {
  const size_t o = off;
  off = (off + n + 255) & ~(size_t)255;
  return o;
}

PsdLayout psd_layout(int64_t L, bool fft) {
  const BandPlan bp = band_plan(L);
  PsdLayout s{};
  size_t off = 0;
  s.cntX = take(off, (size_t)bp.nb * (size_t)L * sizeof(uint32_t));
  s.cntY = take(off, (size_t)L * sizeof(uint32_t));
  if (fft) {
    s.a = take(off, 2 * (size_t)L * sizeof(double2));
    s.tw = take(off, (size_t)(L / 2) * sizeof(double2));
  }
  s.total = off;
  return s;
}

__device__ __forceinline__ long long warp_excl_scan(long long v, int lane) {
  long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long n = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += n;
  }
  return inc - v;
}

__device__ __forceinline__ long long block_sum(long long v, long long *sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  long long t = 0;
  for (int i = 0; i < nw; ++i) t += sh[i];
  __syncthreads();
  return t;
}

// out[i] = base + sum_{i'<i} (2 cnt[i'] - L): each thread a contiguous run.
__device__ void scan_counts(const uint32_t *__restrict__ cnt, int64_t L, long long base,
                            int64_t *__restrict__ out, long long *sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int64_t run_len = (L + blockDim.x - 1) / blockDim.x;
  const int64_t a = tid * run_len < L ? tid * run_len : L;
  const int64_t b = a + run_len < L ? a + run_len : L;
  long long run = 0;
  for (int64_t i = a; i < b; ++i) run += 2LL * cnt[i] - L;
  const long long pre = warp_excl_scan(run, lane);
  if (lane == 31) sh[warp] = pre + run;
  __syncthreads();
  if (warp == 0) {
    const long long v = lane < nw ? sh[lane] : 0;
    const long long p = warp_excl_scan(v, lane);
    if (lane < nw) sh[lane] = p;
  }
  __syncthreads();
  long long h = base + sh[warp] + pre;
  for (int64_t i = a; i < b; ++i) {
    out[i] = h;
    h += 2LL * cnt[i] - L;
  }
  __syncthreads();
}

}  // namespace

// One thread per word column w and band of rows [ya, yb): nX per column
// through nibble counters (bit 4i + j of the X words in nibble i of A[j]),
// nY per row through a warp sum and shared-memory row counters, added to
// cntY once per block. Rows go in batches of 15 (the nibble counters' range):
// the batch's loads are issued together, then its rows are counted and the
// nibbles emptied once; the few remaining rows (and the lattice's last row,
// whose upper neighbour wraps to row 0) take a one-row path.
template <bool PAR>
__device__ __forceinline__ void count_row(uint32_t xw, uint32_t yw, uint32_t A[4],
                                          uint32_t *rowacc_r, int lane) {
#pragma unroll
  for (int j = 0; j < 4; ++j) A[j] += (xw >> j) & 0x11111111u;
  const uint32_t n = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)__popc(yw));
  if (lane == 0 && n) atomicAdd(rowacc_r, n);
}

__device__ __forceinline__ void empty_nibbles(uint32_t A[4], uint32_t cnt[32]) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) cnt[4 * i + j] += (A[j] >> (4 * i)) & 15u;
  A[0] = A[1] = A[2] = A[3] = 0;
}

template <bool PAR>
__global__ void __launch_bounds__(kCountThreads, 3)
profile_count_kernel(const uint32_t *__restrict__ P, int64_t L64, int64_t R,
                     uint32_t *__restrict__ cntX, uint32_t *__restrict__ cntY) {
  constexpr int kBatch = 15;
  __shared__ uint32_t rowacc[kBandMax];
  const int L = (int)L64, W = L >> 5;
  const int tid = threadIdx.x, lane = tid & 31;
  const int w = (int)blockIdx.x * kCountThreads + tid;
  const bool on = w < W;
  const int ya = (int)blockIdx.y * (int)R;
  const int yb = ya + (int)R < L ? ya + (int)R : L;
  const int nrow = yb - ya;
  for (int r = tid; r < nrow; r += kCountThreads) rowacc[r] = 0;
  __syncthreads();

  uint32_t cnt[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) cnt[b] = 0;
  uint32_t A[4] = {0, 0, 0, 0};
  const int wc = on ? w : 0;                         // loads of idle lanes stay in bounds
  const int dn_off = (wc + 1 == W) ? 1 - W : 1;      // word w+1, periodic in x
  const size_t plane = (size_t)L * (size_t)W;
  const uint32_t *pw = P + (size_t)ya * W + wc;      // row y, word w
  uint32_t cur = PAR ? pw[0] : 0u;
  // rows whose upper neighbour does not wrap
  const int ymain = (PAR && yb == L) ? yb - 1 : yb;
  int y = ya;
  for (; y + kBatch <= ymain; y += kBatch, pw += (size_t)kBatch * W) {
    uint32_t la[kBatch], lb[kBatch];
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      if (PAR) {
        la[k] = pw[(k + 1) * W];       // b of row y+k+1
        lb[k] = pw[k * W + dn_off];    // b of word w+1, row y+k
      } else {
        la[k] = pw[k * W];             // X word
        lb[k] = pw[plane + k * W];     // Y word
      }
    }
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      uint32_t xw, yw;
      if (PAR) {
        const uint32_t odd = odd_sites(y + k);
        xw = ~(cur ^ __funnelshift_r(cur, lb[k], 1) ^ odd);
        yw = ~(cur ^ la[k] ^ odd);
        cur = la[k];
      } else {
        xw = la[k];
        yw = lb[k];
      }
      if (!on) xw = yw = 0u;
      count_row<PAR>(xw, yw, A, &rowacc[y + k - ya], lane);
    }
    empty_nibbles(A, cnt);
  }
  for (int k = 0; y < yb; ++y, ++k, pw += W) {  // fewer than kBatch rows, or the wrapping row
    uint32_t xw, yw;
    if (PAR) {
      const uint32_t up = (y + 1 == L) ? P[wc] : pw[W];
      const uint32_t odd = odd_sites(y);
      xw = ~(cur ^ __funnelshift_r(cur, pw[dn_off], 1) ^ odd);
      yw = ~(cur ^ up ^ odd);
      cur = up;
    } else {
      xw = pw[0];
      yw = pw[plane];
    }
    if (!on) xw = yw = 0u;
    count_row<PAR>(xw, yw, A, &rowacc[y - ya], lane);
    if (k == kBatch - 1) {
      empty_nibbles(A, cnt);
      k = -1;
    }
  }
  empty_nibbles(A, cnt);
  __syncthreads();
  for (int r = tid; r < nrow; r += kCountThreads)
    if (rowacc[r]) atomicAdd(&cntY[ya + r], rowacc[r]);
  if (on) {
    uint4 *dst = reinterpret_cast<uint4 *>(cntX + (int64_t)blockIdx.y * L + 32 * w);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      dst[q] = make_uint4(cnt[4 * q], cnt[4 * q + 1], cnt[4 * q + 2], cnt[4 * q + 3]);
  }
}

// cntX[x] = sum over bands (in place into band 0).
__global__ void __launch_bounds__(256)
band_sum_kernel(uint32_t *__restrict__ cntX, int64_t L, int64_t nb) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= L) return;
  uint32_t s = 0;
  for (int64_t b = 0; b < nb; ++b) s += cntX[b * L + x];
  cntX[x] = s;
}

// col[0] and the column scan (block 0), row[0] and the row scan (block 1).
template <bool PAR>
__global__ void __launch_bounds__(1024)
profile_finish_kernel(const uint32_t *__restrict__ P, int64_t L,
                      const int64_t *__restrict__ hcol, const uint32_t *__restrict__ cntX,
                      const uint32_t *__restrict__ cntY, int64_t *__restrict__ col,
                      int64_t *__restrict__ row) {
  __shared__ long long sh[32];
  const int64_t W = L >> 5;
  if (blockIdx.x == 0) {  // columns: col[0] = sum_y (h(0,y) - H0), then the scan
    long long s0 = 0;
    for (int64_t y = threadIdx.x; y < L; y += blockDim.x) s0 += hcol[y];
    scan_counts(cntX, L, block_sum(s0, sh), col, sh);
  } else {  // rows: row[0] = sum_x (L-1-x) sigma_x(x,0), then the scan
    long long s1 = 0;
    for (int64_t w = threadIdx.x; w < W; w += blockDim.x) {
      const uint32_t v = x_word<PAR>(P, W, w, 0);
      for (int b = 0; b < 32; ++b) {
        const long long wgt = L - 1 - (32 * w + b);
        s1 += ((v >> b) & 1u) ? wgt : -wgt;
      }
    }
    scan_counts(cntY, L, block_sum(s1, sh), row, sh);
  }
}

// a[t][bitrev(i)] = (t ? row : col)[i], the input of an in-place radix-2 FFT.
__global__ void __launch_bounds__(256)
fft_load_kernel(const int64_t *__restrict__ col, const int64_t *__restrict__ row, int64_t L,
                int lg, double2 *__restrict__ a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  const int64_t *src = blockIdx.y ? row : col;
  const uint32_t r = __brev((uint32_t)i) >> (32 - lg);
  a[blockIdx.y * L + r] = make_double2((double)src[i], 0.0);
}

// tw[j] = e^{-2 pi i j / L}, j < L/2.
__global__ void __launch_bounds__(256) twiddle_kernel(int64_t L, double2 *__restrict__ tw) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L / 2) return;
  double s, c;
  sincospi(-2.0 * (double)j / (double)L, &s, &c);
  tw[j] = make_double2(c, s);
}

// One butterfly stage with half-length 2^lh, both transforms (blockIdx.y).
__global__ void __launch_bounds__(256)
fft_stage_kernel(double2 *__restrict__ a, const double2 *__restrict__ tw, int64_t L, int lh,
                 int lg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L / 2) return;
  double2 *v = a + blockIdx.y * L;
  const int64_t half = 1LL << lh;
  const int64_t j = i & (half - 1);
  const int64_t i0 = ((i >> lh) << (lh + 1)) | j, i1 = i0 + half;
  const double2 w = tw[j << (lg - 1 - lh)];
  const double2 u = v[i0], x = v[i1];
  const double tr = w.x * x.x - w.y * x.y, ti = w.x * x.y + w.y * x.x;
  v[i0] = make_double2(u.x + tr, u.y + ti);
  v[i1] = make_double2(u.x - tr, u.y - ti);
}

__global__ void __launch_bounds__(256)
psd_finish_kernel(const double2 *__restrict__ a, int64_t L, double *__restrict__ S) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  const double2 c = a[k], r = a[L + k];
  const double inv = 1.0 / (2.0 * (double)L * (double)L);
  S[k] = (k == 0) ? 0.0 : (c.x * c.x + c.y * c.y + r.x * r.x + r.y * r.y) * inv;
}

size_t psd_scratch_bytes(int64_t L, bool fft) { return psd_layout(L, fft).total; }

cudaError_t launch_profiles(const uint32_t *planes, int64_t L, bool parity, int64_t *hcol,
                            void *scratch, int64_t *col, int64_t *row, cudaStream_t st) {
  const BandPlan bp = band_plan(L);
  const PsdLayout lay = psd_layout(L, false);
  char *base = static_cast<char *>(scratch);
  uint32_t *cntX = reinterpret_cast<uint32_t *>(base + lay.cntX);
  uint32_t *cntY = reinterpret_cast<uint32_t *>(base + lay.cntY);
  cudaError_t e = launch_colscan(planes, L, parity, hcol, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cntY, 0, (size_t)L * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)bp.cb, (unsigned)bp.nb);
  if (parity)
    profile_count_kernel<true><<<grid, kCountThreads, 0, st>>>(planes, L, bp.R, cntX, cntY);
  else
    profile_count_kernel<false><<<grid, kCountThreads, 0, st>>>(planes, L, bp.R, cntX, cntY);
  band_sum_kernel<<<(unsigned)((L + 255) / 256), 256, 0, st>>>(cntX, L, bp.nb);
  if (parity)
    profile_finish_kernel<true><<<2, 1024, 0, st>>>(planes, L, hcol, cntX, cntY, col, row);
  else
    profile_finish_kernel<false><<<2, 1024, 0, st>>>(planes, L, hcol, cntX, cntY, col, row);
  return cudaGetLastError();
}

cudaError_t launch_psd(const int64_t *col, const int64_t *row, int64_t L, void *scratch,
                       double *S, cudaStream_t st) {
  const PsdLayout lay = psd_layout(L, true);
  char *base = static_cast<char *>(scratch);
  double2 *a = reinterpret_cast<double2 *>(base + lay.a);
  double2 *tw = reinterpret_cast<double2 *>(base + lay.tw);
  int lg = 0;
  while ((1LL << lg) < L) ++lg;
  const unsigned gL = (unsigned)((L + 255) / 256), gH = (unsigned)((L / 2 + 255) / 256);
  fft_load_kernel<<<dim3(gL, 2), 256, 0, st>>>(col, row, L, lg, a);
  twiddle_kernel<<<gH, 256, 0, st>>>(L, tw);
  for (int lh = 0; lh < lg; ++lh) fft_stage_kernel<<<dim3(gH, 2), 256, 0, st>>>(a, tw, L, lh, lg);
  psd_finish_kernel<<<gL, 256, 0, st>>>(a, L, S);
  return cudaGetLastError();
}

}  // namespace okz
