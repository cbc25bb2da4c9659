// batch.cu -- many independent lattices ("slots") in one persistent launch.
//
// Replicas are the paper's parallelism across independent runs (Kelling &
// Odor, arXiv:1110.6745, Sec. III: 10-1000 independent simulations per size).
// Every slot holds one height-parity plane (parity.cu) in a device arena. A
// launch drains a device work queue of (slot, sweeps) items: one CTA takes an
// item, stages the lattice in shared memory when it fits (else works on it in
// global memory, where a 2^11 lattice stays L2-resident), runs the sweeps in
// place -- a half-sweep updates only one sublattice and a move toggles only
// the site's own bit, so a CTA barrier between half-sweeps is the only
// synchronisation -- and writes the lattice, t and H0 back. Random draws use
// the slot's own seed with the single-lattice counter layout, so every slot
// evolves bit-identically to a simulation of its own.
#include <cuda_runtime.h>

#include "okz_batch_internal.h"

namespace okz {

namespace {

// Philox4x32-10 of counter (c0, c1, c2, c3) with the slot's round keys in
// shared memory (k[2r], k[2r+1] for round r): one 8-byte broadcast load per
// round instead of two adds of the key schedule (the key is the slot's seed,
// the same for the whole CTA).
__device__ __forceinline__ u32x4 philox10_sm(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                             const uint32_t *__restrict__ rks) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t kx, ky;  // loaded round by round (volatile keeps the loads from piling up)
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                 : "=r"(kx), "=r"(ky)
                 : "r"((uint32_t)__cvta_generic_to_shared(rks + 2 * r)));
    const uint2 k = make_uint2(kx, ky);
    const uint64_t pa = (uint64_t)kPhiloxMulA * c0;
    const uint64_t pb = (uint64_t)kPhiloxMulB * c2;
    const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k.x;
    const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k.y;
    c1 = (uint32_t)pb;
    c3 = (uint32_t)pa;
    c0 = n0;
    c2 = n2;
  }
  u32x4 out;
  out.v[0] = c0;
  out.v[1] = c1;
  out.v[2] = c2;
  out.v[3] = c3;
  return out;
}

// One 128-site group (4 words) of half-sweep s, in place on B.
template <bool LAZY>
__device__ __forceinline__ void group_update(uint32_t *B, int L, int W, uint32_t g, int s,
                                             uint32_t t, const uint32_t *rks, const Accept &acc,
                                             int &dH0) {
  uint32_t mn[4], mx[4], ctr[4];
  uint32_t idx[4];
  const uint32_t S = s ? ~0u : 0u;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t gw = 4 * g + j;
    const uint32_t y = gw / (uint32_t)W, w = gw - y * (uint32_t)W;
    const uint32_t wl = (w == 0) ? W - 1 : w - 1, wr = (w == (uint32_t)W - 1) ? 0 : w + 1;
    const uint32_t yd = (y == 0) ? L - 1 : y - 1, yu = (y == (uint32_t)L - 1) ? 0 : y + 1;
    idx[j] = gw;
    ctr[j] = B[gw];
    const uint32_t l = __funnelshift_l(B[y * W + wl], ctr[j], 1);
    const uint32_t r = __funnelshift_r(ctr[j], B[y * W + wr], 1);
    const uint32_t c = ctr[j] ^ S, d = B[yd * W + w], u = B[yu * W + w];
    const uint32_t dl = l ^ c, dr = r ^ c, dd = d ^ c, du = u ^ c;
    const uint32_t a = active_mask(y, s);
    mn[j] = a & ~(dl | dr | dd | du);
    mx[j] = a & dl & dr & dd & du;
  }
  const uint64_t full = 1ull << acc.k;
  uint32_t ltp[4], eqp[4], ltq[4], eqq[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    ltp[j] = (acc.P >= full) ? mn[j] : 0u;
    eqp[j] = (acc.P >= full || acc.P == 0) ? 0u : mn[j];
    ltq[j] = (acc.Q >= full) ? mx[j] : 0u;
    eqq[j] = (acc.Q >= full || acc.Q == 0) ? 0u : mx[j];
  }
  for (int m = 0; m < acc.k; ++m) {
    if (((eqp[0] | eqq[0]) | (eqp[1] | eqq[1]) | (eqp[2] | eqq[2]) | (eqp[3] | eqq[3])) == 0u)
      break;
    const u32x4 rb = philox10_sm(g, 0u, t, (uint32_t)m, rks);
    const uint32_t pb = (uint32_t)(acc.P >> (acc.k - 1 - m)) & 1u;
    const uint32_t qb = (uint32_t)(acc.Q >> (acc.k - 1 - m)) & 1u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      lt_step(rb.v[j], pb, ltp[j], eqp[j]);
      lt_step(rb.v[j], qb, ltq[j], eqq[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t f = ltp[j] | ltq[j];
    if (f != 0u) B[idx[j]] = ctr[j] ^ f;
    if (idx[j] == 0 && (f & 1u)) dH0 += (mn[0] & 1u) ? 2 : -2;  // site (0,0)
  }
}

// Level 0 of a group is the same in both half-sweeps of a sweep (a site is
// active in one of them). CACHE = 1: keep the level-0 words drawn in the
// first half-sweep in cw and mark bit cbit of cvalid; CACHE = 2: take them
// from there in the second (draw them if the first did not).
constexpr int kCacheGroups = 8;  // groups per thread up to which level 0 is kept

// Acceptance of 4 words (lazy, bit-sliced U < P / U < Q) -> flips.
template <int CACHE>
__device__ __forceinline__ void accept4(const uint32_t mn[4], const uint32_t mx[4], uint32_t g,
                                        uint32_t t, const uint32_t *rks, const Accept &acc,
                                        uint32_t f[4], uint32_t *cw, uint32_t &cvalid,
                                        uint32_t cbit) {
  const uint64_t full = 1ull << acc.k;
  uint32_t ltp[4], eqp[4], ltq[4], eqq[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    ltp[j] = (acc.P >= full) ? mn[j] : 0u;
    eqp[j] = (acc.P >= full || acc.P == 0) ? 0u : mn[j];
    ltq[j] = (acc.Q >= full) ? mx[j] : 0u;
    eqq[j] = (acc.Q >= full || acc.Q == 0) ? 0u : mx[j];
  }
  for (int m = 0; m < acc.k; ++m) {
    if (((eqp[0] | eqq[0]) | (eqp[1] | eqq[1]) | (eqp[2] | eqq[2]) | (eqp[3] | eqq[3])) == 0u)
      break;
    u32x4 rb;
    if (CACHE == 2 && m == 0 && (cvalid & cbit)) {
#pragma unroll
      for (int j = 0; j < 4; ++j) rb.v[j] = cw[j];
    } else {
      rb = philox10_sm(g, 0u, t, (uint32_t)m, rks);
      if (CACHE == 1 && m == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) cw[j] = rb.v[j];
        cvalid |= cbit;
      }
    }
    const uint32_t pb = (uint32_t)(acc.P >> (acc.k - 1 - m)) & 1u;
    const uint32_t qb = (uint32_t)(acc.Q >> (acc.k - 1 - m)) & 1u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      lt_step(rb.v[j], pb, ltp[j], eqp[j]);
      lt_step(rb.v[j], qb, ltq[j], eqq[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) f[j] = ltp[j] | ltq[j];
}

// A group of 4 words inside one row (L % 128 == 0): 3 vector loads (row,
// row below, row above), 2 neighbour words, 1 vector store. Whole-word
// stores are safe: every bit another thread reads from these words sits on a
// site this half-sweep does not move.
template <bool POW2, int SP, int CACHE>
__device__ __forceinline__ void row_group_update(uint32_t *B, int L, int W, uint32_t gpr,
                                                 int lg_gpr, uint32_t g, uint32_t t,
                                                 const uint32_t *rks, const Accept &acc,
                                                 int &dH0, uint32_t *cw, uint32_t &cvalid,
                                                 uint32_t cbit) {
  constexpr int s = SP;
  const uint32_t y = POW2 ? (g >> lg_gpr) : (g / gpr);
  const uint32_t w0 = 4 * (g - y * gpr);
  const uint32_t yd = (y == 0) ? L - 1 : y - 1, yu = (y == (uint32_t)L - 1) ? 0 : y + 1;
  uint32_t *row = B + (size_t)y * W;
  const uint4 cv = *(const uint4 *)(row + w0);
  const uint4 dv = *(const uint4 *)(B + (size_t)yd * W + w0);
  const uint4 uv = *(const uint4 *)(B + (size_t)yu * W + w0);
  const uint32_t lw = row[w0 == 0 ? W - 1 : w0 - 1];
  const uint32_t rw = row[w0 + 4 == (uint32_t)W ? 0 : w0 + 4];
  const uint32_t c[4] = {cv.x, cv.y, cv.z, cv.w};
  const uint32_t d[4] = {dv.x, dv.y, dv.z, dv.w};
  const uint32_t u[4] = {uv.x, uv.y, uv.z, uv.w};
  const uint32_t a = active_mask(y, s);
  // a minimum of half-sweep s has all four neighbours equal to its own bit
  // xor s: "both equal" (table 0x81) for s = 0, "both differ" (0x42) for
  // s = 1, on (l, r, c) and (d, u, c); a maximum the reverse
  constexpr uint32_t kMin = SP ? 0x42u : 0x81u;
  constexpr uint32_t kMax = SP ? 0x81u : 0x42u;
  uint32_t mn[4], mx[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t l = __funnelshift_l(j == 0 ? lw : c[j - 1], c[j], 1);
    const uint32_t r = __funnelshift_r(c[j], j == 3 ? rw : c[j + 1], 1);
    mn[j] = lop3<0x80>(lop3<kMin>(l, r, c[j]), lop3<kMin>(d[j], u[j], c[j]), a);
    mx[j] = lop3<0x80>(lop3<kMax>(l, r, c[j]), lop3<kMax>(d[j], u[j], c[j]), a);
  }
  uint32_t f[4];
  accept4<CACHE>(mn, mx, g, t, rks, acc, f, cw, cvalid, cbit);
  if ((f[0] | f[1] | f[2] | f[3]) != 0u)
    *(uint4 *)(row + w0) = make_uint4(c[0] ^ f[0], c[1] ^ f[1], c[2] ^ f[2], c[3] ^ f[3]);
  if (g == 0 && (f[0] & 1u)) dH0 += (mn[0] & 1u) ? 2 : -2;  // site (0,0)
}

// `n` sweeps of one lattice by the whole CTA.
__device__ __forceinline__ void cta_sweeps(uint32_t *B, int L, uint32_t t0, int n,
                                           const uint32_t *rks, const Accept &acc, int &dH0) {
  const int W = L >> 5;
  const uint32_t groups = (uint32_t)L * (uint32_t)W / 4;
  if ((L & 127) == 0) {  // groups never straddle rows
    const uint32_t gpr = (uint32_t)W / 4;
    const bool pow2 = (gpr & (gpr - 1)) == 0;
    const int lg = __ffs(gpr) - 1;
    // a thread takes the same groups in both half-sweeps; with at most
    // kCacheGroups of them it keeps their level-0 words between the two
    // (with k >= 3 the later levels dominate and the local-memory round trip
    // does not pay: -1.5 % on a k = 32 mix, +6 % at k = 1)
    const bool cache = acc.k <= 2 && groups <= kCacheGroups * blockDim.x;
    uint32_t cw[4 * kCacheGroups];
    for (int i = 0; i < n; ++i) {
      const uint32_t t = t0 + (uint32_t)i;
      uint32_t cvalid = 0;
      if (cache && pow2) {
        uint32_t q = 0;
        for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x, ++q)
          row_group_update<true, 0, 1>(B, L, W, gpr, lg, g, t, rks, acc, dH0, cw + 4 * q, cvalid,
                                       1u << q);
        __syncthreads();
        q = 0;
        for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x, ++q)
          row_group_update<true, 1, 2>(B, L, W, gpr, lg, g, t, rks, acc, dH0, cw + 4 * q, cvalid,
                                       1u << q);
      } else if (pow2) {
        for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x)
          row_group_update<true, 0, 0>(B, L, W, gpr, lg, g, t, rks, acc, dH0, cw, cvalid, 0u);
        __syncthreads();
        for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x)
          row_group_update<true, 1, 0>(B, L, W, gpr, lg, g, t, rks, acc, dH0, cw, cvalid, 0u);
      } else {
        for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x)
          row_group_update<false, 0, 0>(B, L, W, gpr, lg, g, t, rks, acc, dH0, cw, cvalid, 0u);
        __syncthreads();
        for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x)
          row_group_update<false, 1, 0>(B, L, W, gpr, lg, g, t, rks, acc, dH0, cw, cvalid, 0u);
      }
      __syncthreads();
    }
    return;
  }
  for (int i = 0; i < n; ++i) {  // L = 32, 64, 96: groups span rows
    const uint32_t t = t0 + (uint32_t)i;
    for (int s = 0; s < 2; ++s) {
      for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x)
        group_update<true>(B, L, W, g, s, t, rks, acc, dH0);
      __syncthreads();
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(1024, 1)
batch_sweep_kernel(uint32_t *__restrict__ arena, SlotDesc *__restrict__ slots,
                   const WorkTable *__restrict__ work, unsigned int *__restrict__ head,
                   uint32_t smem_words) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int item;
  __shared__ __align__(8) uint32_t rks[20];  // round keys of the current slot's seed
  const int nwork = work->count;
  while (true) {
    if (threadIdx.x == 0) item = (int)atomicAdd(head, 1u);
    __syncthreads();
    const int it = item;
    __syncthreads();
    if (it >= nwork) break;
    const int slot = work->item[it].slot;
    const int n = work->item[it].sweeps;
    SlotDesc d = slots[slot];
    const uint32_t words = (uint32_t)d.L * (uint32_t)(d.L >> 5);
    uint32_t *g = arena + d.offset_words;
    Accept acc;
    acc.P = d.P;
    acc.Q = d.Q;
    acc.k = d.k;
    int dH0 = 0;
    if (threadIdx.x < 10) {
      const uint32_t r = threadIdx.x;
      rks[2 * r] = (uint32_t)d.seed + r * kPhiloxWeylA;
      rks[2 * r + 1] = (uint32_t)(d.seed >> 32) + r * kPhiloxWeylB;
    }
    if (words <= smem_words) {
      for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) sm[w] = g[w];
      __syncthreads();
      cta_sweeps(sm, d.L, d.t, n, rks, acc, dH0);
      for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) g[w] = sm[w];
    } else {
      __syncthreads();
      cta_sweeps(g, d.L, d.t, n, rks, acc, dH0);
    }
    if (threadIdx.x == 0) {  // thread 0 owns group 0, the only group with site (0,0)
      slots[slot].t = d.t + (uint32_t)n;
      slots[slot].H0 = d.H0 + dH0;
    }
    __syncthreads();
  }
}

// Exact power sums S_1..S_4 of (h - H0) per slot: one CTA per slot item, a
// warp per row (lanes own contiguous words), slopes formed from the parity
// plane, 128-bit accumulation; results to the slot's sums.
__global__ void __launch_bounds__(256)
batch_moments_kernel(const uint32_t *__restrict__ arena, SlotDesc *__restrict__ slots,
                     const WorkTable *__restrict__ work) {
  __shared__ __int128 red[4][8];
  extern __shared__ long long colh[];  // L entries
  const int it = blockIdx.x;
  if (it >= work->count) return;
  const int slot = work->item[it].slot;
  const SlotDesc d = slots[slot];
  const int L = d.L, W = L >> 5;
  const uint32_t *B = arena + d.offset_words;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // column 0 heights (relative to H0): sigma_y(0,y) = +1 iff b(0,y+1)^b(0,y)^p == 0
  if (tid == 0) {
    long long h = 0;
    for (int y = 0; y < L; ++y) {
      colh[y] = h;
      const int yu = (y == L - 1) ? 0 : y + 1;
      const uint32_t up = ~(B[y * W] ^ B[yu * W] ^ (uint32_t)(y & 1)) & 1u;
      h += 2 * (long long)up - 1;
    }
  }
  __syncthreads();
  __int128 s[4] = {0, 0, 0, 0};
  const int wpl = (W + 31) >> 5;
  const int w0 = lane * wpl < W ? lane * wpl : W;
  const int w1 = w0 + wpl < W ? w0 + wpl : W;
  for (int y = warp; y < L; y += blockDim.x >> 5) {
    const uint32_t *row = B + y * W;
    const uint32_t P = (y & 1) ? 0x55555555u : 0xAAAAAAAAu;
    int c = 0;
    for (int w = w0; w < w1; ++w) {
      const uint32_t v = ~(row[w] ^ __funnelshift_r(row[w], row[w == W - 1 ? 0 : w + 1], 1) ^ P);
      c += __popc(v);
    }
    int d2 = 2 * c - 32 * (w1 - w0), inc = d2;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int nb = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += nb;
    }
    long long a = colh[y] + (inc - d2);
    for (int w = w0; w < w1; ++w) {
      const uint32_t v = ~(row[w] ^ __funnelshift_r(row[w], row[w == W - 1 ? 0 : w + 1], 1) ^ P);
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
  // reduce: warp shuffles of 64-bit halves are awkward for int128; go via smem
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long lo = (unsigned long long)s[n];
      const long long hi = (long long)(s[n] >> 64);
      const unsigned long long olo = __shfl_down_sync(0xFFFFFFFFu, lo, o);
      const long long ohi = __shfl_down_sync(0xFFFFFFFFu, hi, o);
      s[n] += (__int128)(((unsigned __int128)(unsigned long long)ohi << 64) | olo);
    }
    if (lane == 0) red[n][warp] = s[n];
  }
  __syncthreads();
  if (tid < 4) {
    __int128 tot = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[tid][i];
    slots[slot].sum[2 * tid] = (unsigned long long)tot;
    slots[slot].sum[2 * tid + 1] = (unsigned long long)(tot >> 64);
  }
}

cudaError_t launch_batch_sweeps(uint32_t *arena, SlotDesc *slots, const WorkTable *work,
                                unsigned int *head, int grid, int threads, size_t smem_bytes,
                                cudaStream_t st) {
  // the dynamic shared-memory limit was raised by batch_occupancy() before
  cudaError_t e = cudaMemsetAsync(head, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  batch_sweep_kernel<<<grid, threads, smem_bytes, st>>>(arena, slots, work, head,
                                                       (uint32_t)(smem_bytes / 4));
  return cudaGetLastError();
}

cudaError_t launch_batch_moments(const uint32_t *arena, SlotDesc *slots, const WorkTable *work,
                                 int nitems, int64_t max_L, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const size_t smem = (size_t)max_L * sizeof(long long);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void *)batch_moments_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  batch_moments_kernel<<<nitems, 256, smem, st>>>(arena, slots, work);
  return cudaGetLastError();
}

int batch_occupancy(int threads, size_t smem_bytes) {
  int per_sm = 0;
  // one limit for every batch: the largest staging buffer a tiling may ask for
  cudaFuncSetAttribute((const void *)batch_sweep_kernel,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)batch_sweep_kernel,
                                                    threads, smem_bytes) != cudaSuccess)
    return 0;
  return per_sm;
}

}  // namespace okz
