// psd.cu -- interface profiles and the power spectrum on the k axes (Kelling &
// Odor, arXiv:1110.6745, Sec. III, Eqs. (15) and (16)).
//
// With the anchor c = H0: col[x] = sum_y (h(x,y) - c), row[y] = sum_x
// (h(x,y) - c). Zero curl makes every column of sigma_x sum the same way:
//   col[x+1] - col[x] = sum_y sigma_x(x,y) = 2 nX(x) - L,
//   row[y+1] - row[y] = sum_x sigma_y(x,y) = 2 nY(y) - L,
// nX(x) = up-bonds in column x of the X plane, nY(y) = up-bonds in row y of
// the Y plane. The first entries follow from column 0 and row 0 alone: with
// h(0,y) - c = sum_{y'<y} sigma_y(0,y') and h(x,0) - c = sum_{x'<x}
// sigma_x(x',0),
//   col[0] = sum_y (L-1-y) sigma_y(0,y),   row[0] = sum_x (L-1-x) sigma_x(x,0).
// A profile thus costs one pass of bit counting over the state (0.125 B/site
// on the parity plane) and two scans of L counts.
//
// On the axes the transform of Eq. (16) (d = 2, mean removed) is
//   h(k,0) = (1/L) sum_x col[x] e^{-2 pi i k x / L} (k != 0),
// likewise h(0,k) with row, and the spectrum averaged over the two
// directions is S[k] = (|h(k,0)|^2 + |h(0,k)|^2) / 2, S[0] = 0 (the mean is
// removed). The transforms are radix-2 FFTs in fp64 on the exact sums.
#include "okz_internal.h"
#include "okz_planes.cuh"
#include "okz_tma.cuh"

namespace okz {

namespace {

constexpr int kCountThreads = 256;  // word columns per counting block
constexpr int kGroup = 16;          // rows per carry-save group
constexpr int kBandMax = 16 * 255;  // rows per band: byte counters of 16-row units
constexpr int kTile = 256;          // entries per scan tile
constexpr int kStages = 3;                      // bulk-copy ring: slots of one group each
constexpr int kSlotRows = kGroup + 1;           // rows y .. y+16 of a group
constexpr int kSlotWords = kCountThreads + 4;   // a row segment and the 4 words after it
constexpr int kConsumerWarps = kCountThreads / 32;    // one word column per thread
constexpr int kCountTmaThreads = kCountThreads + 32;  // and one producer warp
constexpr size_t kCountTmaSmem = (size_t)kStages * kSlotRows * kSlotWords * 4 +
                                 (size_t)2 * kStages * 8 + (size_t)(kBandMax / 2) * 4;

struct BandPlan {
  int64_t R, nb, cb;  // rows per band, bands, column blocks
};

// Bands of R rows (a multiple of 16, at most 4080) and blocks of 256 word
// columns; R is the largest that gives whole waves of three blocks per SM.
BandPlan band_plan(int64_t L) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    sms = n > 0 ? n : 152;
  }
  const int64_t W = L >> 5;
  const int64_t cb = (W + kCountThreads - 1) / kCountThreads;
  const int64_t slots = 3 * (int64_t)sms;
  int64_t R = kBandMax;
  for (int64_t waves = 1; waves <= 64; ++waves) {
    const int64_t nbt = (waves * slots + cb - 1) / cb;
    int64_t r = (L + nbt - 1) / nbt;
    r = (r + kGroup - 1) / kGroup * kGroup;
    if (r <= kBandMax) {
      R = r;
      break;
    }
  }
  return {R, (L + R - 1) / R, cb};
}

struct PsdLayout {
  size_t cntX, cntY, tiles, a, tw, total;  // cntY is followed by the two anchors
};

size_t take(size_t &off, size_t n) {
  const size_t o = off;
  off = (off + n + 255) & ~(size_t)255;
  return o;
}

int64_t n_tiles(int64_t L) { return (L + kTile - 1) / kTile; }

PsdLayout psd_layout(int64_t L, bool fft) {
  const BandPlan bp = band_plan(L);
  PsdLayout s{};
  size_t off = 0;
  s.cntX = take(off, (size_t)bp.nb * (size_t)L * sizeof(uint32_t));
  s.cntY = take(off, (size_t)L * sizeof(uint32_t) + 2 * sizeof(long long));
  s.tiles = take(off, 2 * (size_t)n_tiles(L) * sizeof(long long));
  if (fft) {
    s.a = take(off, (size_t)L * sizeof(double2));
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

// (h, l) <- carry and sum of l + b + c, bit by bit (a carry-save adder).
__device__ __forceinline__ void csa(uint32_t &h, uint32_t &l, uint32_t b, uint32_t c) {
  const uint32_t a = l;
  l = lop3<0x96>(a, b, c);
  h = lop3<0xE8>(a, b, c);
}

// Per-bit counts of one word column, n_b = 16 S_b + 8 e_b + 4 f_b + 2 t_b +
// o_b: o, t, f, e are carry-save bit planes, S_b is byte b/8 of c8[b%8].
struct ColCount {
  uint32_t o, t, f, e;
  uint32_t c8[8];
};

// Adds 16 words to the counts: a tree of 15 carry-save adders (Harley and
// Seal's population count, applied per bit position) whose weight-16 carry
// goes to the byte counters.
__device__ __forceinline__ void add16(ColCount &cc, const uint32_t d[kGroup]) {
  uint32_t tA, tB, fA, fB, eA, eB, s;
  csa(tA, cc.o, d[0], d[1]);
  csa(tB, cc.o, d[2], d[3]);
  csa(fA, cc.t, tA, tB);
  csa(tA, cc.o, d[4], d[5]);
  csa(tB, cc.o, d[6], d[7]);
  csa(fB, cc.t, tA, tB);
  csa(eA, cc.f, fA, fB);
  csa(tA, cc.o, d[8], d[9]);
  csa(tB, cc.o, d[10], d[11]);
  csa(fA, cc.t, tA, tB);
  csa(tA, cc.o, d[12], d[13]);
  csa(tB, cc.o, d[14], d[15]);
  csa(fB, cc.t, tA, tB);
  csa(eB, cc.f, fA, fB);
  csa(s, cc.e, eA, eB);
#pragma unroll
  for (int i = 0; i < 8; ++i) cc.c8[i] += (s >> i) & 0x01010101u;
}

// *addr += v in shared memory if p (one predicated reduction, no branch).
__device__ __forceinline__ void red_add_if(bool p, uint32_t *addr, uint32_t v) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q red.shared.add.u32 [%1], %2;\n\t}" ::"r"(
          (uint32_t)p),
      "r"((uint32_t)__cvta_generic_to_shared(addr)), "r"(v)
      : "memory");
}

// Row counts of a group: two rows per warp sum (each half at most 1024);
// lane j < 8 keeps the sum of pair j and the eight add it to their rows'
// shared counters in one reduction (each half at most 8192 per block).
__device__ __forceinline__ void add_rows(const uint32_t yw[kGroup], uint32_t *acc, int lane) {
  uint32_t mine = 0;
#pragma unroll
  for (int k = 0; k < kGroup; k += 2) {
    const uint32_t v = (uint32_t)__popc(yw[k]) | ((uint32_t)__popc(yw[k + 1]) << 16);
    const uint32_t s = __reduce_add_sync(0xFFFFFFFFu, v);
    mine = (lane == (k >> 1)) ? s : mine;
  }
  red_add_if(lane < kGroup / 2, &acc[lane & (kGroup / 2 - 1)], mine);
}

// The block's row counts to cntY, its column counts (word column w) to band
// b of cntX.
__device__ __forceinline__ void count_epilogue(const ColCount &cc, const uint32_t *rowacc,
                                               int nrow, int ya, int L, int w, bool on,
                                               uint32_t *__restrict__ cntX,
                                               uint32_t *__restrict__ cntY) {
  __syncthreads();
  for (int r = threadIdx.x; r < nrow; r += blockDim.x) {
    const uint32_t v = (rowacc[r >> 1] >> (16 * (r & 1))) & 0xFFFFu;
    if (v) atomicAdd(&cntY[ya + r], v);
  }
  if (on) {
    uint32_t cnt[32];
#pragma unroll
    for (int b = 0; b < 32; ++b)
      cnt[b] = 16u * ((cc.c8[b & 7] >> (8 * (b >> 3))) & 0xFFu) + 8u * ((cc.e >> b) & 1u) +
               4u * ((cc.f >> b) & 1u) + 2u * ((cc.t >> b) & 1u) + ((cc.o >> b) & 1u);
    uint4 *dst = reinterpret_cast<uint4 *>(cntX + (size_t)blockIdx.y * L + 32 * (size_t)w);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      dst[q] = make_uint4(cnt[4 * q], cnt[4 * q + 1], cnt[4 * q + 2], cnt[4 * q + 3]);
  }
}

}  // namespace

// One thread per word column w and band of rows [ya, yb), in groups of 16
// rows: nX per bit of the column through the carry-save counts, nY per row
// through a warp sum (two rows packed in the halves of one word) and
// shared-memory row counters, added to cntY once per block. A group's loads
// are issued together; the band's last group (and the lattice's last row,
// whose upper neighbour wraps to row 0) takes a checked path.
template <bool PAR>
__global__ void __launch_bounds__(kCountThreads, 3)
profile_count_kernel(const uint32_t *__restrict__ P, int L, int R,
                     uint32_t *__restrict__ cntX, uint32_t *__restrict__ cntY) {
  __shared__ uint32_t rowacc[kBandMax / 2];  // rows 2i (low half) and 2i+1 (high half)
  const int W = L >> 5;
  const int tid = threadIdx.x, lane = tid & 31;
  const int w = (int)blockIdx.x * kCountThreads + tid;
  const bool on = w < W;
  const bool partial = ((int)blockIdx.x + 1) * kCountThreads > W;  // some columns idle
  const int wc = on ? w : 0;                    // loads of idle lanes stay in bounds
  const int wn = (wc + 1 == W) ? 0 : wc + 1;    // word w+1, periodic in x
  const int ya = (int)blockIdx.y * R;
  const int yb = ya + R < L ? ya + R : L;
  const int nrow = yb - ya;
  for (int i = tid; i < (nrow + 1) / 2; i += kCountThreads) rowacc[i] = 0;
  __syncthreads();

  ColCount cc;
  cc.o = cc.t = cc.f = cc.e = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) cc.c8[i] = 0;
  const size_t plane = (size_t)L * (size_t)W;
  // groups start at even offsets from ya, so row y + k has the odd-site mask
  // of ya for even k and its complement for odd k
  const uint32_t oddE = odd_sites(ya), oddO = ~oddE;
  uint32_t cur = PAR ? P[(size_t)ya * W + wc] : 0u;  // b of the current row
  for (int y = ya; y < yb; y += kGroup) {
    const int n = yb - y < kGroup ? yb - y : kGroup;
    const uint32_t *r0 = P + (size_t)y * W;
    uint32_t xw[kGroup], yw[kGroup];
    if (n == kGroup && y + kGroup < L) {  // a whole group, no wrap
      uint32_t la[kGroup], lb[kGroup];
#pragma unroll
      for (int k = 0; k < kGroup; ++k) {
        if (PAR) {
          la[k] = r0[(size_t)(k + 1) * W + wc];  // b of row y+k+1
          lb[k] = r0[(size_t)k * W + wn];        // b of word w+1, row y+k
        } else {
          la[k] = r0[(size_t)k * W + wc];          // X word
          lb[k] = r0[plane + (size_t)k * W + wc];  // Y word
        }
      }
#pragma unroll
      for (int k = 0; k < kGroup; ++k) {
        if (PAR) {
          const uint32_t odd = (k & 1) ? oddO : oddE;
          xw[k] = lop3<0x69>(cur, __funnelshift_r(cur, lb[k], 1), odd);  // ~(c ^ c(x+1) ^ p)
          yw[k] = lop3<0x69>(cur, la[k], odd);                           // ~(c ^ c(y+1) ^ p)
          cur = la[k];
        } else {
          xw[k] = la[k];
          yw[k] = lb[k];
        }
      }
    } else {  // the band's last rows, or the lattice's last row
#pragma unroll
      for (int k = 0; k < kGroup; ++k) {
        xw[k] = yw[k] = 0u;
        if (k < n) {
          const uint32_t *rr = r0 + (size_t)k * W;
          if (PAR) {
            const int yu = (y + k + 1 == L) ? 0 : y + k + 1;
            const uint32_t up = P[(size_t)yu * W + wc];
            const uint32_t odd = (k & 1) ? oddO : oddE;
            xw[k] = lop3<0x69>(cur, __funnelshift_r(cur, rr[wn], 1), odd);
            yw[k] = lop3<0x69>(cur, up, odd);
            cur = up;
          } else {
            xw[k] = rr[wc];
            yw[k] = rr[plane + wc];
          }
        }
      }
    }
    if (partial && !on) {
#pragma unroll
      for (int k = 0; k < kGroup; ++k) xw[k] = yw[k] = 0u;
    }
    add16(cc, xw);
    add_rows(yw, rowacc + ((y - ya) >> 1), lane);
  }
  count_epilogue(cc, rowacc, nrow, ya, L, w, on, cntX, cntY);
}

// The same counts on the parity plane with the rows streamed through shared
// memory by a producer warp: each group's rows y .. y+16 (the block's
// 256-word segment of each and the 4 words after it, periodic in x) go into
// a ring slot by 1-D bulk copies (TMA), one row per lane, completing on the
// slot's "full" mbarrier; the eight consumer warps read their words from the
// slot and arrive on its "empty" mbarrier, which the producer waits for
// before refilling it kStages groups later. No block-wide barrier inside the
// loop. Needs L % 128 == 0 (16-byte copies). Waits are bounded: on a timeout
// the warp sets kErrWaitTimeout in *err and the abort flag, every warp leaves
// its loop, and the producer lets the copies in flight land before exit.
__global__ void __launch_bounds__(kCountTmaThreads, 3)
profile_count_tma_kernel(const uint32_t *__restrict__ P, int L, int R,
                         uint32_t *__restrict__ cntX, uint32_t *__restrict__ cntY,
                         unsigned int *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int abort_flag;
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem);
  uint64_t *full =
      reinterpret_cast<uint64_t *>(smem + (size_t)kStages * kSlotRows * kSlotWords * 4);
  uint64_t *empty = full + kStages;
  uint32_t *rowacc = reinterpret_cast<uint32_t *>(empty + kStages);
  volatile int *abort_v = &abort_flag;
  const int W = L >> 5;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int s0 = (int)blockIdx.x * kCountThreads;  // the segment: words s0 .. s1-1
  const int s1 = s0 + kCountThreads < W ? s0 + kCountThreads : W;
  const int segw = s1 - s0;  // a multiple of 4
  const uint32_t segb = 4u * (uint32_t)segw;
  const int tailw = s1 == W ? 0 : s1;
  const bool on = tid < segw, partial = segw < kCountThreads;
  const int ya = (int)blockIdx.y * R;
  const int yb = ya + R < L ? ya + R : L;
  const int nrow = yb - ya;  // a multiple of 16
  const int ngroups = nrow / kGroup;
  for (int i = tid; i < (nrow + 1) / 2; i += blockDim.x) rowacc[i] = 0;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tma::mbar_init(&full[s], 1);
      tma::mbar_init(&empty[s], kConsumerWarps);
    }
    tma::mbar_init_fence();
    abort_flag = 0;
  }
  __syncthreads();

  ColCount cc;
  cc.o = cc.t = cc.f = cc.e = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) cc.c8[i] = 0;
  int issued = 0;  // producer: groups issued
  if (warp == kConsumerWarps) {
    for (int g = 0; g < ngroups; ++g) {
      const int st = g % kStages;
      if (g >= kStages) {  // wait until the consumers have read group g - kStages
        const bool ok = __all_sync(0xFFFFFFFFu,
                                   tma::mbar_wait(&empty[st], (uint32_t)((g / kStages - 1) & 1)));
        if (!ok) {
          if (lane == 0) {
            atomicOr(err, kErrWaitTimeout);
            *abort_v = 1;
          }
          break;
        }
      }
      if (__any_sync(0xFFFFFFFFu, *abort_v != 0)) break;
      if (lane == 0) tma::mbar_expect_tx(&full[st], (uint32_t)kSlotRows * (segb + 16u));
      __syncwarp();
      if (lane < kSlotRows) {
        const int row = ya + g * kGroup + lane;
        const uint32_t *src = P + (size_t)(row < L ? row : row - L) * W;
        uint32_t *dst = ring + ((size_t)st * kSlotRows + lane) * kSlotWords;
        tma::fence_proxy_async();
        if (tailw != 0) {  // the 4 words after the segment follow it in memory
          tma::load_1d(dst, src + s0, segb + 16u, &full[st]);
        } else {           // the row's last block: they are its first 4 words
          tma::load_1d(dst, src + s0, segb, &full[st]);
          tma::load_1d(dst + segw, src, 16u, &full[st]);
        }
      }
      issued = g + 1;
    }
  } else {
    const uint32_t oddE = odd_sites(ya), oddO = ~oddE;
    for (int g = 0; g < ngroups; ++g) {
      const int st = g % kStages;
      const bool ok =
          __all_sync(0xFFFFFFFFu, tma::mbar_wait(&full[st], (uint32_t)((g / kStages) & 1)));
      if (!ok) {
        if (lane == 0) {
          atomicOr(err, kErrWaitTimeout);
          *abort_v = 1;
        }
        break;
      }
      const uint32_t *sl = ring + (size_t)st * kSlotRows * kSlotWords;
      uint32_t xw[kGroup], yw[kGroup];
      uint32_t cur = sl[tid];
#pragma unroll
      for (int k = 0; k < kGroup; ++k) {
        const uint32_t nxt = sl[(k + 1) * kSlotWords + tid];
        const uint32_t odd = (k & 1) ? oddO : oddE;
        xw[k] = lop3<0x69>(cur, __funnelshift_r(cur, sl[k * kSlotWords + tid + 1], 1), odd);
        yw[k] = lop3<0x69>(cur, nxt, odd);
        cur = nxt;
      }
      __syncwarp();
      if (lane == 0) tma::mbar_arrive(&empty[st]);
      if (partial && !on) {
#pragma unroll
        for (int k = 0; k < kGroup; ++k) xw[k] = yw[k] = 0u;
      }
      add16(cc, xw);
      add_rows(yw, rowacc + g * (kGroup / 2), lane);
    }
  }
  __syncthreads();
  if (warp == kConsumerWarps && lane == 0 && *abort_v) {
    // let the copies of the last groups issued to each slot land
    for (int j = issued - kStages > 0 ? issued - kStages : 0; j < issued; ++j)
      (void)tma::mbar_wait(&full[j % kStages], (uint32_t)((j / kStages) & 1));
  }
  count_epilogue(cc, rowacc, nrow, ya, L, s0 + tid, on, cntX, cntY);
}

// Tiles of 256 columns (blockIdx.y = 0) or rows (1): nX(x) summed over the
// bands (written back into band 0), the tile's sum of 2 n - L, and the
// anchors' terms, (L-1-x) sigma_x(x,0) into row[0] and (L-1-y) sigma_y(0,y)
// into col[0] (anchors[1] and anchors[0]).
template <bool PAR>
__global__ void __launch_bounds__(kTile)
profile_tiles_kernel(const uint32_t *__restrict__ P, int L, int nb, uint32_t *__restrict__ cntX,
                     const uint32_t *__restrict__ cntY, long long *__restrict__ tiles,
                     long long *__restrict__ anchors) {
  __shared__ long long sh[32];
  const int W = L >> 5;
  const int i = (int)blockIdx.x * kTile + threadIdx.x;
  long long v = 0, a = 0;
  if (i < L) {
    const long long wgt = (long long)(L - 1 - i);
    if (blockIdx.y == 0) {
      uint32_t n = 0;
      for (int b = 0; b < nb; ++b) n += cntX[(size_t)b * L + i];
      cntX[i] = n;
      v = 2LL * n - L;
      const uint32_t xw = x_word<PAR>(P, W, i >> 5, 0);
      a = ((xw >> (i & 31)) & 1u) ? wgt : -wgt;
    } else {
      v = 2LL * cntY[i] - L;
      a = col0_up<PAR>(P, L, W, i) ? wgt : -wgt;
    }
  }
  const long long ts = block_sum(v, sh);
  const long long as = block_sum(a, sh);
  if (threadIdx.x == 0) {
    tiles[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = ts;
    atomicAdd(reinterpret_cast<unsigned long long *>(&anchors[1 - blockIdx.y]),
              (unsigned long long)as);
  }
}

// col[x] = anchors[0] + sum_{x'<x} (2 nX(x') - L) (blockIdx.y = 0), row[y]
// likewise from nY and anchors[1]: the tiles before this one, then an
// exclusive scan inside it.
__global__ void __launch_bounds__(kTile)
profile_scan_kernel(const uint32_t *__restrict__ cntX, const uint32_t *__restrict__ cntY, int L,
                    const long long *__restrict__ tiles, const long long *__restrict__ anchors,
                    int64_t *__restrict__ col, int64_t *__restrict__ row) {
  __shared__ long long sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long *ts = tiles + (size_t)blockIdx.y * gridDim.x;
  long long pre = 0;
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += kTile) pre += ts[t];
  const long long off = anchors[blockIdx.y] + block_sum(pre, sh);
  const int i = (int)blockIdx.x * kTile + threadIdx.x;
  const uint32_t *cnt = blockIdx.y ? cntY : cntX;
  const long long v = i < L ? 2LL * cnt[i] - L : 0;
  const long long pw = warp_excl_scan(v, lane);
  if (lane == 31) sh[warp] = pw + v;
  __syncthreads();
  if (warp == 0) {
    const long long s = lane < kTile / 32 ? sh[lane] : 0;
    const long long p = warp_excl_scan(s, lane);
    if (lane < kTile / 32) sh[lane] = p;
  }
  __syncthreads();
  if (i < L) (blockIdx.y ? row : col)[i] = (int64_t)(off + sh[warp] + pw);
}

constexpr int kFftLogBlock = 10;  // points per shared-memory FFT block: 1024

// u, x <- u + w x, u - w x with the rounding of every step fixed, so that all
// FFT kernels compute a butterfly alike.
__device__ __forceinline__ void bfly(double2 &u, double2 &x, double2 w) {
  const double tr = __fma_rn(w.x, x.x, __dmul_rn(-w.y, x.y));
  const double ti = __fma_rn(w.x, x.y, __dmul_rn(w.y, x.x));
  const double2 a = u;
  u = make_double2(__dadd_rn(a.x, tr), __dadd_rn(a.y, ti));
  x = make_double2(__dsub_rn(a.x, tr), __dsub_rn(a.y, ti));
}

__device__ __forceinline__ double power(double2 c) {
  return __fma_rn(c.x, c.x, __dmul_rn(c.y, c.y));
}

// The radix-2 decimation-in-time FFT of z = col + i row, on the bit-reversed
// input a[p] = z[bitrev(p)]; one transform gives both axes, since with
// Z = FFT(z) the transforms of the real col and row satisfy
// |C(k)|^2 + |R(k)|^2 = (|Z(k)|^2 + |Z(L-k)|^2) / 2. The first lb stages
// (half-lengths 1 .. 2^(lb-1)) never leave a block of B = 2^lb points: block
// b loads points b B .. b B + B - 1, runs them in shared memory with
// twiddles e^{-2 pi i k / B}, and writes them to a; if L > B, the blocks also
// write their slice of the table tw[j] = e^{-2 pi i j / L}, j < L/2, for the
// later stages.
__global__ void __launch_bounds__(1 << (kFftLogBlock - 1))
fft_block_kernel(const int64_t *__restrict__ col, const int64_t *__restrict__ row, int64_t L,
                 int lg, int lb, double2 *__restrict__ a, double2 *__restrict__ tw) {
  __shared__ double2 v[1 << kFftLogBlock];
  __shared__ double2 wb[1 << (kFftLogBlock - 1)];
  const int B = 1 << lb, t = threadIdx.x, nt = blockDim.x;
  const int64_t base = (int64_t)blockIdx.x * B;
  for (int i = t; i < B; i += nt) {
    const uint32_t r = __brev((uint32_t)(base + i)) >> (32 - lg);
    v[i] = make_double2((double)col[r], (double)row[r]);
  }
  for (int k = t; k < B / 2; k += nt) {
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)B, &sn, &cs);
    wb[k] = make_double2(cs, sn);
  }
  if (L > B) {
    const int64_t per = (L / 2) / gridDim.x;
    for (int64_t k = t; k < per; k += nt) {
      const int64_t j = (int64_t)blockIdx.x * per + k;
      double sn, cs;
      sincospi(-2.0 * (double)j / (double)L, &sn, &cs);
      tw[j] = make_double2(cs, sn);
    }
  }
  __syncthreads();
  for (int lh = 0; lh < lb; ++lh) {
    const int half = 1 << lh;
    for (int i = t; i < B / 2; i += nt) {
      const int j = i & (half - 1);
      const int p = ((i >> lh) << (lh + 1)) | j;
      double2 u = v[p], x = v[p + half];
      bfly(u, x, wb[j << (lb - 1 - lh)]);
      v[p] = u;
      v[p + half] = x;
    }
    __syncthreads();
  }
  double2 *dst = a + base;
  for (int i = t; i < B; i += nt) dst[i] = v[i];
}

// One radix-2 stage with half-length 2^lh.
__global__ void __launch_bounds__(256)
fft_stage_kernel(double2 *__restrict__ a, const double2 *__restrict__ tw, int64_t L, int lh,
                 int lg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L / 2) return;
  const int64_t half = 1LL << lh;
  const int64_t j = i & (half - 1);
  const int64_t p = ((i >> lh) << (lh + 1)) | j;
  double2 u = a[p], x = a[p + half];
  bfly(u, x, tw[j << (lg - 1 - lh)]);
  a[p] = u;
  a[p + half] = x;
}

// Stages lh and lh+1 (half-lengths h = 2^lh and 2h) as radix-4 steps: thread
// i takes the points p + {0, h, 2h, 3h}, p = its 4h group's start + j
// (j < h), and runs the four radix-2 butterflies of the two stages on them.
__global__ void __launch_bounds__(256)
fft_radix4_kernel(double2 *__restrict__ a, const double2 *__restrict__ tw, int64_t L, int lh,
                  int lg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L / 4) return;
  const int64_t h = 1LL << lh;
  const int64_t j = i & (h - 1);
  const int64_t p = ((i >> lh) << (lh + 2)) | j;
  const double2 w1 = tw[j << (lg - 1 - lh)];
  const double2 w2a = tw[j << (lg - 2 - lh)];
  const double2 w2b = tw[(j + h) << (lg - 2 - lh)];
  double2 x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = a[p + q * h];
  bfly(x[0], x[1], w1);
  bfly(x[2], x[3], w1);
  bfly(x[0], x[2], w2a);
  bfly(x[1], x[3], w2b);
#pragma unroll
  for (int q = 0; q < 4; ++q) a[p + q * h] = x[q];
}

// S[k] = S[L-k] = (|Z(k)|^2 + |Z(L-k)|^2) / (4 L^2) (the axis average of
// |h(k,0)|^2 and |h(0,k)|^2 with h = transform / L), S[0] = 0: thread k
// writes both entries of the pair k, L-k.
__global__ void __launch_bounds__(256)
psd_finish_kernel(const double2 *__restrict__ a, int64_t L, double *__restrict__ S) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k > L / 2) return;
  if (k == 0) {
    S[0] = 0.0;
    return;
  }
  const double v = __dmul_rn(__dadd_rn(power(a[k]), power(a[L - k])),
                             1.0 / (4.0 * (double)L * (double)L));
  S[k] = v;
  S[L - k] = v;
}

size_t psd_scratch_bytes(int64_t L, bool fft) { return psd_layout(L, fft).total; }

cudaError_t launch_profiles(const uint32_t *planes, int64_t L, bool parity, void *scratch,
                            int64_t *col, int64_t *row, unsigned int *err, cudaStream_t st) {
  const BandPlan bp = band_plan(L);
  const PsdLayout lay = psd_layout(L, false);
  char *base = static_cast<char *>(scratch);
  uint32_t *cntX = reinterpret_cast<uint32_t *>(base + lay.cntX);
  uint32_t *cntY = reinterpret_cast<uint32_t *>(base + lay.cntY);
  long long *anchors = reinterpret_cast<long long *>(cntY + L);
  long long *tiles = reinterpret_cast<long long *>(base + lay.tiles);
  cudaError_t e = cudaMemsetAsync(cntY, 0, (size_t)L * sizeof(uint32_t) + 2 * sizeof(long long), st);
  if (e != cudaSuccess) return e;
  const int Li = (int)L, nt = (int)n_tiles(L);
  const dim3 grid((unsigned)bp.cb, (unsigned)bp.nb);
  if (parity) {
    if (L % 128 == 0) {
      static bool attr_set = false;
      if (!attr_set) {
        e = cudaFuncSetAttribute(profile_count_tma_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCountTmaSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
      }
      profile_count_tma_kernel<<<grid, kCountTmaThreads, kCountTmaSmem, st>>>(
          planes, Li, (int)bp.R, cntX, cntY, err);
    } else {
      profile_count_kernel<true><<<grid, kCountThreads, 0, st>>>(planes, Li, (int)bp.R, cntX,
                                                                 cntY);
    }
    profile_tiles_kernel<true><<<dim3(nt, 2), kTile, 0, st>>>(planes, Li, (int)bp.nb, cntX, cntY,
                                                              tiles, anchors);
  } else {
    profile_count_kernel<false><<<grid, kCountThreads, 0, st>>>(planes, Li, (int)bp.R, cntX, cntY);
    profile_tiles_kernel<false><<<dim3(nt, 2), kTile, 0, st>>>(planes, Li, (int)bp.nb, cntX,
                                                               cntY, tiles, anchors);
  }
  profile_scan_kernel<<<dim3(nt, 2), kTile, 0, st>>>(cntX, cntY, Li, tiles, anchors, col, row);
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
  const int lb = lg < kFftLogBlock ? lg : kFftLogBlock;
  const int B = 1 << lb;
  fft_block_kernel<<<(unsigned)(L / B), B / 2 > 0 ? B / 2 : 1, 0, st>>>(col, row, L, lg, lb, a,
                                                                         tw);
  int lh = lb;
  if ((lg - lh) % 2 == 1) {  // an odd number of stages left: one radix-2 stage first
    fft_stage_kernel<<<(unsigned)((L / 2 + 255) / 256), 256, 0, st>>>(a, tw, L, lh, lg);
    ++lh;
  }
  for (; lh < lg; lh += 2)
    fft_radix4_kernel<<<(unsigned)((L / 4 + 255) / 256), 256, 0, st>>>(a, tw, L, lh, lg);
  psd_finish_kernel<<<(unsigned)((L / 2 + 1 + 255) / 256), 256, 0, st>>>(a, L, S);
  return cudaGetLastError();
}

}  // namespace okz
