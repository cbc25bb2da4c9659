// sweep_stream.cu -- one launch per sweep (both half-sweeps), one pass over
// HBM: read 2 bits and write 2 bits per site (0.5 B/site/sweep).
//
// Model: octahedron KPZ lattice gas, Kelling & Odor (arXiv:1110.6745),
// Sec. I, Eq. (2), on the checkerboard schedule (half-sweep s = 0 then 1).
//
// Decomposition. A CTA spans a full row: L/128 threads, each owning 4
// consecutive 32-bit words (one 128-site Philox group) of both planes, so
// periodic wrap in x stays inside the CTA. The CTA owns a band of rows
// [yb, ye) and streams rows yb-2 .. ye+1 through a ring of shared-memory slots
// filled by 1-D TMA bulk copies (cp.async.bulk + mbarrier). The two
// half-sweeps run as a wavefront lagging one row:
//   at row r: F0(r)      (half-sweep 0 flips of row r)
//             F1(r-1)    (half-sweep 1 flips of row r-1)
//   and the bonds are rewritten by their owners ("pull" form):
//     X'(x) = X(x) ^ F(x) ^ F(x+1),   Y'(x,y) = Y(x,y) ^ F(x,y) ^ F(x,y+1).
// A flip of a site in half-sweep s only touches bits that are inactive for
// the neighbouring rows' sites of the same half-sweep, which lets the kernel
// carry "Y(y-1) ^ F(y-1)" instead of Y(y-1) (the extra bits are masked).
// One CTA barrier per row exchanges the edge bits between threads (shuffles
// inside a warp, shared memory across warps) and recycles the ring slot.
// Output goes to the other buffer of a ping-pong pair, so bands never race.
#include <cuda_runtime.h>

#include "okz_internal.h"

namespace okz {

namespace {

constexpr int kWPT = 4;  // words per thread per plane: one 128-site group

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase completed, false after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t start = globaltimer_ns();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - start > kWaitLimitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_1d(void *dst_smem, const void *src_gmem,
                                            uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Acceptance of the flips of one thread's 4 words in half-sweep s of row y.
// KM = 0: k <= 1 and no maxima move (q_eff = 0);  KM = 1: k <= 1;
// KM = 2: any k, lazily evaluated level by level.
// mode values for k <= 1: 0 never, 1 accept iff the level-0 bit is 0
// (threshold 1 of 2), 2 always.
struct Modes {
  uint32_t p1, p2, q1, q2;  // all-ones masks selecting the mode
};

template <int KM>
__device__ __forceinline__ void flips(const uint32_t mn[4], const uint32_t mx[4],
                                      const uint32_t r0[4], uint64_t g, uint32_t t,
                                      uint64_t seed, const Accept &acc, const Modes &md,
                                      uint32_t f[4]) {
  if (KM == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) f[j] = mn[j] & ((~r0[j] & md.p1) | md.p2);
  } else if (KM == 1) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      f[j] = (mn[j] & ((~r0[j] & md.p1) | md.p2)) | (mx[j] & ((~r0[j] & md.q1) | md.q2));
  } else {
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
      if (((eqp[0] | eqq[0]) | (eqp[1] | eqq[1]) | (eqp[2] | eqq[2]) | (eqp[3] | eqq[3])) ==
          0u)
        break;
      uint32_t r[4];
      if (m == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) r[j] = r0[j];
      } else {
        const u32x4 b = group_bits(g, t, (uint32_t)m, seed);
#pragma unroll
        for (int j = 0; j < 4; ++j) r[j] = b.v[j];
      }
      const uint32_t pb = (uint32_t)(acc.P >> (acc.k - 1 - m)) & 1u;
      const uint32_t qb = (uint32_t)(acc.Q >> (acc.k - 1 - m)) & 1u;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        lt_step(r[j], pb, ltp[j], eqp[j]);
        lt_step(r[j], qb, ltq[j], eqq[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) f[j] = ltp[j] | ltq[j];
  }
}

// Extremum masks of 4 words given the left-bond carry of word 0.
__device__ __forceinline__ void extrema(const uint32_t xc[4], uint32_t carry,
                                        const uint32_t yd[4], const uint32_t yc[4],
                                        uint32_t a, uint32_t mn[4], uint32_t mx[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t cin = (j == 0) ? carry : (xc[j - 1] >> 31);
    const uint32_t xl = (xc[j] << 1) | cin;  // sigma_x(x-1) at bit x
    mn[j] = minima(xl, xc[j], yd[j], yc[j]) & a;
    mx[j] = maxima(xl, xc[j], yd[j], yc[j]) & a;
  }
}

// x-bond update of 4 words: X ^ F ^ F(x+1), with F(x+1) of the last bit
// supplied by the right neighbour.
__device__ __forceinline__ void pull_x(uint32_t xc[4], const uint32_t f[4],
                                       uint32_t right_bit0) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t nxt = (j == 3) ? right_bit0 : (f[j + 1] & 1u);
    xc[j] ^= f[j] ^ ((f[j] >> 1) | (nxt << 31));
  }
}

}  // namespace

template <int KM>
__global__ void __launch_bounds__(1024, 1)
sweep_stream_kernel(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                    int64_t L, int stages, uint32_t t, uint64_t seed, Accept acc,
                    Modes md, Ctrl *__restrict__ ctrl) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int nthr = blockDim.x;  // L / 128
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  const int64_t W = L >> 5;  // words per row per plane
  const uint32_t rowbytes = (uint32_t)(L >> 3);
  const int64_t plane_words = L * W;

  unsigned char *ring = smem;  // stages x (X row | Y row)
  uint64_t *full = (uint64_t *)(smem + (size_t)stages * 2 * rowbytes);
  uint32_t *exL = (uint32_t *)(full + stages);  // [2][nwarps]: value of lane 0
  uint32_t *exR = exL + 2 * 32;                 // [2][nwarps]: value of lane 31

  const int64_t yb = (int64_t)blockIdx.x * L / gridDim.x;
  const int64_t ye = (int64_t)(blockIdx.x + 1) * L / gridDim.x;
  const int nin = (int)(ye - yb) + 4;  // rows yb-2 .. ye+1

  auto row_of = [&](int i) -> int64_t {  // wrapped row index of stream position i
    int64_t y = yb - 2 + i;
    if (y < 0) y += L;
    if (y >= L) y -= L;
    return y;
  };
  auto issue = [&](int i) {
    const int slot = i % stages;
    unsigned char *d = ring + (size_t)slot * 2 * rowbytes;
    const int64_t y = row_of(i);
    mbar_expect_tx(&full[slot], 2 * rowbytes);
    tma_load_1d(d, src + y * W, rowbytes, &full[slot]);
    tma_load_1d(d + rowbytes, src + plane_words + y * W, rowbytes, &full[slot]);
  };

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int i = 0; i < stages && i < nin; ++i) issue(i);

  // carried state (see the file comment)
  uint32_t U[4] = {0, 0, 0, 0};    // Y(r-1) ^ F0(r-1)
  uint32_t X0[4] = {0, 0, 0, 0};   // X after half-sweep 0, row r-1
  uint32_t T[4] = {0, 0, 0, 0};    // Y0(r-2) ^ F1(r-2)
  uint32_t Rp[4] = {0, 0, 0, 0};   // level-0 random words of row r-1
  uint32_t x0_left = 0;            // X0(r-1) at x0-1 (left neighbour's last bond)
  const int64_t gw0 = (int64_t)kWPT * tid;  // my first word within a row
  const int64_t wprev = (gw0 == 0) ? W - 1 : gw0 - 1;  // word holding my left bond

  for (int i = 0; i < nin; ++i) {
    const int slot = i % stages;
    const uint32_t parity = (uint32_t)((i / stages) & 1);
    const bool ok = mbar_wait_bounded(&full[slot], parity);
    const unsigned char *d = ring + (size_t)slot * 2 * rowbytes;
    const uint4 xv = *(const uint4 *)(d + 16 * tid);
    const uint4 yv = *(const uint4 *)(d + rowbytes + 16 * tid);
    const uint32_t xprev = *(const uint32_t *)(d + 4 * wprev);
    uint32_t Xr[4] = {xv.x, xv.y, xv.z, xv.w};
    const uint32_t Yr[4] = {yv.x, yv.y, yv.z, yv.w};
    const int64_t r = yb - 2 + i;  // unwrapped row
    const int64_t y = row_of(i);
    const uint64_t g = (uint64_t)y * (uint64_t)nthr + (uint64_t)tid;  // 128-site group

    // level-0 random words of row r (shared by both half-sweeps of the row)
    uint32_t Rr[4];
    {
      const u32x4 b = group_bits(g, t, 0u, seed);
#pragma unroll
      for (int j = 0; j < 4; ++j) Rr[j] = b.v[j];
    }

    // half-sweep 0 at row r
    uint32_t mn[4], mx[4], F0[4];
    extrema(Xr, xprev >> 31, U, Yr, active_mask(y, 0), mn, mx);
    flips<KM>(mn, mx, Rr, g, t, seed, acc, md, F0);

    // half-sweep 1 at row r-1 (needs Y0(r-1) = U ^ F0(r))
    uint32_t Y0[4], F1[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) Y0[j] = U[j] ^ F0[j];
    const int64_t yp = (y == 0) ? L - 1 : y - 1;
    {
      uint32_t mn1[4], mx1[4];
      extrema(X0, x0_left, T, Y0, active_mask(yp, 1), mn1, mx1);
      const uint64_t gp = (uint64_t)yp * (uint64_t)nthr + (uint64_t)tid;
      flips<KM>(mn1, mx1, Rp, gp, t, seed, acc, md, F1);
    }

    if (r == 0 && tid == 0 && (F0[0] & 1u))  // site (0,0), inside CTA 0's band
      ctrl->H0 += (mn[0] & 1u) ? 2 : -2;

    // exchange edge bits: bit0 F0 at my first site, bit1 F0 at my last site,
    // bit2 F1 at my first site
    const uint32_t v = (F0[0] & 1u) | ((F0[3] >> 31) << 1) | ((F1[0] & 1u) << 2);
    uint32_t vr = __shfl_down_sync(0xFFFFFFFFu, v, 1);
    uint32_t vl = __shfl_up_sync(0xFFFFFFFFu, v, 1);
    const int par = i & 1;
    if (lane == 0) exL[par * 32 + warp] = v;
    if (lane == 31) exR[par * 32 + warp] = v;
    const int bad = __syncthreads_or(!ok);
    if (bad) {
      if (tid == 0) {
        atomicOr(&ctrl->err, kErrWaitTimeout);
        // give copies already issued a bounded chance to land before exiting
        for (int k = i + 1; k < nin && k < i + stages; ++k)
          (void)mbar_wait_bounded(&full[k % stages], (uint32_t)((k / stages) & 1));
      }
      return;
    }
    if (lane == 31) vr = exL[par * 32 + (warp + 1 == nwarps ? 0 : warp + 1)];
    if (lane == 0) vl = exR[par * 32 + (warp == 0 ? nwarps - 1 : warp - 1)];

    // the slot of row i is free: refill it with row i + stages
    if (tid == 0 && i + stages < nin) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(i + stages);
    }

    // finish half-sweep 1 of row r-1: X1(r-1) and Y1(r-2)
    {
      uint32_t X1[4] = {X0[0], X0[1], X0[2], X0[3]};
      pull_x(X1, F1, (vr >> 2) & 1u);
      if (i >= 3 && r - 1 < ye)
        *(uint4 *)(dst + yp * W + gw0) = make_uint4(X1[0], X1[1], X1[2], X1[3]);
      if (i >= 4) {
        const int64_t y2 = (yp == 0) ? L - 1 : yp - 1;
        *(uint4 *)(dst + plane_words + y2 * W + gw0) =
            make_uint4(T[0] ^ F1[0], T[1] ^ F1[1], T[2] ^ F1[2], T[3] ^ F1[3]);
      }
    }

    // finish half-sweep 0 of row r: X0(r); roll the carried state
    const uint32_t xl_bit = xprev >> 31;  // X(r) at x0-1
    pull_x(Xr, F0, vr & 1u);
    x0_left = xl_bit ^ ((vl >> 1) & 1u) ^ (F0[0] & 1u);  // X0(r) at x0-1
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      T[j] = Y0[j] ^ F1[j];
      U[j] = Yr[j] ^ F0[j];
      X0[j] = Xr[j];
      Rp[j] = Rr[j];
    }
  }
}

bool stream_kernel_supports(int64_t L) {
  return L >= 4096 && L <= 131072 && (L % 4096) == 0;
}

// Launch plan: ring depth from the shared-memory budget, grid from occupancy,
// at least 64 rows per CTA so the 4-row halo stays small.
struct StreamPlan {
  int threads, stages, grid;
  size_t smem;
};

static StreamPlan plan_for(int64_t L, const void *fn) {
  StreamPlan p;
  p.threads = (int)(L / 128);
  const size_t slot = (size_t)2 * (size_t)(L / 8);
  const size_t budget = 200 * 1024;
  int stages = (int)(budget / slot);
  if (stages > 8) stages = 8;
  if (stages < 2) stages = 2;
  p.stages = stages;
  p.smem = (size_t)stages * slot + (size_t)stages * 8 + 2 * 2 * 32 * 4;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  int dev = 0, sms = 0, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, p.threads, p.smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > L / 64) grid = L / 64;
  if (grid < 1) grid = 1;
  p.grid = (int)grid;
  return p;
}

cudaError_t launch_sweep_stream(const uint32_t *src, uint32_t *dst, int64_t L, uint32_t t,
                                uint64_t seed, const Accept &acc, Ctrl *ctrl,
                                cudaStream_t st) {
  Modes md{0, 0, 0, 0};
  int km = 2;
  if (acc.k <= 1) {
    const uint64_t full = 1ull << acc.k;  // thresholds are in [0, full]
    auto mode = [&](uint64_t T) {         // 0 never, 1 level-0 bit must be 0, 2 always
      if (T == 0) return 0;
      if (T >= full) return 2;
      return 1;
    };
    const int pm = mode(acc.P), qm = mode(acc.Q);
    md.p1 = pm == 1 ? ~0u : 0u;
    md.p2 = pm == 2 ? ~0u : 0u;
    md.q1 = qm == 1 ? ~0u : 0u;
    md.q2 = qm == 2 ? ~0u : 0u;
    km = (qm == 0) ? 0 : 1;
  }
  const void *fn = km == 0   ? (const void *)sweep_stream_kernel<0>
                   : km == 1 ? (const void *)sweep_stream_kernel<1>
                             : (const void *)sweep_stream_kernel<2>;
  static thread_local int64_t cached_L[3] = {0, 0, 0};
  static thread_local StreamPlan cached[3];
  if (cached_L[km] != L) {
    cached[km] = plan_for(L, fn);
    cached_L[km] = L;
  }
  const StreamPlan &p = cached[km];
  if (km == 0)
    sweep_stream_kernel<0><<<p.grid, p.threads, p.smem, st>>>(src, dst, L, p.stages, t, seed,
                                                              acc, md, ctrl);
  else if (km == 1)
    sweep_stream_kernel<1><<<p.grid, p.threads, p.smem, st>>>(src, dst, L, p.stages, t, seed,
                                                              acc, md, ctrl);
  else
    sweep_stream_kernel<2><<<p.grid, p.threads, p.smem, st>>>(src, dst, L, p.stages, t, seed,
                                                              acc, md, ctrl);
  return cudaGetLastError();
}

}  // namespace okz
