// sweep_stream.cu -- F fused sweeps (both half-sweeps each) per launch, one
// pass over HBM: read 2 bits and write 2 bits per site per launch
// (0.5/F B/site/sweep).
//
// Model: octahedron KPZ lattice gas, Kelling & Odor (arXiv:1110.6745),
// Sec. I, Eq. (2), on the checkerboard schedule (half-sweep s = 0 then 1).
//
// Decomposition. A CTA spans a full row: L/(32*WPT) threads, each owning WPT
// consecutive 32-bit words (WPT/4 Philox groups of 128 sites) of both planes,
// so periodic wrap in x stays inside the CTA. The CTA owns a band of rows
// [yb, ye) and streams rows yb-2F .. ye+2F-1 through a ring of shared-memory
// slots filled by 1-D TMA bulk copies (cp.async.bulk + mbarrier).
//
// The 2F half-sweeps ("stages") run as a wavefront: at stream row r, stage h
// (half-sweep h%2 of sweep t + h/2) processes row r-h. Bonds are rewritten by
// their owners ("pull" form):
//     X'(x) = X(x) ^ F(x) ^ F(x+1),   Y'(x,y) = Y(x,y) ^ F(x,y) ^ F(x,y+1).
// Per stage h a thread carries
//   XC[h] = X after stage h of the row it processed last step,
//   E[h]  = Y_in(row) ^ F_h(row) of that row, where Y_in is the Y plane
//           before stage h: it is the "down" bond of the next row (the extra
//           F_h bits sit on sites inactive for the next row, so they are
//           masked), and E[h-1] ^ F_{h-1}(this step) is the "up" bond of
//           stage h,
//   R[j]  = the level-0 random words of sweep t + j, shared by its two
//           half-sweeps (each site is active in exactly one of them).
// One CTA barrier per stream row exchanges two edge bits per stage (shuffles
// inside a warp, shared memory across warps) and recycles the ring slot.
// Output goes to the other buffer of a ping-pong pair, so bands never race.
#include <cuda_runtime.h>

#include "okz_internal.h"
#include "okz_tma.cuh"

namespace okz {

namespace {

// Acceptance modes.
//  kModeHalf: k = 1, P = 1, Q = 0 -- a minimum moves iff its level-0 bit is 0
//             (p_eff = 1/2, q_eff = 0: the growth workloads);
//  kModeK1:   k <= 1, any thresholds (runtime masks md);
//  kModeGen:  any k, levels drawn lazily until every extremum is decided.
constexpr int kModeHalf = 0, kModeK1 = 1, kModeGen = 2;

struct Modes {
  uint32_t p1, p2, q1, q2;  // k <= 1: all-ones masks for "bit must be 0" and "always"
};

template <int WPT, int MODE>
__device__ __forceinline__ void stage_flips(const uint32_t xin[WPT], uint32_t xl_carry,
                                            const uint32_t yd[WPT], const uint32_t yu[WPT],
                                            uint32_t a, const uint32_t r0[WPT], uint32_t g0,
                                            uint32_t t, uint64_t seed, const Accept &acc,
                                            const Modes &md, uint32_t f[WPT],
                                            uint32_t *mn0) {
  uint32_t mn[WPT], mx[WPT];
#pragma unroll
  for (int j = 0; j < WPT; ++j) {
    const uint32_t cin = (j == 0) ? xl_carry : (xin[j - 1] >> 31);
    const uint32_t xl = (xin[j] << 1) | cin;  // sigma_x(x-1) at bit x
    mn[j] = minima(xl, xin[j], yd[j], yu[j]) & a;
    if (MODE != kModeHalf) mx[j] = maxima(xl, xin[j], yd[j], yu[j]) & a;
  }
  *mn0 = mn[0];
  if (MODE == kModeHalf) {
#pragma unroll
    for (int j = 0; j < WPT; ++j) f[j] = mn[j] & ~r0[j];
  } else if (MODE == kModeK1) {
#pragma unroll
    for (int j = 0; j < WPT; ++j)
      f[j] = (mn[j] & ((~r0[j] & md.p1) | md.p2)) | (mx[j] & ((~r0[j] & md.q1) | md.q2));
  } else {
    const uint64_t full = 1ull << acc.k;
    uint32_t ltp[WPT], eqp[WPT], ltq[WPT], eqq[WPT];
    uint32_t any = 0;
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      ltp[j] = (acc.P >= full) ? mn[j] : 0u;
      eqp[j] = (acc.P >= full || acc.P == 0) ? 0u : mn[j];
      ltq[j] = (acc.Q >= full) ? mx[j] : 0u;
      eqq[j] = (acc.Q >= full || acc.Q == 0) ? 0u : mx[j];
      any |= eqp[j] | eqq[j];
    }
    for (int m = 0; m < acc.k && any != 0u; ++m) {
      uint32_t r[WPT];
      if (m == 0) {
#pragma unroll
        for (int j = 0; j < WPT; ++j) r[j] = r0[j];
      } else {
#pragma unroll
        for (int gq = 0; gq < WPT / 4; ++gq) {
          const u32x4 b = group_bits((uint64_t)(g0 + gq), t, (uint32_t)m, seed);
#pragma unroll
          for (int j = 0; j < 4; ++j) r[4 * gq + j] = b.v[j];
        }
      }
      const uint32_t pb = (uint32_t)(acc.P >> (acc.k - 1 - m)) & 1u;
      const uint32_t qb = (uint32_t)(acc.Q >> (acc.k - 1 - m)) & 1u;
      any = 0;
#pragma unroll
      for (int j = 0; j < WPT; ++j) {
        lt_step(r[j], pb, ltp[j], eqp[j]);
        lt_step(r[j], qb, ltq[j], eqq[j]);
        any |= eqp[j] | eqq[j];
      }
    }
#pragma unroll
    for (int j = 0; j < WPT; ++j) f[j] = ltp[j] | ltq[j];
  }
}

}  // namespace

template <int WPT, int F, int MODE>
__global__ void __launch_bounds__(WPT == 4 ? 1024 : 512, 1)
sweep_stream_kernel(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, int L,
                    int stages, uint32_t t0, uint64_t seed, Accept acc, Modes md,
                    Ctrl *__restrict__ ctrl) {
  constexpr int NST = 2 * F;     // half-sweep stages per pass
  constexpr int NG = WPT / 4;    // Philox groups per thread
  extern __shared__ __align__(128) unsigned char smem[];
  const int nthr = blockDim.x;  // L / (32 * WPT)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  const uint32_t W = (uint32_t)L >> 5;   // words per row per plane
  const uint32_t rowbytes = (uint32_t)L >> 3;
  const uint32_t plane_words = (uint32_t)L * W;
  const uint32_t groups_per_row = (uint32_t)L >> 7;

  unsigned char *ring = smem;  // stages x (X row | Y row)
  uint64_t *full = (uint64_t *)(smem + (size_t)stages * 2 * rowbytes);
  uint32_t *exL = (uint32_t *)(full + stages);  // [2][32]: value of lane 0
  uint32_t *exR = exL + 2 * 32;                 // [2][32]: value of lane 31

  const int yb = (int)((int64_t)blockIdx.x * L / gridDim.x);
  const int ye = (int)((int64_t)(blockIdx.x + 1) * L / gridDim.x);
  const int nin = ye - yb + 4 * F;  // rows yb-2F .. ye+2F-1

  // producer state (thread 0): next stream row to load and its ring position
  int p_row = yb - 2 * F;
  if (p_row < 0) p_row += L;
  int p_slot = 0;
  auto issue = [&]() {
    unsigned char *d = ring + (size_t)p_slot * 2 * rowbytes;
    tma::mbar_expect_tx(&full[p_slot], 2 * rowbytes);
    tma::load_1d(d, src + (size_t)p_row * W, rowbytes, &full[p_slot]);
    tma::load_1d(d + rowbytes, src + plane_words + (size_t)p_row * W, rowbytes, &full[p_slot]);
    if (++p_row == L) p_row = 0;
    if (++p_slot == stages) p_slot = 0;
  };

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) tma::mbar_init(&full[s], 1);
    tma::mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0)
    for (int i = 0; i < stages && i < nin; ++i) issue();

  // carried state (see the file comment)
  uint32_t XC[NST > 1 ? NST - 1 : 1][WPT];
  uint32_t XLC[NST > 1 ? NST - 1 : 1];
  uint32_t E[NST][WPT];
  uint32_t R[F][WPT];
#pragma unroll
  for (int h = 0; h < NST; ++h) {
#pragma unroll
    for (int j = 0; j < WPT; ++j) E[h][j] = 0;
    if (h < NST - 1) {
      XLC[h] = 0;
#pragma unroll
      for (int j = 0; j < WPT; ++j) XC[h][j] = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < F; ++q)
#pragma unroll
    for (int j = 0; j < WPT; ++j) R[q][j] = 0;

  const uint32_t w0 = (uint32_t)(WPT * tid);         // my first word within a row
  const uint32_t wprev = (w0 == 0) ? W - 1 : w0 - 1;  // word holding my left bond
  int slot = 0;
  uint32_t phase = 0;
  int y = yb - 2 * F;  // wrapped row of the current stream position
  if (y < 0) y += L;
  const int r_origin = yb - 2 * F;  // unwrapped row of stream position 0

  for (int i = 0; i < nin; ++i) {
    const bool ok = tma::mbar_wait(&full[slot], phase);
    const unsigned char *d = ring + (size_t)slot * 2 * rowbytes;
    uint32_t Xr[WPT], Yr[WPT];
#pragma unroll
    for (int gq = 0; gq < NG; ++gq) {
      const uint4 xv = *(const uint4 *)(d + 4 * (w0 + 4 * gq));
      const uint4 yv = *(const uint4 *)(d + rowbytes + 4 * (w0 + 4 * gq));
      Xr[4 * gq + 0] = xv.x; Xr[4 * gq + 1] = xv.y; Xr[4 * gq + 2] = xv.z; Xr[4 * gq + 3] = xv.w;
      Yr[4 * gq + 0] = yv.x; Yr[4 * gq + 1] = yv.y; Yr[4 * gq + 2] = yv.z; Yr[4 * gq + 3] = yv.w;
    }
    const uint32_t xl_raw = *(const uint32_t *)(d + 4 * wprev) >> 31;  // X(r) at x0-1

    // ---- stages: F_h for row y - h ------------------------------------
    uint32_t Fs[NST][WPT];
    uint32_t Rn[F][WPT];
    uint32_t mn0[NST];
    uint32_t yup[WPT];
#pragma unroll
    for (int j = 0; j < WPT; ++j) yup[j] = Yr[j];
#pragma unroll
    for (int h = 0; h < NST; ++h) {
      int q = y - h;
      if (q < 0) q += L;
      const int s = h & 1;
      const uint32_t t = t0 + (uint32_t)(h >> 1);
      const uint32_t g0 = (uint32_t)q * groups_per_row + (uint32_t)(NG * tid);
      // level-0 words of row q, sweep t: fresh for s = 0 (kept in Rn until
      // the s = 1 stage of this step has used the previous row's R)
      if (s == 0) {
#pragma unroll
        for (int gq = 0; gq < NG; ++gq) {
          const u32x4 b = group_bits((uint64_t)(g0 + gq), t, 0u, seed);
#pragma unroll
          for (int j = 0; j < 4; ++j) Rn[h >> 1][4 * gq + j] = b.v[j];
        }
      }
      const uint32_t *xin = (h == 0) ? Xr : XC[h > 0 ? h - 1 : 0];
      const uint32_t xlc = (h == 0) ? xl_raw : XLC[h > 0 ? h - 1 : 0];
      stage_flips<WPT, MODE>(xin, xlc, E[h], yup, active_mask(q, s),
                             s == 0 ? Rn[h >> 1] : R[h >> 1], g0, t, seed, acc, md, Fs[h],
                             &mn0[h]);
      if (s == 1) {
#pragma unroll
        for (int j = 0; j < WPT; ++j) R[h >> 1][j] = Rn[h >> 1][j];
      }
      // next stage's up bond (uses the old E[h]), then the new E[h]
      uint32_t nxt[WPT];
#pragma unroll
      for (int j = 0; j < WPT; ++j) {
        nxt[j] = E[h][j] ^ Fs[h][j];
        E[h][j] = yup[j] ^ Fs[h][j];
        yup[j] = nxt[j];
      }
      // after the loop yup = old E[NST-1] ^ F_last = final Y of row y - NST
    }

    // H0 = h(0,0): only CTA 0 sees unwrapped row 0; site (0,0) is active in s = 0
    if (tid == 0) {
      const int r = r_origin + i;
#pragma unroll
      for (int h = 0; h < NST; h += 2)
        if (r - h == 0 && (Fs[h][0] & 1u)) ctrl->H0 += (mn0[h] & 1u) ? 2 : -2;
    }

    // ---- exchange edge bits: bit 2h = F_h at my first site (for the left
    // neighbour), bit 2h+1 = F_h at my last site (for the right neighbour)
    uint32_t v = 0;
#pragma unroll
    for (int h = 0; h < NST; ++h)
      v |= ((Fs[h][0] & 1u) << (2 * h)) | ((Fs[h][WPT - 1] >> 31) << (2 * h + 1));
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
        // (positions i .. i + stages - 1; the wait on position i itself
        // failed, so it gets one more bounded wait as well)
        int sl = slot;
        uint32_t ph = phase;
        for (int k = i; k < nin && k < i + stages; ++k) {
          (void)tma::mbar_wait(&full[sl], ph);
          if (++sl == stages) {
            sl = 0;
            ph ^= 1u;
          }
        }
      }
      return;
    }
    if (lane == 31) vr = exL[par * 32 + (warp + 1 == nwarps ? 0 : warp + 1)];
    if (lane == 0) vl = exR[par * 32 + (warp == 0 ? nwarps - 1 : warp - 1)];

    // the slot of this row is free: refill it with row i + stages
    if (tid == 0 && i + stages < nin) {
      tma::fence_proxy_async();
      issue();
    }

    // ---- X updates: X_h = X_in ^ F_h ^ F_h(x+1); carry or store ----------
#pragma unroll
    for (int h = NST - 1; h >= 0; --h) {
      const uint32_t *xin = (h == 0) ? Xr : XC[h > 0 ? h - 1 : 0];
      const uint32_t xlc = (h == 0) ? xl_raw : XLC[h > 0 ? h - 1 : 0];
      uint32_t xo[WPT];
#pragma unroll
      for (int j = 0; j < WPT; ++j) {
        const uint32_t nb = (j == WPT - 1) ? ((vr >> (2 * h)) & 1u) : (Fs[h][j + 1] & 1u);
        xo[j] = xin[j] ^ Fs[h][j] ^ ((Fs[h][j] >> 1) | (nb << 31));
      }
      if (h == NST - 1) {  // final X of row y - (NST-1)
        const int r = r_origin + i - (NST - 1);
        if (r >= yb && r < ye) {
          int q = y - (NST - 1);
          if (q < 0) q += L;
          uint32_t *o = dst + (size_t)q * W + w0;
#pragma unroll
          for (int gq = 0; gq < NG; ++gq)
            *(uint4 *)(o + 4 * gq) =
                make_uint4(xo[4 * gq], xo[4 * gq + 1], xo[4 * gq + 2], xo[4 * gq + 3]);
        }
      } else {
        // X_h at x0-1 = X_in at x0-1 ^ F_h(x0-1) (left neighbour) ^ F_h(x0)
        XLC[h] = xlc ^ ((vl >> (2 * h + 1)) & 1u) ^ (Fs[h][0] & 1u);
#pragma unroll
        for (int j = 0; j < WPT; ++j) XC[h][j] = xo[j];
      }
    }
    // final Y of row y - NST
    {
      const int r = r_origin + i - NST;
      if (r >= yb && r < ye) {
        int q = y - NST;
        if (q < 0) q += L;
        uint32_t *o = dst + plane_words + (size_t)q * W + w0;
#pragma unroll
        for (int gq = 0; gq < NG; ++gq)
          *(uint4 *)(o + 4 * gq) =
              make_uint4(yup[4 * gq], yup[4 * gq + 1], yup[4 * gq + 2], yup[4 * gq + 3]);
      }
    }

    if (++slot == stages) {
      slot = 0;
      phase ^= 1u;
    }
    if (++y == L) y = 0;
  }
}

bool stream_kernel_supports(int64_t L) {
  return L >= 4096 && L <= 131072 && (L % 4096) == 0;
}

namespace {

struct StreamPlan {
  int threads, stages, grid;
  size_t smem;
};

// Launch plan: ring depth from the shared-memory budget, grid from occupancy
// and the band height (stream_grid).
StreamPlan plan_for(int L, int wpt, int F, int band_rows, const void *fn) {
  StreamPlan p;
  p.threads = L / (32 * wpt);
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
  p.grid = stream_grid(L, F, band_rows, sms * per_sm);
  return p;
}

template <int WPT, int F, int MODE>
cudaError_t launch_cfg(const uint32_t *src, uint32_t *dst, int L, uint32_t t, uint64_t seed,
                       const Accept &acc, const Modes &md, int band_rows, Ctrl *ctrl,
                       cudaStream_t st) {
  static thread_local int cached_L = 0, cached_band = -1;
  static thread_local StreamPlan plan;
  const void *fn = (const void *)sweep_stream_kernel<WPT, F, MODE>;
  if (cached_L != L || cached_band != band_rows) {
    plan = plan_for(L, WPT, F, band_rows, fn);
    cached_L = L;
    cached_band = band_rows;
  }
  sweep_stream_kernel<WPT, F, MODE><<<plan.grid, plan.threads, plan.smem, st>>>(
      src, dst, L, plan.stages, t, seed, acc, md, ctrl);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode(const uint32_t *src, uint32_t *dst, int L, uint32_t t, uint64_t seed,
                        const Accept &acc, const Modes &md, int wpt, int fuse, int band_rows,
                        Ctrl *ctrl, cudaStream_t st) {
  if (wpt == 8) {
    if (fuse == 2) return launch_cfg<8, 2, MODE>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
    return launch_cfg<8, 1, MODE>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
  }
  if (fuse == 2) return launch_cfg<4, 2, MODE>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
  return launch_cfg<4, 1, MODE>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
}

}  // namespace

bool stream_wpt_valid(int64_t L, int wpt) {
  if (!stream_kernel_supports(L)) return false;
  if (wpt == 4) return true;
  if (wpt == 8) return L % 8192 == 0;  // L/256 threads, a whole number of warps
  return false;
}

cudaError_t launch_sweep_stream(const uint32_t *src, uint32_t *dst, int64_t L, uint32_t t,
                                uint64_t seed, const Accept &acc, int wpt, int fuse,
                                int band_rows, Ctrl *ctrl, cudaStream_t st) {
  Modes md{0, 0, 0, 0};
  int mode = kModeGen;
  if (acc.k <= 1) {
    const uint64_t full = 1ull << acc.k;  // thresholds are in [0, full]
    auto sel = [&](uint64_t T) {          // 0 never, 1 level-0 bit must be 0, 2 always
      if (T == 0) return 0;
      if (T >= full) return 2;
      return 1;
    };
    const int pm = sel(acc.P), qm = sel(acc.Q);
    md.p1 = pm == 1 ? ~0u : 0u;
    md.p2 = pm == 2 ? ~0u : 0u;
    md.q1 = qm == 1 ? ~0u : 0u;
    md.q2 = qm == 2 ? ~0u : 0u;
    mode = (pm == 1 && qm == 0) ? kModeHalf : kModeK1;
  }
  const int Li = (int)L;
  if (mode == kModeHalf)
    return launch_mode<kModeHalf>(src, dst, Li, t, seed, acc, md, wpt, fuse, band_rows, ctrl, st);
  if (mode == kModeK1)
    return launch_mode<kModeK1>(src, dst, Li, t, seed, acc, md, wpt, fuse, band_rows, ctrl, st);
  return launch_mode<kModeGen>(src, dst, Li, t, seed, acc, md, wpt, fuse, band_rows, ctrl, st);
}

}  // namespace okz
