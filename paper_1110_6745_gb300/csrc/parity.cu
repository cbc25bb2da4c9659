// parity.cu -- the octahedron model on a single height-parity bit-plane.
//
// Heights of the octahedron model satisfy h(x,y) == x + y (mod 2) (Kelling &
// Odor, arXiv:1110.6745, Sec. I: neighbours differ by exactly 1). Writing
// h = p + 2k with p = (x+y) mod 2, one bit per site, b = k mod 2 (h mod 4
// given p), fixes every slope:
//     sigma_x(x,y) = +1  <=>  b(x+1,y) ^ b(x,y) ^ p(x,y) == 0,
//     sigma_y(x,y) = +1  <=>  b(x,y+1) ^ b(x,y) ^ p(x,y) == 0,
// so the two slope planes of Sec. II carry one redundant bit per site. In
// this encoding the rule of Eq. (2) reads: a site of half-sweep s (p = s) is
// a local minimum iff all four neighbours have b == b(x,y) ^ s, a local
// maximum iff all four have b == !(b(x,y) ^ s), and a move (h += 2 or
// h -= 2) toggles only the site's own bit. A sweep therefore reads one bit
// and writes one bit per site (0.25 B/site) and no bond is shared.
//
// Layout: L rows of L/32 little-endian uint32 words; bit b of word w of row y
// is site x = 32w + b. The C-ABI state format stays the slope planes;
// convert.cu converts at the boundary.
#include <cuda_runtime.h>

#include "okz_internal.h"
#include "okz_tma.cuh"

namespace okz {

namespace {

// Sites of row y with p(x,y) = (x+y) mod 2 == 1.
__device__ __forceinline__ uint32_t odd_mask(int64_t y) {
  return (y & 1) ? 0x55555555u : 0xAAAAAAAAu;
}

// Minima and maxima of 32 sites: c = own bits ^ S (S = all ones for s = 1),
// l, r, d, u = the left, right, lower and upper neighbours' bits.
__device__ __forceinline__ void parity_extrema(uint32_t c, uint32_t l, uint32_t r, uint32_t d,
                                               uint32_t u, uint32_t a, uint32_t &mn,
                                               uint32_t &mx) {
  const uint32_t dl = l ^ c, dr = r ^ c, dd = d ^ c, du = u ^ c;
  mn = a & ~(dl | dr | dd | du);
  mx = a & dl & dr & dd & du;
}

}  // namespace

// ---------------------------------------------------------------------------
// In-place half-sweep, one thread per 128-site group. A flip changes only the
// site's own bit, and every bit a thread reads from a neighbouring word sits
// on a site of the other sublattice, which nobody writes in this half-sweep;
// whole-word stores therefore never change a bit another thread uses.
// ---------------------------------------------------------------------------
// (t_base: as in the slope-plane half-sweep, the first sweep of a graph
// chunk read from device memory; t is then the offset within the chunk)
__global__ void __launch_bounds__(256)
parity_halfsweep_kernel(uint32_t *__restrict__ B, int64_t L, int s, uint32_t t_off,
                        const unsigned int *__restrict__ t_base, const RoundKeys rk, Accept acc,
                        Ctrl *__restrict__ ctrl) {
  const uint32_t t = t_off + (t_base ? *t_base : 0u);
  const int64_t W = L >> 5;
  const int64_t groups = L * W >> 2;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= groups) return;
  uint32_t mn[4], mx[4], ctr[4];
  int64_t idx[4];
  const uint32_t S = s ? ~0u : 0u;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t gw = 4 * g + j;
    const int64_t y = gw / W, w = gw - y * W;
    const int64_t wl = (w == 0) ? W - 1 : w - 1, wr = (w == W - 1) ? 0 : w + 1;
    const int64_t yd = (y == 0) ? L - 1 : y - 1, yu = (y == L - 1) ? 0 : y + 1;
    idx[j] = gw;
    ctr[j] = B[gw];
    const uint32_t l = __funnelshift_l(B[y * W + wl], ctr[j], 1);  // b(x-1)
    const uint32_t r = __funnelshift_r(ctr[j], B[y * W + wr], 1);  // b(x+1)
    parity_extrema(ctr[j] ^ S, l, r, B[yd * W + w], B[yu * W + w], active_mask(y, s), mn[j],
                   mx[j]);
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
    const u32x4 r = philox10_rk((uint32_t)g, (uint32_t)((uint64_t)g >> 32), t, (uint32_t)m, rk);
    const uint32_t pb = (uint32_t)(acc.P >> (acc.k - 1 - m)) & 1u;
    const uint32_t qb = (uint32_t)(acc.Q >> (acc.k - 1 - m)) & 1u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      lt_step(r.v[j], pb, ltp[j], eqp[j]);
      lt_step(r.v[j], qb, ltq[j], eqq[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t f = ltp[j] | ltq[j];
    if (f == 0u) continue;
    B[idx[j]] = ctr[j] ^ f;
    if (idx[j] == 0 && (f & 1u)) ctrl->H0 += (mn[0] & 1u) ? 2 : -2;  // site (0,0)
  }
}

cudaError_t launch_parity_halfsweep(uint32_t *B, int64_t L, int s, uint32_t t, uint64_t seed,
                                    const Accept &acc, Ctrl *ctrl, cudaStream_t st,
                                    const unsigned int *t_base) {
  const int64_t groups = L * (L >> 5) / 4;
  parity_halfsweep_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(
      B, L, s, t, t_base, round_keys(seed), acc, ctrl);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Streaming kernel: F sweeps (2F half-sweep "stages") per launch; a CTA spans
// full rows (L/(32*WPT) threads, WPT words each) and owns a band [yb, ye).
// Stream row r (one 1-D TMA copy into a ring slot) drives a wavefront:
//   stage 0 (half-sweep 0 of sweep t) processes row r-1 from the ring rows
//       r-2, r-1, r;
//   stage h > 0 processes row r-1-h from stage h-1's outputs: two carried
//       rows (Wd = two steps ago, Wc = one step ago) and this step's output.
// Output rows depend only on their own inputs (a move toggles only the site's
// own bit), so nothing is masked or pulled. The x-neighbour bits of each
// carried row are exchanged once per stream row (warp shuffles, shared memory
// across warps, one CTA barrier that also recycles the ring slot of row r-2).
// ---------------------------------------------------------------------------
namespace {

constexpr int kPModeHalf = 0, kPModeK1 = 1, kPModeGen = 2;

struct PModes {
  uint32_t p1, p2, q1, q2;  // k <= 1: all-ones masks for "bit must be 0" and "always"
};

// New words (o) of WPT words of one stage of half-sweep parity SP. The neighbour
// tests use 3-input logic: for SP = 0 a minimum has all four neighbours equal
// to its own bit ("both equal" table 0x81 on (l, r, c) and on (d, u, c)),
// for SP = 1 all four differ (table 0x42); maxima are the reverse.
template <int WPT, int MODE, int SP, int KC>
__device__ __forceinline__ void pstage(const uint32_t c[WPT], uint32_t lbit, uint32_t rbit,
                                       const uint32_t d[WPT], const uint32_t u[WPT], uint32_t a,
                                       const uint32_t (&lv)[KC][WPT], uint32_t g0, uint32_t t,
                                       const RoundKeys &rk, const Accept &acc,
                                       const PModes &md, uint32_t o[WPT], uint32_t *mn0) {
  const uint32_t *r0 = lv[0];
  constexpr uint32_t kMin = SP ? 0x42u : 0x81u;
  constexpr uint32_t kMax = SP ? 0x81u : 0x42u;
  uint32_t mn[WPT], mx[WPT];
#pragma unroll
  for (int j = 0; j < WPT; ++j) {
    const uint32_t l = __funnelshift_l(j == 0 ? (lbit << 31) : c[j - 1], c[j], 1);
    const uint32_t r = __funnelshift_r(c[j], j == WPT - 1 ? rbit : c[j + 1], 1);
    if (MODE == kPModeHalf) {
      // new word = c ^ (x & y & a & ~r0): y & a & ~r0 (table 0x40), then
      // c ^ (x & that) (table 0x78) -- 2 funnel shifts + 4 logic ops per word
      const uint32_t ysel = lop3<0x40>(lop3<kMin>(d[j], u[j], c[j]), a, r0[j]);
      o[j] = lop3<0x78>(c[j], lop3<kMin>(l, r, c[j]), ysel);
    } else {
      mn[j] = lop3<0x80>(lop3<kMin>(l, r, c[j]), lop3<kMin>(d[j], u[j], c[j]), a);
      mx[j] = lop3<0x80>(lop3<kMax>(l, r, c[j]), lop3<kMax>(d[j], u[j], c[j]), a);
    }
  }
  if (MODE == kPModeHalf) {  // q = 0: every move is a minimum rising by 2
    *mn0 = 1u;
    return;
  }
  *mn0 = mn[0];
  if (MODE == kPModeK1) {
#pragma unroll
    for (int j = 0; j < WPT; ++j)
      o[j] = c[j] ^ ((mn[j] & ((~r0[j] & md.p1) | md.p2)) | (mx[j] & ((~r0[j] & md.q1) | md.q2)));
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
    if constexpr (KC > 1) {
      // levels 0..KC-1: drawn once per sweep and carried between its stages
      // (compile-time indices, so the cache stays in registers)
#pragma unroll
      for (int m = 0; m < KC; ++m) {
        if (m >= acc.k || any == 0u) break;
        const uint32_t pb = (uint32_t)(acc.P >> (acc.k - 1 - m)) & 1u;
        const uint32_t qb = (uint32_t)(acc.Q >> (acc.k - 1 - m)) & 1u;
        any = 0;
#pragma unroll
        for (int j = 0; j < WPT; ++j) {
          lt_step(lv[m][j], pb, ltp[j], eqp[j]);
          lt_step(lv[m][j], qb, ltq[j], eqq[j]);
          any |= eqp[j] | eqq[j];
        }
      }
    }
    // level 0 from the cache when KC == 1; further levels drawn when needed
    for (int m = (KC > 1 ? KC : 0); m < acc.k && any != 0u; ++m) {
      uint32_t rr[WPT];
      if (KC == 1 && m == 0) {
#pragma unroll
        for (int j = 0; j < WPT; ++j) rr[j] = lv[0][j];
      } else {
#pragma unroll
        for (int gq = 0; gq < WPT / 4; ++gq) {
          const u32x4 b = philox10_rk(g0 + gq, 0u, t, (uint32_t)m, rk);
#pragma unroll
          for (int j = 0; j < 4; ++j) rr[4 * gq + j] = b.v[j];
        }
      }
      const uint32_t pb = (uint32_t)(acc.P >> (acc.k - 1 - m)) & 1u;
      const uint32_t qb = (uint32_t)(acc.Q >> (acc.k - 1 - m)) & 1u;
      any = 0;
#pragma unroll
      for (int j = 0; j < WPT; ++j) {
        lt_step(rr[j], pb, ltp[j], eqp[j]);
        lt_step(rr[j], qb, ltq[j], eqq[j]);
        any |= eqp[j] | eqq[j];
      }
    }
#pragma unroll
    for (int j = 0; j < WPT; ++j) o[j] = c[j] ^ (ltp[j] | ltq[j]);
  }
}

// Thresholds of the general-k stage: P and Q with level 0 at bit 31, and the
// comparison state every site starts from (lt: decided below, eq: undecided;
// a threshold of 0 or 2^k decides every site at once).
struct GenBits {
  uint32_t pw, qw, lp0, ep0, lq0, eq0;
};

__device__ __forceinline__ GenBits gen_bits(const Accept &acc) {
  const uint64_t full = 1ull << acc.k;
  GenBits b;
  b.pw = (uint32_t)(acc.P << (32 - acc.k));
  b.qw = (uint32_t)(acc.Q << (32 - acc.k));
  b.lp0 = (acc.P >= full) ? ~0u : 0u;
  b.ep0 = (acc.P >= full || acc.P == 0) ? 0u : ~0u;
  b.lq0 = (acc.Q >= full) ? ~0u : 0u;
  b.eq0 = (acc.Q >= full || acc.Q == 0) ? 0u : ~0u;
  return b;
}

__device__ __forceinline__ uint32_t rotl1(uint32_t x) { return __funnelshift_l(x, x, 1); }
__device__ __forceinline__ uint32_t rotr1(uint32_t x) { return __funnelshift_r(x, x, 1); }

// General k (random levels drawn lazily), one stage of half-sweep parity SP.
// The random words of level m of 128-site group g in sweep t are Philox
// (g, 0, t, m): keyed by group, sweep and level, never by the half-sweep, and
// a site is active in one half-sweep only, so the levels the first half draws
// for its candidates decide the second half's sites as far as they go. SP = 0
// starts every site of the words undecided and draws levels while any lane
// of the warp has an undecided candidate (every lane runs every stage, and a
// warp runs to its last lane anyway); it leaves the second-half state packed
// in LT, EQ (word j: the P comparison at the second-half positions, the Q
// comparison rotated left by one bit into the first-half positions) with the
// next level in m. SP = 1, one stream row later on the same row and sweep,
// starts from that state and draws only the levels beyond it.
template <int WPT, int SP>
__device__ __forceinline__ void pstage_gen(const uint32_t c[WPT], uint32_t lbit, uint32_t rbit,
                                           const uint32_t d[WPT], const uint32_t u[WPT],
                                           uint32_t a, uint32_t g0, uint32_t t,
                                           const RoundKeys &rk, const Accept &acc,
                                           const GenBits &gb, uint32_t o[WPT], uint32_t *mn0,
                                           uint32_t LT[WPT], uint32_t EQ[WPT], int &m) {
  constexpr int NG = WPT / 4;
  constexpr uint32_t kMin = SP ? 0x42u : 0x81u;
  constexpr uint32_t kMax = SP ? 0x81u : 0x42u;
  uint32_t mn[WPT], mx[WPT], lp[WPT], ep[WPT], lq[WPT], eq[WPT];
#pragma unroll
  for (int j = 0; j < WPT; ++j) {
    const uint32_t l = __funnelshift_l(j == 0 ? (lbit << 31) : c[j - 1], c[j], 1);
    const uint32_t r = __funnelshift_r(c[j], j == WPT - 1 ? rbit : c[j + 1], 1);
    mn[j] = lop3<0x80>(lop3<kMin>(l, r, c[j]), lop3<kMin>(d[j], u[j], c[j]), a);
    mx[j] = lop3<0x80>(lop3<kMax>(l, r, c[j]), lop3<kMax>(d[j], u[j], c[j]), a);
    if (SP == 0) {
      lp[j] = gb.lp0;
      ep[j] = gb.ep0;
      lq[j] = gb.lq0;
      eq[j] = gb.eq0;
    } else {  // only the second-half positions are read below
      lp[j] = LT[j];
      ep[j] = EQ[j];
      lq[j] = rotr1(LT[j]);
      eq[j] = rotr1(EQ[j]);
    }
  }
  *mn0 = mn[0];
  if (SP == 0) m = 0;
  // the first half draws two levels per test at 4 words per thread: two
  // independent Philox chains in flight (a level drawn beyond the last
  // undecided candidate changes nothing decided)
  constexpr int LV = (SP == 0 && WPT == 4) ? 2 : 1;
  while (m < acc.k) {
    uint32_t open = 0;
#pragma unroll
    for (int j = 0; j < WPT; ++j) open |= (ep[j] & mn[j]) | (eq[j] & mx[j]);
    if (SP == 0 ? !__any_sync(0xFFFFFFFFu, open != 0u) : open == 0u) break;
    const int nl = (LV == 2 && m + 1 < acc.k) ? 2 : 1;
    u32x4 bl[LV][NG];
#pragma unroll
    for (int v = 0; v < LV; ++v)
#pragma unroll
      for (int gq = 0; gq < NG; ++gq)
        if (v < nl) bl[v][gq] = philox10_rk(g0 + gq, 0u, t, (uint32_t)(m + v), rk);
#pragma unroll
    for (int v = 0; v < LV; ++v) {
      if (v >= nl) break;
      const int mv = m + v;
      const uint32_t pb = (gb.pw >> (31 - mv)) & 1u, qb = (gb.qw >> (31 - mv)) & 1u;
#pragma unroll
      for (int gq = 0; gq < NG; ++gq)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          lt_step(bl[v][gq].v[j], pb, lp[4 * gq + j], ep[4 * gq + j]);
          lt_step(bl[v][gq].v[j], qb, lq[4 * gq + j], eq[4 * gq + j]);
        }
    }
    m += nl;
  }
#pragma unroll
  for (int j = 0; j < WPT; ++j) o[j] = c[j] ^ ((lp[j] & mn[j]) | (lq[j] & mx[j]));
  if (SP == 0) {
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      LT[j] = (lp[j] & ~a) | (rotl1(lq[j]) & a);
      EQ[j] = (ep[j] & ~a) | (rotl1(eq[j]) & a);
    }
  }
}

}  // namespace

// SMALL: rows of at most 256 threads (L <= 32768 at 4 words per thread, any
// L at 16), so the register budget is not capped by a 512- or 1024-thread
// bound.
template <int WPT, int F, int MODE, bool SMALL>
__global__ void __launch_bounds__(SMALL ? 256 : (WPT == 4 ? 1024 : 512), 1)
parity_stream_kernel(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, int L,
                     int stages, uint32_t t0, const RoundKeys rk, Accept acc, PModes md,
                     Ctrl *__restrict__ ctrl) {
  constexpr int NST = 2 * F;
  constexpr int NC = NST > 1 ? NST - 1 : 1;  // stages whose output is carried
  constexpr int NG = WPT / 4;
  constexpr bool GEN = MODE == kPModeGen;
  constexpr int KC = 1;            // k <= 1: level 0 drawn once per sweep
  constexpr int FG = GEN ? F : 1;  // general k: comparison state carried per sweep
  extern __shared__ __align__(128) unsigned char smem[];
  const int nthr = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  const uint32_t W = (uint32_t)L >> 5;
  const uint32_t rowbytes = (uint32_t)L >> 3;
  const uint32_t groups_per_row = (uint32_t)L >> 7;

  unsigned char *ring = smem;  // stages x one row of b
  uint64_t *full = (uint64_t *)(smem + (size_t)stages * rowbytes);
  uint32_t *exL = (uint32_t *)(full + stages);  // [2][32]: value of lane 0
  uint32_t *exR = exL + 2 * 32;                 // [2][32]: value of lane 31

  const int yb = (int)((int64_t)blockIdx.x * L / gridDim.x);
  const int ye = (int)((int64_t)(blockIdx.x + 1) * L / gridDim.x);
  const int nin = ye - yb + 4 * F;  // stream rows yb-2F .. ye+2F-1

  int p_row = yb - 2 * F;  // producer (thread 0): next row to load, its slot
  if (p_row < 0) p_row += L;
  int p_slot = 0;
  auto issue = [&]() {
    tma::mbar_expect_tx(&full[p_slot], rowbytes);
    tma::load_1d(ring + (size_t)p_slot * rowbytes, src + (size_t)p_row * W, rowbytes,
                 &full[p_slot]);
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

  uint32_t Wd[NC][WPT], Wc[NC][WPT];  // stage h's outputs two / one steps ago
  uint32_t WL[NC], WR[NC];            // x-neighbour bits of Wc[h]
  uint32_t R[F][KC][WPT];             // k <= 1: level 0 of the row stage 2j saw last step
  uint32_t CL[FG][WPT], CE[FG][WPT];  // general k: that row's packed second-half state
  int Cm[FG];
  const GenBits gb = gen_bits(acc);
#pragma unroll
  for (int h = 0; h < NC; ++h) {
    WL[h] = 0;
    WR[h] = 0;
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      Wd[h][j] = 0;
      Wc[h][j] = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < F; ++q)
#pragma unroll
    for (int m = 0; m < KC; ++m)
#pragma unroll
      for (int j = 0; j < WPT; ++j) R[q][m][j] = 0;
#pragma unroll
  for (int q = 0; q < FG; ++q) {
    Cm[q] = 0;
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      CL[q][j] = 0;
      CE[q][j] = 0;
    }
  }

  const uint32_t w0 = (uint32_t)(WPT * tid);
  const uint32_t wprev = (w0 == 0) ? W - 1 : w0 - 1;
  const uint32_t wnext = (w0 + WPT == W) ? 0 : w0 + WPT;
  int slot = 0, sl1 = stages - 1, sl2 = stages - 2;  // slots of positions i, i-1, i-2
  uint32_t phase = 0;
  int y = yb - 2 * F;  // wrapped row of stream position i
  if (y < 0) y += L;
  const int r_origin = yb - 2 * F;
  // every stage of a step shares one active mask: stage h works on row
  // y-1-h in half-sweep h%2, and (y - 1 - h + h%2) has the parity of y - 1
  uint32_t am = ((y - 1) & 1) ? 0xAAAAAAAAu : 0x55555555u;
  // first group of this thread in row y-1 (stage 0); stage h: - h rows
  int q0 = (y == 0) ? L - 1 : y - 1;
  uint32_t gq0 = (uint32_t)q0 * groups_per_row + (uint32_t)(NG * tid);
  const uint32_t wrap_groups = (uint32_t)L * groups_per_row;

  for (int i = 0; i < nin; ++i) {
    const bool ok = tma::mbar_wait(&full[slot], phase);
    uint32_t out[NST][WPT];
    uint32_t fbit[NST], mn0[NST];
    const bool active = i >= 2;  // rows r-2, r-1, r are in the ring
    if (active) {
      const unsigned char *ru = ring + (size_t)slot * rowbytes;  // row r   (above)
      const unsigned char *rc = ring + (size_t)sl1 * rowbytes;   // row r-1
      const unsigned char *rd = ring + (size_t)sl2 * rowbytes;   // row r-2 (below)
      uint32_t cu[WPT], cc[WPT], cd[WPT];
#pragma unroll
      for (int gq = 0; gq < NG; ++gq) {
        const uint4 a = *(const uint4 *)(ru + 4 * (w0 + 4 * gq));
        const uint4 b = *(const uint4 *)(rc + 4 * (w0 + 4 * gq));
        const uint4 e = *(const uint4 *)(rd + 4 * (w0 + 4 * gq));
        cu[4 * gq] = a.x; cu[4 * gq + 1] = a.y; cu[4 * gq + 2] = a.z; cu[4 * gq + 3] = a.w;
        cc[4 * gq] = b.x; cc[4 * gq + 1] = b.y; cc[4 * gq + 2] = b.z; cc[4 * gq + 3] = b.w;
        cd[4 * gq] = e.x; cd[4 * gq + 1] = e.y; cd[4 * gq + 2] = e.z; cd[4 * gq + 3] = e.w;
      }
      const uint32_t lb = *(const uint32_t *)(rc + 4 * wprev) >> 31;
      const uint32_t rb = *(const uint32_t *)(rc + 4 * wnext) & 1u;
      uint32_t Rn[F][KC][WPT];
      uint32_t CnL[FG][WPT], CnE[FG][WPT];
      int Cnm[FG];
#pragma unroll
      for (int h = 0; h < NST; ++h) {
        const int s = h & 1;
        const uint32_t t = t0 + (uint32_t)(h >> 1);
        uint32_t g0 = gq0 - (uint32_t)h * groups_per_row;  // row y-1-h, wrapped
        if (q0 < h) g0 += wrap_groups;
        if (!GEN && s == 0) {  // fresh words of row y-1-h, sweep t: level 0
#pragma unroll
          for (int gq = 0; gq < NG; ++gq) {
            const u32x4 b = philox10_rk(g0 + gq, 0u, t, 0u, rk);
#pragma unroll
            for (int j = 0; j < 4; ++j) Rn[h >> 1][0][4 * gq + j] = b.v[j];
          }
        }
        const uint32_t *c = (h == 0) ? cc : Wc[h > 0 ? h - 1 : 0];
        const uint32_t *d = (h == 0) ? cd : Wd[h > 0 ? h - 1 : 0];
        const uint32_t *u = (h == 0) ? cu : out[h > 0 ? h - 1 : 0];
        const uint32_t lbit = (h == 0) ? lb : WL[h > 0 ? h - 1 : 0];
        const uint32_t rbit = (h == 0) ? rb : WR[h > 0 ? h - 1 : 0];
        uint32_t o[WPT];
        // s = 1 uses what stage h-1 drew for the same row last step
        if (GEN && s == 0)
          pstage_gen<WPT, 0>(c, lbit, rbit, d, u, am, g0, t, rk, acc, gb, o, &mn0[h],
                             CnL[(h >> 1) % FG], CnE[(h >> 1) % FG], Cnm[(h >> 1) % FG]);
        else if (GEN)
          pstage_gen<WPT, 1>(c, lbit, rbit, d, u, am, g0, t, rk, acc, gb, o, &mn0[h],
                             CL[(h >> 1) % FG], CE[(h >> 1) % FG], Cm[(h >> 1) % FG]);
        else if (s == 0)
          pstage<WPT, MODE, 0, KC>(c, lbit, rbit, d, u, am, Rn[h >> 1], g0, t, rk, acc, md,
                                   o, &mn0[h]);
        else
          pstage<WPT, MODE, 1, KC>(c, lbit, rbit, d, u, am, R[h >> 1], g0, t, rk, acc, md,
                                   o, &mn0[h]);
        fbit[h] = (o[0] ^ c[0]) & 1u;
#pragma unroll
        for (int j = 0; j < WPT; ++j) out[h][j] = o[j];
        if (s == 1 && GEN) {
          const int q = (h >> 1) % FG;
          Cm[q] = Cnm[q];
#pragma unroll
          for (int j = 0; j < WPT; ++j) {
            CL[q][j] = CnL[q][j];
            CE[q][j] = CnE[q][j];
          }
        } else if (s == 1) {
#pragma unroll
          for (int m = 0; m < KC; ++m)
#pragma unroll
            for (int j = 0; j < WPT; ++j) R[h >> 1][m][j] = Rn[h >> 1][m][j];
        }
      }
      // H0 = h(0,0): site (0,0) moves in the s = 0 stages; only CTA 0 meets
      // the unwrapped row 0 (bands are at least 4F + 1 rows high, so the
      // next CTA's stream starts above row 2F)
      if (tid == 0) {
        const int r = r_origin + i;
#pragma unroll
        for (int h = 0; h < NST; h += 2)
          if (r - 1 - h == 0 && fbit[h]) ctrl->H0 += (mn0[h] & 1u) ? 2 : -2;
      }
    }

    // exchange: bits 2h / 2h+1 = first / last bit of stage h's output row
    uint32_t v = 0;
    if (active) {
#pragma unroll
      for (int h = 0; h < NC; ++h)
        v |= ((out[h][0] & 1u) << (2 * h)) | ((out[h][WPT - 1] >> 31) << (2 * h + 1));
    }
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
        int issued = (i >= 2 ? i - 2 : 0) + stages;
        if (issued > nin) issued = nin;
        for (int k = i; k < issued; ++k)
          (void)tma::mbar_wait(&full[k % stages], (uint32_t)((k / stages) & 1));
      }
      return;
    }
    if (lane == 31) vr = exL[par * 32 + (warp + 1 == nwarps ? 0 : warp + 1)];
    if (lane == 0) vl = exR[par * 32 + (warp == 0 ? nwarps - 1 : warp - 1)];

    // the slot of stream row r-2 is free: refill it with row r-2+stages
    if (tid == 0 && active && i - 2 + stages < nin) {
      tma::fence_proxy_async();
      issue();
    }

    if (active) {
      const int rr = r_origin + i - NST;  // the last stage finished row r-NST
      if (rr >= yb && rr < ye) {
        int q = y - NST;
        if (q < 0) q += L;
        uint32_t *o = dst + (size_t)q * W + w0;
#pragma unroll
        for (int gq = 0; gq < NG; ++gq)
          *(uint4 *)(o + 4 * gq) = make_uint4(out[NST - 1][4 * gq], out[NST - 1][4 * gq + 1],
                                              out[NST - 1][4 * gq + 2],
                                              out[NST - 1][4 * gq + 3]);
      }
#pragma unroll
      for (int h = 0; h < NC; ++h) {
#pragma unroll
        for (int j = 0; j < WPT; ++j) {
          Wd[h][j] = Wc[h][j];
          Wc[h][j] = out[h][j];
        }
        WL[h] = (vl >> (2 * h + 1)) & 1u;  // left neighbour's last bit
        WR[h] = (vr >> (2 * h)) & 1u;      // right neighbour's first bit
      }
    }

    if (++slot == stages) {
      slot = 0;
      phase ^= 1u;
    }
    if (++sl1 == stages) sl1 = 0;
    if (++sl2 == stages) sl2 = 0;
    if (++y == L) y = 0;
    am = ~am;
    if (++q0 == L) {
      q0 = 0;
      gq0 = (uint32_t)(NG * tid);
    } else {
      gq0 += groups_per_row;
    }
  }
}

namespace {

struct PPlan {
  int threads, stages, grid;
  size_t smem;
};

PPlan pplan_for(int L, int wpt, int F, int band_rows, const void *fn) {
  PPlan p;
  p.threads = L / (32 * wpt);
  const size_t slot = (size_t)(L / 8);
  int stages = (int)((200 * 1024) / slot);
  if (stages > 12) stages = 12;
  if (stages < 4) stages = 4;
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

template <int WPT, int F, int MODE, bool SMALL = false>
cudaError_t plaunch(const uint32_t *src, uint32_t *dst, int L, uint32_t t, uint64_t seed,
                    const Accept &acc, const PModes &md, int band_rows, Ctrl *ctrl,
                    cudaStream_t st) {
  static thread_local int cached_L = 0, cached_band = -1;
  static thread_local PPlan plan;
  const void *fn = (const void *)parity_stream_kernel<WPT, F, MODE, SMALL>;
  if (cached_L != L || cached_band != band_rows) {
    plan = pplan_for(L, WPT, F, band_rows, fn);
    cached_L = L;
    cached_band = band_rows;
  }
  parity_stream_kernel<WPT, F, MODE, SMALL><<<plan.grid, plan.threads, plan.smem, st>>>(
      src, dst, L, plan.stages, t, round_keys(seed), acc, md, ctrl);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t plaunch_mode(const uint32_t *src, uint32_t *dst, int L, uint32_t t, uint64_t seed,
                         const Accept &acc, const PModes &md, int wpt, int fuse, int band_rows,
                         Ctrl *ctrl, cudaStream_t st) {
  if (wpt == 16) {  // rows of at most 256 threads (parity_wpt_valid)
    if (fuse == 2) return plaunch<16, 2, MODE, true>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
    return plaunch<16, 1, MODE, true>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
  }
  if (wpt == 8) {
    if (fuse == 2) return plaunch<8, 2, MODE>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
    return plaunch<8, 1, MODE>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
  }
  if (L / 128 <= 256) {  // rows of at most 256 threads
    if (fuse == 2) return plaunch<4, 2, MODE, true>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
    return plaunch<4, 1, MODE, true>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
  }
  if (fuse == 2) return plaunch<4, 2, MODE>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
  return plaunch<4, 1, MODE>(src, dst, L, t, seed, acc, md, band_rows, ctrl, st);
}

}  // namespace

bool parity_wpt_valid(int64_t L, int wpt) {
  if (wpt == 16)  // L/512 threads: whole warps, at most 256 (the SMALL bound)
    return stream_kernel_supports(L) && L % 16384 == 0 && L / 512 <= 256;
  return stream_wpt_valid(L, wpt);
}

cudaError_t launch_parity_stream(const uint32_t *src, uint32_t *dst, int64_t L, uint32_t t,
                                 uint64_t seed, const Accept &acc, int wpt, int fuse,
                                 int band_rows, Ctrl *ctrl, cudaStream_t st) {
  PModes md{0, 0, 0, 0};
  int mode = kPModeGen;
  if (acc.k <= 1) {
    const uint64_t full = 1ull << acc.k;
    auto sel = [&](uint64_t T) { return T == 0 ? 0 : (T >= full ? 2 : 1); };
    const int pm = sel(acc.P), qm = sel(acc.Q);
    md.p1 = pm == 1 ? ~0u : 0u;
    md.p2 = pm == 2 ? ~0u : 0u;
    md.q1 = qm == 1 ? ~0u : 0u;
    md.q2 = qm == 2 ? ~0u : 0u;
    mode = (pm == 1 && qm == 0) ? kPModeHalf : kPModeK1;
  }
  const int Li = (int)L;
  if (mode == kPModeHalf)
    return plaunch_mode<kPModeHalf>(src, dst, Li, t, seed, acc, md, wpt, fuse, band_rows, ctrl, st);
  if (mode == kPModeK1)
    return plaunch_mode<kPModeK1>(src, dst, Li, t, seed, acc, md, wpt, fuse, band_rows, ctrl, st);
  return plaunch_mode<kPModeGen>(src, dst, Li, t, seed, acc, md, wpt, fuse, band_rows, ctrl, st);
}

}  // namespace okz
