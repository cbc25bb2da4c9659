// batch.cu -- many independent lattices ("slots") in one persistent launch.
//
// Replicas are the paper's parallelism across independent runs (Kelling &
// Odor, arXiv:1110.6745, Sec. III: 10-1000 independent simulations per size).
// Every slot holds one height-parity plane (parity.cu) in a device arena. A
// launch drains a device work queue of (slot, sweeps) items: one CTA takes an
// item, stages the lattice in shared memory when it fits (else works on it in
// global memory, where a 2^11 lattice stays L2-resident), runs the sweeps in
// place -- a half-sweep updates only one sublattice and a move toggles only
// the site's own bit, so CTA barriers between the half-sweeps of bands of
// rows are the only synchronisation -- and writes the lattice, t and H0 back.
// Random draws use the slot's own seed with the single-lattice counter
// layout, so every slot evolves bit-identically to a simulation of its own.
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

// ---- band wavefront (lattices with L % 128 == 0) ----
//
// The random words of level m of 128-site group g in sweep t are Philox
// (g, 0, t, m): every level is keyed by group, sweep and level, never by the
// half-sweep, and a site is active in one half-sweep only: the levels a group
// draws for its first-half candidates decide its second-half sites just as
// well, as far as they go. So the first half-sweep of a group advances the
// comparisons U < P and U < Q of all 128 sites, and the second half-sweep
// starts from that state and draws only the levels beyond it (the first-half
// loop runs to the warp's last undecided candidate, which usually leaves
// none). Carrying the state needs the thread that did a group's first half to
// do its second half too, one barrier later, which a band wavefront gives:
// per band step of R rows, the first half of rows y0 .. y0+R-1, a barrier,
// the second half of rows y0-1 .. y0+R-2, a barrier. That is the checkerboard
// order (a first-half site reads only second-half neighbours, and those of
// rows y0-1 and y0+R have not moved yet), with two rows held back: a band's
// last row waits for the next band step (its state goes through shared
// memory), and row 0 waits for the end of the sweep, after the first half of
// row L-1, which reads it.

constexpr int kBandCols = (int)(kBatchMaxL / 128);  // 128-site groups per row, at most
constexpr int kCarryWords = 9;                      // LT[4], EQ[4], next level

// [0], [1]: a band's last row, by band parity; [2]: row 0.
struct BandCarry {
  uint32_t w[3][kCarryWords][kBandCols];
};

__device__ __forceinline__ void carry_put(BandCarry &bc, int b, uint32_t col, const uint32_t LT[4],
                                          const uint32_t EQ[4], int m) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    bc.w[b][j][col] = LT[j];
    bc.w[b][4 + j][col] = EQ[j];
  }
  bc.w[b][8][col] = (uint32_t)m;
}

__device__ __forceinline__ void carry_get(const BandCarry &bc, int b, uint32_t col, uint32_t LT[4],
                                          uint32_t EQ[4], int &m) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    LT[j] = bc.w[b][j][col];
    EQ[j] = bc.w[b][4 + j][col];
  }
  m = (int)bc.w[b][8][col];
}

// philox(g, 0, t, m) for the successive levels m of one group in one sweep:
// the first two rounds depend on m only through c2 = hi(A g) ^ k1 ^ m, so the
// rest of them is formed once per group (same rounds and keys as
// philox10_sm).
struct LevelPhilox {
  uint32_t X, Z, V1, V3;
};

__device__ __forceinline__ LevelPhilox level_philox_init(uint32_t g, uint32_t t,
                                                         const uint32_t *rks) {
  const uint64_t pa = (uint64_t)kPhiloxMulA * g, pb = (uint64_t)kPhiloxMulB * t;
  const uint32_t U0 = (uint32_t)(pb >> 32) ^ rks[0];  // round 0: c0, c1 from t only
  const uint64_t pa1 = (uint64_t)kPhiloxMulA * U0;    // round 1: c2, c3 from g, t only
  LevelPhilox lp;
  lp.X = (uint32_t)(pa >> 32) ^ rks[1];
  lp.Z = (uint32_t)(pa1 >> 32) ^ (uint32_t)pa ^ rks[3];
  lp.V1 = (uint32_t)pb ^ rks[2];
  lp.V3 = (uint32_t)pa1;
  return lp;
}

__device__ __forceinline__ u32x4 level_philox(const LevelPhilox &lp, uint32_t m,
                                              const uint32_t *__restrict__ rks) {
  const uint64_t p1 = (uint64_t)kPhiloxMulB * (lp.X ^ m);
  uint32_t c0 = (uint32_t)(p1 >> 32) ^ lp.V1, c1 = (uint32_t)p1, c2 = lp.Z, c3 = lp.V3;
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    uint32_t kx, ky;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                 : "=r"(kx), "=r"(ky)
                 : "r"((uint32_t)__cvta_generic_to_shared(rks + 2 * r)));
    const uint64_t pa = (uint64_t)kPhiloxMulA * c0;
    const uint64_t pb = (uint64_t)kPhiloxMulB * c2;
    const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ kx;
    const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ ky;
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

// Thresholds as 32-bit words with level 0 at bit 31 (P < 2^k; a P of 0 or
// 2^k never reaches a level: its comparisons start decided).
struct LevelBits {
  uint32_t pw, qw;
};

__device__ __forceinline__ LevelBits level_bits(const Accept &acc) {
  LevelBits b;
  b.pw = (uint32_t)(acc.P << (32 - acc.k));
  b.qw = (uint32_t)(acc.Q << (32 - acc.k));
  return b;
}

// Level m of the group's random words rb applied to the comparisons of all
// 128 sites with both thresholds.
__device__ __forceinline__ void cmp_level(const u32x4 &rb, const LevelBits &tb, int m,
                                          uint32_t lp[4], uint32_t ep[4], uint32_t lq[4],
                                          uint32_t eq[4]) {
  const uint32_t pb = (tb.pw >> (31 - m)) & 1u, qb = (tb.qw >> (31 - m)) & 1u;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    lt_step(rb.v[j], pb, lp[j], ep[j]);
    lt_step(rb.v[j], qb, lq[j], eq[j]);
  }
}

__device__ __forceinline__ uint32_t rotl1(uint32_t x) { return __funnelshift_l(x, x, 1); }
__device__ __forceinline__ uint32_t rotr1(uint32_t x) { return __funnelshift_r(x, x, 1); }

__device__ __forceinline__ uint32_t open_candidates(const uint32_t ep[4], const uint32_t eq[4],
                                                   const uint32_t mn[4], const uint32_t mx[4]) {
  return ((ep[0] & mn[0]) | (eq[0] & mx[0])) | ((ep[1] & mn[1]) | (eq[1] & mx[1])) |
         ((ep[2] & mn[2]) | (eq[2] & mx[2])) | ((ep[3] & mn[3]) | (eq[3] & mx[3]));
}

// Minima and maxima of half-sweep SP among the group's 4 words c (row y,
// words w0 .. w0+3), from the rows below and above and the words either side.
template <int SP>
__device__ __forceinline__ void group_extrema(const uint32_t *B, int L, int W, uint32_t y,
                                              uint32_t w0, const uint32_t c[4], uint32_t mn[4],
                                              uint32_t mx[4]) {
  const uint32_t yd = (y == 0) ? L - 1 : y - 1, yu = (y == (uint32_t)L - 1) ? 0 : y + 1;
  const uint32_t *row = B + (size_t)y * W;
  const uint4 dv = *(const uint4 *)(B + (size_t)yd * W + w0);
  const uint4 uv = *(const uint4 *)(B + (size_t)yu * W + w0);
  const uint32_t lw = row[w0 == 0 ? W - 1 : w0 - 1];
  const uint32_t rw = row[w0 + 4 == (uint32_t)W ? 0 : w0 + 4];
  const uint32_t d[4] = {dv.x, dv.y, dv.z, dv.w};
  const uint32_t u[4] = {uv.x, uv.y, uv.z, uv.w};
  const uint32_t a = active_mask(y, SP);
  // a minimum of half-sweep SP has all four neighbours equal to its own bit
  // xor SP: "both equal" (table 0x81) for SP = 0, "both differ" (0x42) for
  // SP = 1, on (l, r, c) and (d, u, c); a maximum the reverse
  constexpr uint32_t kMin = SP ? 0x42u : 0x81u;
  constexpr uint32_t kMax = SP ? 0x81u : 0x42u;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t l = __funnelshift_l(j == 0 ? lw : c[j - 1], c[j], 1);
    const uint32_t r = __funnelshift_r(c[j], j == 3 ? rw : c[j + 1], 1);
    mn[j] = lop3<0x80>(lop3<kMin>(l, r, c[j]), lop3<kMin>(d[j], u[j], c[j]), a);
    mx[j] = lop3<0x80>(lop3<kMax>(l, r, c[j]), lop3<kMax>(d[j], u[j], c[j]), a);
  }
}

__device__ __forceinline__ void load_group(const uint32_t *B, int W, uint32_t y, uint32_t w0,
                                           uint32_t c[4]) {
  const uint4 v = *(const uint4 *)(B + (size_t)y * W + w0);
  c[0] = v.x;
  c[1] = v.y;
  c[2] = v.z;
  c[3] = v.w;
}

// First half-sweep of group g at (y, w0). Levels are drawn while any lane of
// `lanes` has an undecided candidate (the warp runs to its last one anyway),
// LV levels per test (a level drawn beyond the last undecided candidate
// changes nothing decided). Out: the group's words after the moves in c; the
// second-half state packed in LT, EQ -- word j holds the P comparison at the
// second-half positions and the Q comparison rotated left by one bit into the
// first-half positions -- and the next level in m.
template <int LV>
__device__ __forceinline__ void band_first_half(uint32_t *B, int L, int W, uint32_t y,
                                                uint32_t w0, uint32_t g, uint32_t t,
                                                const uint32_t *rks, const Accept &acc,
                                                unsigned lanes, int &dH0, uint32_t c[4],
                                                uint32_t LT[4], uint32_t EQ[4], int &m) {
  load_group(B, W, y, w0, c);
  uint32_t mn[4], mx[4];
  group_extrema<0>(B, L, W, y, w0, c, mn, mx);
  const uint64_t full = 1ull << acc.k;
  const uint32_t lp0 = (acc.P >= full) ? ~0u : 0u, ep0 = (acc.P >= full || acc.P == 0) ? 0u : ~0u;
  const uint32_t lq0 = (acc.Q >= full) ? ~0u : 0u, eq0 = (acc.Q >= full || acc.Q == 0) ? 0u : ~0u;
  uint32_t lp[4], ep[4], lq[4], eq[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    lp[j] = lp0;
    ep[j] = ep0;
    lq[j] = lq0;
    eq[j] = eq0;
  }
  const LevelPhilox ph = level_philox_init(g, t, rks);
  const LevelBits tb = level_bits(acc);
  m = 0;
  while (m < acc.k) {
    if (!__any_sync(lanes, open_candidates(ep, eq, mn, mx) != 0u)) break;
    cmp_level(level_philox(ph, (uint32_t)m, rks), tb, m, lp, ep, lq, eq);
    if (++m < acc.k && LV == 2) {
      cmp_level(level_philox(ph, (uint32_t)m, rks), tb, m, lp, ep, lq, eq);
      ++m;
    }
  }
  uint32_t f[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) f[j] = (lp[j] & mn[j]) | (lq[j] & mx[j]);
  if ((f[0] | f[1] | f[2] | f[3]) != 0u)
    *(uint4 *)(B + (size_t)y * W + w0) =
        make_uint4(c[0] ^ f[0], c[1] ^ f[1], c[2] ^ f[2], c[3] ^ f[3]);
  if (g == 0 && (f[0] & 1u)) dH0 += (mn[0] & 1u) ? 2 : -2;  // site (0,0)
  const uint32_t a0 = active_mask(y, 0);  // first-half positions
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    c[j] ^= f[j];
    LT[j] = (lp[j] & ~a0) | (rotl1(lq[j]) & a0);
    EQ[j] = (ep[j] & ~a0) | (rotl1(eq[j]) & a0);
  }
}

// Second half-sweep of group g at (y, w0), its words c as the first half left
// them, from the packed state (LT, EQ, m) that half left.
__device__ __forceinline__ void band_second_half(uint32_t *B, int L, int W, uint32_t y,
                                                 uint32_t w0, uint32_t g, uint32_t t,
                                                 const uint32_t *rks, const Accept &acc,
                                                 int &dH0, const uint32_t c[4],
                                                 const uint32_t LT[4], const uint32_t EQ[4],
                                                 int m) {
  uint32_t mn[4], mx[4];
  group_extrema<1>(B, L, W, y, w0, c, mn, mx);
  uint32_t lp[4], ep[4], lq[4], eq[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {  // only the second-half positions are read below
    lp[j] = LT[j];
    ep[j] = EQ[j];
    lq[j] = rotr1(LT[j]);
    eq[j] = rotr1(EQ[j]);
  }
  if (m < acc.k && open_candidates(ep, eq, mn, mx) != 0u) {  // rare
    const LevelPhilox ph = level_philox_init(g, t, rks);
    const LevelBits tb = level_bits(acc);
    for (; m < acc.k && open_candidates(ep, eq, mn, mx) != 0u; ++m)
      cmp_level(level_philox(ph, (uint32_t)m, rks), tb, m, lp, ep, lq, eq);
  }
  uint32_t f[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) f[j] = (lp[j] & mn[j]) | (lq[j] & mx[j]);
  if ((f[0] | f[1] | f[2] | f[3]) != 0u)
    *(uint4 *)(B + (size_t)y * W + w0) =
        make_uint4(c[0] ^ f[0], c[1] ^ f[1], c[2] ^ f[2], c[3] ^ f[3]);
  if (g == 0 && (f[0] & 1u)) dH0 += (mn[0] & 1u) ? 2 : -2;  // site (0,0)
}

// `n` sweeps of one lattice (L % 128 == 0) by the whole CTA in band steps of
// R = blockDim.x / (L/128) rows (all rows for small L), thread (ry, col)
// taking group col of row y0 + ry. Thread 0 takes group 0 of row 0 in both
// halves, so it alone sees site (0,0).
template <int LV>
__device__ __forceinline__ void cta_sweeps_band(uint32_t *B, int L, uint32_t t0, int n,
                                                const uint32_t *rks, const Accept &acc, int &dH0,
                                                BandCarry &bc) {
  const int W = L >> 5;
  const uint32_t G = (uint32_t)W >> 2;
  const uint32_t tid = threadIdx.x;
  const uint32_t R = min(blockDim.x / G, (uint32_t)L);
  const uint32_t nb = ((uint32_t)L + R - 1) / R;
  const uint32_t ry = tid / G, col = tid - ry * G, w0 = 4 * col;
  for (int i = 0; i < n; ++i) {
    const uint32_t t = t0 + (uint32_t)i;
    for (uint32_t j = 0; j < nb; ++j) {
      const uint32_t y0 = j * R, rc = min(R, (uint32_t)L - y0), y = y0 + ry;
      const bool mine = ry < rc;
      const unsigned lanes = __ballot_sync(0xFFFFFFFFu, mine);
      uint32_t c[4], LT[4], EQ[4];
      int m = 0;
      if (mine) {
        band_first_half<LV>(B, L, W, y, w0, y * G + col, t, rks, acc, lanes, dH0, c, LT, EQ,
                            m);
        if (ry + 1 == rc) carry_put(bc, (int)(j & 1), col, LT, EQ, m);
        if (y == 0) carry_put(bc, 2, col, LT, EQ, m);
      }
      __syncthreads();
      if (mine && ry + 1 < rc && y != 0) {
        band_second_half(B, L, W, y, w0, y * G + col, t, rks, acc, dH0, c, LT, EQ, m);
      } else if (mine && ry + 1 == rc && j > 0 && y0 - 1 != 0) {
        const uint32_t yp = y0 - 1;  // the previous band's last row
        carry_get(bc, (int)((j - 1) & 1), col, LT, EQ, m);
        load_group(B, W, yp, w0, c);
        band_second_half(B, L, W, yp, w0, yp * G + col, t, rks, acc, dH0, c, LT, EQ, m);
      }
      __syncthreads();
    }
    if (tid < 2 * G) {  // row 0 (threads 0 .. G-1) and row L-1, held back to here
      const bool r0 = tid < G;
      const uint32_t cl = r0 ? tid : tid - G, yy = r0 ? 0u : (uint32_t)L - 1;
      uint32_t c[4], LT[4], EQ[4];
      int m = 0;
      carry_get(bc, r0 ? 2 : (int)((nb - 1) & 1), cl, LT, EQ, m);
      load_group(B, W, yy, 4 * cl, c);
      band_second_half(B, L, W, yy, 4 * cl, yy * G + cl, t, rks, acc, dH0, c, LT, EQ, m);
    }
    __syncthreads();
  }
}

// `n` sweeps of one lattice by the whole CTA.
template <int LV>
__device__ __forceinline__ void cta_sweeps(uint32_t *B, int L, uint32_t t0, int n,
                                           const uint32_t *rks, const Accept &acc, int &dH0,
                                           BandCarry &bc) {
  if ((L & 127) == 0) {  // groups never straddle rows
    cta_sweeps_band<LV>(B, L, t0, n, rks, acc, dH0, bc);
    return;
  }
  const int W = L >> 5;
  const uint32_t groups = (uint32_t)L * (uint32_t)W / 4;
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

template <int MAXT, int MINB>
constexpr int kLevelsPerTest = (65536 / (MAXT * MINB) >= 128) ? 2 : 1;

// CTAs of MAXT threads, MINB of them per SM: 1024 x 1 and 512 x 2 leave 64
// registers a thread (one random level per candidate test), 256 x 2 leave
// 128 (two). Several CTAs per SM fill one another's barrier waits.
template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
batch_sweep_kernel(uint32_t *__restrict__ arena, SlotDesc *__restrict__ slots,
                   const WorkTable *__restrict__ work, unsigned int *__restrict__ head,
                   uint32_t smem_words) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int item;
  __shared__ __align__(8) uint32_t rks[20];  // round keys of the current slot's seed
  __shared__ BandCarry carry;
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
      cta_sweeps<kLevelsPerTest<MAXT, MINB>>(sm, d.L, d.t, n, rks, acc, dH0, carry);
      for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) g[w] = sm[w];
    } else {
      __syncthreads();
      cta_sweeps<kLevelsPerTest<MAXT, MINB>>(g, d.L, d.t, n, rks, acc, dH0, carry);
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
  const uint32_t words = (uint32_t)(smem_bytes / 4);
  if (threads > 512)
    batch_sweep_kernel<1024, 1><<<grid, threads, smem_bytes, st>>>(arena, slots, work, head, words);
  else if (threads > 256)
    batch_sweep_kernel<512, 2><<<grid, threads, smem_bytes, st>>>(arena, slots, work, head, words);
  else
    batch_sweep_kernel<256, 2><<<grid, threads, smem_bytes, st>>>(arena, slots, work, head, words);
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

// One lattice swept in place by one CTA out of shared memory: the band
// wavefront of the batch kernel (bit-identical to every other sweep kernel),
// all n sweeps in one launch. For lattices too small to spread over the GPU,
// where a launch per half-sweep costs more than the sweep itself.
__global__ void __launch_bounds__(1024, 1)
cta_lattice_kernel(uint32_t *__restrict__ B, int L, uint32_t t0, int n, uint64_t seed, Accept acc,
                   Ctrl *__restrict__ ctrl) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ __align__(8) uint32_t rks[20];
  __shared__ BandCarry carry;
  const uint32_t words = (uint32_t)L * (uint32_t)(L >> 5);
  if (threadIdx.x < 10) {
    const uint32_t r = threadIdx.x;
    rks[2 * r] = (uint32_t)seed + r * kPhiloxWeylA;
    rks[2 * r + 1] = (uint32_t)(seed >> 32) + r * kPhiloxWeylB;
  }
  for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) sm[w] = B[w];
  __syncthreads();
  int dH0 = 0;
  cta_sweeps<1>(sm, L, t0, n, rks, acc, dH0, carry);
  for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) B[w] = sm[w];
  if (threadIdx.x == 0) ctrl->H0 += dH0;  // thread 0 owns site (0,0)
}

bool cta_kernel_supports(int64_t L) { return L >= 32 && L % 32 == 0 && L <= kCtaMaxL; }

cudaError_t launch_cta_sweeps(uint32_t *B, int64_t L, uint32_t t, int64_t n, uint64_t seed,
                              const Accept &acc, Ctrl *ctrl, cudaStream_t st) {
  const size_t smem = (size_t)L * (size_t)L / 8;
  // threads: one per 128-site group, whole warps, at least 2 groups' rows
  int threads = (int)((L * (L / 32) / 4 + 31) / 32 * 32);
  if (threads > 1024) threads = 1024;
  if (threads < 64) threads = 64;
  cudaError_t e = cudaFuncSetAttribute((const void *)cta_lattice_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((size_t)kCtaMaxL * kCtaMaxL / 8));
  if (e != cudaSuccess) return e;
  for (int64_t done = 0; done < n;) {  // launches of at most 2^20 sweeps
    const int64_t m = (n - done < (1 << 20)) ? n - done : (1 << 20);
    cta_lattice_kernel<<<1, threads, smem, st>>>(B, (int)L, t + (uint32_t)done, (int)m, seed, acc,
                                                 ctrl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    done += m;
  }
  return cudaSuccess;
}

int batch_occupancy(int threads, size_t smem_bytes) {
  int per_sm = 0;
  const void *fn = threads > 512   ? (const void *)batch_sweep_kernel<1024, 1>
                   : threads > 256 ? (const void *)batch_sweep_kernel<512, 2>
                                   : (const void *)batch_sweep_kernel<256, 2>;
  // one limit for every batch: the largest staging buffer a tiling may ask for
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem_bytes) !=
      cudaSuccess)
    return 0;
  return per_sm;
}

}  // namespace okz
