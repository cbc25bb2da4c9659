// okz_device.cuh -- device building blocks of the octahedron-model kernels.
//
// Bit-plane conventions (Kelling & Odor, arXiv:1110.6745, Sec. II: two bits
// per site): bit b of 32-bit word w of row y is the bond at x = 32w + b.
// Plane X holds sigma_x(x,y) = h(x+1,y) - h(x,y), plane Y holds
// sigma_y(x,y) = h(x,y+1) - h(x,y); a set bit is +1.
#pragma once

#include <cstdint>

namespace okz {

// ---------------------------------------------------------------------------
// Philox4x32-10 (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64-bit
// products (counter words 0 and 2 by the two multipliers), output
// (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), with the key advanced by the two
// Weyl increments between rounds.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u;
constexpr uint32_t kPhiloxWeylB = 0xBB67AE85u;

struct u32x4 {
  uint32_t v[4];
};

__device__ __forceinline__ u32x4 philox10(uint32_t c0, uint32_t c1, uint32_t c2,
                                          uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t pa = (uint64_t)kPhiloxMulA * c0;
    const uint64_t pb = (uint64_t)kPhiloxMulB * c2;
    const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)pb;
    c3 = (uint32_t)pa;
    c0 = n0;
    c2 = n2;
    k0 += kPhiloxWeylA;
    k1 += kPhiloxWeylB;
  }
  u32x4 out;
  out.v[0] = c0;
  out.v[1] = c1;
  out.v[2] = c2;
  out.v[3] = c3;
  return out;
}

// The 4 x 32 random bits of 128-site group g at sweep t, level m: one Philox
// block with counter (g lo, g hi, t, m) and key (seed lo, seed hi). Word j
// serves sites 128g + 32j .. 128g + 32j + 31 (bit b = site 128g + 32j + b).
__device__ __forceinline__ u32x4 group_bits(uint64_t g, uint32_t t, uint32_t m,
                                            uint64_t seed) {
  return philox10((uint32_t)g, (uint32_t)(g >> 32), t, m, (uint32_t)seed,
                  (uint32_t)(seed >> 32));
}

// Philox4x32-10 round keys of one seed: k[2r] = seed_lo + r*W_A,
// k[2r+1] = seed_hi + r*W_B (r = 0..9). Passed to kernels by value, so the
// rounds read them as constant-bank operands instead of recomputing them.
struct RoundKeys {
  uint32_t k[20];
};

inline RoundKeys round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k[2 * r] = k0;
    rk.k[2 * r + 1] = k1;
    k0 += kPhiloxWeylA;
    k1 += kPhiloxWeylB;
  }
  return rk;
}

// Philox4x32-10 of counter (c0, c1, c2, c3) with precomputed round keys.
__device__ __forceinline__ u32x4 philox10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                             const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t pa = (uint64_t)kPhiloxMulA * c0;
    const uint64_t pb = (uint64_t)kPhiloxMulB * c2;
    const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ rk.k[2 * r];
    const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ rk.k[2 * r + 1];
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

// Three-input bitwise function with an explicit truth table (lop3.b32):
// bit i of the result is bit ((a_i << 2) | (b_i << 1) | c_i) of LUT.
template <uint32_t LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}

// Acceptance thresholds of a simulation: accept a minimum iff U < P and a
// maximum iff U < Q, U a k-bit uniform read most significant level first.
struct Accept {
  uint64_t P, Q;
  int k;
};

// Sites of row y that are active in half-sweep s: (x + y) mod 2 == s. Words
// hold 32 sites starting at an even x, so the pattern depends on y and s only.
__device__ __forceinline__ uint32_t active_mask(int64_t y, int s) {
  return ((y + s) & 1) ? 0xAAAAAAAAu : 0x55555555u;
}

// Eq. (2): a site is a local minimum when sigma_x(x-1) = -1, sigma_x(x) = +1,
// sigma_y(y-1) = -1, sigma_y(y) = +1, and a local maximum for the reverse.
// xl holds sigma_x(x-1,y) at bit x, xc sigma_x(x,y), yd sigma_y(x,y-1),
// yc sigma_y(x,y).
__device__ __forceinline__ uint32_t minima(uint32_t xl, uint32_t xc, uint32_t yd,
                                           uint32_t yc) {
  return ~xl & xc & ~yd & yc;
}
__device__ __forceinline__ uint32_t maxima(uint32_t xl, uint32_t xc, uint32_t yd,
                                           uint32_t yc) {
  return xl & ~xc & yd & ~yc;
}

// Bit-sliced comparison U < T for up to 32 sites at once, one level of random
// bits at a time. lt collects sites already decided "less", eq those still
// equal on every level so far. Levels are fed most significant first; a site
// with T = 2^k is accepted before any level (handled by the caller).
__device__ __forceinline__ void lt_step(uint32_t r, uint32_t tbit, uint32_t &lt,
                                        uint32_t &eq) {
  if (tbit) {
    lt |= eq & ~r;
    eq &= r;
  } else {
    eq &= ~r;
  }
}

// Bounded spin budget of every device-side wait (nanoseconds of %globaltimer).
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Device-side error bits reported through the control block.
constexpr uint32_t kErrWaitTimeout = 1u;
constexpr uint32_t kErrHeightRange = 2u;

// Control block in device memory (256 bytes, one per simulation).
struct Ctrl {
  long long H0;           // h(0,0)
  unsigned int err;       // kErr* bits
  unsigned int t_base;     // sweep counter read by graph-replayed half-sweeps
  unsigned long long sum[8];  // exact sums as (lo, hi) pairs: S1, S2, S3, S4
  unsigned long long pad1[22];
};
static_assert(sizeof(Ctrl) == 256, "control block is 256 bytes");

}  // namespace okz
