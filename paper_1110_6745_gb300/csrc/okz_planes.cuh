// okz_planes.cuh -- slope words of the two state encodings.
//
// Slope planes (Sec. II): X plane then Y plane, L rows of L/32 words each,
// bit b of word w of row y = [sigma(32w + b, y) = +1]. Height-parity plane:
// one bit b(x,y) = floor(h/2) mod 2 per site, with
//   sigma_x(x,y) = +1 <=> b(x+1,y) ^ b(x,y) ^ p(x,y) == 0,
//   sigma_y(x,y) = +1 <=> b(x,y+1) ^ b(x,y) ^ p(x,y) == 0,
// p(x,y) = (x+y) mod 2. The helpers return a word of X or Y bits from either.
#pragma once

#include <cstdint>

namespace okz {

// Sites of word w in row y with x + y odd (32w is even, so only y matters).
__device__ __forceinline__ uint32_t odd_sites(int64_t y) {
  return (y & 1) ? 0x55555555u : 0xAAAAAAAAu;
}

// sigma_y(0, y) as a bit.
template <bool PAR>
__device__ __forceinline__ uint32_t col0_up(const uint32_t *__restrict__ P, int64_t L,
                                            int64_t W, int64_t y) {
  if (!PAR) return P[L * W + y * W] & 1u;
  const int64_t yu = (y == L - 1) ? 0 : y + 1;
  return ~(P[y * W] ^ P[yu * W] ^ (uint32_t)(y & 1)) & 1u;
}

// X-plane word w of row y: stored, or (parity plane) ~(b ^ b(x+1) ^ p).
template <bool PAR>
__device__ __forceinline__ uint32_t x_word(const uint32_t *__restrict__ row, int64_t W,
                                           int64_t w, int64_t y) {
  if (!PAR) return row[w];
  const uint32_t c = row[w], n = row[w == W - 1 ? 0 : w + 1];
  return ~(c ^ __funnelshift_r(c, n, 1) ^ odd_sites(y));
}

}  // namespace okz
