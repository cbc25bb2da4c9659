// ddrs.cu -- the paper's own GPU dynamics on the height-parity plane
// (Kelling & Odor, arXiv:1110.6745, Sec. II and Fig. 1): random-sequential
// update attempts inside dead-border domains whose origin moves every MCS.
#include <cuda_runtime.h>

#include "okz_internal.h"

namespace okz {

// ---------------------------------------------------------------------------
// Domain-decomposed random-sequential sweeps (the paper's own GPU dynamics,
// Sec. II: blocks with dead borders, the origin moved at random every MCS,
// random update attempts inside each block). Sweep t: offsets (ox, oy) =
// (r0, r1) mod 32 of Philox(ctr = (0, 0, t, 768)); 32 x 32 cells with origins
// (ox + 32i, oy + 32j) mod L and ids c = j*(L/32) + i; cell c receives 1024
// attempts, attempt a drawing words (r0, r1) (a even) or (r2, r3) (a odd) of
// Philox(ctr = (c, a/2, t, 1024)): local x = first & 31, local y =
// (first >> 16) & 31, u = second; attempts on the dead first column or first
// row do nothing, otherwise a minimum moves iff u < P32 and a maximum iff
// u < Q32. As in Fig. 1 of the paper two dead edges suffice: a cell's last
// column and row read only the next cells' dead first column and row, which
// do not change during the sweep. One thread per cell: the cell (33 rows of
// 33 bits: its own sites plus those frozen neighbours) is staged in shared
// memory, swept, and its changed bits are xor-ed back (neighbouring cells
// share the words at their x edges).
// ---------------------------------------------------------------------------
constexpr int kCell = 32;
constexpr int kCellStride = kCell + 3;  // rows 0..32, then the column x0+32; odd stride

__global__ void __launch_bounds__(128)
ddrs_kernel(uint32_t *__restrict__ B, int L, uint32_t t, const RoundKeys rk, uint32_t Pm1,
            uint32_t Qm1, uint32_t pq_on, Ctrl *__restrict__ ctrl) {
  __shared__ uint32_t cell_sm[128][kCellStride];
  uint32_t *cell = cell_sm[threadIdx.x];
  const int ncell = L / kCell;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (uint32_t)ncell * (uint32_t)ncell) return;
  const u32x4 o = philox10_rk(0u, 0u, t, 768u, rk);
  const int ox = (int)(o.v[0] & (kCell - 1)), oy = (int)(o.v[1] & (kCell - 1));
  const int ci = (int)(c % (uint32_t)ncell), cj = (int)(c / (uint32_t)ncell);
  const int x0 = (ox + ci * kCell) % L, y0 = (oy + cj * kCell) % L;
  const int W = L >> 5;
  const int wA = x0 >> 5, sh = x0 & 31, wB = (wA + 1 == W) ? 0 : wA + 1;
  uint32_t next_col = 0;  // bit ly = b(x0 + 32, y0 + ly)
  for (int ly = 0; ly <= kCell; ++ly) {
    const int y = (y0 + ly) % L;
    const uint32_t a = B[(size_t)y * W + wA], b = B[(size_t)y * W + wB];
    cell[ly] = __funnelshift_r(a, b, sh);
    if (ly < kCell) next_col |= ((b >> sh) & 1u) << ly;
  }
  // loop invariants: the sites of parity (x0 + lx + y0 + ly) mod 2 = 1 (L is
  // even) are pm0 in rows of even ly and its complement in odd rows, and the
  // local coordinates of site (0,0) if this cell holds it (else 64)
  const uint32_t pm0 = ((uint32_t)(x0 + y0) & 1u) ? 0x55555555u : 0xAAAAAAAAu;
  const int lx00 = (L - x0) % L < kCell ? (L - x0) % L : 64;
  const int ly00 = (L - y0) % L < kCell ? (L - y0) % L : 64;
  const bool p_on = pq_on & 1u, q_on = pq_on & 2u;
  uint32_t touched = 0;
  int dH0 = 0;
  uint32_t r2 = 0, r3 = 0;
  for (uint32_t a = 0; a < kCell * kCell; ++a) {
    uint32_t first, u;
    if ((a & 1u) == 0) {
      const u32x4 r = philox10_rk(c, a >> 1, t, 1024u, rk);
      first = r.v[0];
      u = r.v[1];
      r2 = r.v[2];
      r3 = r.v[3];
    } else {
      first = r2;
      u = r3;
    }
    const int lx = (int)(first & (kCell - 1)), ly = (int)((first >> 16) & (kCell - 1));
    if (lx == 0 || ly == 0) continue;  // dead border
    const uint32_t row = cell[ly];
    // the whole row at once: bit lx of l / r is the left / right neighbour
    // (bit 31 of r: the next cell's column), then three-input truth tables
    // for "all four neighbours equal the own bit" (E) and "all four differ"
    // (N); a site of parity 0 is a minimum iff E and a maximum iff N,
    // parity 1 the reverse
    const uint32_t l = row << 1, r = __funnelshift_r(row, next_col >> ly, 1);
    const uint32_t dn = cell[ly - 1], up = cell[ly + 1];
    const uint32_t E = lop3<0x81>(l, r, row) & lop3<0x81>(dn, up, row);
    const uint32_t N = lop3<0x42>(l, r, row) & lop3<0x42>(dn, up, row);
    const uint32_t pm = (ly & 1) ? ~pm0 : pm0, m = 1u << lx;
    const bool is_min = (lop3<0xCA>(pm, N, E) & m) != 0u;  // pm ? N : E
    const bool is_max = (lop3<0xCA>(pm, E, N) & m) != 0u;
    const bool accept = (is_min && p_on && u <= Pm1) || (is_max && q_on && u <= Qm1);
    if (!accept) continue;
    cell[ly] = row ^ (1u << lx);
    touched |= 1u << ly;
    if (lx == lx00 && ly == ly00) dH0 += is_min ? 2 : -2;
  }
  while (touched) {
    const int ly = __ffs(touched) - 1;
    touched &= touched - 1;
    const int y = (y0 + ly) % L;
    uint32_t *pa = B + (size_t)y * W + wA, *pb = B + (size_t)y * W + wB;
    const uint32_t old = __funnelshift_r(*pa, *pb, sh);  // this cell's bits are its own
    const uint32_t delta = old ^ cell[ly];
    atomicXor(pa, delta << sh);
    if (sh) atomicXor(pb, delta >> (32 - sh));
  }
  if (dH0) atomicAdd((unsigned long long *)&ctrl->H0, (unsigned long long)(long long)dH0);
}

cudaError_t launch_ddrs(uint32_t *B, int64_t L, uint32_t t, uint64_t seed, uint64_t P32,
                        uint64_t Q32, Ctrl *ctrl, cudaStream_t st) {
  // u < P32 with P32 in [0, 2^32] as u <= P32 - 1 in 32 bits, P32 = 0 never
  const uint32_t Pm1 = P32 ? (uint32_t)(P32 - 1) : 0u, Qm1 = Q32 ? (uint32_t)(Q32 - 1) : 0u;
  const uint32_t pq_on = (P32 ? 1u : 0u) | (Q32 ? 2u : 0u);
  const int64_t cells = (L / kCell) * (L / kCell);
  ddrs_kernel<<<(unsigned)((cells + 127) / 128), 128, 0, st>>>(B, (int)L, t, round_keys(seed),
                                                              Pm1, Qm1, pq_on, ctrl);
  return cudaGetLastError();
}

}  // namespace okz
