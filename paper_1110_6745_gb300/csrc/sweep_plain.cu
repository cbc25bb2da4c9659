// sweep_plain.cu -- striped start and the in-place half-sweep kernel.
//
// One launch updates one sublattice (half-sweep s of sweep t) of the
// octahedron model (Kelling & Odor, arXiv:1110.6745, Sec. I, Eq. (2)). Each
// thread owns one 128-site group (four 32-bit words of the flattened
// row-major lattice), draws the group's Philox block level by level, and
// applies its flips with atomicXor. In-place updates are race-free at the bit
// level: every bond touches exactly one site of the active sublattice, so a
// bond is read and written only by the thread owning that site; other threads
// may xor other bits of the same word, which atomicXor keeps intact.
#include "okz_internal.h"

namespace okz {

// Striped start (Sec. III): h(x,y) = (x+y) mod 2, so sigma_x(x,y) and
// sigma_y(x,y) are +1 exactly where x + y is even.
__global__ void init_flat_kernel(uint32_t *__restrict__ planes, int64_t L) {
  const int64_t W = L >> 5;
  const int64_t words = L * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / W;
    const uint32_t v = (y & 1) ? 0xAAAAAAAAu : 0x55555555u;
    planes[i] = v;          // X plane
    planes[words + i] = v;  // Y plane
  }
}

cudaError_t launch_init_flat(uint32_t *planes, int64_t L, cudaStream_t st) {
  const int64_t words = L * (L >> 5);
  int64_t blocks = (words + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  init_flat_kernel<<<(unsigned)blocks, 256, 0, st>>>(planes, L);
  return cudaGetLastError();
}

// Half-sweep s of sweep t (plus *t_base when t_base is set: the launches of a
// CUDA graph replayed for consecutive chunks of sweeps read the chunk's first
// sweep from device memory). acc.k levels of random bits at most; the level
// loop stops as soon as no extremum of the group is still undecided.
__global__ void __launch_bounds__(256)
halfsweep_plain_kernel(uint32_t *__restrict__ planes, int64_t L, int s, uint32_t t_off,
                       const unsigned int *__restrict__ t_base, uint64_t seed, Accept acc,
                       Ctrl *__restrict__ ctrl) {
  const uint32_t t = t_off + (t_base ? *t_base : 0u);
  const int64_t W = L >> 5;
  const int64_t words = L * W;
  const int64_t groups = words >> 2;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= groups) return;
  uint32_t *X = planes;
  uint32_t *Y = planes + words;

  uint32_t mn[4], mx[4];
  int64_t idx[4], idx_left[4], idx_down[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t gw = 4 * g + j;  // flattened word index
    const int64_t y = gw / W, w = gw - y * W;
    const int64_t wl = (w == 0) ? W - 1 : w - 1;
    const int64_t yd = (y == 0) ? L - 1 : y - 1;
    idx[j] = gw;
    idx_left[j] = y * W + wl;
    idx_down[j] = yd * W + w;
    const uint32_t xc = X[gw];
    const uint32_t xl = (xc << 1) | (X[idx_left[j]] >> 31);  // sigma_x(x-1)
    const uint32_t yc = Y[gw];
    const uint32_t ydn = Y[idx_down[j]];
    const uint32_t a = active_mask(y, s);
    mn[j] = minima(xl, xc, ydn, yc) & a;
    mx[j] = maxima(xl, xc, ydn, yc) & a;
  }

  // Acceptance: U < P for minima, U < Q for maxima (bit-sliced, lazy).
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
    const u32x4 r = group_bits((uint64_t)g, t, (uint32_t)m, seed);
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
    const uint32_t f = ltp[j] | ltq[j];  // flipped sites (subsets of mn, mx)
    if (f == 0u) continue;
    // a flip at x toggles sigma_x(x-1), sigma_x(x), sigma_y(x,y-1), sigma_y(x,y)
    atomicXor(&X[idx[j]], f ^ (f >> 1));
    if (f & 1u) atomicXor(&X[idx_left[j]], 0x80000000u);
    atomicXor(&Y[idx[j]], f);
    atomicXor(&Y[idx_down[j]], f);
    if (idx[j] == 0 && (f & 1u)) ctrl->H0 += (mn[0] & 1u) ? 2 : -2;  // site (0,0)
  }
}

cudaError_t launch_halfsweep_plain(uint32_t *planes, int64_t L, int s, uint32_t t,
                                   uint64_t seed, const Accept &acc, Ctrl *ctrl,
                                   cudaStream_t st, const unsigned int *t_base) {
  const int64_t groups = L * (L >> 5) / 4;
  const int64_t blocks = (groups + 255) / 256;
  halfsweep_plain_kernel<<<(unsigned)blocks, 256, 0, st>>>(planes, L, s, t, t_base, seed, acc,
                                                           ctrl);
  return cudaGetLastError();
}

namespace {
__global__ void sweep_counter_kernel(Ctrl *__restrict__ ctrl, uint32_t v, int add) {
  if (add)
    ctrl->t_base += v;
  else
    ctrl->t_base = v;
}
}  // namespace

cudaError_t launch_set_sweep_counter(Ctrl *ctrl, uint32_t t, cudaStream_t st) {
  sweep_counter_kernel<<<1, 1, 0, st>>>(ctrl, t, 0);
  return cudaGetLastError();
}

cudaError_t launch_advance_sweep_counter(Ctrl *ctrl, uint32_t n, cudaStream_t st) {
  sweep_counter_kernel<<<1, 1, 0, st>>>(ctrl, n, 1);
  return cudaGetLastError();
}

}  // namespace okz
