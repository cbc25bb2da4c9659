// okz_internal.h -- host-side declarations shared by the library's .cu files.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/okz.h"
#include "okz_device.cuh"

namespace okz {

// Upper bound on the blocks of the row-reduction kernel; its per-block
// partial sums live in the simulation's device buffer.
constexpr int kMaxReduceBlocks = 2048;

struct Layout {
  size_t planes_bytes;  // one state buffer: X plane then Y plane
  size_t off_planes0, off_planes1, off_hcol, off_partials, off_ctrl, total;
};
Layout layout_for(int64_t L);

void set_error(const std::string &msg);
okz_status cuda_fail(cudaError_t e, const char *what);

// ---- launchers (each returns cudaGetLastError() of its launches) ----------
cudaError_t launch_init_flat(uint32_t *planes, int64_t L, cudaStream_t st);
// t_base (device, may be null): added to t, for graph-replayed chunks of sweeps.
cudaError_t launch_halfsweep_plain(uint32_t *planes, int64_t L, int s, uint32_t t,
                                   uint64_t seed, const Accept &acc, Ctrl *ctrl,
                                   cudaStream_t st, const unsigned int *t_base = nullptr);
// ctrl->t_base = t, and ctrl->t_base += n (one-thread kernels, stream-ordered).
cudaError_t launch_set_sweep_counter(Ctrl *ctrl, uint32_t t, cudaStream_t st);
cudaError_t launch_advance_sweep_counter(Ctrl *ctrl, uint32_t n, cudaStream_t st);
bool stream_kernel_supports(int64_t L);
// Words per thread the stream kernel can use for L (4 or 8; 0 = not valid).
bool stream_wpt_valid(int64_t L, int wpt);
// Runs `fuse` (1 or 2) sweeps t, t+1, .. in one pass from src to dst.
cudaError_t launch_sweep_stream(const uint32_t *src, uint32_t *dst, int64_t L,
                                uint32_t t, uint64_t seed, const Accept &acc,
                                int wpt, int fuse, int band_rows, Ctrl *ctrl,
                                cudaStream_t st);
// Measurement: column heights, then exact power sums about H0 into ctrl->sum.
// nmom = 2 (S1, S2) or 4 (S1..S4). parity: the state is a height-parity plane.
cudaError_t launch_power_sums(const uint32_t *planes, int64_t L, bool parity, int nmom,
                              int64_t *hcol, unsigned long long *partials,
                              Ctrl *ctrl, cudaStream_t st);
// hcol[y] = h(0,y) - H0 (the column-0 scan of the height reconstruction).
cudaError_t launch_colscan(const uint32_t *planes, int64_t L, bool parity, int64_t *hcol,
                           cudaStream_t st);
cudaError_t launch_heights(const uint32_t *planes, int64_t L, bool parity, int64_t y0,
                           int64_t ny, int64_t *hcol, int32_t *out, Ctrl *ctrl,
                           cudaStream_t st);
// Height-parity plane: half-sweeps and fused stream sweeps (parity.cu), the
// blocked random-sequential sweep (ddrs.cu), and the conversions to and from
// the slope planes of the C-ABI state format (convert.cu).
cudaError_t launch_parity_halfsweep(uint32_t *B, int64_t L, int s, uint32_t t, uint64_t seed,
                                    const Accept &acc, Ctrl *ctrl, cudaStream_t st,
                                    const unsigned int *t_base = nullptr);
// Grid of a stream-kernel launch (both kernels): bands of band_rows rows,
// or (band_rows = 0) as many bands as the GPU holds at once (`capacity`
// CTAs), each at least 4F + 1 rows -- a band streams 2F rows either side of
// its own, and only the first band's stream may meet the unwrapped rows
// 0 .. 2F, where the tracking of h(0,0) looks.
inline int stream_min_band(int F) { return 4 * F + 1; }
inline int stream_grid(int L, int F, int band_rows, int capacity) {
  int grid = band_rows > 0 ? L / band_rows : capacity;
  if (band_rows <= 0 && grid > L / stream_min_band(F)) grid = L / stream_min_band(F);
  return grid < 1 ? 1 : grid;
}

// One-CTA kernel (batch.cu): the parity plane swept out of shared memory,
// n sweeps in one launch; L % 32 == 0 and L <= kCtaMaxL (128 KiB).
constexpr int64_t kCtaMaxL = 1024;
bool cta_kernel_supports(int64_t L);
cudaError_t launch_cta_sweeps(uint32_t *B, int64_t L, uint32_t t, int64_t n, uint64_t seed,
                              const Accept &acc, Ctrl *ctrl, cudaStream_t st);

// The parity stream kernel also takes 16 words per thread: L % 16384 == 0.
bool parity_wpt_valid(int64_t L, int wpt);
cudaError_t launch_parity_stream(const uint32_t *src, uint32_t *dst, int64_t L, uint32_t t,
                                 uint64_t seed, const Accept &acc, int wpt, int fuse,
                                 int band_rows, Ctrl *ctrl, cudaStream_t st);
cudaError_t launch_ddrs(uint32_t *B, int64_t L, uint32_t t, uint64_t seed, uint64_t P32,
                        uint64_t Q32, Ctrl *ctrl, cudaStream_t st);
cudaError_t launch_to_slopes(const uint32_t *B, int64_t L, uint32_t *out, cudaStream_t st);
cudaError_t launch_from_slopes(const uint32_t *slopes, int64_t L, long long H0, int64_t *bcol,
                               uint32_t *B, cudaStream_t st);

// Stream-ordered device scratch from the library's per-device memory pool
// (capi.cu); freed memory stays mapped for the next call.
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t st);
void scratch_free(void *p, cudaStream_t st);

// Interface profiles and power spectrum (psd.cu). Scratch for L: see
// psd_scratch_bytes; col, row (L int64 each) are device arrays.
size_t psd_scratch_bytes(int64_t L, bool fft);
cudaError_t launch_profiles(const uint32_t *planes, int64_t L, bool parity, void *scratch,
                            int64_t *col, int64_t *row, unsigned int *err, cudaStream_t st);
// S[k], k = 0..L-1 (device array) from col and row; L a power of two.
cudaError_t launch_psd(const int64_t *col, const int64_t *row, int64_t L, void *scratch,
                       double *S, cudaStream_t st);

}  // namespace okz
