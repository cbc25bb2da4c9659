/*
 * okz.h -- C-ABI of the GB300 octahedron-model library.
 *
 * The library simulates the 2+1-dimensional octahedron model of
 * J. Kelling and G. Odor, "Extremely large scale simulation of a
 * Kardar-Parisi-Zhang model using graphics cards" (arXiv:1110.6745):
 * integer heights h(x,y) on an L x L periodic lattice whose neighbours differ
 * by exactly 1, held as two slope bit-planes (Sec. II: two bits per site).
 * A local minimum is raised by 2 with probability p, a local maximum lowered
 * by 2 with probability q (Sec. I, Eq. (2)).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an okz_status. Output arguments are written only when
 *    the call returns OKZ_OK. okz_last_error() gives a thread-local message
 *    for the most recent failure of the calling thread.
 *  - A simulation is owned by the library (opaque handle). Caller buffers
 *    passed in are only read or written during the call, unless stated.
 *  - Work is ordered on the simulation's CUDA stream. Calls marked
 *    "synchronizing" wait for that stream before returning.
 *  - Pointers are plain host or device addresses as stated per argument;
 *    "device" means memory of the CUDA device current when the simulation was
 *    created.
 *
 * Bit-plane layout (the only state format that crosses this boundary):
 *   plane X holds sigma_x(x,y) = h(x+1,y) - h(x,y), plane Y holds
 *   sigma_y(x,y) = h(x,y+1) - h(x,y); a set bit means +1, a clear bit -1.
 *   Each plane is L rows of L/32 little-endian uint32 words, row-major; bit b
 *   of word w of row y is the bond at x = 32*w + b. A state buffer is the X
 *   plane followed by the Y plane: 2 * L * L / 8 bytes.
 *
 * Dynamics (one sweep = one Monte Carlo step, Sec. II):
 *   sweep t runs half-sweep s = 0 (every site with (x+y) even) and then
 *   half-sweep s = 1. A site touches only its four bonds, and sites of one
 *   sublattice share no bond, so a half-sweep is order independent.
 *   Every active site is selected with probability s_sel; a selected minimum
 *   (maximum) moves when U < P (U < Q). U is a k-bit uniform, and k, P, Q
 *   come from p_eff = s_sel * p, q_eff = s_sel * q: k is the smallest k <=
 *   k_max with p_eff 2^k and q_eff 2^k integral, else k = k_max with
 *   round-half-even thresholds.
 *   Random draws: for site index i = y*L + x, group g = i / 128, word
 *   j = (i mod 128) / 32, bit b = i mod 32, level m of the draw at sweep t is
 *   bit b of word j of Philox4x32-10 (Salmon et al., SC'11) with counter
 *   (g mod 2^32, g / 2^32, t, m) and key (seed mod 2^32, seed / 2^32);
 *   U = sum_m bit_m 2^(k-1-m), most significant level first.
 */
#ifndef OKZ_H
#define OKZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum okz_status {
    OKZ_OK = 0,
    OKZ_EINVAL = 1,       /* bad argument (odd L, p > 1, null pointer, ...)        */
    OKZ_ENOMEM = 2,       /* device or host allocation failed / buffer too small    */
    OKZ_ECUDA = 3,        /* a CUDA call failed; see okz_last_error()               */
    OKZ_ETIMEOUT = 4,     /* a bounded device-side wait gave up                     */
    OKZ_EBUSY = 5,        /* no free slot or memory for admission                   */
    OKZ_EOVERFLOW = 6,    /* sweep counter would pass 2^32 - 1                      */
    OKZ_EUNSUPPORTED = 7  /* valid request this build does not handle (e.g. L % 32) */
} okz_status;

/* Two's-complement 128-bit integer: value = hi * 2^64 + lo. */
typedef struct okz_i128 {
    uint64_t lo;
    int64_t hi;
} okz_i128;

/* Which sweep kernel (and device representation) a simulation uses. All
 * give bit-identical results; the state format of okz_state/okz_restore is
 * always the two slope planes.
 *  - PLAIN, STREAM keep the two slope planes of Sec. II on the device.
 *  - PARITY_PLAIN, PARITY_STREAM keep one height-parity plane: since
 *    h(x,y) == x + y (mod 2), the bit b = floor(h/2) mod 2 fixes h mod 4
 *    and with it every slope (sigma_x(x,y) = +1 iff b(x+1,y) ^ b(x,y) ^
 *    ((x+y) mod 2) == 0, likewise sigma_y), and a move toggles only the
 *    site's own bit: one bit read and one written per site and sweep.
 * AUTO picks PARITY_STREAM when L is a multiple of 4096 and at most
 * 131072, else PARITY_CTA up to L = 512 (L % 32 == 0), else PARITY_PLAIN. */
enum {
    OKZ_KERNEL_AUTO = 0,
    OKZ_KERNEL_PLAIN = 1,          /* slope planes, one in-place launch per half-sweep */
    OKZ_KERNEL_STREAM = 2,         /* slope planes, TMA-staged rows, ping-pong         */
    OKZ_KERNEL_PARITY_PLAIN = 3,   /* parity plane, one in-place launch per half-sweep */
    OKZ_KERNEL_PARITY_STREAM = 4,  /* parity plane, TMA-staged rows, ping-pong         */
    OKZ_KERNEL_PARITY_CTA = 5      /* parity plane swept by one CTA out of shared
                                      memory, all sweeps of a call in one launch;
                                      L % 32 == 0 and L <= 1024. AUTO: the stream
                                      kernel where it runs (L % 4096 == 0), else
                                      this one up to L = 512, else PARITY_PLAIN     */
};

typedef struct okz_params {
    int64_t L;      /* linear size; the GPU needs L % 32 == 0 and L >= 32         */
    double p;       /* attachment probability, minimum -> maximum, in [0, 1]      */
    double q;       /* detachment probability, maximum -> minimum, in [0, 1]      */
    uint64_t seed;  /* Philox key                                                  */
    double s_sel;   /* selection probability of an active site, (0, 1]; 0.5      */
    int32_t k_max;  /* largest acceptance precision in bits, 1..32; 32            */
    int32_t kernel; /* OKZ_KERNEL_*                                                */
    int32_t words_per_thread; /* STREAM: 4, 8 (or 16, parity plane) words of 32 sites
                                 per thread; 0 = auto                                */
    int32_t sweeps_per_pass;  /* STREAM: 1 or 2 sweeps fused per launch; 0 = auto      */
    int32_t band_rows;        /* STREAM: rows per CTA band, at least 4F + 1 (F the
                                 sweeps per pass) and at most L; 0 = auto: as many
                                 bands as the GPU holds at once, each at least
                                 4F + 1 rows. A band streams 4F rows beyond its
                                 own, so smaller bands trade work for parallelism.
                                 Results do not depend on it.                      */
} okz_params;

typedef struct okz_info {
    int64_t L;
    uint64_t t;           /* completed sweeps                                  */
    int64_t H0;           /* h(0,0)                                            */
    int32_t k;            /* acceptance precision in bits                      */
    int32_t kernel;       /* the OKZ_KERNEL_* in use (never AUTO)              */
    uint64_t P, Q;        /* thresholds: accept iff U < P (min) / U < Q (max)  */
    size_t device_bytes;  /* device memory held by the simulation              */
    int32_t words_per_thread;  /* stream kernels: words per thread (else 0)    */
    int32_t sweeps_per_pass;   /* sweeps per launch                             */
    int32_t graph_chunk;       /* in-place kernels: sweeps per replay of the
                                  simulation's CUDA graph (0 = not built)       */
    uint64_t graph_replays;    /* replays of that graph so far                  */
    int32_t band_rows;         /* stream kernels: the band_rows in use (0 = auto) */
} okz_info;

typedef struct okz_sim okz_sim;

/* Fills *prm with the defaults: L = 0, p = 1, q = 0, seed = 0, s_sel = 0.5,
 * k_max = 32, kernel = AUTO, words_per_thread = 0, sweeps_per_pass = 0,
 * band_rows = 0. The
 * last two only choose how the stream kernel tiles the work; results are
 * bit-identical for every choice. 8 words per thread needs L % 8192 == 0,
 * 16 (parity stream kernel only) L % 16384 == 0. Their automatic values
 * (measured best on GB300): parity plane -- with k = 1, 16 words per thread
 * from L = 32768 up, with k >= 2, 8 from L = 65536 up, else 4 (or the next
 * smaller valid choice); two sweeps per pass with k = 1, one with k >= 2;
 * slope planes -- 8 words per thread where L % 8192 == 0, else 4; one sweep
 * per pass. */
void okz_params_init(okz_params *prm);

/* Device bytes a simulation of size L needs when memory is passed to
 * okz_create_ex: two state buffers (ping-pong, L*L/4 bytes each), L int64 of
 * column heights and a 256-byte control block, each 256-byte aligned.
 * Returns 0 for an invalid L. */
size_t okz_device_bytes(int64_t L);

/* Creates a simulation on the current CUDA device with the striped start
 * h(x,y) = (x+y) mod 2, H0 = 0, t = 0 (Sec. III: "half filled (striped)",
 * W^2 = 1/4), s_sel = 0.5 and k_max = 32. The library allocates the device
 * memory and a non-blocking stream. L even, L % 32 == 0, L >= 32; p, q in
 * [0, 1]. Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA. */
okz_status okz_create(int64_t L, double p, double q, uint64_t seed, okz_sim **out);

/* As okz_create with every parameter given. If dev_buf is not NULL it must
 * be a device buffer of at least okz_device_bytes(L) bytes, 256-byte
 * aligned, which the caller keeps alive until okz_destroy; otherwise the
 * library allocates. stream is a cudaStream_t (NULL = the library creates
 * its own non-blocking stream); all work of this simulation is ordered on
 * it. With a caller's stream the call returns once the initialisation (the
 * striped start) is enqueued on that stream; with the library's own stream
 * it waits for it. Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA. */
okz_status okz_create_ex(const okz_params *prm, void *dev_buf, size_t bytes,
                         void *stream, okz_sim **out);

/* Enqueues n >= 0 sweeps (Sec. II: one sweep = one MCS) on the simulation's
 * stream and returns without waiting. The stream kernels take one launch per
 * sweeps_per_pass sweeps. The in-place kernels (PLAIN, PARITY_PLAIN: two
 * launches per sweep) run whole chunks of 32 sweeps by replaying one CUDA
 * graph, captured on the first call with n >= 32, whose launches read the
 * chunk's first sweep index from the simulation's device control block; the
 * rest of n goes as direct launches. Results do not depend on the split.
 * Errors: EINVAL (n < 0), EOVERFLOW (t + n > 2^32 - 1; nothing is
 * enqueued), ECUDA (launch failure). */
okz_status okz_sweep(okz_sim *sim, int64_t n);

/* Enqueues n sweeps of the domain-decomposed random-sequential dynamics, the
 * paper's own GPU update (Sec. II: blocks with dead borders, the origin moved
 * at random every MCS, random attempts inside each block), as a statistical
 * counterpart of the checkerboard sweep. Sweep t: offsets (ox, oy) = (r0, r1)
 * mod 32 of Philox(counter (0, 0, t, 768)); 32 x 32 cells with origins
 * (ox + 32i, oy + 32j) mod L, ids c = j*(L/32) + i; cell c receives 1024
 * attempts, attempt a using words (r0, r1) (a even) or (r2, r3) (a odd) of
 * Philox(counter (c, a/2, t, 1024)): local x = first & 31, local y =
 * (first >> 16) & 31, u = second. Attempts on a cell's dead first column or
 * first row do nothing (two dead edges, as in Fig. 1 of the paper);
 * elsewhere a minimum moves iff u < round(p 2^32), a maximum iff
 * u < round(q 2^32) (round half to even; no selection factor). Needs a
 * parity-plane simulation (EUNSUPPORTED otherwise) and L % 32 == 0; shares t
 * with okz_sweep. Errors: EINVAL (n < 0), EUNSUPPORTED, EOVERFLOW (t + n >
 * 2^32 - 1), ECUDA (launch failure). */
okz_status okz_sweep_rs(okz_sim *sim, int64_t n);

/* Synchronizing. Reconstructs the heights from the slopes (Sec. I, Eq. (3),
 * anchored at H0 = h(0,0)) and returns the exact sums S1 = sum h,
 * S2 = sum h^2 and the squared width of Sec. I, Eq. (4),
 *   W2 = (N*S2 - S1^2) / N^2,  N = L*L,
 * with the numerator formed exactly in 128-bit integers and rounded once to
 * double. Any output pointer may be NULL. Errors: ECUDA, ETIMEOUT. */
okz_status okz_width2(okz_sim *sim, okz_i128 *S1, okz_i128 *S2, double *W2);

/* Synchronizing. Exact central power sums S_n = sum (h - H0)^n, n = 1..4
 * (Sk[0..3]), and from them W2, the skewness m3/m2^1.5 and the excess
 * kurtosis m4/m2^2 - 3 of the height distribution, with mu = S1/N,
 * m2 = S2/N - mu^2, m3 = S3/N - 3 mu S2/N + 2 mu^3,
 * m4 = S4/N - 4 mu S3/N + 6 mu^2 S2/N - 3 mu^4 in long double.
 * Needs L <= 131072. Any output pointer may be NULL. */
okz_status okz_moments(okz_sim *sim, okz_i128 Sk[4], double *W2, double *skew,
                       double *kurt);

/* The growth run of Sec. III in one call: sweeps the simulation to each of
 * the n sample times (ascending from its current sweep count) and takes at
 * each the exact S1 = sum h, S2 = sum h^2 and W^2 of okz_width2 (Eq. (4))
 * and H0 = h(0,0). Sweeps and measurements are queued on the simulation's
 * stream; each sample's sums are copied aside on the device, and the call
 * synchronizes once at the end. Outputs are host arrays of n entries (any may
 * be NULL). Errors: EINVAL (times not ascending), EOVERFLOW (a time past
 * 2^32 - 1), ENOMEM, ECUDA, ETIMEOUT. */
okz_status okz_growth_series(okz_sim *sim, int32_t n, const uint64_t *times, okz_i128 *S1,
                             okz_i128 *S2, double *W2, int64_t *H0);

/* okz_moments in two halves, for callers that must not block while other
 * streams work: okz_moments_enqueue launches the power-sum kernels on the
 * simulation's stream and returns at once; okz_moments_fetch waits for that
 * stream (record an event after enqueue and poll it to know when the wait is
 * free) and returns what okz_moments would have. Sweeps enqueued in between
 * do not change the result of the enqueued sums; a later measurement call
 * overwrites them. Errors: as okz_moments. */
okz_status okz_moments_enqueue(okz_sim *sim);
okz_status okz_moments_fetch(okz_sim *sim, okz_i128 Sk[4], double *W2, double *skew,
                             double *kurt);

/* Synchronizing. Writes h(x, y) for rows y0 .. y0+ny-1 (Sec. I, Eq. (3)) as
 * int32, row-major, ny * L values, to out (device memory if out_is_device,
 * else host memory). 0 <= y0, y0 + ny <= L. Errors: EINVAL, EOVERFLOW (some
 * |h| >= 2^31; out is then undefined), ECUDA. */
okz_status okz_heights(okz_sim *sim, int64_t y0, int64_t ny, int32_t *out,
                       int out_is_device);

/* Synchronizing. Interface profiles for the power spectrum of Sec. III
 * (Eqs. (15)-(16)): col[x] = sum_y (h(x,y) - H0) and row[y] = sum_x
 * (h(x,y) - H0), x, y = 0 .. L-1, exact int64, into caller-owned host arrays
 * of L values (either may be NULL). Allocates about 4 L ceil(L/R) + 29 L
 * bytes (plus 40 L for okz_psd) of stream-ordered device scratch for the
 * call, R being the rows per counting band (a multiple of 16, at most 4080;
 * 2304 at L = 131072 on a 152-SM GPU, i.e. 32 MiB). Errors: EINVAL, ENOMEM,
 * ECUDA, ETIMEOUT (a bounded wait of the streaming counting kernel gave up;
 * the outputs are then undefined). */
okz_status okz_profiles(okz_sim *sim, int64_t *col, int64_t *row);

/* Synchronizing. The power spectrum of Sec. III, Eqs. (15)-(16), on the two
 * k axes, averaged over the x and y directions:
 *   S[k] = (|h(k,0)|^2 + |h(0,k)|^2) / 2,  k = 0 .. L-1 (wave number 2 pi k / L),
 *   h(k,0) = (1/L) sum_{x,y} (h(x,y) - <h>) e^{-2 pi i k x / L},
 * (the d = 2 normalisation L^{-d/2}; S[0] = 0 as the mean is removed; the
 * sign of the exponent does not change |h(k)|). Computed from the exact
 * profiles (okz_profiles) by one fp64 FFT of col + i row on the device
 * (radix-2 decimation in time; S is symmetric, S[k] = S[L-k]). S is a
 * caller-owned host array of L doubles. Needs a power-of-two L (EUNSUPPORTED
 * otherwise). Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA, ETIMEOUT (as
 * okz_profiles). */
okz_status okz_psd(okz_sim *sim, double *S);

/* Synchronizing. Copies the state buffer (X plane then Y plane, layout
 * above) to planes_out (device memory if out_is_device, else host) and
 * returns H0 and t (either pointer may be NULL). */
okz_status okz_state(okz_sim *sim, uint32_t *planes_out, int out_is_device,
                     int64_t *H0, uint64_t *t);

/* Replaces the state with planes (same layout; device memory if
 * in_is_device, else host), H0 and t. The planes must describe a height
 * function (zero row sums of sigma_x, zero column sums of sigma_y, zero
 * curl); this is not checked. Synchronizing. */
okz_status okz_restore(okz_sim *sim, const uint32_t *planes, int in_is_device,
                       int64_t H0, uint64_t t);

/* okz_restore from host memory in two halves, so that the host-to-device
 * copy of the next state can run while the simulation sweeps (the state is
 * the slope planes of Sec. II; the paper has no counterpart to the split).
 * okz_stage_host starts copying planes (layout above, 2*L*L/8 bytes) into a
 * staging buffer of that size that the simulation owns (made on first use,
 * counted in okz_info's device_bytes, freed by okz_destroy) on a copy stream
 * of its own, after the previous staged planes have been converted, and
 * returns at once.
 * okz_restore_staged makes the simulation's stream wait for that copy, then
 * replaces the state with the staged planes, H0 and t (as okz_restore) on
 * that stream, and returns at once. The host planes must stay unchanged until
 * the copy has run: any later synchronizing call on the simulation
 * (okz_synchronize, okz_width2, ...) guarantees it. Pinned host memory makes
 * the copy asynchronous. Errors: EINVAL (null arguments, odd H0, t past
 * 2^32 - 1, nothing staged), ENOMEM, ECUDA. */
okz_status okz_stage_host(okz_sim *sim, const uint32_t *planes);
okz_status okz_restore_staged(okz_sim *sim, int64_t H0, uint64_t t);

/* okz_tune_stream -- the paper has no counterpart to this entry point (the
 * tiling of the update is this build's). Autotuner of the stream kernels'
 * launch shape for one workload: for every valid words_per_thread (4, 8, 16),
 * sweeps_per_pass (1, 2) and band_rows (0 = auto, 16, 32) it creates a
 * scratch simulation of prm (kernel STREAM or PARITY_STREAM; AUTO means
 * PARITY_STREAM), runs 4 sweeps, then times probe_sweeps (>= 2) sweeps with
 * CUDA events, and keeps the fastest per sweep. The choice is remembered for
 * (device, L, kernel, acceptance mode: k = 1 with minima only, other k <= 1,
 * k >= 2) and used by every later okz_create / okz_create_ex that leaves
 * words_per_thread and sweeps_per_pass automatic (0), band_rows too when that
 * is 0 (a band_rows given with a tuned two-sweep pass it does not fit makes
 * the pass one sweep). Results are
 * bit-identical for every tiling, so tuning never changes a result. Writes
 * the choice and its time per sweep (any output may be NULL). Synchronizing; each scratch simulation holds
 * okz_device_bytes(L) for its run. Errors: EINVAL, EUNSUPPORTED (L outside the
 * stream kernels' range), ENOMEM, ECUDA, ETIMEOUT. */
okz_status okz_tune_stream(const okz_params *prm, int32_t probe_sweeps, int32_t *wpt_out,
                           int32_t *fuse_out, int32_t *band_out, double *ms_per_sweep);

/* Fills *info. Synchronizing (H0 lives on the device). */
okz_status okz_get_info(okz_sim *sim, okz_info *info);

/* Waits for the simulation's stream and reports device-side errors
 * (ETIMEOUT when a bounded wait inside a kernel gave up). */
okz_status okz_synchronize(okz_sim *sim);

/* The simulation's stream (a cudaStream_t). */
void *okz_stream(okz_sim *sim);

/* Waits for outstanding work, frees what the library allocated, and
 * destroys the handle. NULL is accepted. */
okz_status okz_destroy(okz_sim *sim);

/* Message of the calling thread's most recent failure ("" if none). */
const char *okz_last_error(void);

/* okz_selftest_wait_timeout -- the paper has no counterpart to this entry
 * point. Self-test of the bounded device-side wait the streaming kernels use
 * for their TMA copies: one block arms an mbarrier for a 16-byte transaction
 * that is never issued and waits on it with the library's wait limit (2 s
 * of %globaltimer). Returns OKZ_ETIMEOUT when the bound works -- the kernel
 * gives up, reports the timeout and exits, and the context stays usable --
 * and OKZ_OK if the wait completed (a defect). stream is a cudaStream_t (NULL
 * = the legacy default stream); synchronizing; uses 4 bytes of
 * stream-ordered device memory. Errors: ENOMEM, ECUDA. */
okz_status okz_selftest_wait_timeout(void *stream);

/* okz_alu_peak -- the paper has no counterpart to this entry point. A
 * diagnostic that measures the INT32 ALU-pipe throughput of the current
 * device, the denominator of the sweep kernels' roofline (their update logic
 * and most of the Philox work are three-input logic ops and funnel shifts,
 * which issue to that pipe). Launches 8 blocks of 256 threads per SM, each
 * thread running 8 independent chains of `iters` lop3.b32 ops (no memory
 * traffic in the loop); one warm-up launch, then the best of three timed
 * launches (CUDA events on `stream`, a cudaStream_t, NULL = the legacy
 * default stream). Writes the rate in thread-ops per second to *ops_per_s and
 * the best launch time to *best_ms (may be NULL). Synchronizing; allocates
 * nothing. iters of 20000 give launches of about 2.5 ms on GB300. Errors:
 * EINVAL (iters < 1 or ops_per_s NULL), ECUDA. */
okz_status okz_alu_peak(void *stream, int32_t iters, double *ops_per_s, double *best_ms);

/* okz_width2_noalloc -- the paper has no counterpart to this entry point; it
 * serves callers that cannot allocate device memory when they measure, e.g.
 * because a framework's caching allocator already holds all free device
 * memory, because an allocation (and the synchronisation it can cause) is not
 * allowed on their latency-critical path, or because their policy forbids
 * allocating after start-up.
 *
 * Computes the same exact sums and W^2 as okz_width2 for a state the caller
 * owns: `planes` is a 16-byte aligned device pointer to the slope-plane
 * layout above (X plane then Y plane; an unaligned pointer is rejected with
 * OKZ_EINVAL before any kernel runs), `H0` its h(0,0), `stream` the cudaStream_t to run on
 * (NULL = the legacy default stream). 32 <= L <= 131072 and L % 32 == 0;
 * a larger L is rejected with OKZ_EINVAL ("exceeds the fixed scratch size").
 * Outputs as okz_width2; any may be NULL. Synchronizing: waits for `stream`.
 *
 * It allocates nothing (no cudaMalloc, cudaFree or pinned buffers). Its
 * scratch is one fixed device array of 1 MiB + 128 KiB + 256 B, present on
 * every device that loads this library until the process exits. The first
 * call on a device looks up that array's address (cudaGetSymbolAddress, with
 * the device current); make that first call before any stream capture. All
 * calls share the one array: calls whose work overlaps on the GPU (different
 * streams, or several host threads) race and return wrong sums -- serialise
 * them. */
okz_status okz_width2_noalloc(const uint32_t *planes, int64_t L, int64_t H0, void *stream,
                              okz_i128 *S1, okz_i128 *S2, double *W2);

/* ---------------------------------------------------------------------------
 * Batched and pooled lattices (Sec. III: many independent runs per size).
 *
 * An okz_batch is a slot table of independent lattices (32 <= L <= 8192,
 * L % 32 == 0) kept on the device as height-parity planes in one arena.
 * okz_batch_run advances any subset of slots by per-slot sweep counts in one
 * persistent kernel launch (a CUDA graph replayed each run): CTAs take
 * (slot, sweeps) items longest-first from a device queue, stage a lattice in
 * shared memory when it fits, and sweep it in place. Every slot evolves
 * bit-identically to an okz_sim with the same (L, p, q, seed, s_sel, k_max).
 * --------------------------------------------------------------------------- */
typedef struct okz_batch okz_batch;

/* An empty slot table: `arena_bytes` of device memory for lattices
 * (L*L/8 bytes each, 256-byte granules), `max_slots` slots, selection
 * probability and acceptance precision shared by all slots, `stream` a
 * cudaStream_t (NULL = own stream). Errors: EINVAL, ENOMEM, ECUDA. */
okz_status okz_pool_create(size_t arena_bytes, int32_t max_slots, double s_sel,
                           int32_t k_max, void *stream, okz_batch **out);

/* n slots with the given sizes, probabilities and seeds (s_sel = 0.5,
 * k_max = 32), each at the striped start; slot i is replica i. */
okz_status okz_batch_create(int32_t n, const int64_t *L, const double *p, const double *q,
                            const uint64_t *seed, okz_batch **out);

/* Admits a lattice into a free slot (striped start, t = 0, H0 = 0).
 * Synchronizing. Errors: EBUSY (no free slot or no arena space -- the caller
 * may retry after removing slots), EINVAL, EUNSUPPORTED. */
okz_status okz_batch_add(okz_batch *b, int64_t L, double p, double q, uint64_t seed,
                         int32_t *slot);

/* Frees a slot and its arena space. Synchronizing. */
okz_status okz_batch_remove(okz_batch *b, int32_t slot);

/* Advances slot i by sweeps[i] sweeps (array of max_slots entries; 0 = leave
 * the slot alone) in one launch on the batch's stream and returns without
 * waiting for it (it waits for the previous run first). Errors: EINVAL
 * (negative count or an empty slot with work), EOVERFLOW, ECUDA. */
okz_status okz_batch_run(okz_batch *b, const int64_t *sweeps);

/* Waits for the batch's stream. */
okz_status okz_batch_sync(okz_batch *b);

/* Synchronizing. Per slot (arrays of max_slots entries; NaN for empty slots):
 * W^2 of Eq. (4) from exact sums, and the skewness and excess kurtosis of
 * the heights (formulas of okz_moments). Any pointer may be NULL. */
okz_status okz_batch_stats(okz_batch *b, double *W2, double *skew, double *kurt);

/* Synchronizing. Exact S_n = sum (h - H0)^n, n = 1..4, H0 and t of a slot. */
okz_status okz_batch_sums(okz_batch *b, int32_t slot, okz_i128 Sk[4], int64_t *H0,
                          uint64_t *t);

/* Synchronizing. Exact sums of n listed slots in one launch: Sk[4*j + m] =
 * S_{m+1} of slots[j], H0[j], t[j] (any output may be NULL). */
okz_status okz_batch_measure(okz_batch *b, int32_t n, const int32_t *slots, okz_i128 *Sk,
                             int64_t *H0, uint64_t *t);

/* Synchronizing. The slot's state as slope planes (layout above) in host
 * memory (2*L*L/8 bytes), H0 and t. */
okz_status okz_batch_state(okz_batch *b, int32_t slot, uint32_t *planes_out, int64_t *H0,
                           uint64_t *t);

/* Launch shape of okz_batch_run: threads per CTA (256, 512 or 1024) and the
 * shared-memory staging size (lattices up to that many bytes are swept in
 * shared memory). Results do not depend on it. */
okz_status okz_batch_set_tiling(okz_batch *b, int32_t threads, size_t smem_bytes);
okz_status okz_batch_get_tiling(okz_batch *b, int32_t *threads, size_t *smem_bytes,
                                int32_t *grid);

/* Times every tiling on a scratch copy of the slot mix (fresh lattices,
 * probe_sweeps sweeps each) and keeps the fastest. Synchronizing; the
 * batch's own lattices are untouched. */
okz_status okz_batch_autotune(okz_batch *b, int32_t probe_sweeps);

/* The batch's stream (a cudaStream_t). */
void *okz_batch_stream(okz_batch *b);

/* Waits for outstanding work and frees everything. NULL is accepted. */
okz_status okz_batch_destroy(okz_batch *b);

/* Acceptance precision and thresholds for (p, q, s_sel, k_max), the rule
 * stated above; the host computation every simulation uses. */
okz_status okz_thresholds(double p, double q, double s_sel, int32_t k_max,
                          int32_t *k, uint64_t *P, uint64_t *Q);

#ifdef __cplusplus
}
#endif

#endif /* OKZ_H */
