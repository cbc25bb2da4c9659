// capi.cu -- the C-ABI of include/okz.h: simulation handles, argument checks,
// stream-ordered launches and the exact host-side finalization of W^2.
#include <cuda_runtime.h>

#include <cfenv>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstddef>
#include <vector>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "okz_internal.h"

struct okz_sim {
  okz_params prm;
  okz::Accept acc;
  int kernel;
  bool parity;  // device state is one height-parity plane (else two slope planes)
  int wpt;   // stream kernel: words per thread
  int fuse;  // stream kernel: sweeps per launch
  int band_rows;  // stream kernel: rows per CTA band (0 = auto)
  int device;
  cudaStream_t stream;
  bool own_stream;
  char *base;
  bool own_mem;
  okz::Layout lay;
  uint32_t *planes[2];
  int cur;
  int64_t *hcol;
  unsigned long long *partials;
  okz::Ctrl *ctrl;
  uint64_t t;
  // in-place (plain) kernels: a CUDA graph of kGraphChunk sweeps that reads
  // its first sweep from ctrl->t_base and advances it; 0 = not built yet,
  // 1 = built, -1 = capture failed (direct launches only)
  cudaGraphExec_t sweep_graph;
  int graph_state;
  uint64_t graph_replays;
  // okz_stage_host / okz_restore_staged (made on first use): a device copy of
  // caller planes taken on copy_stream; `staged` is recorded after the copy,
  // `consumed` on the simulation's stream after the conversion has read it
  uint32_t *stage_buf;
  cudaStream_t copy_stream;
  cudaEvent_t staged_ev, consumed_ev;
  bool stage_pending;
};

namespace okz {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

okz_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
            ")");
  return OKZ_ECUDA;
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Stream-ordered scratch comes from a memory pool owned by the library, one
// per device, that keeps up to 1 GiB of freed memory mapped between calls
// (the default pool returns it to the driver at every synchronization, so
// each call would map its scratch afresh). Falls back to the default pool if
// the pool cannot be created.
static cudaMemPool_t scratch_pool(int dev) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
    uint64_t keep = 1ull << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  } else {
    cudaGetLastError();
    pool = nullptr;
  }
  pools[dev] = pool;
  return pool;
}

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool = scratch_pool(dev);
  return pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
}

void scratch_free(void *p, cudaStream_t st) { cudaFreeAsync(p, st); }

Layout layout_for(int64_t L) {
  Layout lay{};
  lay.planes_bytes = (size_t)L * (size_t)L / 4;  // 2 bits per site
  size_t off = 0;
  lay.off_planes0 = off;
  off = align256(off + lay.planes_bytes);
  lay.off_planes1 = off;
  off = align256(off + lay.planes_bytes);
  lay.off_hcol = off;
  off = align256(off + (size_t)L * sizeof(int64_t));
  lay.off_partials = off;
  off = align256(off + (size_t)kMaxReduceBlocks * 8 * sizeof(unsigned long long));
  lay.off_ctrl = off;
  off = align256(off + sizeof(Ctrl));
  lay.total = off;
  return lay;
}

static okz_status check_L(int64_t L) {
  if (L < 2 || (L & 1)) {
    set_error("L must be even and >= 2");
    return OKZ_EINVAL;
  }
  if (L % 32 != 0 || L > (int64_t)1 << 20) {
    set_error("this build needs L % 32 == 0 and L <= 2^20");
    return OKZ_EUNSUPPORTED;
  }
  return OKZ_OK;
}

// Kernel mode of the stream kernels for thresholds (k, P, Q): 0 = k = 1 with
// only minima moving at one random level (P < 2^k, Q = 0), 1 = other k <= 1,
// 2 = k >= 2 (lazily drawn levels).
static int stream_mode(int k, uint64_t P, uint64_t Q) {
  if (k >= 2) return 2;
  const uint64_t full = 1ull << k;
  const bool half = P != 0 && P < full && Q == 0;
  return half ? 0 : 1;
}

// Tilings chosen by okz_tune_stream, per (device, L, kernel, mode).
struct TuneKey {
  int dev;
  int64_t L;
  int kernel, mode;
  bool operator<(const TuneKey &o) const {
    if (dev != o.dev) return dev < o.dev;
    if (L != o.L) return L < o.L;
    if (kernel != o.kernel) return kernel < o.kernel;
    return mode < o.mode;
  }
};
static std::mutex g_tune_mu;
struct Tiling {
  int wpt, fuse, band_rows;
};
static std::map<TuneKey, Tiling> g_tuned;

static bool tuned_tiling(int64_t L, int kernel, int mode, int *wpt, int *fuse, int *band_rows) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(TuneKey{dev, L, kernel, mode});
  if (it == g_tuned.end()) return false;
  *wpt = it->second.wpt;
  *fuse = it->second.fuse;
  *band_rows = it->second.band_rows;
  return true;
}

}  // namespace okz

using namespace okz;

static okz_i128 from_i128(__int128 v) {
  okz_i128 r;
  r.lo = (uint64_t)(unsigned __int128)v;
  r.hi = (int64_t)(uint64_t)((unsigned __int128)v >> 64);
  return r;
}

extern "C" {

const char *okz_last_error(void) { return g_last_error.c_str(); }

void okz_params_init(okz_params *prm) {
  if (!prm) return;
  prm->L = 0;
  prm->p = 1.0;
  prm->q = 0.0;
  prm->seed = 0;
  prm->s_sel = 0.5;
  prm->k_max = 32;
  prm->kernel = OKZ_KERNEL_AUTO;
  prm->words_per_thread = 0;
  prm->sweeps_per_pass = 0;
  prm->band_rows = 0;
}

okz_status okz_thresholds(double p, double q, double s_sel, int32_t k_max, int32_t *k,
                          uint64_t *P, uint64_t *Q) {
  if (!(p >= 0.0 && p <= 1.0 && q >= 0.0 && q <= 1.0)) {
    set_error("p and q must lie in [0, 1]");
    return OKZ_EINVAL;
  }
  if (!(s_sel > 0.0 && s_sel <= 1.0) || k_max < 1 || k_max > 32) {
    set_error("s_sel must lie in (0, 1] and k_max in 1..32");
    return OKZ_EINVAL;
  }
  const double pe = s_sel * p, qe = s_sel * q;
  int kk = -1;
  double a = 0, b = 0;
  for (int j = 0; j <= k_max; ++j) {  // smallest exact precision
    a = std::ldexp(pe, j);
    b = std::ldexp(qe, j);
    if (a == std::floor(a) && b == std::floor(b)) {
      kk = j;
      break;
    }
  }
  if (kk < 0) {  // round half to even at k_max bits
    const int mode = std::fegetround();
    std::fesetround(FE_TONEAREST);
    a = std::nearbyint(std::ldexp(pe, k_max));
    b = std::nearbyint(std::ldexp(qe, k_max));
    std::fesetround(mode);
    kk = k_max;
  }
  if (k) *k = kk;
  if (P) *P = (uint64_t)a;
  if (Q) *Q = (uint64_t)b;
  return OKZ_OK;
}

size_t okz_device_bytes(int64_t L) {
  if (check_L(L) != OKZ_OK) return 0;
  return layout_for(L).total;
}

okz_status okz_create_ex(const okz_params *prm, void *dev_buf, size_t bytes, void *stream,
                         okz_sim **out) {
  if (!prm || !out) {
    set_error("null argument");
    return OKZ_EINVAL;
  }
  okz_status st = check_L(prm->L);
  if (st != OKZ_OK) return st;
  int32_t k;
  uint64_t P, Q;
  st = okz_thresholds(prm->p, prm->q, prm->s_sel, prm->k_max, &k, &P, &Q);
  if (st != OKZ_OK) return st;
  int kernel = prm->kernel;
  if (kernel == OKZ_KERNEL_AUTO)  // one CTA up to L = 512 (measured: 2.3x faster at 256)
    kernel = stream_kernel_supports(prm->L)      ? OKZ_KERNEL_PARITY_STREAM
             : (prm->L <= 512 && cta_kernel_supports(prm->L)) ? OKZ_KERNEL_PARITY_CTA
                                                              : OKZ_KERNEL_PARITY_PLAIN;
  if (kernel < OKZ_KERNEL_PLAIN || kernel > OKZ_KERNEL_PARITY_CTA) {
    set_error("unknown kernel selector");
    return OKZ_EINVAL;
  }
  if (kernel == OKZ_KERNEL_PARITY_CTA && !cta_kernel_supports(prm->L)) {
    set_error("the one-CTA kernel needs L % 32 == 0 and L <= 1024");
    return OKZ_EUNSUPPORTED;
  }
  const bool streamed = kernel == OKZ_KERNEL_STREAM || kernel == OKZ_KERNEL_PARITY_STREAM;
  if (streamed && !stream_kernel_supports(prm->L)) {
    set_error("the streaming kernels need L % 4096 == 0 and L <= 131072");
    return OKZ_EUNSUPPORTED;
  }
  int wpt = prm->words_per_thread, fuse = prm->sweeps_per_pass, band = prm->band_rows;
  if (streamed && wpt == 0 && fuse == 0) {  // okz_tune_stream's best tiling
    int tw = 0, tf = 0, tb = 0;
    if (tuned_tiling(prm->L, kernel, stream_mode(k, P, Q), &tw, &tf, &tb)) {
      wpt = tw;
      fuse = tf;
      if (band == 0) band = tb;
      else if (band < stream_min_band(fuse)) fuse = 1;  // the caller's band decides
    }
  }
  if (streamed) {
    // defaults measured on GB300. Slope planes: 8 words per thread where the
    // row allows it, one sweep per pass. Parity plane with one random level
    // per site (k = 1): 16 words per thread from L = 32768 up (256 threads
    // a row at L = 2^17, each with twice the independent words of the
    // 8-word kernel: 8-12 % faster), 4 below (a CTA spans one short row, and
    // 4 words per thread gives it the most threads); with k >= 2, 8 words per
    // thread from L = 65536 up, else 4 (the 16-word general-k kernels are
    // 5-15 % slower). Two sweeps per pass with k = 1, one with k >= 2 (the
    // fused general-k kernels hold too many registers: one pass per sweep is
    // 8-30 % faster)
    if (kernel == OKZ_KERNEL_PARITY_STREAM) {
      if (wpt == 0) {
        const int64_t L = prm->L;
        if (k <= 1 && L >= 32768 && parity_wpt_valid(L, 16))
          wpt = 16;
        else if (L >= (k <= 1 ? 32768 : 65536) && stream_wpt_valid(L, 8))
          wpt = 8;
        else
          wpt = 4;
      }
      if (fuse == 0) fuse = (k >= 2) ? 1 : 2;
    } else {
      if (wpt == 0) wpt = stream_wpt_valid(prm->L, 8) ? 8 : 4;
      if (fuse == 0) fuse = 1;
    }
    const bool wpt_ok = kernel == OKZ_KERNEL_PARITY_STREAM ? parity_wpt_valid(prm->L, wpt)
                                                          : stream_wpt_valid(prm->L, wpt);
    if (!wpt_ok || (fuse != 1 && fuse != 2)) {
      set_error("words_per_thread must be 4 or 8 (8 needs L % 8192 == 0; the parity "
                "stream kernel also takes 16 with L % 16384 == 0) and sweeps_per_pass 1 or 2");
      return OKZ_EINVAL;
    }
    if (band != 0 && (band < stream_min_band(fuse) || band > prm->L)) {
      set_error("band_rows must be 0 (auto) or lie in [4F + 1, L], F the sweeps per pass");
      return OKZ_EINVAL;
    }
  } else {
    wpt = 0;
    fuse = 1;
    band = 0;
  }
  const Layout lay = layout_for(prm->L);
  if (dev_buf && (bytes < lay.total || ((uintptr_t)dev_buf & 255u))) {
    set_error("external device buffer too small or not 256-byte aligned");
    return OKZ_ENOMEM;
  }

  okz_sim *sim = new (std::nothrow) okz_sim();
  if (!sim) {
    set_error("host allocation failed");
    return OKZ_ENOMEM;
  }
  sim->prm = *prm;
  sim->acc.P = P;
  sim->acc.Q = Q;
  sim->acc.k = k;
  sim->kernel = kernel;
  sim->parity = kernel == OKZ_KERNEL_PARITY_PLAIN || kernel == OKZ_KERNEL_PARITY_STREAM ||
                kernel == OKZ_KERNEL_PARITY_CTA;
  sim->wpt = wpt;
  sim->fuse = fuse;
  sim->band_rows = band;
  sim->lay = lay;
  sim->t = 0;
  sim->cur = 0;
  cudaError_t e = cudaGetDevice(&sim->device);
  if (e != cudaSuccess) {
    delete sim;
    return cuda_fail(e, "cudaGetDevice");
  }
  if (stream) {
    sim->stream = (cudaStream_t)stream;
    sim->own_stream = false;
  } else {
    e = cudaStreamCreateWithFlags(&sim->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete sim;
      return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    sim->own_stream = true;
  }
  if (dev_buf) {
    sim->base = (char *)dev_buf;
    sim->own_mem = false;
  } else {
    e = cudaMalloc((void **)&sim->base, lay.total);
    if (e != cudaSuccess) {
      if (sim->own_stream) cudaStreamDestroy(sim->stream);
      delete sim;
      cudaGetLastError();
      set_error("cudaMalloc of " + std::to_string(lay.total) + " bytes failed");
      return OKZ_ENOMEM;
    }
    sim->own_mem = true;
  }
  sim->planes[0] = (uint32_t *)(sim->base + lay.off_planes0);
  sim->planes[1] = (uint32_t *)(sim->base + lay.off_planes1);
  sim->hcol = (int64_t *)(sim->base + lay.off_hcol);
  sim->partials = (unsigned long long *)(sim->base + lay.off_partials);
  sim->ctrl = (Ctrl *)(sim->base + lay.off_ctrl);

  e = cudaMemsetAsync(sim->ctrl, 0, sizeof(Ctrl), sim->stream);
  if (e == cudaSuccess) {
    if (sim->parity)  // striped start: h = (x+y) mod 2, so b = 0 everywhere
      e = cudaMemsetAsync(sim->planes[0], 0, lay.planes_bytes / 2, sim->stream);
    else
      e = launch_init_flat(sim->planes[0], prm->L, sim->stream);
  }
  // on a caller's stream the initialisation stays enqueued (stream order covers
  // every later call); on the library's own stream creation waits for it
  if (e == cudaSuccess && sim->own_stream) e = cudaStreamSynchronize(sim->stream);
  if (e != cudaSuccess) {
    okz_status r = cuda_fail(e, "initialisation");
    if (sim->own_mem) cudaFree(sim->base);
    if (sim->own_stream) cudaStreamDestroy(sim->stream);
    delete sim;
    return r;
  }
  *out = sim;
  return OKZ_OK;
}

okz_status okz_create(int64_t L, double p, double q, uint64_t seed, okz_sim **out) {
  okz_params prm;
  okz_params_init(&prm);
  prm.L = L;
  prm.p = p;
  prm.q = q;
  prm.seed = seed;
  return okz_create_ex(&prm, nullptr, 0, nullptr, out);
}

namespace {

// Sweeps replayed per launch of a simulation's sweep graph.
constexpr int64_t kGraphChunk = 32;

// The two half-sweeps of sweep t (t_base set: of sweep t + *t_base) of an
// in-place (plain) kernel.
cudaError_t enqueue_inplace_sweep(okz_sim *sim, uint32_t t, cudaStream_t st,
                                  const unsigned int *t_base) {
  const int64_t L = sim->prm.L;
  cudaError_t e;
  if (sim->parity) {
    e = launch_parity_halfsweep(sim->planes[sim->cur], L, 0, t, sim->prm.seed, sim->acc,
                                sim->ctrl, st, t_base);
    if (e == cudaSuccess)
      e = launch_parity_halfsweep(sim->planes[sim->cur], L, 1, t, sim->prm.seed, sim->acc,
                                  sim->ctrl, st, t_base);
  } else {
    e = launch_halfsweep_plain(sim->planes[sim->cur], L, 0, t, sim->prm.seed, sim->acc,
                               sim->ctrl, st, t_base);
    if (e == cudaSuccess)
      e = launch_halfsweep_plain(sim->planes[sim->cur], L, 1, t, sim->prm.seed, sim->acc,
                                 sim->ctrl, st, t_base);
  }
  return e;
}

// Captures kGraphChunk in-place sweeps (2 launches each, sweep indices read
// from ctrl->t_base) plus the advance of ctrl->t_base into one CUDA graph.
// The graph's pointers are the simulation's own (in-place kernels never swap
// buffers), so it is built once and replayed for every later chunk.
void build_sweep_graph(okz_sim *sim) {
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    sim->graph_state = -1;
    return;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  for (int64_t k = 0; k < kGraphChunk && e == cudaSuccess; ++k)
    e = enqueue_inplace_sweep(sim, (uint32_t)k, cs, &sim->ctrl->t_base);
  if (e == cudaSuccess) e = launch_advance_sweep_counter(sim->ctrl, (uint32_t)kGraphChunk, cs);
  const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&sim->sweep_graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sim->sweep_graph = nullptr;
    sim->graph_state = -1;
    return;
  }
  sim->graph_state = 1;
}

}  // namespace

okz_status okz_sweep(okz_sim *sim, int64_t n) {
  if (!sim || n < 0) {
    set_error("null simulation or negative sweep count");
    return OKZ_EINVAL;
  }
  if ((uint64_t)n > 0xFFFFFFFFull - sim->t) {
    set_error("sweep counter would pass 2^32 - 1");
    return OKZ_EOVERFLOW;
  }
  const int64_t L = sim->prm.L;
  if (sim->kernel == OKZ_KERNEL_PARITY_CTA) {  // every sweep of the call in one launch
    if (n == 0) return OKZ_OK;
    cudaError_t e = launch_cta_sweeps(sim->planes[sim->cur], L, (uint32_t)sim->t, n,
                                      sim->prm.seed, sim->acc, sim->ctrl, sim->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    sim->t += (uint64_t)n;
    return OKZ_OK;
  }
  int64_t done = 0;
  const bool inplace = sim->kernel == OKZ_KERNEL_PLAIN || sim->kernel == OKZ_KERNEL_PARITY_PLAIN;
  if (inplace && n >= kGraphChunk) {  // whole chunks by graph replay
    if (sim->graph_state == 0) build_sweep_graph(sim);
    if (sim->graph_state == 1) {
      cudaError_t e = launch_set_sweep_counter(sim->ctrl, (uint32_t)sim->t, sim->stream);
      const int64_t chunks = n / kGraphChunk;
      for (int64_t c = 0; c < chunks && e == cudaSuccess; ++c)
        e = cudaGraphLaunch(sim->sweep_graph, sim->stream);
      if (e != cudaSuccess) return cuda_fail(e, "sweep graph launch");
      sim->graph_replays += (uint64_t)chunks;
      done = chunks * kGraphChunk;
      sim->t += (uint64_t)done;
    }
  }
  while (done < n) {
    const uint32_t t = (uint32_t)sim->t;
    cudaError_t e;
    int64_t step = 1;
    if (sim->kernel == OKZ_KERNEL_STREAM || sim->kernel == OKZ_KERNEL_PARITY_STREAM) {
      step = (sim->fuse == 2 && n - done >= 2) ? 2 : 1;
      if (sim->parity)
        e = launch_parity_stream(sim->planes[sim->cur], sim->planes[1 - sim->cur], L, t,
                                 sim->prm.seed, sim->acc, sim->wpt, (int)step,
                                 sim->band_rows, sim->ctrl, sim->stream);
      else
        e = launch_sweep_stream(sim->planes[sim->cur], sim->planes[1 - sim->cur], L, t,
                                sim->prm.seed, sim->acc, sim->wpt, (int)step, sim->band_rows,
                                sim->ctrl, sim->stream);
      if (e == cudaSuccess) sim->cur = 1 - sim->cur;
    } else {
      e = enqueue_inplace_sweep(sim, t, sim->stream, nullptr);
    }
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    sim->t += (uint64_t)step;
    done += step;
  }
  return OKZ_OK;
}

okz_status okz_sweep_rs(okz_sim *sim, int64_t n) {
  if (!sim || n < 0) {
    set_error("null simulation or negative sweep count");
    return OKZ_EINVAL;
  }
  if (!sim->parity) {
    set_error("okz_sweep_rs needs a parity-plane simulation (kernel PARITY_PLAIN, "
              "PARITY_STREAM or PARITY_CTA)");
    return OKZ_EUNSUPPORTED;
  }
  if (sim->prm.L % 32 != 0) {
    set_error("okz_sweep_rs needs L % 32 == 0");
    return OKZ_EUNSUPPORTED;
  }
  if ((uint64_t)n > 0xFFFFFFFFull - sim->t) {
    set_error("sweep counter would pass 2^32 - 1");
    return OKZ_EOVERFLOW;
  }
  // 32-bit thresholds, round half to even, no selection factor
  const int mode = std::fegetround();
  std::fesetround(FE_TONEAREST);
  const uint64_t P32 = (uint64_t)std::nearbyint(std::ldexp(sim->prm.p, 32));
  const uint64_t Q32 = (uint64_t)std::nearbyint(std::ldexp(sim->prm.q, 32));
  std::fesetround(mode);
  for (int64_t i = 0; i < n; ++i) {
    cudaError_t e = launch_ddrs(sim->planes[sim->cur], sim->prm.L, (uint32_t)sim->t,
                                sim->prm.seed, P32, Q32, sim->ctrl, sim->stream);
    if (e != cudaSuccess) return cuda_fail(e, "random-sequential sweep launch");
    sim->t += 1;
  }
  return OKZ_OK;
}

static okz_status sync_and_check(okz_sim *sim) {
  cudaError_t e = cudaStreamSynchronize(sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  unsigned int err = 0;
  e = cudaMemcpy(&err, &sim->ctrl->err, sizeof(err), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
  if (err & kErrWaitTimeout) {
    set_error("a bounded device-side wait timed out");
    return OKZ_ETIMEOUT;
  }
  return OKZ_OK;
}

okz_status okz_synchronize(okz_sim *sim) {
  if (!sim) {
    set_error("null simulation");
    return OKZ_EINVAL;
  }
  return sync_and_check(sim);
}

void *okz_stream(okz_sim *sim) { return sim ? (void *)sim->stream : nullptr; }

// Reads back H0 and S_1..S_4 (about H0) once the stream is done.
static okz_status read_sums(okz_sim *sim, long long *H0, __int128 S[4]) {
  cudaError_t e;
  okz_status st = sync_and_check(sim);
  if (st != OKZ_OK) return st;
  Ctrl c;
  e = cudaMemcpy(&c, sim->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading the sums");
  *H0 = c.H0;
  for (int n = 0; n < 4; ++n)
    S[n] = (__int128)(((unsigned __int128)c.sum[2 * n + 1] << 64) |
                      (unsigned __int128)c.sum[2 * n]);
  return OKZ_OK;
}

// Runs the power-sum kernels and reads back H0 and S_1..S_nmom (about H0).
static okz_status power_sums(okz_sim *sim, int nmom, long long *H0, __int128 S[4]) {
  cudaError_t e = launch_power_sums(sim->planes[sim->cur], sim->prm.L, sim->parity, nmom,
                                    sim->hcol, sim->partials, sim->ctrl, sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "power-sum launch");
  return read_sums(sim, H0, S);
}

okz_status okz_width2(okz_sim *sim, okz_i128 *S1, okz_i128 *S2, double *W2) {
  if (!sim) {
    set_error("null simulation");
    return OKZ_EINVAL;
  }
  long long H0 = 0;
  __int128 S[4];
  okz_status st = power_sums(sim, 2, &H0, S);
  if (st != OKZ_OK) return st;
  const __int128 N = (__int128)sim->prm.L * sim->prm.L;
  // W^2 = (N S2 - S1^2) / N^2 with sums about H0 (the numerator is shift-free)
  const __int128 num = N * S[1] - S[0] * S[0];
  const double w2 = (double)num / ((double)N * (double)N);
  // absolute sums: sum h = S1c + N H0, sum h^2 = S2c + 2 H0 S1c + N H0^2
  const __int128 h0 = H0;
  if (S1) *S1 = from_i128(S[0] + N * h0);
  if (S2) *S2 = from_i128(S[1] + 2 * h0 * S[0] + N * h0 * h0);
  if (W2) *W2 = w2;
  return OKZ_OK;
}

okz_status okz_growth_series(okz_sim *sim, int32_t n, const uint64_t *times, okz_i128 *S1,
                             okz_i128 *S2, double *W2, int64_t *H0) {
  if (!sim || n < 0 || (n > 0 && !times)) {
    set_error("okz_growth_series: null simulation, negative count or null times");
    return OKZ_EINVAL;
  }
  for (int32_t i = 0; i < n; ++i) {
    if (times[i] < (i ? times[i - 1] : sim->t)) {
      set_error("okz_growth_series: sample times must ascend from the current sweep count");
      return OKZ_EINVAL;
    }
    if (times[i] > 0xFFFFFFFFull) {
      set_error("sweep counter would pass 2^32 - 1");
      return OKZ_EOVERFLOW;
    }
  }
  if (n == 0) return OKZ_OK;
  // each sample's H0 and sums (the control block's first 80 bytes) are copied
  // aside on the device; one read-back and one synchronisation at the end
  constexpr size_t kRec = offsetof(Ctrl, sum) + sizeof(((Ctrl *)nullptr)->sum);
  void *dev = nullptr;
  cudaError_t e = scratch_alloc(&dev, (size_t)n * kRec, sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "okz_growth_series scratch");
  okz_status st = OKZ_OK;
  for (int32_t i = 0; i < n && st == OKZ_OK && e == cudaSuccess; ++i) {
    st = okz_sweep(sim, (int64_t)(times[i] - sim->t));
    if (st != OKZ_OK) break;
    e = launch_power_sums(sim->planes[sim->cur], sim->prm.L, sim->parity, 2, sim->hcol,
                          sim->partials, sim->ctrl, sim->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char *)dev + (size_t)i * kRec, sim->ctrl, kRec,
                          cudaMemcpyDeviceToDevice, sim->stream);
  }
  std::vector<unsigned char> host((size_t)n * kRec);
  if (st == OKZ_OK && e == cudaSuccess)
    e = cudaMemcpyAsync(host.data(), dev, host.size(), cudaMemcpyDeviceToHost, sim->stream);
  scratch_free(dev, sim->stream);
  if (st != OKZ_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "okz_growth_series");
  st = sync_and_check(sim);
  if (st != OKZ_OK) return st;
  const __int128 N = (__int128)sim->prm.L * sim->prm.L;
  for (int32_t i = 0; i < n; ++i) {
    Ctrl c;
    memcpy(&c, host.data() + (size_t)i * kRec, kRec);
    const __int128 s1 = (__int128)(((unsigned __int128)c.sum[1] << 64) | c.sum[0]);
    const __int128 s2 = (__int128)(((unsigned __int128)c.sum[3] << 64) | c.sum[2]);
    const __int128 h0 = c.H0;
    // as okz_width2: sums about H0, the numerator N S2 - S1^2 shift-free
    if (W2) W2[i] = (double)(N * s2 - s1 * s1) / ((double)N * (double)N);
    if (S1) S1[i] = from_i128(s1 + N * h0);
    if (S2) S2[i] = from_i128(s2 + 2 * h0 * s1 + N * h0 * h0);
    if (H0) H0[i] = c.H0;
  }
  return OKZ_OK;
}

static okz_status moments_check(okz_sim *sim) {
  if (!sim) {
    set_error("null simulation");
    return OKZ_EINVAL;
  }
  if (sim->prm.L > 131072) {
    set_error("okz_moments needs L <= 131072");
    return OKZ_EUNSUPPORTED;
  }
  return OKZ_OK;
}

static okz_status moments_finish(okz_sim *sim, const __int128 S[4], okz_i128 Sk[4],
                                 double *W2, double *skew, double *kurt);

okz_status okz_moments(okz_sim *sim, okz_i128 Sk[4], double *W2, double *skew,
                       double *kurt) {
  okz_status st = moments_check(sim);
  if (st != OKZ_OK) return st;
  long long H0 = 0;
  __int128 S[4];
  st = power_sums(sim, 4, &H0, S);
  if (st != OKZ_OK) return st;
  return moments_finish(sim, S, Sk, W2, skew, kurt);
}

okz_status okz_moments_enqueue(okz_sim *sim) {
  okz_status st = moments_check(sim);
  if (st != OKZ_OK) return st;
  cudaError_t e = launch_power_sums(sim->planes[sim->cur], sim->prm.L, sim->parity, 4,
                                    sim->hcol, sim->partials, sim->ctrl, sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "power-sum launch");
  return OKZ_OK;
}

okz_status okz_moments_fetch(okz_sim *sim, okz_i128 Sk[4], double *W2, double *skew,
                             double *kurt) {
  okz_status st = moments_check(sim);
  if (st != OKZ_OK) return st;
  long long H0 = 0;
  __int128 S[4];
  st = read_sums(sim, &H0, S);
  if (st != OKZ_OK) return st;
  return moments_finish(sim, S, Sk, W2, skew, kurt);
}

static okz_status moments_finish(okz_sim *sim, const __int128 S[4], okz_i128 Sk[4],
                                 double *W2, double *skew, double *kurt) {
  const __int128 N = (__int128)sim->prm.L * sim->prm.L;
  if (Sk)
    for (int n = 0; n < 4; ++n) Sk[n] = from_i128(S[n]);
  if (W2) *W2 = (double)(N * S[1] - S[0] * S[0]) / ((double)N * (double)N);
  const long double n_ = (long double)N;
  const long double mu = (long double)S[0] / n_;
  const long double a2 = (long double)S[1] / n_, a3 = (long double)S[2] / n_,
                    a4 = (long double)S[3] / n_;
  const long double m2 = a2 - mu * mu;
  const long double m3 = a3 - 3.0L * mu * a2 + 2.0L * mu * mu * mu;
  const long double m4 = a4 - 4.0L * mu * a3 + 6.0L * mu * mu * a2 - 3.0L * mu * mu * mu * mu;
  if (skew) *skew = (double)(m3 / powl(m2, 1.5L));
  if (kurt) *kurt = (double)(m4 / (m2 * m2) - 3.0L);
  return OKZ_OK;
}

okz_status okz_heights(okz_sim *sim, int64_t y0, int64_t ny, int32_t *out,
                       int out_is_device) {
  if (!sim || !out || y0 < 0 || ny < 0 || y0 + ny > sim->prm.L) {
    set_error("bad heights request");
    return OKZ_EINVAL;
  }
  if (ny == 0) return OKZ_OK;
  const int64_t L = sim->prm.L;
  const size_t bytes = (size_t)ny * (size_t)L * sizeof(int32_t);
  int32_t *dst = out;
  cudaError_t e;
  if (!out_is_device) {
    e = scratch_alloc((void **)&dst, bytes, sim->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("device staging allocation for heights failed");
      return OKZ_ENOMEM;
    }
  }
  unsigned int zero = 0;
  e = cudaMemcpyAsync(&sim->ctrl->err, &zero, sizeof(zero), cudaMemcpyHostToDevice,
                      sim->stream);
  if (e == cudaSuccess)
    e = launch_heights(sim->planes[sim->cur], L, sim->parity, y0, ny, sim->hcol, dst,
                       sim->ctrl, sim->stream);
  if (e == cudaSuccess && !out_is_device)
    e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, sim->stream);
  if (!out_is_device) scratch_free(dst, sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "heights");
  e = cudaStreamSynchronize(sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "heights synchronize");
  unsigned int err = 0;
  e = cudaMemcpy(&err, &sim->ctrl->err, sizeof(err), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "heights error word");
  if (err & kErrHeightRange) {
    set_error("a height does not fit in int32");
    return OKZ_EOVERFLOW;
  }
  return OKZ_OK;
}

// Profiles (and optionally the axis power spectrum) into host arrays.
static okz_status profiles_and_psd(okz_sim *sim, int64_t *col, int64_t *row, double *S) {
  const int64_t L = sim->prm.L;
  const bool fft = S != nullptr;
  const size_t scratch = psd_scratch_bytes(L, fft);
  const size_t vec = ((size_t)L * sizeof(int64_t) + 255) & ~(size_t)255;
  const size_t bytes = scratch + 3 * vec;
  char *buf = nullptr;
  cudaError_t e = scratch_alloc((void **)&buf, bytes, sim->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device scratch allocation for the profiles failed");
    return OKZ_ENOMEM;
  }
  int64_t *dcol = reinterpret_cast<int64_t *>(buf + scratch);
  int64_t *drow = reinterpret_cast<int64_t *>(buf + scratch + vec);
  double *dS = reinterpret_cast<double *>(buf + scratch + 2 * vec);
  e = launch_profiles(sim->planes[sim->cur], L, sim->parity, buf, dcol, drow, &sim->ctrl->err,
                      sim->stream);
  if (e == cudaSuccess && fft) e = launch_psd(dcol, drow, L, buf, dS, sim->stream);
  if (e == cudaSuccess && col)
    e = cudaMemcpyAsync(col, dcol, (size_t)L * sizeof(int64_t), cudaMemcpyDeviceToHost,
                        sim->stream);
  if (e == cudaSuccess && row)
    e = cudaMemcpyAsync(row, drow, (size_t)L * sizeof(int64_t), cudaMemcpyDeviceToHost,
                        sim->stream);
  if (e == cudaSuccess && fft)
    e = cudaMemcpyAsync(S, dS, (size_t)L * sizeof(double), cudaMemcpyDeviceToHost,
                        sim->stream);
  scratch_free(buf, sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "profiles");
  return sync_and_check(sim);
}

okz_status okz_profiles(okz_sim *sim, int64_t *col, int64_t *row) {
  if (!sim) {
    set_error("null simulation");
    return OKZ_EINVAL;
  }
  return profiles_and_psd(sim, col, row, nullptr);
}

okz_status okz_psd(okz_sim *sim, double *S) {
  if (!sim || !S) {
    set_error("null simulation or output");
    return OKZ_EINVAL;
  }
  const int64_t L = sim->prm.L;
  if ((L & (L - 1)) != 0) {
    set_error("okz_psd needs a power-of-two L");
    return OKZ_EUNSUPPORTED;
  }
  return profiles_and_psd(sim, nullptr, nullptr, S);
}

okz_status okz_state(okz_sim *sim, uint32_t *planes_out, int out_is_device, int64_t *H0,
                     uint64_t *t) {
  if (!sim) {
    set_error("null simulation");
    return OKZ_EINVAL;
  }
  cudaError_t e = cudaSuccess;
  if (planes_out) {
    const uint32_t *slopes = sim->planes[sim->cur];
    if (sim->parity) {  // convert into the idle ping-pong buffer, then copy out
      if (out_is_device) {
        e = launch_to_slopes(sim->planes[sim->cur], sim->prm.L, planes_out, sim->stream);
        slopes = nullptr;
      } else {
        e = launch_to_slopes(sim->planes[sim->cur], sim->prm.L, sim->planes[1 - sim->cur],
                             sim->stream);
        slopes = sim->planes[1 - sim->cur];
      }
    }
    if (e == cudaSuccess && slopes)
      e = cudaMemcpyAsync(planes_out, slopes, sim->lay.planes_bytes,
                          out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          sim->stream);
  }
  long long h0 = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h0, &sim->ctrl->H0, sizeof(h0), cudaMemcpyDeviceToHost, sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "state copy");
  okz_status st = sync_and_check(sim);
  if (st != OKZ_OK) return st;
  if (H0) *H0 = h0;
  if (t) *t = sim->t;
  return OKZ_OK;
}

okz_status okz_restore(okz_sim *sim, const uint32_t *planes, int in_is_device, int64_t H0,
                       uint64_t t) {
  if (!sim || !planes || t > 0xFFFFFFFFull) {
    set_error("bad restore request");
    return OKZ_EINVAL;
  }
  if (H0 & 1) {
    set_error("H0 = h(0,0) must be even (h(x,y) == x + y mod 2)");
    return OKZ_EINVAL;
  }
  long long h0 = H0;
  // parity plane: stage the slopes in the idle ping-pong buffer, then convert
  uint32_t *landing = sim->parity ? sim->planes[1 - sim->cur] : sim->planes[sim->cur];
  cudaError_t e = cudaMemcpyAsync(landing, planes, sim->lay.planes_bytes,
                                  in_is_device ? cudaMemcpyDeviceToDevice
                                               : cudaMemcpyHostToDevice,
                                  sim->stream);
  if (e == cudaSuccess && sim->parity)
    e = launch_from_slopes(landing, sim->prm.L, h0, sim->hcol, sim->planes[sim->cur],
                           sim->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&sim->ctrl->H0, &h0, sizeof(h0), cudaMemcpyHostToDevice, sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "restore copy");
  e = cudaStreamSynchronize(sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "restore synchronize");
  sim->t = t;
  return OKZ_OK;
}

okz_status okz_stage_host(okz_sim *sim, const uint32_t *planes) {
  if (!sim || !planes) {
    set_error("okz_stage_host: null simulation or planes");
    return OKZ_EINVAL;
  }
  cudaError_t e = cudaSuccess;
  if (!sim->stage_buf) {
    e = cudaMalloc((void **)&sim->stage_buf, sim->lay.planes_bytes);
    if (e != cudaSuccess) {
      sim->stage_buf = nullptr;
      cudaGetLastError();
      set_error("okz_stage_host: cannot allocate the staging buffer");
      return OKZ_ENOMEM;
    }
    e = cudaStreamCreateWithFlags(&sim->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sim->staged_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sim->consumed_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(sim->consumed_ev, sim->stream);
    if (e != cudaSuccess) return cuda_fail(e, "okz_stage_host set-up");
  }
  // the previous staged planes must have been converted before they are overwritten
  e = cudaStreamWaitEvent(sim->copy_stream, sim->consumed_ev, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sim->stage_buf, planes, sim->lay.planes_bytes, cudaMemcpyHostToDevice,
                        sim->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(sim->staged_ev, sim->copy_stream);
  if (e != cudaSuccess) return cuda_fail(e, "okz_stage_host copy");
  sim->stage_pending = true;
  return OKZ_OK;
}

okz_status okz_restore_staged(okz_sim *sim, int64_t H0, uint64_t t) {
  if (!sim || t > 0xFFFFFFFFull) {
    set_error("bad restore request");
    return OKZ_EINVAL;
  }
  if (!sim->stage_pending) {
    set_error("okz_restore_staged: nothing staged (okz_stage_host first)");
    return OKZ_EINVAL;
  }
  if (H0 & 1) {
    set_error("H0 = h(0,0) must be even (h(x,y) == x + y mod 2)");
    return OKZ_EINVAL;
  }
  long long h0 = H0;
  cudaError_t e = cudaStreamWaitEvent(sim->stream, sim->staged_ev, 0);
  if (e == cudaSuccess) {
    if (sim->parity)
      e = launch_from_slopes(sim->stage_buf, sim->prm.L, h0, sim->hcol, sim->planes[sim->cur],
                             sim->stream);
    else
      e = cudaMemcpyAsync(sim->planes[sim->cur], sim->stage_buf, sim->lay.planes_bytes,
                          cudaMemcpyDeviceToDevice, sim->stream);
  }
  // a pageable source: the value is taken before the call returns
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&sim->ctrl->H0, &h0, sizeof(h0), cudaMemcpyHostToDevice, sim->stream);
  if (e == cudaSuccess) e = cudaEventRecord(sim->consumed_ev, sim->stream);
  if (e != cudaSuccess) return cuda_fail(e, "okz_restore_staged");
  sim->stage_pending = false;
  sim->t = t;
  return OKZ_OK;
}

okz_status okz_get_info(okz_sim *sim, okz_info *info) {
  if (!sim || !info) {
    set_error("null argument");
    return OKZ_EINVAL;
  }
  int64_t H0 = 0;
  okz_status st = okz_state(sim, nullptr, 0, &H0, nullptr);
  if (st != OKZ_OK) return st;
  info->L = sim->prm.L;
  info->graph_chunk = sim->graph_state == 1 ? (int32_t)kGraphChunk : 0;
  info->graph_replays = sim->graph_replays;
  info->t = sim->t;
  info->H0 = H0;
  info->k = sim->acc.k;
  info->kernel = sim->kernel;
  info->P = sim->acc.P;
  info->Q = sim->acc.Q;
  info->device_bytes = sim->lay.total + (sim->stage_buf ? sim->lay.planes_bytes : 0);
  info->words_per_thread = sim->wpt;
  info->sweeps_per_pass = sim->fuse;
  info->band_rows = sim->band_rows;
  return OKZ_OK;
}

okz_status okz_tune_stream(const okz_params *prm, int32_t probe_sweeps, int32_t *wpt_out,
                           int32_t *fuse_out, int32_t *band_out, double *ms_per_sweep) {
  if (!prm || probe_sweeps < 2) {
    set_error("okz_tune_stream: null parameters or probe_sweeps < 2");
    return OKZ_EINVAL;
  }
  okz_status st = check_L(prm->L);
  if (st != OKZ_OK) return st;
  int32_t k;
  uint64_t P, Q;
  st = okz_thresholds(prm->p, prm->q, prm->s_sel, prm->k_max, &k, &P, &Q);
  if (st != OKZ_OK) return st;
  int kernel = prm->kernel;
  if (kernel == OKZ_KERNEL_AUTO && stream_kernel_supports(prm->L)) kernel = OKZ_KERNEL_PARITY_STREAM;
  if ((kernel != OKZ_KERNEL_STREAM && kernel != OKZ_KERNEL_PARITY_STREAM) ||
      !stream_kernel_supports(prm->L)) {
    set_error("okz_tune_stream: the stream kernels need L % 4096 == 0 and L <= 131072");
    return OKZ_EUNSUPPORTED;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  double best = 1e300;
  int bw = 0, bf = 0, bb = 0;
  const int wpts[3] = {4, 8, 16}, bands[3] = {0, 16, 32};
  for (int wi = 0; wi < 3; ++wi)
    for (int f = 1; f <= 2; ++f)
      for (int bi = 0; bi < 3; ++bi) {
        const int w = wpts[wi];
        const bool ok = kernel == OKZ_KERNEL_PARITY_STREAM ? parity_wpt_valid(prm->L, w)
                                                           : stream_wpt_valid(prm->L, w);
        if (!ok || (bands[bi] != 0 && bands[bi] < stream_min_band(f))) continue;
        okz_params q = *prm;
        q.kernel = kernel;
        q.words_per_thread = w;
        q.sweeps_per_pass = f;
        q.band_rows = bands[bi];
        okz_sim *sim = nullptr;
        st = okz_create_ex(&q, nullptr, 0, nullptr, &sim);
        if (st != OKZ_OK) return st;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        float ms = 0.0f;
        if (e == cudaSuccess) {
          // past the striped start (its first sweeps move every site), then timed
          okz_status s2 = okz_sweep(sim, 4);
          if (s2 == OKZ_OK) e = cudaEventRecord(e0, sim->stream);
          if (s2 == OKZ_OK && e == cudaSuccess) s2 = okz_sweep(sim, probe_sweeps);
          if (s2 == OKZ_OK && e == cudaSuccess) e = cudaEventRecord(e1, sim->stream);
          if (s2 == OKZ_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
          if (s2 == OKZ_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (s2 != OKZ_OK) st = s2;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        const okz_status s3 = sync_and_check(sim);
        okz_destroy(sim);
        if (st != OKZ_OK) return st;
        if (e != cudaSuccess) return cuda_fail(e, "okz_tune_stream timing");
        if (s3 != OKZ_OK) return s3;
        const double per = ms / probe_sweeps;
        if (per < best) {
          best = per;
          bw = w;
          bf = f;
          bb = bands[bi];
        }
      }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[TuneKey{dev, prm->L, kernel, stream_mode(k, P, Q)}] = Tiling{bw, bf, bb};
  }
  if (wpt_out) *wpt_out = bw;
  if (fuse_out) *fuse_out = bf;
  if (band_out) *band_out = bb;
  if (ms_per_sweep) *ms_per_sweep = best;
  return OKZ_OK;
}

okz_status okz_destroy(okz_sim *sim) {
  if (!sim) return OKZ_OK;
  cudaError_t e = cudaStreamSynchronize(sim->stream);
  if (sim->copy_stream) {
    cudaError_t e2 = cudaStreamSynchronize(sim->copy_stream);
    if (e == cudaSuccess) e = e2;
    cudaStreamDestroy(sim->copy_stream);
  }
  if (sim->staged_ev) cudaEventDestroy(sim->staged_ev);
  if (sim->consumed_ev) cudaEventDestroy(sim->consumed_ev);
  if (sim->stage_buf) cudaFree(sim->stage_buf);
  if (sim->sweep_graph) cudaGraphExecDestroy(sim->sweep_graph);
  if (sim->own_mem) cudaFree(sim->base);
  if (sim->own_stream) cudaStreamDestroy(sim->stream);
  delete sim;
  if (e != cudaSuccess) return cuda_fail(e, "destroy synchronize");
  return OKZ_OK;
}

}  // extern "C"
