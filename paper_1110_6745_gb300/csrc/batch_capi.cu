// batch_capi.cu -- okz_batch_*: a slot table of independent lattices in one
// device arena, driven by one graph-captured persistent launch per run.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "okz_batch_internal.h"

namespace {

struct HostSlot {
  bool active = false;
  int64_t L = 0;
  size_t offset = 0;  // bytes into the arena
  size_t bytes = 0;
  double p = 0, q = 0;
  uint64_t seed = 0;
};

size_t lattice_bytes(int64_t L) { return (((size_t)L * (size_t)L / 8) + 255) & ~(size_t)255; }

}  // namespace

struct okz_batch {
  int max_slots = 0;
  double s_sel = 0.5;
  int32_t k_max = 32;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  std::map<size_t, size_t> free_list;  // offset -> size (bytes), coalesced
  std::vector<HostSlot> slots;
  okz::SlotDesc *d_slots = nullptr;
  okz::WorkTable *d_work = nullptr;
  okz::WorkTable *h_work = nullptr;  // pinned
  unsigned int *d_head = nullptr;
  int threads = 512;
  size_t smem = 32 * 1024;
  int grid = 0;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;
};

using namespace okz;

namespace {

okz_status arena_alloc(okz_batch *b, size_t bytes, size_t *off) {
  for (auto it = b->free_list.begin(); it != b->free_list.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes, at = it->first + bytes;
      b->free_list.erase(it);
      if (rest) b->free_list[at] = rest;
      return OKZ_OK;
    }
  }
  return OKZ_EBUSY;
}

void arena_free(okz_batch *b, size_t off, size_t bytes) {
  auto it = b->free_list.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != b->free_list.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    b->free_list.erase(nx);
  }
  if (it != b->free_list.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      b->free_list.erase(it);
    }
  }
}

void plan_grid(okz_batch *b) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = batch_occupancy(b->threads, b->smem);
  if (per_sm < 1) per_sm = 1;
  b->grid = sms * per_sm;
}

void drop_graph(okz_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->graph_ok = false;
}

// Capture: upload the work table, reset the queue head, run the kernel.
okz_status build_graph(okz_batch *b) {
  drop_graph(b);
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "capture stream");
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_work, b->h_work, work_table_bytes(b->max_slots),
                        cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = launch_batch_sweeps((uint32_t *)b->arena, b->d_slots, b->d_work, b->d_head, b->grid,
                            b->threads, b->smem, cs);
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
  b->graph_ok = true;
  return OKZ_OK;
}

}  // namespace

extern "C" {

okz_status okz_pool_create(size_t arena_bytes, int32_t max_slots, double s_sel, int32_t k_max,
                           void *stream, okz_batch **out) {
  if (!out || max_slots < 1 || arena_bytes < 256 || !(s_sel > 0 && s_sel <= 1) || k_max < 1 ||
      k_max > 32) {
    set_error("okz_pool_create: bad arguments");
    return OKZ_EINVAL;
  }
  okz_batch *b = new (std::nothrow) okz_batch();
  if (!b) {
    set_error("host allocation failed");
    return OKZ_ENOMEM;
  }
  b->max_slots = max_slots;
  b->s_sel = s_sel;
  b->k_max = k_max;
  b->arena_bytes = (arena_bytes + 255) & ~(size_t)255;
  b->slots.resize(max_slots);
  cudaError_t e = cudaSuccess;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->arena, b->arena_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_slots, sizeof(SlotDesc) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_work, work_table_bytes(max_slots));
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_head, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_work, work_table_bytes(max_slots));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_slots, 0, sizeof(SlotDesc) * max_slots, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    okz_status r = (e == cudaErrorMemoryAllocation) ? OKZ_ENOMEM : cuda_fail(e, "okz_pool_create");
    if (r == OKZ_ENOMEM) set_error("device allocation for the batch arena failed");
    cudaGetLastError();
    cudaFree(b->arena);
    cudaFree(b->d_slots);
    cudaFree(b->d_work);
    cudaFree(b->d_head);
    cudaFreeHost(b->h_work);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return r;
  }
  b->free_list[0] = b->arena_bytes;
  b->h_work->count = 0;
  plan_grid(b);
  *out = b;
  return OKZ_OK;
}

okz_status okz_batch_add(okz_batch *b, int64_t L, double p, double q, uint64_t seed,
                         int32_t *slot_out) {
  if (!b || !slot_out) {
    set_error("null argument");
    return OKZ_EINVAL;
  }
  if (L < 32 || (L % 32) != 0 || L > kBatchMaxL) {
    set_error("batch slots need L % 32 == 0 and 32 <= L <= 8192");
    return (L < 2 || (L & 1)) ? OKZ_EINVAL : OKZ_EUNSUPPORTED;
  }
  int32_t k;
  uint64_t P, Q;
  okz_status st = okz_thresholds(p, q, b->s_sel, b->k_max, &k, &P, &Q);
  if (st != OKZ_OK) return st;
  int slot = -1;
  for (int i = 0; i < b->max_slots; ++i)
    if (!b->slots[i].active) {
      slot = i;
      break;
    }
  if (slot < 0) {
    set_error("no free slot");
    return OKZ_EBUSY;
  }
  const size_t bytes = lattice_bytes(L);
  size_t off = 0;
  if (arena_alloc(b, bytes, &off) != OKZ_OK) {
    set_error("no arena space for this lattice");
    return OKZ_EBUSY;
  }
  SlotDesc d{};
  d.seed = seed;
  d.P = P;
  d.Q = Q;
  d.k = k;
  d.L = (int32_t)L;
  d.t = 0;
  d.active = 1;
  d.offset_words = off / 4;
  d.H0 = 0;
  cudaError_t e = cudaMemsetAsync(b->arena + off, 0, bytes, b->stream);  // striped start: b = 0
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&b->d_slots[slot], &d, sizeof(d), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    arena_free(b, off, bytes);
    return cuda_fail(e, "okz_batch_add");
  }
  HostSlot &h = b->slots[slot];
  h.active = true;
  h.L = L;
  h.offset = off;
  h.bytes = bytes;
  h.p = p;
  h.q = q;
  h.seed = seed;
  *slot_out = slot;
  return OKZ_OK;
}

okz_status okz_batch_remove(okz_batch *b, int32_t slot) {
  if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].active) {
    set_error("okz_batch_remove: no such active slot");
    return OKZ_EINVAL;
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);  // its lattice may still be in use
  if (e != cudaSuccess) return cuda_fail(e, "okz_batch_remove");
  HostSlot &h = b->slots[slot];
  arena_free(b, h.offset, h.bytes);
  h = HostSlot();
  unsigned int zero = 0;
  e = cudaMemcpyAsync(&b->d_slots[slot].active, &zero, sizeof(zero), cudaMemcpyHostToDevice,
                      b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "okz_batch_remove");
  return OKZ_OK;
}

okz_status okz_batch_create(int32_t n, const int64_t *L, const double *p, const double *q,
                            const uint64_t *seed, okz_batch **out) {
  if (n < 1 || !L || !p || !q || !seed || !out) {
    set_error("okz_batch_create: bad arguments");
    return OKZ_EINVAL;
  }
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    if (L[i] < 32 || (L[i] % 32) != 0 || L[i] > kBatchMaxL) {
      set_error("batch slots need L % 32 == 0 and 32 <= L <= 8192");
      return (L[i] < 2 || (L[i] & 1)) ? OKZ_EINVAL : OKZ_EUNSUPPORTED;
    }
    total += lattice_bytes(L[i]);
  }
  okz_batch *b = nullptr;
  okz_status st = okz_pool_create(total, n, 0.5, 32, nullptr, &b);
  if (st != OKZ_OK) return st;
  for (int i = 0; i < n; ++i) {
    int32_t slot;
    st = okz_batch_add(b, L[i], p[i], q[i], seed[i], &slot);
    if (st != OKZ_OK) {
      okz_batch_destroy(b);
      return st;
    }
  }
  *out = b;
  return OKZ_OK;
}

okz_status okz_batch_run(okz_batch *b, const int64_t *sweeps) {
  if (!b || !sweeps) {
    set_error("null argument");
    return OKZ_EINVAL;
  }
  // the pinned table is read by the previous graph launch until it finishes
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "okz_batch_run");
  std::vector<std::pair<double, int>> order;
  for (int i = 0; i < b->max_slots; ++i) {
    if (sweeps[i] < 0) {
      set_error("negative sweep count");
      return OKZ_EINVAL;
    }
    if (sweeps[i] == 0) continue;
    if (!b->slots[i].active) {
      set_error("sweeps requested for an empty slot");
      return OKZ_EINVAL;
    }
    if (sweeps[i] > 0x7FFFFFFF) {
      set_error("at most 2^31 - 1 sweeps per slot and run");
      return OKZ_EOVERFLOW;
    }
    const double cost = (double)b->slots[i].L * (double)b->slots[i].L * (double)sweeps[i];
    order.emplace_back(-cost, i);
  }
  std::sort(order.begin(), order.end());  // longest first: balances the queue
  b->h_work->count = (int32_t)order.size();
  for (size_t j = 0; j < order.size(); ++j) {
    b->h_work->item[j].slot = order[j].second;
    b->h_work->item[j].sweeps = (int32_t)sweeps[order[j].second];
  }
  if (order.empty()) return OKZ_OK;
  if (!b->graph_ok) {
    okz_status st = build_graph(b);
    if (st != OKZ_OK) return st;
  }
  e = cudaGraphLaunch(b->exec, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
  return OKZ_OK;
}

okz_status okz_batch_sync(okz_batch *b) {
  if (!b) {
    set_error("null batch");
    return OKZ_EINVAL;
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "okz_batch_sync");
  return OKZ_OK;
}

// Exact sums of the listed slots (all active slots when list is empty), read
// back to `out` (max_slots descriptors).
static okz_status batch_sums(okz_batch *b, std::vector<SlotDesc> &out,
                             const std::vector<int> &list = {}) {
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch sums");
  int n = 0;
  int64_t max_L = 32;
  for (int i = 0; i < b->max_slots; ++i) {
    const int slot = list.empty() ? i : (i < (int)list.size() ? list[i] : -1);
    if (slot < 0) break;
    if (!b->slots[slot].active) continue;
    b->h_work->item[n].slot = slot;
    b->h_work->item[n].sweeps = 0;
    max_L = std::max(max_L, b->slots[slot].L);
    ++n;
  }
  b->h_work->count = n;
  e = cudaMemcpyAsync(b->d_work, b->h_work, work_table_bytes(b->max_slots),
                      cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = launch_batch_moments((const uint32_t *)b->arena, b->d_slots, b->d_work, n, max_L,
                             b->stream);
  out.resize(b->max_slots);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out.data(), b->d_slots, sizeof(SlotDesc) * b->max_slots,
                        cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch sums");
  return OKZ_OK;
}

okz_status okz_batch_stats(okz_batch *b, double *W2, double *skew, double *kurt) {
  if (!b) {
    set_error("null batch");
    return OKZ_EINVAL;
  }
  std::vector<SlotDesc> d;
  okz_status st = batch_sums(b, d);
  if (st != OKZ_OK) return st;
  for (int i = 0; i < b->max_slots; ++i) {
    double w = NAN, sk = NAN, ku = NAN;
    if (b->slots[i].active) {
      __int128 S[4];
      for (int n = 0; n < 4; ++n)
        S[n] = (__int128)(((unsigned __int128)d[i].sum[2 * n + 1] << 64) |
                          (unsigned __int128)d[i].sum[2 * n]);
      const __int128 N = (__int128)d[i].L * d[i].L;
      w = (double)(N * S[1] - S[0] * S[0]) / ((double)N * (double)N);
      const long double nn = (long double)N;
      const long double mu = (long double)S[0] / nn;
      const long double a2 = (long double)S[1] / nn, a3 = (long double)S[2] / nn,
                        a4 = (long double)S[3] / nn;
      const long double m2 = a2 - mu * mu;
      const long double m3 = a3 - 3.0L * mu * a2 + 2.0L * mu * mu * mu;
      const long double m4 = a4 - 4.0L * mu * a3 + 6.0L * mu * mu * a2 - 3.0L * mu * mu * mu * mu;
      sk = (double)(m3 / powl(m2, 1.5L));
      ku = (double)(m4 / (m2 * m2) - 3.0L);
    }
    if (W2) W2[i] = w;
    if (skew) skew[i] = sk;
    if (kurt) kurt[i] = ku;
  }
  return OKZ_OK;
}

okz_status okz_batch_sums(okz_batch *b, int32_t slot, okz_i128 Sk[4], int64_t *H0,
                          uint64_t *t) {
  if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].active) {
    set_error("okz_batch_sums: no such active slot");
    return OKZ_EINVAL;
  }
  std::vector<SlotDesc> d;
  okz_status st = batch_sums(b, d, {slot});
  if (st != OKZ_OK) return st;
  if (Sk)
    for (int n = 0; n < 4; ++n) {
      Sk[n].lo = d[slot].sum[2 * n];
      Sk[n].hi = (int64_t)d[slot].sum[2 * n + 1];
    }
  if (H0) *H0 = d[slot].H0;
  if (t) *t = d[slot].t;
  return OKZ_OK;
}

okz_status okz_batch_measure(okz_batch *b, int32_t n, const int32_t *slots, okz_i128 *Sk,
                             int64_t *H0, uint64_t *t) {
  if (!b || n < 0 || (n > 0 && !slots) || n > b->max_slots) {
    set_error("okz_batch_measure: bad arguments");
    return OKZ_EINVAL;
  }
  std::vector<int> list(slots, slots + n);
  for (int s : list)
    if (s < 0 || s >= b->max_slots || !b->slots[s].active) {
      set_error("okz_batch_measure: no such active slot");
      return OKZ_EINVAL;
    }
  if (n == 0) return OKZ_OK;
  std::vector<SlotDesc> d;
  okz_status st = batch_sums(b, d, list);
  if (st != OKZ_OK) return st;
  for (int j = 0; j < n; ++j) {
    const SlotDesc &x = d[list[j]];
    if (Sk)
      for (int m = 0; m < 4; ++m) {
        Sk[4 * j + m].lo = x.sum[2 * m];
        Sk[4 * j + m].hi = (int64_t)x.sum[2 * m + 1];
      }
    if (H0) H0[j] = x.H0;
    if (t) t[j] = x.t;
  }
  return OKZ_OK;
}

okz_status okz_batch_state(okz_batch *b, int32_t slot, uint32_t *planes_out, int64_t *H0,
                           uint64_t *t) {
  if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].active) {
    set_error("okz_batch_state: no such active slot");
    return OKZ_EINVAL;
  }
  const HostSlot &h = b->slots[slot];
  const size_t out_bytes = (size_t)h.L * (size_t)h.L / 4;
  uint32_t *tmp = nullptr;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = scratch_alloc((void **)&tmp, out_bytes, b->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("staging allocation for okz_batch_state failed");
    return OKZ_ENOMEM;
  }
  SlotDesc d;
  e = launch_to_slopes((const uint32_t *)(b->arena + h.offset), h.L, tmp, b->stream);
  if (e == cudaSuccess && planes_out)
    e = cudaMemcpyAsync(planes_out, tmp, out_bytes, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&d, &b->d_slots[slot], sizeof(d), cudaMemcpyDeviceToHost, b->stream);
  scratch_free(tmp, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "okz_batch_state");
  if (H0) *H0 = d.H0;
  if (t) *t = d.t;
  return OKZ_OK;
}

okz_status okz_batch_set_tiling(okz_batch *b, int32_t threads, size_t smem_bytes) {
  if (!b || (threads != 256 && threads != 512 && threads != 1024) || smem_bytes > 200 * 1024 ||
      (smem_bytes & 15)) {
    set_error("threads must be 256, 512 or 1024 and smem_bytes <= 200 KiB, a multiple of 16");
    return OKZ_EINVAL;
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "okz_batch_set_tiling");
  if (batch_occupancy(threads, smem_bytes) < 1) {
    set_error("tiling does not fit on an SM");
    return OKZ_EINVAL;
  }
  b->threads = threads;
  b->smem = smem_bytes;
  plan_grid(b);
  drop_graph(b);
  return OKZ_OK;
}

okz_status okz_batch_get_tiling(okz_batch *b, int32_t *threads, size_t *smem_bytes,
                                int32_t *grid) {
  if (!b) {
    set_error("null batch");
    return OKZ_EINVAL;
  }
  if (threads) *threads = b->threads;
  if (smem_bytes) *smem_bytes = b->smem;
  if (grid) *grid = b->grid;
  return OKZ_OK;
}

// Autotuner: time each tiling on a scratch pool with the same lattice sizes
// (fresh lattices, `probe_sweeps` sweeps each) and keep the fastest. Results
// are bit-identical for every tiling, so tuning never changes a result.
okz_status okz_batch_autotune(okz_batch *b, int32_t probe_sweeps) {
  if (!b || probe_sweeps < 1) {
    set_error("okz_batch_autotune: bad arguments");
    return OKZ_EINVAL;
  }
  std::vector<int> idx;
  size_t need = 0;
  for (int i = 0; i < b->max_slots; ++i)
    if (b->slots[i].active) {
      idx.push_back(i);
      need += b->slots[i].bytes;
    }
  if (idx.empty()) return OKZ_OK;
  okz_batch *s = nullptr;
  okz_status st = okz_pool_create(need, (int32_t)idx.size(), b->s_sel, b->k_max, nullptr, &s);
  if (st != OKZ_OK) return st;
  std::vector<int64_t> sw(idx.size(), probe_sweeps);
  for (int i : idx) {
    int32_t slot;
    st = okz_batch_add(s, b->slots[i].L, b->slots[i].p, b->slots[i].q, b->slots[i].seed, &slot);
    if (st != OKZ_OK) {
      okz_batch_destroy(s);
      return st;
    }
  }
  const int thr[3] = {256, 512, 1024};
  const size_t sm[3] = {32 * 1024, 64 * 1024, 128 * 1024};
  double best = 1e300;
  int bt = b->threads;
  size_t bs = b->smem;
  for (int ti = 0; ti < 3; ++ti)
    for (int si = 0; si < 3; ++si) {
      if (okz_batch_set_tiling(s, thr[ti], sm[si]) != OKZ_OK) continue;
      if (okz_batch_run(s, sw.data()) != OKZ_OK) continue;  // warm-up (and capture)
      okz_batch_sync(s);
      const auto t0 = std::chrono::steady_clock::now();
      okz_batch_run(s, sw.data());
      if (okz_batch_sync(s) != OKZ_OK) continue;
      const double dt =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (dt < best) {
        best = dt;
        bt = thr[ti];
        bs = sm[si];
      }
    }
  okz_batch_destroy(s);
  return okz_batch_set_tiling(b, bt, bs);
}

okz_status okz_batch_destroy(okz_batch *b) {
  if (!b) return OKZ_OK;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  drop_graph(b);
  cudaFree(b->arena);
  cudaFree(b->d_slots);
  cudaFree(b->d_work);
  cudaFree(b->d_head);
  cudaFreeHost(b->h_work);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  if (e != cudaSuccess) return cuda_fail(e, "okz_batch_destroy");
  return OKZ_OK;
}

void *okz_batch_stream(okz_batch *b) { return b ? (void *)b->stream : nullptr; }

}  // extern "C"
