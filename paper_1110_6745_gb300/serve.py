"""Continuous batching of simulation requests on one GPU (host loop only).

A request asks for one lattice (L, p, q, seed) run for `budget` sweeps from the
striped start, and gets back its exact sums and W^2 (Sec. I, Eq. (4)). The
loop admits arrived requests whenever a slot and device memory are free, so
requests that arrive while others run join at the next tick:

* L <= 2048: a slot of an okz_batch pool (the arena is the HBM budget for
  small lattices); every tick advances all active slots in one
  graph-captured persistent launch, each by about the site updates of
  `tick_sweeps` sweeps of an L = 2048 lattice (so the tick's CTAs work about
  equally long and small lattices finish in few ticks);
* L >= 4096: a simulation of its own (parity-plane stream kernel) on its own
  CUDA stream, admitted while its okz_device_bytes fit in the large-lattice
  budget and a stream is free. Its budget is enqueued in chunks of about
  `chunk_attempts` site updates, at most `ahead` chunks in flight, each
  closed by an event, so the stream never drains while the host loop runs
  and the host never blocks on a full launch queue; its exact sums are
  enqueued behind the last chunk (okz_moments_enqueue) and read once their
  event has fired.

The loop never waits on the device: the batched launch is also closed by an
event and its slots are retired, and new small requests admitted, when that
event has fired. Both kinds run concurrently on the device. Every request
evolves exactly as it would alone (same counter-based random stream), which
tests check. All arithmetic runs in the CUDA library; this module only
schedules.
"""
import dataclasses
import time
from collections import deque

import numpy as np

import paper_1110_6745_gb300 as okz


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float  # seconds after the start of the session
    L: int
    p: float
    q: float
    seed: int
    budget: int


@dataclasses.dataclass
class Result:
    rid: int
    Sk: list        # exact sums of (h - H0)^n, n = 1..4
    H0: int
    W2: float
    admitted: float
    finished: float
    latency: float  # finished - arrival


def poisson_requests(n=10000, rate=200.0, seed=2027, log_budget=(2.0, 4.0), exponents=(7, 13)):
    """The served workload: Poisson arrivals at `rate`/s, L = 2^e with
    e ~ U{exponents}, p ~ U{1.0, 0.75, 0.5}, q = 1 - p, budget =
    round(10^U(log_budget)) sweeps, numpy PCG64 seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    e = rng.integers(exponents[0], exponents[1] + 1, size=n)
    p = rng.choice(np.array([1.0, 0.75, 0.5]), size=n)
    budgets = np.round(10.0 ** rng.uniform(log_budget[0], log_budget[1], size=n)).astype(np.int64)
    return [Request(i, float(arrivals[i]), int(1 << e[i]), float(p[i]), float(1.0 - p[i]),
                    5000 + i, int(max(1, budgets[i]))) for i in range(n)]


class Server:
    def __init__(self, small_arena_bytes=1 << 31, max_slots=1024, large_bytes=8 << 30,
                 max_large=16, tick_sweeps=128, large_threshold=4096, chunk_attempts=2e10,
                 ahead=2, max_chunk_sweeps=256, equal_ticks=True, large_band_rows=16):
        import torch
        self._torch = torch
        # the pool's stream has the higher priority: its short synchronous
        # steps (admission, exact sums) then do not queue behind the large
        # lattices' kernels
        self.pool_stream = torch.cuda.Stream(priority=-1)
        self.pool = okz.Batch(arena_bytes=small_arena_bytes, max_slots=max_slots,
                              stream=self.pool_stream.cuda_stream)
        self.small_event = None
        self.max_slots = max_slots
        self.tick_sweeps = int(tick_sweeps)
        # equal_ticks: every slot gets about the site updates of tick_sweeps
        # sweeps of an L = 2048 lattice per tick, so a tick's CTAs work about
        # equally long and small lattices finish in few ticks
        self.equal_ticks = bool(equal_ticks)
        self.tick_attempts = float(tick_sweeps) * 2048.0 ** 2
        self.large_threshold = int(large_threshold)
        # band height of the large lattices' stream kernels. The library's
        # automatic height (0) makes one lattice fill the GPU with short
        # bands; the server runs several at once, where taller bands stream
        # fewer halo rows (measured on the served mix: 0 / 32 / 16 rows ->
        # 5.06 / 5.25 / 5.26e12 attempts/s, p99 3.9 / 2.4 / 1.9 s)
        self.large_band_rows = int(large_band_rows)
        self.large_bytes = int(large_bytes)
        self.large_used = 0
        self.max_large = int(max_large)
        self.chunk_attempts = float(chunk_attempts)
        self.ahead = int(ahead)
        self.max_chunk_sweeps = int(max_chunk_sweeps)
        self.streams = [torch.cuda.Stream() for _ in range(self.max_large)]
        self.free_streams = list(range(self.max_large))
        self.queue = deque()
        self.small = {}   # slot -> [request, remaining, admitted]
        self.large = {}   # rid -> _Large
        self.results = {}
        self.attempts = 0.0

    def tune(self, classes):
        """Autotunes the stream kernels (okz_tune_stream) once for every
        large-lattice class (L, p, q) the session will see, before it starts:
        the simulations admitted later pick the measured best tiling up."""
        done = {}
        for L, p, q in classes:
            if L >= self.large_threshold and (L, p, q) not in done:
                done[(L, p, q)] = okz.okz_tune_stream(L, p, q, probe_sweeps=8)
        return {"%d,%g,%g" % k: list(v[:3]) for k, v in done.items()}

    # -- admission ----------------------------------------------------------
    def _admit(self, now, small_ok):
        blocked = deque()
        while self.queue:
            r = self.queue.popleft()
            if r.L >= self.large_threshold:
                nbytes = okz.okz_device_bytes(r.L)
                if self.free_streams and self.large_used + nbytes <= self.large_bytes:
                    si = self.free_streams.pop()
                    # device memory from torch's caching allocator, tied to the
                    # request's stream: creating and closing a simulation then
                    # never calls cudaMalloc / cudaFree, which would stall the
                    # other streams
                    with self._torch.cuda.stream(self.streams[si]):
                        sim = okz.Simulation(r.L, r.p, r.q, seed=r.seed,
                                             kernel=okz.OKZ_KERNEL_PARITY_STREAM,
                                             torch_buffer=True,
                                             stream=self.streams[si].cuda_stream,
                                             band_rows=self.large_band_rows)
                    self.large_used += nbytes
                    chunk = int(min(self.max_chunk_sweeps,
                                    max(1, round(self.chunk_attempts / (r.L * r.L)))))
                    self.large[r.rid] = _Large(r, sim, si, r.budget, deque(), now, nbytes,
                                               chunk)
                    continue
            elif small_ok:
                try:
                    slot = self.pool.add(r.L, r.p, r.q, r.seed)
                    self.small[slot] = [r, r.budget, now]
                    continue
                except okz.OkzError as e:
                    if e.status != okz.OKZ_EBUSY:
                        raise
            blocked.append(r)  # no room yet (or the pool is busy): keep arrival order
        self.queue = blocked

    # -- large lattices: keep `ahead` chunks in flight ------------------------
    def _pump_large(self):
        torch = self._torch
        moved = False
        for ent in self.large.values():
            while ent.inflight and ent.inflight[0].query():
                ent.inflight.popleft()
                moved = True
            while ent.remaining > 0 and len(ent.inflight) < self.ahead:
                n = min(ent.remaining, ent.chunk)
                ent.sim.sweep(n)
                ent.remaining -= n
                ev = torch.cuda.Event()
                ev.record(self.streams[ent.si])
                ent.inflight.append(ev)
                self.attempts += float(ent.r.L) ** 2 * n
                moved = True
        return moved

    def _retire_large(self, t0):
        moved = False
        # budget done: enqueue the exact sums behind the last chunk, close by an event
        for ent in self.large.values():
            if ent.remaining == 0 and not ent.inflight and ent.measured is None:
                ent.sim.moments_enqueue()
                ev = self._torch.cuda.Event()
                ev.record(self.streams[ent.si])
                ent.measured = ev
                moved = True
        done = [rid for rid, ent in self.large.items()
                if ent.measured is not None and ent.measured.query()]
        for rid in done:
            ent = self.large.pop(rid)
            Sk, W2, _, _ = ent.sim.moments_fetch()
            H0 = ent.sim.info().H0
            ent.sim.close()
            self.large_used -= ent.nbytes
            self.free_streams.append(ent.si)
            fin = time.perf_counter() - t0
            self.results[rid] = Result(rid, Sk, H0, W2, ent.admitted, fin, fin - ent.r.arrival)
        return moved or bool(done)

    # -- small lattices: one batched launch at a time -------------------------
    def _retire_small(self, t0):
        now = time.perf_counter() - t0
        done = [slot for slot, ent in self.small.items() if ent[1] == 0]
        for slot, (Sk, H0, _) in zip(done, self.pool.measure(done)):
            r, _, adm = self.small.pop(slot)
            N = r.L * r.L
            W2 = float(N * Sk[1] - Sk[0] * Sk[0]) / (float(N) * float(N))
            self.pool.remove(slot)
            self.results[r.rid] = Result(r.rid, Sk, H0, W2, adm, now, now - r.arrival)

    def _launch_small(self):
        sweeps = np.zeros(self.max_slots, np.int64)
        for slot, ent in self.small.items():
            per_tick = (max(1, int(self.tick_attempts // (ent[0].L * ent[0].L)))
                        if self.equal_ticks else self.tick_sweeps)
            n = min(ent[1], per_tick)
            sweeps[slot] = n
            ent[1] -= n
            self.attempts += float(ent[0].L) ** 2 * n
        if not sweeps.any():
            return False
        self.pool.run(sweeps)
        ev = self._torch.cuda.Event()
        ev.record(self.pool_stream)
        self.small_event = ev
        return True

    def run(self, requests):
        """Serve `requests` (sorted by arrival) in real time; returns results by id."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        t0 = time.perf_counter()
        while pending or self.queue or self.small or self.large or self.small_event:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                self.queue.append(pending.popleft())
            busy = False
            pool_idle = self.small_event is None or self.small_event.query()
            if pool_idle and self.small_event is not None:
                self.small_event = None
                self._retire_small(t0)
                busy = True
            self._admit(now, small_ok=pool_idle)
            if pool_idle:
                busy |= self._launch_small()
            busy |= self._pump_large()
            busy |= self._retire_large(t0)
            if not busy:
                if not self.small and not self.large and pending and not self.queue:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival - now)))
                else:
                    time.sleep(0.00005)
        self.makespan = time.perf_counter() - t0
        return self.results

    def close(self):
        for ent in self.large.values():
            ent.sim.close()
        self.pool.close()


@dataclasses.dataclass
class _Large:
    r: Request
    sim: object
    si: int
    remaining: int      # sweeps not yet enqueued
    inflight: deque     # events closing the enqueued chunks
    admitted: float
    nbytes: int
    chunk: int
    measured: object = None  # event closing the enqueued exact sums


def run_alone(r):
    """The reference for one request: its lattice on its own."""
    kernel = (okz.OKZ_KERNEL_PARITY_STREAM if r.L >= 4096 else okz.OKZ_KERNEL_PARITY_PLAIN)
    with okz.Simulation(r.L, r.p, r.q, seed=r.seed, kernel=kernel) as sim:
        sim.sweep(r.budget)
        Sk, W2, _, _ = sim.moments()
        return Sk, sim.info().H0, W2


def served_record(unit, n=10000, rate=200.0, alone_sample=200):
    """The served workload (n Poisson requests at `rate` per second) through
    one Server; aggregate attempts per second over the makespan, latency
    percentiles (overall and per L), whether the offered load was sustained,
    and the same requests run alone one after another on a sample."""
    reqs = poisson_requests(n=n, rate=rate)
    srv = Server()
    tuned = srv.tune(sorted(set((r.L, r.p, r.q) for r in reqs)))
    res = srv.run(reqs)
    lat = np.array([res[r.rid].latency for r in reqs])
    attempts = sum(float(r.L) ** 2 * r.budget for r in reqs)
    value = attempts / srv.makespan / 1e9
    arrivals_s = max(r.arrival for r in reqs)
    sample = reqs[:: max(1, len(reqs) // alone_sample)]
    t0 = time.perf_counter()
    for r in sample:
        run_alone(r)
    alone_s = time.perf_counter() - t0
    alone = sum(float(r.L) ** 2 * r.budget for r in sample) / alone_s / 1e9
    tick = srv.tick_sweeps
    equal = srv.equal_ticks
    srv.close()
    return {
        "value": value, "unit": unit, "requests": len(reqs), "makespan_s": srv.makespan,
        "offered": attempts / arrivals_s / 1e9, "arrival_window_s": arrivals_s,
        "sustained": bool(srv.makespan <= 1.1 * arrivals_s),
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(lat.max())},
        "latency_by_L_s": {str(L): [float(np.percentile(lat[m], 50)),
                                    float(np.percentile(lat[m], 99))]
                           for L in sorted(set(r.L for r in reqs))
                           for m in [np.array([r.L == L for r in reqs])]},
        "per_request_alone": {"value": alone, "unit": unit, "sample": len(sample),
                              "seconds": alone_s},
        "served_over_alone": value / alone,
        "tick_sweeps": tick,
        "tuned_tilings": tuned,
        "tick": ("equal site updates per slot (tick_sweeps sweeps of L = 2048)"
                 if equal else "tick_sweeps sweeps per slot"),
    }


def bench(args, world, rank, local, unit):
    """bench.py --workload served: 10^4 Poisson requests at 200/s."""
    import json

    import torch
    torch.cuda.set_device(local)
    rec = served_record(unit)
    if rank != 0:
        return
    line = {
        "metric": "aggregate site-update attempts/s, served requests", "value": rec["value"],
        "unit": unit, "n_gpus": world, "steps": 1, "warmup": 0,
        "ms_per_step": rec["makespan_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic", "impl": "okz-serve",
        "config": {"workload": "10^4 requests, Poisson 200/s (PCG64 2027), L = 2^e, "
                               "e ~ U{7..13}, p ~ U{1, 0.75, 0.5}, q = 1 - p, budgets "
                               "round(10^U(2,4)) sweeps, admitted by slot and HBM footprint",
                   "requests": rec["requests"]},
    }
    line.update({k: v for k, v in rec.items() if k not in ("value", "unit")})
    print(json.dumps(line), flush=True)
