"""Benchmark of the octahedron-model hot path on GB300.

Workload (the L = 2^17 growth run): L = 131072 periodic lattice (2^34 sites,
4 GiB of bond planes), striped start, p = 1, q = 0, selection 1/2, Philox seed
11. One step = 256 sweeps (one fused sweep-kernel launch each) followed by one
measurement: height reconstruction and the exact sums sum h, sum h^2 that give
W^2. 32 steps = the full 2^13-sweep run; the timed steps start from t = 0.

Metric: site-update attempts per second (every active-sublattice visit counts
as one attempt), reported in GUPS = 1e9 attempts/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). Under torchrun (N > 1) every rank runs its own
independent lattice (replicas, no data-path collective; weak scaling).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_DEFAULT = 1 << 17
SEED = 11
SWEEPS_PER_STEP = 256
METRIC = "site-update attempts/s (GUPS)"
UNIT = "GUPS (1e9 site-update attempts/s)"
# algorithmic bytes per site per launch: read + write every stored bit once
BYTES_PER_SITE_LAUNCH = {"slope": 0.5, "parity": 0.25}
KERNELS = {"auto": 0, "slope": 2, "parity": 4}

# Integer work of one sweep of the parity-plane kernel, per site (the ALU roof):
# per 32-site word and half-sweep 2 funnel shifts (left and right neighbours)
# + 4 three-input logic ops (the two neighbour tests, then y & a & ~r0 and
# c ^ (x & that): the new word depends on 7 inputs with c used five times, so
# no 3-op form exists) = 6 ALU-pipe ops; per 128-site Philox4x32-10 block 20
# three-input xors (ALU pipe) and 20 32x32->64 multiplies (FMA pipe).
ALU_OPS_PER_SITE_SWEEP = {"parity": 2 * 6 / 32 + 20 / 128,
                          "slope": 2 * 9 / 32 + 20 / 128}
# Other thresholds (the batched, served and steady forms): both half-sweeps
# test minima and maxima and flip (2 funnel shifts, 6 three-input ops and 2
# ops per 32-site word and half-sweep), and every random level a 128-site
# group needs costs one Philox block (20 three-input xors) and the comparison
# steps with both thresholds (4 words x 3 ops). A group needs the deepest
# comparison among its candidates of both half-sweeps (the levels are shared
# between them): all k levels for k <= 3, else the expected maximum of
# CANDIDATES_PER_GROUP_SWEEP depths (geometric with ratio 1/2, capped at k).
CANDIDATES_PER_GROUP_SWEEP = 50  # minima + maxima per 128 sites and sweep: about 25
                                 # per half-sweep on oracle states of the p = 0.95,
                                 # q = 0.05 mix
ALU_LANES_PER_SM = 64  # INT32 ALU-pipe lanes per SM per clock (16 per sub-partition)
N_SMS = 152

# dram__bytes_read.sum + dram__bytes_write.sum per site of one launch of each
# dominant kernel (ncu on a small case, profiles/ gives the commands), valid
# only for the kernel source with the recorded SHA-256: traffic is reported as
# null once the source changes.
#   parity_stream_kernel  L = 65536, one launch = 2 sweeps
#   ddrs_kernel           L = 32768, one launch = 1 sweep
#   profile_count_tma_kernel  L = 65536, one profile pass
TRAFFIC = {
    "parity": ((556842496 + 485700608) / 65536 ** 2, "parity.cu",
               "e885ebdca0a5071622570b2e9ae60d759de864158c4595e2eadbb60e3896aa8a"),
    "ddrs": ((134544640 + 73219072) / 32768 ** 2, "ddrs.cu",
             "c2f242e7e5e1b6fc82f8f918aac71218c2f2182050306070f95ae2ed2e30a831"),
    "profile": ((546672384 + 8760064) / 65536 ** 2, "psd.cu",
                "3f9759eae0ced78fce621bcd7e32102d0a5400f4681801d3a991cb01838fd513"),
}


def alu_ops_per_attempt(okz, p, q, s_sel=0.5, k_max=32):
    """Algorithmic ALU-pipe ops per site-update attempt for (p, q)."""
    k, P, Q = okz.okz_thresholds(p, q, s_sel, k_max)
    full = 1 << k
    if k == 1 and 0 < P < full and Q == 0:
        return ALU_OPS_PER_SITE_SWEEP["parity"]
    if not any(0 < T < full for T in (P, Q)):
        levels = 0.0
    elif k <= 3:
        levels = float(k)
    else:
        levels = sum(1.0 - (1.0 - 2.0 ** -m) ** CANDIDATES_PER_GROUP_SWEEP for m in range(k))
    return 2 * 10 / 32 + levels * (20 + 12) / 128


def alu_roofline(ops_per_attempt, attempts_per_s, peak, note):
    """An ALU roofline record: algorithmic ops per attempt x attempts/s
    against the measured ALU-pipe peak."""
    achieved = ops_per_attempt * attempts_per_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak["value"], "unit": "Tops/s",
            "frac": achieved / peak["value"], "ops_per_attempt": ops_per_attempt,
            "peak_kind": "measured (okz_alu_peak)", "note": note}


def _traffic(name, sites):
    """Measured DRAM bytes of one launch of kernel `name` over `sites` sites,
    or None if its source has changed since the measurement."""
    if name not in TRAFFIC:
        return None
    per_site, src, sha = TRAFFIC[name]
    path = os.path.join(ROOT, "paper_1110_6745_gb300", "csrc", src)
    if hashlib.sha256(open(path, "rb").read()).hexdigest() != sha:
        return None
    return per_site * sites


def _size_label(L):
    """'2^17 (2^34 sites)' for a power of two, else '98304 (9663676416 sites)'."""
    if L & (L - 1) == 0:
        e = L.bit_length() - 1
        return "2^%d (2^%d sites)" % (e, 2 * e)
    return "%d (%d sites)" % (L, L * L)


def _bytes_label(n):
    for unit, size in (("GiB", 1 << 30), ("MiB", 1 << 20), ("KiB", 1 << 10)):
        if n >= size:
            return "%g %s" % (n / size, unit)
    return "%d B" % n


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "sm_min_mhz": min(sm),
                "reasons": sorted(reasons), "samples": len(sm)}


def measure_alu_peak(okz, local, stream=None):
    """The INT32 ALU-pipe rate of this GPU measured by the library's
    okz_alu_peak (independent lop3.b32 chains), with the SM clock sampled
    while it runs, and the derived figure (152 SMs x 64 lanes x that clock)
    beside it as a cross-check."""
    okz.okz_alu_peak(stream, 2000)  # warm-up (module load, clocks up)
    clk = ClockSampler(local)
    clk.start()
    best = 0.0
    for _ in range(20):  # about 1 s, so that the clock sampler sees the run
        ops, _ = okz.okz_alu_peak(stream, 20000)
        best = max(best, ops)
    c = clk.stop()
    mhz = (c or {}).get("sm_mhz") or 2070.0
    return {"value": best / 1e12, "unit": "Tops/s", "sm_mhz": mhz,
            "ops_per_sm_per_clk": best / N_SMS / (mhz * 1e6),
            "derived": N_SMS * ALU_LANES_PER_SM * mhz * 1e6 / 1e12,
            "clocks": c, "kernel": "okz_alu_peak (8 independent lop3.b32 chains per thread)"}


def _alu_peak_at(peak, sm_mhz):
    """The measured ALU-pipe rate scaled to the SM clock of a timed region."""
    return peak["value"] * sm_mhz / peak["sm_mhz"]


def _dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(world, v, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(L=16384, sweeps=40):
    """The CPU oracle as it stands on a bounded sample of the workload."""
    import oracle
    sim = oracle.Sim(L, 1.0, 0.0, SEED)
    t0 = time.perf_counter()
    sim.sweep(sweeps)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": L * L * sweeps / dt / 1e9, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": "L=%d striped start, p=1, q=0, s_sel=1/2, seed=%d, %d sweeps "
                      "(%.3g attempts, %.1f s), OpenMP over rows" % (L, SEED, sweeps,
                                                                     L * L * sweeps, dt)}


def cpu_serial_baseline(L=4096, sweeps=8):
    """The same oracle on one host thread (the paper's CPU reference was
    serial), in a child process so that OpenMP starts with one thread."""
    code = ("import sys, time; sys.path.insert(0, %r); import oracle; "
            "s = oracle.Sim(%d, 1.0, 0.0, %d); s.sweep(1); t = time.perf_counter(); "
            "s.sweep(%d); print(time.perf_counter() - t)" % (ROOT, L, SEED, sweeps))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=600)
    dt = float(out.stdout.strip().splitlines()[-1])
    return {"value": L * L * sweeps / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "L=%d, %d sweeps after one, one thread (%.1f s)" % (L, sweeps, dt)}


def run_reference(args, world, rank):
    """--impl reference: the CPU oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    L, per_step = 8192, 2
    sim = oracle.Sim(L, 1.0, 0.0, SEED)
    sim.sweep(per_step * args.warmup)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.sweep(per_step)
        sim.width2()
    dt = time.perf_counter() - t0
    attempts = L * L * per_step * args.steps
    value = attempts / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": "octahedron growth, striped start, p=1 q=0 s_sel=1/2 "
                               "(bounded CPU sample: L=8192, 2 sweeps + W^2 per step)",
                   "L": L, "sweeps_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "L=8192, %d sweeps + one W^2 per step, %d steps"
                                   % (per_step, args.steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    import paper_1110_6745_gb300 as okz

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = args.L
    N = L * L
    stream = torch.cuda.Stream(device=dev)
    # the tiling (words per thread x sweeps per pass x band rows) by the
    # library's autotuner, unless given on the command line; every choice gives
    # the same lattice
    tuned = None
    if args.wpt == 0 and args.fuse == 0:
        w, f, b, ms = okz.okz_tune_stream(L, 1.0, 0.0, kernel=KERNELS[args.kernel],
                                          probe_sweeps=8)
        tuned = {"words_per_thread": w, "sweeps_per_pass": f, "band_rows": b, "ms_per_sweep": ms,
                 "candidates": "words per thread {4, 8, 16} x sweeps per pass {1, 2} x band "
                               "rows {auto, 16, 32}, 8 timed sweeps each (okz_tune_stream)"}
    with torch.cuda.stream(stream):
        sim = okz.Simulation(L, 1.0, 0.0, seed=SEED + rank, torch_buffer=True,
                             kernel=KERNELS[args.kernel], words_per_thread=args.wpt,
                             sweeps_per_pass=args.fuse)
    peak_meas = measure_alu_peak(okz, local, stream.cuda_stream)
    kind = sim.info().kernel
    assert kind in (okz.OKZ_KERNEL_STREAM, okz.OKZ_KERNEL_PARITY_STREAM)
    repr_name = "parity" if kind == okz.OKZ_KERNEL_PARITY_STREAM else "slope"
    fuse = sim.fuse
    wpt = sim.wpt
    # checkpoint of the striped start, kept on the device
    start_planes = torch.empty(2 * L * L // 32, dtype=torch.int32, device=dev)
    sim.state(out=start_planes)

    def step(ev_a=None, ev_b=None):
        if ev_a is not None:
            ev_a.record(stream)
        sim.sweep(SWEEPS_PER_STEP)
        if ev_b is not None:
            ev_b.record(stream)
        return sim.width2()

    for _ in range(args.warmup):
        step()
    sim.restore(start_planes, 0, 0)
    torch.cuda.synchronize(dev)

    sweep_evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    _barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    t_start.record(stream)
    records = []
    for k in range(args.steps):
        records.append(step(*sweep_evs[k]))
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    _barrier(world)
    elapsed_ms = t_start.elapsed_time(t_end)
    sweep_ms = sum(a.elapsed_time(b) for a, b in sweep_evs)
    elapsed_ms = _max_over_ranks(world, elapsed_ms, dev)
    sweeps = SWEEPS_PER_STEP * args.steps
    value = world * N * sweeps / (elapsed_ms / 1e3) / 1e9
    sweep_launches = SWEEPS_PER_STEP // fuse
    launches = args.steps * (sweep_launches + 3)  # sweep launches + 3 measurement kernels

    # roofline of the sweep kernel: algorithmic bytes per launch / launch time
    per_launch_s = sweep_ms / 1e3 / (args.steps * sweep_launches)
    alg_bytes = BYTES_PER_SITE_LAUNCH[repr_name] * N
    achieved = alg_bytes / per_launch_s / 1e9
    peak, peak_kind = _peaks()
    traffic = _traffic(repr_name, N) if fuse == 2 else None  # measured at 2 sweeps/launch
    # ALU roof: algorithmic ALU-pipe ops per launch / launch time, against
    # the ALU-pipe rate measured on this GPU (okz_alu_peak) at the SM clock
    # sampled during the timed region
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    alu_peak = _alu_peak_at(peak_meas, sm_mhz)
    alu_ops = ALU_OPS_PER_SITE_SWEEP[repr_name] * N * fuse
    alu_achieved = alu_ops / per_launch_s / 1e12

    # end to end through the C-ABI with host buffers: every step's input, the
    # whole lattice state (both slope planes, 4 GiB), goes in from pinned host
    # memory, then 256 sweeps, then the exact sums come back (okz_width2). The
    # input copy of step k + 1 (okz_stage_host: the library's own copy stream)
    # runs while step k sweeps, and okz_restore_staged makes step k + 1 wait
    # for it before converting to the parity plane. All copies lie inside the
    # timed region (the first one not overlapped); one untimed step first
    # (the first copy from freshly pinned memory pays a one-time mapping cost).
    e2e_steps = min(args.steps, 8)
    host_planes = torch.empty(2 * L * L // 32, dtype=torch.int32, pin_memory=True)
    host_planes.copy_(start_planes.cpu())
    del start_planes

    def e2e_run(nsteps):
        sim.stage_host(host_planes)
        for k in range(nsteps):
            sim.restore_staged(0, 0)
            if k + 1 < nsteps:
                sim.stage_host(host_planes)  # overlaps this step's sweeps
            sim.sweep(SWEEPS_PER_STEP)
            sim.width2()  # the step's result to the host (synchronizing)

    e2e_run(1)
    torch.cuda.synchronize(dev)
    # context, not part of the number: this box's rate for a plain copy of
    # the same pinned buffer to the device (the copy the pipeline hides
    # behind each step's sweeps)
    probe = torch.empty_like(host_planes, device=dev)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record()
    probe.copy_(host_planes, non_blocking=True)
    c1.record()
    c1.synchronize()
    h2d_probe_gbs = host_planes.numel() * 4 / (c0.elapsed_time(c1) / 1e3) / 1e9
    del probe
    _barrier(world)
    e2e_clocks = ClockSampler(local)
    e2e_clocks.start()
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    torch.cuda.synchronize(dev)
    e2e_s = _max_over_ranks(world, time.perf_counter() - t0, dev)
    e2e_clk = e2e_clocks.stop()
    e2e_value = world * N * SWEEPS_PER_STEP * e2e_steps / e2e_s / 1e9
    h2d = L * L // 4 + 8            # both planes + H0
    d2h = 256 + 4                   # control block (sums, H0) + error word

    w2_final = records[-1][2]
    sim.close()

    # the two smaller growth workloads, timed as whole runs from t = 0: the
    # launch-bound L = 256 run (1000 sweeps, 20 samples) and the L2-resident
    # L = 2^14 run (10^4 sweeps, 40 samples; two 32 MiB ping-pong planes)
    small = {}
    for name, (Ls, T, ns, sd) in (("growth_L256", (256, 1000, 20, 1)),
                                  ("growth_L16384", (16384, 10000, 40, 7))):
        rec = growth_line(okz, Ls, T, ns, sd + rank)
        rate = rec["value"] * 1e9
        rec["roofline"] = {"bound": "alu", "achieved": ALU_OPS_PER_SITE_SWEEP["parity"] * rate / 1e12,
                           "peak": peak_meas["value"], "unit": "Tops/s",
                           "frac": ALU_OPS_PER_SITE_SWEEP["parity"] * rate / 1e12
                           / peak_meas["value"],
                           "note": "whole run incl. the W^2 samples, against the measured "
                                   "ALU-pipe rate"}
        if Ls == 16384:
            rec["l2"] = "L2-resident (2 x 32 MiB parity planes < 126 MiB L2): not an HBM case"
        small[name] = rec
    # the batched and served forms (compact records; --workload batched /
    # served print the same as lines of their own)
    batched = served = general_k = None
    if not args.no_forms:
        general_k = general_k_record(okz, peak_meas)
        batched = batched_record(okz, args.budget_frac, args.plain_stride, rank, world,
                                 peak=peak_meas)
        from paper_1110_6745_gb300 import serve
        served = serve.served_record(UNIT)
        reqs = serve.poisson_requests()
        att = np.array([float(r.L) ** 2 * r.budget for r in reqs])
        ops = np.array([alu_ops_per_attempt(okz, r.p, r.q) for r in reqs])
        served["roofline"] = alu_roofline(
            float((att * ops).sum() / att.sum()), served["value"] * 1e9, peak_meas,
            "attempt-weighted over the request mix (p = 1, 0.75, 0.5: k = 1 minima only, 3, 2)")
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "octahedron growth run L=%s, striped start, "
                               "p=1 q=0 s_sel=1/2, seed=11; step = %d sweeps + exact W^2"
                               % (_size_label(L), SWEEPS_PER_STEP),
                   "L": L, "sweeps_per_step": SWEEPS_PER_STEP, "t_range": [0, sweeps],
                   "l2": "inputs larger than L2 (2 x %s ping-pong planes)"
                         % _bytes_label(L * L // (8 if repr_name == "parity" else 4)),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak,
                     "unit": "Tops/s", "frac": alu_achieved / alu_peak,
                     "traffic": traffic,
                     "kernel": ("parity_stream_kernel" if repr_name == "parity"
                                else "sweep_stream_kernel"),
                     "peak_kind": "measured: okz_alu_peak on this GPU, scaled to the timed "
                                  "region's SM clock",
                     "peak_measured": peak_meas,
                     "peak_derived": N_SMS * ALU_LANES_PER_SM * sm_mhz * 1e6 / 1e12,
                     "ops_per_launch": alu_ops, "sweeps_per_launch": fuse,
                     "words_per_thread": wpt, "launch_ms": per_launch_s * 1e3},
        "roofline_hbm": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "bytes_per_launch": alg_bytes, "peak_kind": peak_kind},
        "sweep_gups": N * fuse / per_launch_s / 1e9,
        # not a roofline: the rate the paper's two-plane encoding (0.5 B per
        # site and sweep) would need from HBM at this attempt rate
        "slope_plane_equiv_bw_frac": (N * fuse / per_launch_s) * 0.5 / (peak * 1e9),
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps, "clocks": e2e_clk,
                "ms_per_step": e2e_s / e2e_steps * 1e3,
                "h2d_probe_gbs": h2d_probe_gbs,

                "path": "okz_stage_host(pinned host planes; the next step's copy overlaps "
                        "this step's sweeps) + okz_restore_staged + okz_sweep + okz_width2 "
                        "(synchronizing read of each step's sums)"},
        "w2_final": w2_final,
        "clocks": clk,
        "smaller_growth_workloads": small,
        "autotune": tuned,
    }
    if batched is not None:
        line["batched"] = batched
        line["served"] = served
        line["general_k"] = general_k
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_baseline_serial"] = cpu_serial_baseline()
    print(json.dumps(line), flush=True)


def growth_line(okz, L, T, nsamp, seed, reps=3):
    """A whole growth run as the paper times it (Sec. III): the striped start
    swept to n log-spaced sample times over T sweeps, the exact W^2 taken at
    every sample, through okz_growth_series (sweeps and measurements queued
    on the device, each sample's sums kept there, one read-back at the end).
    Timed on the host clock from t = 0, best of `reps` runs after one untimed
    run. Returns attempts/s and the time per run and per sample."""
    from paper_1110_6745_gb300.analysis import sample_times
    times = sample_times(T, nsamp)
    best, info, w2_last = None, None, None
    for rep in range(reps + 1):
        with okz.Simulation(L, 1.0, 0.0, seed=seed) as sim:
            sim.width2()  # the lattice is initialised before the clock starts
            t0 = time.perf_counter()
            rec = sim.growth_series(times)
            dt = time.perf_counter() - t0
            w2_last = rec[-1][4]
            info = sim.info()
        if rep > 0 and (best is None or dt < best):
            best = dt
    return {"value": L * L * T / best / 1e9, "unit": UNIT, "L": L, "sweeps": T,
            "samples": len(times), "ms_per_run": best * 1e3,
            "us_per_sample": best * 1e6 / len(times), "w2_final": w2_last,
            "kernel": {1: "slope plain", 2: "slope stream", 3: "parity plain",
                       4: "parity stream", 5: "parity one-CTA (shared memory, one launch per "
                                              "sample interval)"}[info.kernel],
            "words_per_thread": info.words_per_thread, "sweeps_per_pass": info.sweeps_per_pass,
            "graph_chunk": info.graph_chunk, "graph_replays_per_run": info.graph_replays,
            "timing": "host clock around the whole run (okz_growth_series: sweeps and "
                      "exact W^2 samples queued on the device, one synchronisation), "
                      "best of %d" % reps}


def replica_mix(n=4096, seed=2026):
    """The batched workload: L_r = 2^e_r, e_r ~ U{6..11} (PCG64), p = 0.95, q = 0.05,
    seed_r = 1000 + r, full budgets T_r = ceil(4 L_r^1.61) sweeps."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    e = rng.integers(6, 12, size=n)
    L = (1 << e).astype(np.int64)
    T = np.ceil(4 * L.astype(np.float64) ** 1.61).astype(np.int64)
    seeds = (1000 + np.arange(n)).astype(np.uint64)
    return L, T, seeds


def general_k_record(okz, peak, sweeps=64):
    """One lattice through the general-k stream kernel (the large lattices of
    the served form): L = 8192 and 4096 at p = 0.75, q = 0.25 (k = 3), the
    library's tiling, 8 warm-up sweeps, then `sweeps` timed with CUDA events
    on the simulation's stream."""
    import torch
    out = {}
    for L in (8192, 4096):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            sim = okz.Simulation(L, 0.75, 0.25, seed=31, kernel=okz.OKZ_KERNEL_PARITY_STREAM,
                                 stream=stream.cuda_stream)
        sim.sweep(8)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.sweep(sweeps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        rate = float(L) * L * sweeps / (ms / 1e3)
        out["L%d" % L] = {
            "value": rate / 1e9, "unit": UNIT, "sweeps": sweeps, "ms": ms, "p": 0.75, "q": 0.25,
            "k": 3, "words_per_thread": sim.wpt, "sweeps_per_pass": sim.fuse,
            "band_rows": sim.band_rows,
            "roofline": alu_roofline(alu_ops_per_attempt(okz, 0.75, 0.25), rate, peak,
                                     "3 random levels per 128-site group and sweep; one "
                                     "lattice alone on the GPU")}
        sim.close()
    return out


def batched_record(okz, frac, plain_stride, rank=0, world=1, peak=None):
    """The batched workload: all 4096 replicas in one graph-captured
    persistent launch (tiling autotuned first) at budgets ceil(4 L^1.61)/frac,
    against per-replica plain launches (the in-place parity kernel, one
    okz_sim per replica, every launch enqueued back to back on one stream and
    one synchronisation at the end) of every plain_stride-th replica at the
    same budgets. Both rates are aggregate attempts per second."""
    import numpy as np
    import torch
    L, T, seeds = replica_mix()
    n = len(L)
    budgets = np.maximum(1, T // frac)
    b = okz.Batch(L, [0.95] * n, [0.05] * n, [int(x) + rank for x in seeds])
    tune = b.autotune(probe_sweeps=2)
    st = torch.cuda.ExternalStream(b.stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    _barrier(world)
    e0.record(st)
    b.run(budgets)
    b.sync()
    W2, sk, ku = b.stats()
    e1.record(st)
    torch.cuda.synchronize()
    ms = _max_over_ranks(world, e0.elapsed_time(e1))
    tiling = b.tiling()
    b.close()
    attempts = float(np.sum(L.astype(np.float64) ** 2 * budgets))
    batched = world * attempts / (ms / 1e3) / 1e9
    # per-replica plain launches, same budgets, a strided subset of the mix
    idx = list(range(0, n, plain_stride))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sims = [okz.Simulation(int(L[r]), 0.95, 0.05, seed=int(seeds[r]) + rank,
                               kernel=okz.OKZ_KERNEL_PARITY_PLAIN, torch_buffer=True)
                for r in idx]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, r in enumerate(idx):
        sims[k].sweep(int(budgets[r]))
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_attempts = float(np.sum(L[idx].astype(np.float64) ** 2 * budgets[idx]))
    plain = plain_attempts / plain_s / 1e9
    for s_ in sims:
        s_.close()
    rec = {"value": batched, "unit": UNIT, "ms": ms, "replicas": n, "attempts": attempts,
            "budgets": "ceil(4 L^1.61)/%d sweeps" % frac,
            "tiling": {"threads": tiling[0], "smem_bytes": tiling[1], "grid": tiling[2]},
            "autotune": tune,
            "per_replica_plain": {"value": plain, "unit": UNIT, "replicas": len(idx),
                                  "budgets": "the same",
                                  "kernel": "parity plain (graph-replayed sweeps), one okz_sim "
                                            "per replica, launches back to back on one stream, "
                                            "one synchronisation at the end",
                                  "seconds": plain_s},
            "batched_over_plain": batched / plain,
            "w2_mean_by_L": {int(l): float(np.nanmean(W2[L == l])) for l in np.unique(L)}}
    if peak is not None:
        rec["roofline"] = alu_roofline(
            alu_ops_per_attempt(okz, 0.95, 0.05), batched * 1e9, peak,
            "k = 32 with lazily drawn levels: about 7.0 levels per 128-site group and sweep "
            "(the expected deepest of ~50 candidate comparisons)")
    return rec


def run_batched(args, world, rank, local):
    """--workload batched: the batched line of its own."""
    import torch

    import paper_1110_6745_gb300 as okz
    torch.cuda.set_device(local)
    peak = measure_alu_peak(okz, local, None)
    rec = batched_record(okz, args.budget_frac, args.plain_stride, rank, world, peak=peak)
    if rank != 0:
        return
    line = {
        "metric": "aggregate site-update attempts/s, batched replicas", "value": rec["value"],
        "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": rec["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "impl": "okz-batch",
        "config": {"workload": "4096 replicas, L = 2^e, e ~ U{6..11} (PCG64 2026), p=0.95 "
                               "q=0.05 s_sel=1/2, seeds 1000+r, striped start, budgets "
                               "ceil(4 L^1.61)/%d sweeps; final W^2, skewness, kurtosis"
                               % args.budget_frac}}
    line.update({k: v for k, v in rec.items() if k not in ("value", "unit")})
    print(json.dumps(line), flush=True)


# Integer work of one attempt of the blocked random-sequential sweep (ALU
# pipe): half a Philox4x32-10 block (10 three-input xors; its 10 wide
# multiplies run on the FMA pipe), decoding the site (2), the dead-border test
# (2), the five neighbour/own bits (3 shifts), the extremum tests (4 logic
# ops), the acceptance compare (2), the flip and the touched-row mask (4).
RS_ALU_OPS_PER_ATTEMPT = 10 + 2 + 2 + 3 + 4 + 2 + 4


def run_rs(args, world, rank, local):
    """--workload rs: the paper's own dynamics (blocked random-sequential
    sweeps, okz_sweep_rs) on the L = 2^17 lattice; a step = 2 sweeps + exact W^2."""
    import torch

    import paper_1110_6745_gb300 as okz

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = args.L
    N = L * L
    per_step = 2
    steps = min(args.steps, 8)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        sim = okz.Simulation(L, 1.0, 0.0, seed=SEED + rank, torch_buffer=True,
                             kernel=okz.OKZ_KERNEL_PARITY_PLAIN)
    peak_meas = measure_alu_peak(okz, local, stream.cuda_stream)
    for _ in range(args.warmup):
        sim.sweep_rs(per_step)
        sim.width2()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    _barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    t0.record(stream)
    for k in range(steps):
        evs[k][0].record(stream)
        sim.sweep_rs(per_step)
        evs[k][1].record(stream)
        sim.width2()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    _barrier(world)
    ms = _max_over_ranks(world, t0.elapsed_time(t1), dev)
    launch_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3 / (steps * per_step)
    value = world * N * per_step * steps / (ms / 1e3) / 1e9
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    alu_peak = _alu_peak_at(peak_meas, sm_mhz)
    alu_ops = RS_ALU_OPS_PER_ATTEMPT * N
    sim.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "impl": "okz-rs",
        "config": {"workload": "blocked random-sequential dynamics (32x32 cells, two dead "
                               "edges, origin moved every sweep), L=2^17, striped start, "
                               "p=1 q=0, seed=11; step = 2 sweeps + exact W^2",
                   "L": L, "sweeps_per_step": per_step,
                   "l2": "inputs larger than L2 (2 GiB parity plane)"},
        "roofline": {"bound": "alu", "achieved": alu_ops / launch_s / 1e12, "peak": alu_peak,
                     "unit": "Tops/s", "frac": alu_ops / launch_s / 1e12 / alu_peak,
                     "traffic": _traffic("ddrs", N), "kernel": "ddrs_kernel",
                     "peak_kind": "measured: okz_alu_peak on this GPU, scaled to the timed "
                                  "region's SM clock",
                     "peak_measured": peak_meas,
                     "peak_derived": N_SMS * ALU_LANES_PER_SM * sm_mhz * 1e6 / 1e12,
                     "ops_per_launch": alu_ops, "launch_ms": launch_s * 1e3},
        "gpu_launches": steps * (per_step + 3),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def _fft_launches(L):
    """Kernels of okz_psd's transform: the shared-memory block of the first
    min(log2 L, 10) stages, a radix-2 stage if an odd number is left, radix-4
    steps for the rest, and the finish that writes S."""
    lg = int(L).bit_length() - 1
    rem = lg - min(lg, 10)
    return 1 + rem % 2 + rem // 2 + 1


def run_spectrum(args, world, rank, local):
    """--workload spectrum: interface profiles and the axis power spectrum
    (okz_psd) of the L = 2^17 lattice after 64 sweeps; a step = one spectrum."""
    import torch

    import paper_1110_6745_gb300 as okz

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = args.L
    N = L * L
    steps = min(args.steps, 16)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        sim = okz.Simulation(L, 1.0, 0.0, seed=SEED + rank, torch_buffer=True)
    sim.sweep(64)
    for _ in range(args.warmup):
        sim.psd()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    clocks = ClockSampler(local)
    _barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    w0 = time.perf_counter()
    for k in range(steps):
        evs[k][0].record(stream)
        S = sim.psd()
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = _max_over_ranks(world, time.perf_counter() - w0, dev)
    clk = clocks.stop()
    _barrier(world)
    gpu_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3 / steps
    peak, peak_kind = _peaks()
    alg = 0.125 * N  # the parity plane read once by the counting pass
    sim.close()
    if rank != 0:
        return
    line = {
        "metric": "sites/s through profiles + axis spectrum", "value": world * N * steps / wall / 1e9,
        "unit": "1e9 sites/s", "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": wall / steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32/f64", "data": "synthetic", "impl": "okz-spectrum",
        "config": {"workload": "okz_psd of the L=2^17 lattice after 64 growth sweeps "
                               "(p=1 q=0 s_sel=1/2, seed=11); host-synchronous call, the 1 MiB "
                               "device-to-host copy of S included", "L": L,
                   "l2": "inputs larger than L2 (2 GiB parity plane)"},
        "roofline": {"bound": "hbm", "achieved": alg / gpu_s / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": alg / gpu_s / 1e9 / peak,
                     "traffic": _traffic("profile", N),
                     "kernel": "profile_count_tma_kernel (+ tiles, scan and FFT kernels, all "
                               "in the interval)",
                     "bytes_per_call": alg, "gpu_ms_per_call": gpu_s * 1e3,
                     "peak_kind": peak_kind},
        "S_k1": float(S[1]),
        "gpu_launches": steps * (3 + _fft_launches(L)),  # count, tiles, scan + the FFT's
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# Steady-state plan per L: replicas, burn-in and sample spacing in units of
# L^1.61 sweeps (about the saturation time at s_sel = 1/2), samples.
STEADY_PLAN = {128: (304, 4, 1, 8), 256: (304, 4, 1, 8), 512: (304, 4, 1, 8),
               1024: (304, 4, 1, 8), 2048: (152, 3, 1, 5)}


def run_steady(args, world, rank, local):
    """--workload steady: the steady-state statistics of Secs. III-IV on the
    batched kernels -- replicas at L = 128 .. 2048 (STEADY_PLAN) run from the
    striped start, then sampled (exact W^2 per sample); alpha_eff(L) (Eq.
    (13)) with jackknife errors, the fit of Eq. (14) at the paper's
    correction exponent, and kappa_2 / kappa_1^2 per L."""
    import numpy as np
    import torch

    import paper_1110_6745_gb300 as okz
    from paper_1110_6745_gb300.analysis import alpha_fss, steady_state_w2, w2_cumulants

    torch.cuda.set_device(local)
    okz.lib()
    peak = measure_alu_peak(okz, local, None)
    samples, ratios, attempts, secs = {}, {}, 0.0, {}
    _barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for L, (R, burn_tx, every_tx, nsamp) in sorted(STEADY_PLAN.items()):
        tx = L ** 1.61
        burn, every = int(burn_tx * tx), int(every_tx * tx)
        t1 = time.perf_counter()
        w = steady_state_w2(L, R, burn, nsamp, every, seed0=100000 + 1000 * L + 10 ** 6 * rank,
                            tune=True)
        secs[L] = time.perf_counter() - t1
        k = w2_cumulants(w)
        samples[L], ratios[L] = w, k[1] / k[0] ** 2
        attempts += float(L) ** 2 * R * (burn + nsamp * every)
    torch.cuda.synchronize()
    dt = _max_over_ranks(world, time.perf_counter() - t0)
    fss = alpha_fss(samples, omega=1.16)
    if rank != 0:
        return
    line = {
        "metric": "aggregate site-update attempts/s, steady-state sampling", "unit": UNIT,
        "value": world * attempts / dt / 1e9, "n_gpus": world, "steps": 1, "warmup": 0,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic", "impl": "okz-steady",
        "config": {"workload": "steady state, p=1 q=0 s_sel=1/2, striped start; per L: "
                               "(replicas, burn-in and spacing in L^1.61 sweeps, samples)",
                   "plan": {str(L): v for L, v in sorted(STEADY_PLAN.items())}},
        "w2_mean_by_L": {str(L): float(samples[L].mean()) for L in samples},
        "seconds_by_L": {str(L): secs[L] for L in secs},
        "alpha_fss": fss,
        "roofline": alu_roofline(alu_ops_per_attempt(okz, 1.0, 0.0), world * attempts / dt, peak,
                                 "whole run incl. burn-in, sampling and the exact W^2 per "
                                 "sample; per GPU for n_gpus > 1 divide by n_gpus"),
        "kappa2_over_kappa1_sq": {str(L): float(ratios[L]) for L in ratios},
        "paper_alpha": "0.393(4), correction exponent 1.16 (Sec. III)",
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="okz", choices=["okz", "reference"])
    ap.add_argument("--L", type=int, default=L_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="growth line only: skip the batched and served records")
    ap.add_argument("--kernel", default="auto", choices=sorted(KERNELS))
    ap.add_argument("--wpt", type=int, default=0, help="words per thread (0 = library choice)")
    ap.add_argument("--fuse", type=int, default=0, help="sweeps per launch (0 = library choice)")
    ap.add_argument("--workload", default="growth",
                    choices=["growth", "batched", "served", "rs", "spectrum", "steady"])
    ap.add_argument("--budget-frac", type=int, default=64,
                    help="batched: run ceil(4 L^1.61)/frac sweeps per replica")
    ap.add_argument("--plain-stride", type=int, default=16,
                    help="batched: time the per-replica plain launches on every n-th replica")
    args = ap.parse_args()
    world, rank, local = _dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batched":
        run_batched(args, world, rank, local)
    elif args.workload == "served":
        from paper_1110_6745_gb300 import serve
        serve.bench(args, world, rank, local, UNIT)
    elif args.workload == "rs":
        run_rs(args, world, rank, local)
    elif args.workload == "spectrum":
        run_spectrum(args, world, rank, local)
    elif args.workload == "steady":
        run_steady(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
