"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

Integer state (bond planes, H0, t, exact sums) must match bit for bit; W^2
is finalized from exact integers on both sides and must be equal as doubles;
skewness and kurtosis (long-double finalization) agree to 1e-12 relative.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def okz():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1110_6745_gb300 import _build
    _build.build()
    import paper_1110_6745_gb300 as m
    m.lib()
    return m


def _compare(sim, ref):
    planes, H0, t = sim.state()
    Xw, Yw = ref.packed()
    assert np.array_equal(planes[0], Xw), "X plane differs"
    assert np.array_equal(planes[1], Yw), "Y plane differs"
    assert (H0, t) == (ref.H0, ref.t)


MODES = [  # p, q, s_sel: k and kernel path
    (1.0, 0.0, 0.5),     # k = 1, only minima move (the growth workloads)
    (0.75, 0.25, 0.5),   # k = 3
    (1.0, 1.0, 0.5),     # k = 1, minima and maxima
    (0.95, 0.05, 0.5),   # k = 32, rounded thresholds
    (1.0, 0.0, 1.0),     # k = 0, deterministic growth
    (0.0, 1.0, 1.0),     # k = 0, deterministic etching
    (0.5, 0.5, 0.5),     # k = 2
]


PLAIN_KINDS = [1, 3]   # OKZ_KERNEL_PLAIN (slope planes), OKZ_KERNEL_PARITY_PLAIN
STREAM_KINDS = [2, 4]  # OKZ_KERNEL_STREAM, OKZ_KERNEL_PARITY_STREAM
SMALL_KINDS = [1, 3, 5]  # in-place kinds and OKZ_KERNEL_PARITY_CTA (one CTA, L <= 1024)


@pytest.mark.parametrize("kernel", SMALL_KINDS)
@pytest.mark.parametrize("L", [32, 64, 96, 128, 256, 480])
@pytest.mark.parametrize("p,q,s_sel", MODES)
def test_plain_kernel_matches_oracle(okz, orc, L, p, q, s_sel, kernel):
    seed = 1000 + L
    ref = orc.Sim(L, p, q, seed, s_sel=s_sel)
    with okz.Simulation(L, p, q, seed=seed, s_sel=s_sel, kernel=kernel) as sim:
        for n in (1, 2, 7):
            ref.sweep(n)
            sim.sweep(n)
            _compare(sim, ref)
            S1, S2, W2 = sim.width2()
            assert (S1, S2) == ref.sums() and W2 == ref.width2()


@pytest.mark.parametrize("kernel", STREAM_KINDS)
@pytest.mark.parametrize("L", [4096, 12288])
@pytest.mark.parametrize("p,q,s_sel", MODES)
def test_stream_kernel_matches_oracle(okz, orc, L, p, q, s_sel, kernel):
    seed = 77 + L
    ref = orc.Sim(L, p, q, seed, s_sel=s_sel)
    with okz.Simulation(L, p, q, seed=seed, s_sel=s_sel, kernel=kernel) as sim:
        for n in (1, 3):
            ref.sweep(n)
            sim.sweep(n)
            _compare(sim, ref)
        S1, S2, W2 = sim.width2()
        assert (S1, S2) == ref.sums() and W2 == ref.width2()


@pytest.mark.parametrize("kernel", STREAM_KINDS)
@pytest.mark.parametrize("wpt,fuse", [(4, 1), (8, 1), (4, 2), (8, 2)])
@pytest.mark.parametrize("p,q,s_sel", [(1.0, 0.0, 0.5), (0.75, 0.25, 0.5), (1.0, 1.0, 0.5),
                                       (0.95, 0.05, 0.5)])
def test_stream_variants_match_oracle(okz, orc, wpt, fuse, p, q, s_sel, kernel):
    """Every tiling (words per thread) and temporal-blocking depth (sweeps per
    launch) gives the oracle's lattice, including odd sweep counts."""
    L, seed = 8192, 31
    ref = orc.Sim(L, p, q, seed, s_sel=s_sel)
    with okz.Simulation(L, p, q, seed=seed, s_sel=s_sel, kernel=kernel,
                        words_per_thread=wpt, sweeps_per_pass=fuse) as sim:
        for n in (1, 2, 3):
            ref.sweep(n)
            sim.sweep(n)
            _compare(sim, ref)
        S1, S2, W2 = sim.width2()
        assert (S1, S2) == ref.sums() and W2 == ref.width2()


@pytest.mark.parametrize("kernel", STREAM_KINDS)
@pytest.mark.parametrize("wpt,fuse", [(4, 2), (8, 2), (8, 1)])
def test_stream_variants_long_run_L32768(okz, wpt, fuse, kernel):
    """Long runs at L = 2^15 (several CTA bands per SM) agree with the plain kernel."""
    L = 32768
    a = okz.Simulation(L, 1.0, 0.0, seed=8, kernel=kernel,
                       words_per_thread=wpt, sweeps_per_pass=fuse)
    b = okz.Simulation(L, 1.0, 0.0, seed=8, kernel=okz.OKZ_KERNEL_PLAIN)
    a.sweep(37)
    b.sweep(37)
    pa, ha, ta = a.state()
    pb, hb, tb = b.state()
    assert np.array_equal(pa, pb) and (ha, ta) == (hb, tb)
    a.close()
    b.close()


@pytest.mark.parametrize("fuse", [1, 2])
@pytest.mark.parametrize("p,q,s_sel", [(1.0, 0.0, 0.5), (0.75, 0.25, 0.5), (1.0, 1.0, 0.5),
                                       (0.95, 0.05, 0.5)])
def test_parity_stream_wpt16_matches_oracle(okz, orc, p, q, s_sel, fuse):
    """16 words per thread (the smallest row it allows, L = 2^14: one warp per
    row) gives the oracle's lattice in every acceptance mode."""
    L, seed = 16384, 41
    ref = orc.Sim(L, p, q, seed, s_sel=s_sel)
    with okz.Simulation(L, p, q, seed=seed, s_sel=s_sel, kernel=okz.OKZ_KERNEL_PARITY_STREAM,
                        words_per_thread=16, sweeps_per_pass=fuse) as sim:
        assert sim.wpt == 16
        for n in (1, 2):
            ref.sweep(n)
            sim.sweep(n)
            _compare(sim, ref)
        S1, S2, W2 = sim.width2()
        assert (S1, S2) == ref.sums() and W2 == ref.width2()


@pytest.mark.parametrize("L,p,q,fuse", [(32768, 1.0, 0.0, 2), (65536, 0.95, 0.05, 1),
                                        (131072, 1.0, 0.0, 2), (131072, 1.0, 1.0, 2)])
def test_parity_stream_wpt16_long_run(okz, L, p, q, fuse):
    """16 words per thread against the 8-word kernel over many sweeps, up to
    the largest lattice (256 threads per row)."""
    a = okz.Simulation(L, p, q, seed=12, kernel=okz.OKZ_KERNEL_PARITY_STREAM,
                       words_per_thread=16, sweeps_per_pass=fuse)
    b = okz.Simulation(L, p, q, seed=12, kernel=okz.OKZ_KERNEL_PARITY_STREAM,
                       words_per_thread=8, sweeps_per_pass=fuse)
    a.sweep(21)
    b.sweep(21)
    assert a.width2() == b.width2()
    pa, ha, ta = a.state()
    pb, hb, tb = b.state()
    assert np.array_equal(pa, pb) and (ha, ta) == (hb, tb)
    a.close()
    b.close()


@pytest.mark.parametrize("L,p,q,kernel", [(16384, 1.0, 0.0, 4), (8192, 0.75, 0.25, 4),
                                          (16384, 1.0, 1.0, 4), (8192, 1.0, 0.0, 2)])
def test_tuned_tiling_is_bit_identical(okz, orc, L, p, q, kernel):
    """okz_tune_stream's choice is used by simulations with automatic tiling
    and gives the same lattice as the untuned default and, at L = 8192, as the
    oracle."""
    base = okz.Simulation(L, p, q, seed=61, kernel=kernel)
    default = (base.wpt, base.fuse)
    base.close()
    wpt, fuse, band, ms = okz.okz_tune_stream(L, p, q, kernel=kernel, probe_sweeps=4)
    assert ms > 0 and (wpt, fuse) != (0, 0) and band in (0, 16, 32)
    a = okz.Simulation(L, p, q, seed=61, kernel=kernel)
    assert (a.wpt, a.fuse, a.band_rows) == (wpt, fuse, band)
    b = okz.Simulation(L, p, q, seed=61, kernel=kernel, words_per_thread=default[0],
                       sweeps_per_pass=default[1], band_rows=32)
    a.sweep(9)
    b.sweep(9)
    pa, ha, ta = a.state()
    pb, hb, tb = b.state()
    assert np.array_equal(pa, pb) and (ha, ta) == (hb, tb)
    if L == 8192:
        ref = orc.Sim(L, p, q, 61)
        ref.sweep(9)
        _compare(a, ref)
    a.close()
    b.close()


@pytest.mark.parametrize("L,p,q", [(8192, 0.75, 0.25), (4096, 1.0, 0.0), (4096, 0.95, 0.05)])
def test_band_heights_are_bit_identical(okz, orc, L, p, q):
    """The stream kernels' band height (okz_params.band_rows) is a launch
    shape only: bands of 5 and 13 rows (one sweep per pass), 9 and 32 (two)
    and the automatic choice give the same lattice in both stream kernels,
    and at L = 4096 the oracle's (7 sweeps: a fused pass and a single one)."""
    n = 7
    ref = None
    if L == 4096:
        ref = orc.Sim(L, p, q, 73)
        ref.sweep(n)
    first = None
    for kernel, fuse, band in [(okz.OKZ_KERNEL_PARITY_STREAM, 1, 0),
                               (okz.OKZ_KERNEL_PARITY_STREAM, 1, 5),
                               (okz.OKZ_KERNEL_PARITY_STREAM, 1, 13),
                               (okz.OKZ_KERNEL_PARITY_STREAM, 2, 9),
                               (okz.OKZ_KERNEL_PARITY_STREAM, 2, 32),
                               (okz.OKZ_KERNEL_STREAM, 1, 5),
                               (okz.OKZ_KERNEL_STREAM, 2, 0)]:
        with okz.Simulation(L, p, q, seed=73, kernel=kernel, words_per_thread=4,
                            sweeps_per_pass=fuse, band_rows=band) as sim:
            assert sim.band_rows == band
            sim.sweep(n)
            planes, H0, t = sim.state()
            if first is None:
                first = (planes, H0, t)
            else:
                assert np.array_equal(planes, first[0]) and (H0, t) == first[1:], (kernel, fuse, band)
            if ref is not None:
                _compare(sim, ref)


def test_wpt16_rejected_where_invalid(okz):
    """16 words per thread needs L % 16384 == 0 and the parity stream kernel."""
    for L, kernel in ((8192, okz.OKZ_KERNEL_PARITY_STREAM), (12288, okz.OKZ_KERNEL_PARITY_STREAM),
                      (16384, okz.OKZ_KERNEL_STREAM)):
        with pytest.raises(okz.OkzError):
            okz.Simulation(L, 1.0, 0.0, seed=1, kernel=kernel, words_per_thread=16)


@pytest.mark.parametrize("kernel", [2, 3, 4])
@pytest.mark.parametrize("L", [4096, 8192, 16384])
def test_stream_equals_plain_long_run(okz, L, kernel):
    """All kernels give identical lattices over many sweeps (no oracle needed)."""
    a = okz.Simulation(L, 0.75, 0.25, seed=5, kernel=kernel)
    b = okz.Simulation(L, 0.75, 0.25, seed=5, kernel=okz.OKZ_KERNEL_PLAIN)
    for n in (10, 40):
        a.sweep(n)
        b.sweep(n)
        pa, ha, ta = a.state()
        pb, hb, tb = b.state()
        assert np.array_equal(pa, pb) and (ha, ta) == (hb, tb)
        assert a.width2() == b.width2()
    a.close()
    b.close()


@pytest.mark.parametrize("L,kernel", [(64, 1), (256, 1), (4096, 2), (64, 3), (256, 3),
                                      (4096, 4), (256, 5), (1024, 5)])
def test_moments_and_heights_match_oracle(okz, orc, L, kernel):
    ref = orc.Sim(L, 0.95, 0.05, 3)
    with okz.Simulation(L, 0.95, 0.05, seed=3, kernel=kernel) as sim:
        ref.sweep(25)
        sim.sweep(25)
        Sk, W2, sk, ku = sim.moments()
        assert Sk == ref.power_sums()
        assert W2 == ref.width2()
        rsk, rku = ref.skew_kurt()
        assert sk == pytest.approx(rsk, rel=1e-12, abs=1e-15)
        assert ku == pytest.approx(rku, rel=1e-12, abs=1e-15)
        h = ref.heights()
        assert np.array_equal(sim.heights(), h)
        assert np.array_equal(sim.heights(y0=L // 2 - 3, ny=5), h[L // 2 - 3:L // 2 + 2])


@pytest.mark.parametrize("kernel", [0, 1, 2, 3, 4, 5])
def test_flat_start_width(okz, kernel):
    for L in (32, 256, 4096):
        if (kernel in (2, 4) and L < 4096) or (kernel == 5 and L > 1024):
            continue
        with okz.Simulation(L, 1.0, 0.0, seed=1, kernel=kernel) as sim:
            S1, S2, W2 = sim.width2()
            assert W2 == 0.25 and S1 == L * L // 2 and S2 == L * L // 2


@pytest.mark.parametrize("kernel", SMALL_KINDS)
def test_growth_series_L256(okz, orc, kernel):
    """L = 256, p = 1, q = 0, seed 1, 1000 sweeps, W^2 at 20 log-spaced times:
    every record equal to the oracle's."""
    times = orc.sample_times(1000, 20)
    ref = orc.Sim(256, 1.0, 0.0, 1)
    with okz.Simulation(256, 1.0, 0.0, seed=1, kernel=kernel) as sim:
        for t in times:
            ref.sweep(t - ref.t)
            sim.sweep(t - sim.info().t)
            S1, S2, W2 = sim.width2()
            assert (S1, S2) == ref.sums() and W2 == ref.width2(), t
            assert sim.info().H0 == ref.H0
        _compare(sim, ref)


@pytest.mark.parametrize("kernel", PLAIN_KINDS)
@pytest.mark.parametrize("L,p,q", [(64, 0.75, 0.25), (256, 1.0, 0.0), (480, 0.95, 0.05)])
def test_inplace_sweeps_by_graph_replay(okz, orc, L, p, q, kernel):
    """n >= 32 sweeps of the in-place kernels go as replays of one CUDA graph
    of 32 sweeps (sweep index from device memory) plus direct launches for
    the rest: 100 = 3 x 32 + 4, then 37 = 32 + 5; lattice, H0 and sums equal
    the oracle's after each call."""
    seed = 300 + L
    ref = orc.Sim(L, p, q, seed)
    with okz.Simulation(L, p, q, seed=seed, kernel=kernel) as sim:
        for n, replays in ((100, 3), (37, 4)):
            ref.sweep(n)
            sim.sweep(n)
            _compare(sim, ref)
            info = sim.info()
            assert (info.graph_chunk, info.graph_replays) == (32, replays)
            S1, S2, W2 = sim.width2()
            assert (S1, S2) == ref.sums() and W2 == ref.width2()


@pytest.mark.parametrize("L,p,q,n", [(1024, 0.95, 0.05, 40), (512, 0.75, 0.25, 300),
                                     (384, 1.0, 1.0, 1000)])
def test_one_cta_kernel_long_calls(okz, orc, L, p, q, n):
    """The one-CTA kernel runs every sweep of a call in one launch: long
    calls at the largest sizes it takes, against the oracle."""
    ref = orc.Sim(L, p, q, 77)
    with okz.Simulation(L, p, q, seed=77, kernel=okz.OKZ_KERNEL_PARITY_CTA) as sim:
        ref.sweep(n)
        sim.sweep(n)
        _compare(sim, ref)
        assert sim.width2()[2] == ref.width2()


def test_one_cta_kernel_size_rule(okz):
    for L in (2048, 1000):
        with pytest.raises(okz.OkzError) as e:
            okz.Simulation(L, 1.0, 0.0, seed=1, kernel=okz.OKZ_KERNEL_PARITY_CTA)
        assert e.value.status == okz.OKZ_EUNSUPPORTED


@pytest.mark.parametrize("L,kernel,p,q", [(4096, 4, 1.0, 0.0), (4096, 4, 0.75, 0.25),
                                          (480, 3, 0.95, 0.05), (256, 5, 1.0, 1.0)])
def test_growth_series_call_matches_per_sample_reads(okz, orc, L, kernel, p, q):
    """okz_growth_series (sweeps and sums queued, one synchronisation)
    gives, at every sample time, the sums okz_width2 reads one by one, and
    the oracle's."""
    times = [0, 1, 3, 4, 9, 16, 17, 30]
    with okz.Simulation(L, p, q, seed=91, kernel=kernel) as a, \
            okz.Simulation(L, p, q, seed=91, kernel=kernel) as b:
        rec = a.growth_series(times)
        ref = orc.Sim(L, p, q, 91)
        for (t, H0, S1, S2, W2) in rec:
            b.sweep(t - b.info().t)
            ref.sweep(t - ref.t)
            assert (S1, S2, W2) == b.width2() and H0 == b.info().H0, t
            assert (S1, S2) == ref.sums() and W2 == ref.width2() and H0 == ref.H0, t
        assert a.info().t == 30
        with pytest.raises(okz.OkzError) as e:
            a.growth_series([29])  # before the current sweep count
        assert e.value.status == okz.OKZ_EINVAL


def test_growth_series_helper_matches_oracle(okz, orc):
    """analysis.growth_series (the product's sampling loop) at L = 256,
    1000 sweeps, 20 samples: every record equals the oracle's."""
    from paper_1110_6745_gb300.analysis import growth_series
    rec = growth_series(256, 1000, 20, p=1.0, q=0.0, seed=1)
    ref = orc.Sim(256, 1.0, 0.0, 1)
    for t, H0, S1, S2, W2 in rec:
        ref.sweep(t - ref.t)
        assert (H0, S1, S2, W2) == (ref.H0, *ref.sums(), ref.width2()), t


def test_checkpoint_resume_is_exact(okz):
    for L, kernel in [(256, 1), (8192, 2), (256, 3), (8192, 4)]:
        a = okz.Simulation(L, 0.75, 0.25, seed=9, kernel=kernel)
        a.sweep(30)
        planes, H0, t = a.state()
        a.sweep(30)
        b = okz.Simulation(L, 0.75, 0.25, seed=9, kernel=kernel)
        b.restore(planes, H0, t)
        b.sweep(30)
        pa, ha, ta = a.state()
        pb, hb, tb = b.state()
        assert np.array_equal(pa, pb) and (ha, ta) == (hb, tb) == (ha, 60)
        a.close()
        b.close()


def test_restore_across_representations(okz, orc):
    """A checkpoint taken from the slope planes resumes on the parity plane and
    vice versa; an odd H0 is rejected (h(0,0) is even)."""
    L = 8192
    ref = orc.Sim(L, 0.75, 0.25, 12)
    ref.sweep(20)
    a = okz.Simulation(L, 0.75, 0.25, seed=12, kernel=okz.OKZ_KERNEL_STREAM)
    a.sweep(10)
    planes, H0, t = a.state()
    b = okz.Simulation(L, 0.75, 0.25, seed=12, kernel=okz.OKZ_KERNEL_PARITY_STREAM)
    b.restore(planes, H0, t)
    b.sweep(5)
    c = okz.Simulation(L, 0.75, 0.25, seed=12, kernel=okz.OKZ_KERNEL_PLAIN)
    pb, hb, tb = b.state()
    c.restore(pb, hb, tb)
    c.sweep(5)
    _compare(c, ref)
    with pytest.raises(okz.OkzError) as e:
        b.restore(planes, H0 + 1, t)
    assert e.value.status == okz.OKZ_EINVAL
    for sim in (a, b, c):
        sim.close()


def test_torch_buffer_and_stream(okz):
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = okz.Simulation(4096, 1.0, 0.0, seed=4, torch_buffer=True)
    assert a.stream == s.cuda_stream
    b = okz.Simulation(4096, 1.0, 0.0, seed=4)
    a.sweep(12)
    b.sweep(12)
    assert np.array_equal(a.state()[0], b.state()[0])
    # device-side state and heights outputs
    dev = torch.empty(2 * 4096 * 4096 // 32, dtype=torch.int32, device="cuda")
    a.state(out=dev)
    assert np.array_equal(dev.cpu().numpy().view(np.uint32).reshape(2, 4096, 128),
                          b.state()[0])
    hd = torch.empty(3 * 4096, dtype=torch.int32, device="cuda")
    a.heights(y0=100, ny=3, out=hd)
    assert np.array_equal(hd.cpu().numpy().reshape(3, 4096), b.heights(y0=100, ny=3))
    a.close()
    b.close()


def test_sweep_counter_overflow(okz):
    with okz.Simulation(64, 1.0, 0.0, seed=1) as sim:
        planes, H0, _ = sim.state()
        sim.restore(planes, H0, 2**32 - 2)
        sim.sweep(1)
        with pytest.raises(okz.OkzError) as e:
            sim.sweep(1)
        assert e.value.status == okz.OKZ_EOVERFLOW


def test_exact_sums_beyond_64_bits(okz, orc):
    """A surface lifted by 2^40: S2 ~ 2^92 stays exact (128-bit)."""
    ref = orc.Sim(64, 0.75, 0.25, 2)
    ref.sweep(9)
    with okz.Simulation(64, 0.75, 0.25, seed=2) as sim:
        sim.sweep(9)
        planes, H0, t = sim.state()
        sim.restore(planes, H0 + 2**40, t)
        ref.H0 += 2**40
        S1, S2, W2 = sim.width2()
        assert (S1, S2) == ref.sums() and S2 > 2**64
        assert W2 == ref.width2()
        with pytest.raises(okz.OkzError) as e:
            sim.heights()
        assert e.value.status == okz.OKZ_EOVERFLOW


# --------------------------------------------------------------------------
# Full-size checks at L = 2^17 (16 GiB lattice state pair on the device)
# --------------------------------------------------------------------------
def _unpack_window(planes_dev, L, x0, y0, w, h):
    """Bits of a w x h window (with periodic wrap) from device planes (2, L, L/32)."""
    import torch
    rows = (torch.arange(h, device=planes_dev.device) + y0) % L
    xs = (torch.arange(w, device=planes_dev.device) + x0) % L
    out = []
    for plane in (0, 1):
        words = planes_dev[plane][rows][:, xs // 32]
        bits = (words >> (xs % 32).to(torch.int32)) & 1
        out.append(bits.to(torch.uint8).cpu().numpy())
    return out


def _invariants_on_device(planes_dev, L):
    """Every row of sigma_x and every column of sigma_y sums to zero, and the
    curl vanishes on every plaquette (bitwise, on the device)."""
    import torch
    Xp, Yp = planes_dev[0], planes_dev[1]
    lut = torch.tensor([bin(i).count("1") for i in range(256)], dtype=torch.int64,
                       device=planes_dev.device)
    colsum = torch.zeros(L, dtype=torch.int64, device=planes_dev.device)
    chunk = 1024
    for y0 in range(0, L, chunk):
        xs = Xp[y0:y0 + chunk]
        ones = lut[xs.contiguous().view(torch.uint8).long()].view(xs.shape[0], -1).sum(1)
        assert bool((ones == L // 2).all()), "row of sigma_x does not sum to 0"
        ys = Yp[y0:y0 + chunk]
        for b in range(32):
            colsum[b::32] += ((ys >> b) & 1).sum(0)
        # curl: X(x,y) + Y(x+1,y) == Y(x,y) + X(x,y+1), as bits
        yn = torch.roll(ys, shifts=-1, dims=1)
        yr = ((ys >> 1) & 0x7FFFFFFF) | ((yn & 1) << 31)  # Y(x+1, y)
        xu = Xp[(torch.arange(y0, y0 + xs.shape[0], device=xs.device) + 1) % L]
        a, c = xs, ys
        assert bool((((a ^ yr) == (c ^ xu)) & ((a & yr) == (c & xu))).all()), "curl"
    assert bool((colsum == L // 2).all()), "column of sigma_y does not sum to 0"


def _check_windows(orc, planes, L, p, q, seed, n, windows):
    """Each window's core (farther than 2n + 1 from its edges) equals the
    oracle's light-cone simulation of the same window, site by site."""
    m = 2 * n + 2
    for (x0, y0, cw, ch) in windows:
        w, h = cw + 2 * m, ch + 2 * m
        x0, y0 = (x0 - m) % L, (y0 - m) % L
        WX, WY = orc.window_flat_sweeps(L, x0, y0, w, h, p, q, seed, n)
        GX, GY = _unpack_window(planes, L, x0, y0, w, h)
        assert np.array_equal(GX[m:h - m, m:w - m], WX[m:h - m, m:w - m]), (x0, y0)
        assert np.array_equal(GY[m:h - m, m:w - m], WY[m:h - m, m:w - m]), (x0, y0)


# Window cores (x, y, width, height) at L = 2^17 for the benchmark's launch
# shape (152 bands of ~862 rows, 256 threads of 16 words per row, 2 sweeps
# per launch): two band boundaries (y = 862, 1724) and a warp boundary
# (x = 16384); the periodic corner (both wraps); the last band boundary
# (y = 130209) with a thread boundary (x = 70144).
WINDOWS_L131072 = [(16300, 780, 200, 1020), ((1 << 17) - 100, (1 << 17) - 100, 200, 200),
                   (70100, 130100, 200, 200)]


def test_full_size_L131072(okz, orc):
    """The headline lattice in the benchmark's launch configuration after 512
    sweeps: windows checked site by site against the oracle's light-cone
    simulation across CTA band, warp and thread boundaries and both periodic
    wraps, global invariants on the device, sampled heights against Eq. (3)
    evaluated by the oracle, and the exact sums against an independent
    chunked reduction."""
    import torch
    L, n, seed = 1 << 17, 512, 11
    with okz.Simulation(L, 1.0, 0.0, seed=seed) as sim:
        info = sim.info()
        assert info.kernel == okz.OKZ_KERNEL_PARITY_STREAM
        assert (info.words_per_thread, info.sweeps_per_pass) == (16, 2)
        sim.sweep(n)
        planes = torch.empty((2, L, L // 32), dtype=torch.int32, device="cuda")
        _, H0, t = sim.state(out=planes)
        assert t == n
        _check_windows(orc, planes, L, 1.0, 0.0, seed, n, WINDOWS_L131072)
        _invariants_on_device(planes, L)
        # sampled heights against the oracle's path sum on the host copy
        host = planes.cpu().numpy().view(np.uint32)
        for y in (0, 1, 863, 65536, L - 1):
            row = sim.heights(y0=y, ny=1)[0]
            for x in (0, 1, 31, 32, 4095, 4096, 99999, L - 1):
                assert row[x] == orc.height_packed(L, host[0], host[1], H0, x, y), (x, y)
        # exact sums against a chunked reduction of the materialised heights
        S1, S2, W2 = sim.width2()
        s1 = s2 = 0
        buf = torch.empty((2048, L), dtype=torch.int32, device="cuda")
        for y0 in range(0, L, 2048):
            sim.heights(y0=y0, ny=2048, out=buf)
            hh = buf.long()
            s1 += int(hh.sum())
            s2 += int((hh * hh).sum())
        assert (S1, S2) == (s1, s2)
        N = L * L
        assert W2 == float(N * s2 - s1 * s1) / (float(N) * float(N)) or \
            W2 == pytest.approx((N * s2 - s1 * s1) / N / N, rel=1e-15)


def test_full_size_L131072_minima_and_maxima(okz, orc):
    """p = q = 1 (k = 1, both branches of the rule, the two-threshold kernel)
    at L = 2^17 in the benchmark's launch shape: 512 sweeps, windows across
    band, warp and thread boundaries and the periodic corner against the
    oracle, and the device invariants."""
    import torch
    L, n, seed = 1 << 17, 512, 13
    with okz.Simulation(L, 1.0, 1.0, seed=seed) as sim:
        info = sim.info()
        assert (info.words_per_thread, info.sweeps_per_pass) == (16, 2)
        sim.sweep(n)
        planes = torch.empty((2, L, L // 32), dtype=torch.int32, device="cuda")
        sim.state(out=planes)
        _check_windows(orc, planes, L, 1.0, 1.0, seed, n, WINDOWS_L131072[:2])
        _invariants_on_device(planes, L)


def test_wpt16_two_sweep_kernel_against_oracle_L32768(okz, orc):
    """The 16-word, two-sweeps-per-launch kernel at L = 2^15 (152 bands of
    ~215 rows, two warps per row) against the full-lattice oracle after 64
    sweeps: every bond, H0 and the exact sums."""
    L, n, seed = 32768, 64, 19
    ref = orc.Sim(L, 1.0, 0.0, seed)
    ref.sweep(n)
    with okz.Simulation(L, 1.0, 0.0, seed=seed) as sim:
        info = sim.info()
        assert (info.words_per_thread, info.sweeps_per_pass) == (16, 2)
        sim.sweep(n)
        _compare(sim, ref)
        S1, S2, W2 = sim.width2()
        assert (S1, S2) == ref.sums() and W2 == ref.width2()


def _golden_rows(path):
    rows, digest = [], None
    for line in open(path):
        if line.startswith("# final_planes_sha256"):
            digest = line.split()[-1]
        elif line.strip() and not line.startswith("#"):
            t, H0, S1, S2, W2 = line.split()
            rows.append((int(t), int(H0), int(S1), int(S2), float(W2)))
    return rows, digest


def test_growth_series_L16384_golden(okz):
    """L = 2^14, p = 1, q = 0, seed 7, 10^4 sweeps, 40 log-spaced samples:
    every (t, H0, S1, S2, W^2) record and the final planes equal the oracle's
    stored run (tests/golden/make_growth_golden.py)."""
    import hashlib
    path = os.path.join(GOLDEN, "growth_L16384_p1_q0_seed7.txt")
    if not os.path.exists(path):
        pytest.fail("golden series missing: run tests/golden/make_growth_golden.py")
    rows, digest = _golden_rows(path)
    with okz.Simulation(16384, 1.0, 0.0, seed=7) as sim:
        assert sim.info().kernel == okz.OKZ_KERNEL_PARITY_STREAM
        for (t, H0, S1, S2, W2) in rows:
            sim.sweep(t - sim.info().t)
            s1, s2, w2 = sim.width2()
            assert (sim.info().t, sim.info().H0, s1, s2, w2) == (t, H0, S1, S2, W2)
        planes, _, _ = sim.state()
        assert hashlib.sha256(planes.tobytes()).hexdigest() == digest


# --------------------------------------------------------------------------
# Domain-decomposed random-sequential sweeps (okz_sweep_rs)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L,p,q,seed", [(32, 1.0, 0.0, 1), (64, 0.75, 0.25, 2),
                                         (128, 1.0, 1.0, 3), (96, 0.5, 0.5, 4),
                                         (320, 0.95, 0.05, 5), (512, 1.0, 0.0, 6)])
def test_random_sequential_sweeps_match_oracle(okz, orc, L, p, q, seed):
    ref = orc.Sim(L, p, q, seed)
    with okz.Simulation(L, p, q, seed=seed, kernel=okz.OKZ_KERNEL_PARITY_PLAIN) as sim:
        for n in (1, 4):
            ref.ddrs_sweep(n)
            sim.sweep_rs(n)
            _compare(sim, ref)
        # interleaved with checkerboard sweeps, sharing the sweep counter
        ref.sweep(2)
        sim.sweep(2)
        ref.ddrs_sweep(1)
        sim.sweep_rs(1)
        _compare(sim, ref)
        S1, S2, W2 = sim.width2()
        assert (S1, S2) == ref.sums() and W2 == ref.width2()


def test_random_sequential_needs_parity_plane(okz):
    with okz.Simulation(64, 1.0, 0.0, seed=1, kernel=okz.OKZ_KERNEL_PLAIN) as sim:
        with pytest.raises(okz.OkzError) as e:
            sim.sweep_rs(1)
        assert e.value.status == okz.OKZ_EUNSUPPORTED


def test_random_sequential_growth_exponent(okz):
    """The paper's own (random-sequential, blocked) dynamics and the
    checkerboard schedule give compatible growth exponents at L = 2048."""
    def beta(step_rs):
        ts = [0] + [int(round(10 ** (1 + 2 * j / 19))) for j in range(20)]
        acc = np.zeros(len(ts))
        for sd in range(3):
            with okz.Simulation(2048, 1.0, 0.0, seed=40 + sd) as sim:
                w, done = [], 0
                for t in ts:
                    (sim.sweep_rs if step_rs else sim.sweep)(t - done)
                    done = t
                    w.append(sim.width2()[2])
            acc += np.array(w)
        acc /= 3
        tt, ww = np.array(ts[1:], float), acc[1:]
        m = tt >= 100
        return np.polyfit(np.log(tt[m]), 0.5 * np.log(ww[m] - 0.25), 1)[0]
    b_rs, b_cb = beta(True), beta(False)
    assert 0.20 <= b_rs <= 0.28 and 0.20 <= b_cb <= 0.28, (b_rs, b_cb)
    assert abs(b_rs - b_cb) < 0.04, (b_rs, b_cb)


def test_moments_enqueue_then_fetch(okz, orc):
    """okz_moments_enqueue / okz_moments_fetch return what okz_moments returns
    at the enqueue point, even with sweeps enqueued in between."""
    ref = orc.Sim(480, 0.75, 0.25, 77)
    ref.sweep(9)
    with okz.Simulation(480, 0.75, 0.25, seed=77, kernel=okz.OKZ_KERNEL_PARITY_PLAIN) as sim:
        sim.sweep(9)
        direct = sim.moments()
        sim.moments_enqueue()
        sim.sweep(3)
        assert sim.moments_fetch() == direct
        assert direct[0] == ref.power_sums()
        assert sim.moments() != direct  # the later sweeps are there


@pytest.mark.parametrize("L,kernel", [(4096, 4), (4096, 2), (256, 5), (480, 3)])
def test_staged_restore_equals_restore(okz, orc, L, kernel):
    """okz_stage_host + okz_restore_staged give the state okz_restore gives,
    also when the next copy is staged while the simulation sweeps."""
    ref = orc.Sim(L, 0.75, 0.25, 5)
    ref.sweep(6)
    Xw, Yw = ref.packed()
    planes = np.stack([Xw, Yw]).astype(np.uint32)
    with okz.Simulation(L, 0.75, 0.25, seed=5, kernel=kernel) as a, \
            okz.Simulation(L, 0.75, 0.25, seed=5, kernel=kernel) as b:
        a.stage_host(planes)
        a.restore_staged(ref.H0, ref.t)
        a.stage_host(planes)        # staged while the sweeps below run
        a.sweep(5)
        b.restore(planes, ref.H0, ref.t)
        b.sweep(5)
        assert a.width2() == b.width2()
        pa, ha, ta = a.state()
        pb, hb, tb = b.state()
        assert np.array_equal(pa, pb) and (ha, ta) == (hb, tb)
        a.restore_staged(ref.H0, ref.t)  # the second copy: the same input again
        _compare(a, ref)
        with pytest.raises(okz.OkzError) as e:
            a.restore_staged(ref.H0, ref.t)  # nothing staged
        assert e.value.status == okz.OKZ_EINVAL
