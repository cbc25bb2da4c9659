"""Batched and pooled lattices: every slot evolves exactly like its own simulation."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def okz():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1110_6745_gb300 import _build
    _build.build()
    import paper_1110_6745_gb300 as m
    m.lib()
    return m


def _single(okz, L, p, q, seed, n):
    """The same lattice run on its own (parity plane, plain kernel)."""
    with okz.Simulation(L, p, q, seed=seed, kernel=okz.OKZ_KERNEL_PARITY_PLAIN) as sim:
        sim.sweep(n)
        planes, H0, t = sim.state()
        Sk, W2, sk, ku = sim.moments()
    return planes, H0, t, Sk, W2, sk, ku


MIX = [(64, 1.0, 0.0, 1), (128, 0.95, 0.05, 2), (96, 0.75, 0.25, 3), (256, 1.0, 1.0, 4),
       (512, 0.5, 0.5, 5), (1024, 0.95, 0.05, 6), (2048, 1.0, 0.0, 7), (32, 0.3, 0.6, 8)]


@pytest.mark.parametrize("threads,smem", [(1024, 32 * 1024), (512, 128 * 1024), (256, 0)])
def test_batch_matches_single_runs(okz, threads, smem):
    L = [m[0] for m in MIX]
    with okz.Batch(L, [m[1] for m in MIX], [m[2] for m in MIX], [m[3] for m in MIX]) as b:
        b.set_tiling(threads, smem)
        first = [3, 5, 0, 2, 7, 1, 4, 9]
        second = [4, 0, 6, 1, 1, 3, 2, 0]
        b.run(first)
        b.run(second)
        W2, sk, ku = b.stats()
        for i, (Li, p, q, seed) in enumerate(MIX):
            n = first[i] + second[i]
            planes, H0, t, Sk, w2, s1, k1 = _single(okz, Li, p, q, seed, n)
            bp, bH0, bt = b.state(i)
            assert np.array_equal(bp, planes) and (bH0, bt) == (H0, t), i
            assert b.sums(i)[0] == Sk
            assert W2[i] == w2
            assert sk[i] == pytest.approx(s1, rel=1e-12, abs=1e-15)
            assert ku[i] == pytest.approx(k1, rel=1e-12, abs=1e-15)


def test_batch_matches_oracle(okz, orc):
    cases = [(64, 0.95, 0.05, 1000), (96, 1.0, 0.0, 1001), (128, 0.75, 0.25, 1002)]
    with okz.Batch([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases],
                   [c[3] for c in cases]) as b:
        b.run([40, 25, 31])
        for i, (L, p, q, seed) in enumerate(cases):
            ref = orc.Sim(L, p, q, seed)
            ref.sweep([40, 25, 31][i])
            planes, H0, t = b.state(i)
            Xw, Yw = ref.packed()
            assert np.array_equal(planes[0], Xw) and np.array_equal(planes[1], Yw)
            assert (H0, t) == (ref.H0, ref.t)
            Sk, _, _ = b.sums(i)
            assert Sk == ref.power_sums()


def test_pool_admission_and_reuse(okz):
    """Slots and arena space are admitted, refused when full, freed and reused;
    untouched slots keep their state across other slots' runs."""
    one = 256 * 256 // 8
    with okz.Batch(arena_bytes=3 * one, max_slots=4) as b:
        a = b.add(256, 1.0, 0.0, 11)
        c = b.add(256, 0.75, 0.25, 12)
        d = b.add(128, 1.0, 0.0, 13)
        with pytest.raises(okz.OkzError) as e:  # arena full
            b.add(256, 1.0, 0.0, 14)
        assert e.value.status == okz.OKZ_EBUSY
        b.run({a: 10, c: 4})
        b.remove(a)
        e2 = b.add(256, 1.0, 0.0, 15)
        b.run({e2: 6, c: 3, d: 2})
        b.sync()
        for slot, (L, p, q, seed, n) in {c: (256, 0.75, 0.25, 12, 7), e2: (256, 1.0, 0.0, 15, 6),
                                         d: (128, 1.0, 0.0, 13, 2)}.items():
            planes, H0, t, *_ = _single(okz, L, p, q, seed, n)
            bp, bH0, bt = b.state(slot)
            assert np.array_equal(bp, planes) and (bH0, bt) == (H0, t)
        with pytest.raises(okz.OkzError):
            b.run({a: 1} if a != e2 else {3: 1})  # empty slot with work


def test_autotune_keeps_results(okz):
    L = [2048, 1024, 256, 64]
    with okz.Batch(L, [1.0] * 4, [0.0] * 4, [1, 2, 3, 4]) as b:
        b.autotune(probe_sweeps=2)
        th, sm, grid = b.tiling()
        assert th in (256, 512, 1024) and grid >= 152
        b.run([3, 3, 3, 3])
        for i in range(4):
            planes, H0, t, *_ = _single(okz, L[i], 1.0, 0.0, i + 1, 3)
            assert np.array_equal(b.state(i)[0], planes)


def test_replica_mix_matches_single_runs(okz):
    """The 4096-replica workload's mix -- L = 2^e, e ~ U{6..11} (numpy PCG64,
    seed 2026), seeds 1000 + r, p = 0.95, q = 0.05 -- with budgets of
    ceil(4 L^1.61) / 4096 sweeps: a 48-replica sample checked against runs of
    their own, all six sizes included."""
    rng = np.random.Generator(np.random.PCG64(2026))
    e = rng.integers(6, 12, size=4096)
    L = (1 << e).astype(np.int64)
    T = np.ceil(4 * L.astype(np.float64) ** 1.61).astype(np.int64)
    pick = []
    for size in range(6, 12):
        pick += list(np.nonzero(e == size)[0][:8])
    Ls = [int(L[r]) for r in pick]
    sweeps = [max(1, int(T[r] // 4096)) for r in pick]
    with okz.Batch(Ls, [0.95] * len(pick), [0.05] * len(pick), [1000 + int(r) for r in pick]) as b:
        b.run(sweeps)
        W2, _, _ = b.stats()
        for j, r in enumerate(pick):
            planes, H0, t, Sk, w2, *_ = _single(okz, Ls[j], 0.95, 0.05, 1000 + int(r), sweeps[j])
            assert np.array_equal(b.state(j)[0], planes) and W2[j] == w2, (j, Ls[j])


def test_full_replica_mix_against_single_runs_and_oracle(okz, orc):
    """All 4096 replicas of the batched workload's mix (budgets
    ceil(4 L^1.61) / 4096 sweeps) in one batch: every replica's exact sums
    S1..S4 and H0 equal a run of its own with the in-place parity kernel, and
    a 66-replica subset (11 of each size L = 64 .. 2048) equals the CPU
    oracle bit for bit."""
    rng = np.random.Generator(np.random.PCG64(2026))
    e = rng.integers(6, 12, size=4096)
    L = (1 << e).astype(np.int64)
    T = np.ceil(4 * L.astype(np.float64) ** 1.61).astype(np.int64)
    sweeps = np.maximum(1, T // 4096)
    n = len(L)
    with okz.Batch([int(x) for x in L], [0.95] * n, [0.05] * n,
                   [1000 + r for r in range(n)]) as b:
        b.run(sweeps)
        got = b.measure(range(n))
    for r in range(n):
        Sk, H0, t = got[r]
        with okz.Simulation(int(L[r]), 0.95, 0.05, seed=1000 + r,
                            kernel=okz.OKZ_KERNEL_PARITY_PLAIN) as sim:
            sim.sweep(int(sweeps[r]))
            ref_Sk, _, _, _ = sim.moments()
            assert (Sk, H0, t) == (ref_Sk, sim.info().H0, int(sweeps[r])), r
    subset = []
    for size in range(6, 12):
        subset += [int(r) for r in np.nonzero(e == size)[0][:11]]
    for r in subset:
        ref = orc.Sim(int(L[r]), 0.95, 0.05, 1000 + r)
        ref.sweep(int(sweeps[r]))
        Sk, H0, t = got[r]
        assert Sk == ref.power_sums() and H0 == ref.H0 and t == ref.t, r


@pytest.mark.parametrize("threads,smem", [(1024, 32 * 1024), (512, 64 * 1024), (256, 0)])
def test_band_wavefront_sizes_match_single_runs(okz, threads, smem):
    """The band wavefront at the sizes the replica mix does not reach: bands
    that do not divide L (L = 384, 640: 3 and 5 groups a row), lattices swept
    in global memory at 4096 and 8192 (bands of 4 rows at 256 threads), and
    the k = 32, k = 3 and k = 1 acceptance paths, against runs of their own."""
    cases = [(384, 0.95, 0.05, 21), (640, 0.75, 0.25, 22), (4096, 0.95, 0.05, 23),
             (8192, 1.0, 0.0, 24), (8192, 0.5, 0.5, 25), (1152, 1.0, 1.0, 26)]
    sweeps = [7, 5, 3, 2, 3, 6]
    with okz.Batch([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases],
                   [c[3] for c in cases]) as b:
        b.set_tiling(threads, smem)
        b.run(sweeps)
        for i, (L, p, q, seed) in enumerate(cases):
            planes, H0, t, *_ = _single(okz, L, p, q, seed, sweeps[i])
            bp, bH0, bt = b.state(i)
            assert np.array_equal(bp, planes) and (bH0, bt) == (H0, t), (L, p, q)
