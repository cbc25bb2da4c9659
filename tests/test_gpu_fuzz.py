"""Seeded random configurations against the oracle: sizes, (p, q, s_sel,
k_max), seeds, sweep counts and kernels drawn from a fixed generator, each
run compared bit for bit (planes, H0, t, exact sums, W^2)."""
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


def _configs(n=40, seed=20261204):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        kernel = int(rng.choice([1, 3, 3, 2, 4]))
        if kernel in (2, 4):
            L = 4096
        else:
            L = int(32 * rng.integers(1, 17))          # 32 .. 512, any multiple of 32
        p = float(rng.choice([0.0, 0.1, 0.5, 0.75, 0.9, 1.0, rng.uniform(0, 1)]))
        q = float(rng.choice([0.0, 0.25, 0.5, 1.0, rng.uniform(0, 1)]))
        s_sel = float(rng.choice([0.5, 0.5, 1.0, 0.25, 0.8]))
        k_max = int(rng.choice([32, 32, 8, 3, 1]))
        sweeps = int(rng.integers(1, 12 if L == 4096 else 40))
        out.append((i, L, kernel, p, q, s_sel, k_max, int(rng.integers(0, 2 ** 40)), sweeps))
    return out


@pytest.mark.parametrize("i,L,kernel,p,q,s_sel,k_max,seed,sweeps", _configs())
def test_random_configuration(okz, orc, i, L, kernel, p, q, s_sel, k_max, seed, sweeps):
    ref = orc.Sim(L, p, q, seed, s_sel=s_sel, k_max=k_max)
    ref.sweep(sweeps)
    with okz.Simulation(L, p, q, seed=seed, s_sel=s_sel, k_max=k_max, kernel=kernel) as sim:
        sim.sweep(sweeps)
        planes, H0, t = sim.state()
        S1, S2, W2 = sim.width2()
    Xw, Yw = ref.packed()
    assert np.array_equal(planes[0], Xw) and np.array_equal(planes[1], Yw)
    assert (H0, t) == (ref.H0, ref.t)
    assert (S1, S2) == ref.sums() and W2 == ref.width2()


@pytest.mark.parametrize("j", range(8))
def test_random_sequential_random_configuration(okz, orc, j):
    rng = np.random.Generator(np.random.PCG64(777 + j))
    L = int(32 * rng.integers(1, 9))
    p, q = float(rng.uniform(0, 1)), float(rng.uniform(0, 1))
    seed, n = int(rng.integers(0, 2 ** 40)), int(rng.integers(1, 6))
    ref = orc.Sim(L, p, q, seed)
    ref.ddrs_sweep(n)
    with okz.Simulation(L, p, q, seed=seed, kernel=okz.OKZ_KERNEL_PARITY_PLAIN) as sim:
        sim.sweep_rs(n)
        planes, H0, t = sim.state()
    Xw, Yw = ref.packed()
    assert np.array_equal(planes[0], Xw) and np.array_equal(planes[1], Yw)
    assert (H0, t) == (ref.H0, ref.t)
