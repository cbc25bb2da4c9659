"""GPU parity of the interface profiles and the power spectrum (Sec. III,
Eqs. (15)-(16)) against the oracle.

The profiles are exact integers and must match bit for bit. The spectrum is
fp64 on both sides: the device runs radix-2 FFTs on the exact profiles, the
oracle a 2-D FFT of the heights. For an FFT of length L the normwise error
is at most about 5 log2(L) eps ||x|| (eps = 2^-53), so each |h(k)|^2 is off
by at most ~1.4e-14 of the spectrum's total on the axes; the tests allow
1e-12 of that total per k.
"""
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


def _oracle_heights(orc, sim, L, p, q, seed):
    planes, H0, t = sim.state()
    ref = orc.Sim(L, p, q, seed)
    ref.load_packed(planes[0], planes[1], H0, t)
    return ref.heights(), H0


CASES = [  # L, kernel, p, q, sweeps
    (32, 1, 1.0, 0.0, 7),
    (32, 3, 0.75, 0.25, 9),
    (96, 3, 0.5, 0.5, 20),
    (96, 1, 1.0, 0.0, 13),
    (256, 3, 1.0, 0.0, 50),
    (256, 1, 0.95, 0.05, 31),
    (4096, 4, 1.0, 0.0, 12),
    (4096, 2, 0.75, 0.25, 5),
    (8192, 4, 1.0, 1.0, 6),
]


@pytest.mark.parametrize("L,kernel,p,q,n", CASES)
def test_profiles_match_oracle(okz, orc, L, kernel, p, q, n):
    from oracle import psd
    with okz.Simulation(L, p, q, seed=L + n, kernel=kernel) as sim:
        sim.sweep(n)
        col, row = sim.profiles()
        h, H0 = _oracle_heights(orc, sim, L, p, q, L + n)
    rc, rr = psd.profile_sums(h, H0)
    assert np.array_equal(col, rc)
    assert np.array_equal(row, rr)


@pytest.mark.parametrize("L,kernel,p,q,n", [c for c in CASES if (c[0] & (c[0] - 1)) == 0
                                             and c[0] <= 4096])
def test_psd_matches_oracle(okz, orc, L, kernel, p, q, n):
    from oracle import psd
    with okz.Simulation(L, p, q, seed=3 * L + n, kernel=kernel) as sim:
        sim.sweep(n)
        S = sim.psd()
        h, _ = _oracle_heights(orc, sim, L, p, q, 3 * L + n)
    ref = psd.psd_axes(h)
    tol = 1e-12 * ref.sum()
    assert S[0] == 0.0
    assert np.max(np.abs(S - ref)) <= tol, (np.max(np.abs(S - ref)), tol)


def test_psd_of_the_striped_start(okz):
    """h = (x+y) mod 2: every column and row has the same sum, so the spectrum
    on the axes vanishes."""
    with okz.Simulation(256, 1.0, 0.0, seed=1) as sim:
        col, row = sim.profiles()
        assert np.all(col == 128) and np.all(row == 128)
        assert np.all(sim.psd() == 0.0)


def test_psd_needs_power_of_two(okz):
    with okz.Simulation(96, 1.0, 0.0, seed=1, kernel=okz.OKZ_KERNEL_PARITY_PLAIN) as sim:
        with pytest.raises(okz.OkzError) as e:
            sim.psd()
        assert e.value.status == okz.OKZ_EUNSUPPORTED
        sim.profiles()  # profiles work for any L


def test_profiles_sum_to_the_height_sum(okz):
    """sum col = sum row = S1 - N H0 at the size of the growth benchmark's
    lattice family (L = 2^15, parity stream kernel)."""
    L = 32768
    with okz.Simulation(L, 1.0, 0.0, seed=5) as sim:
        sim.sweep(20)
        S1, _, _ = sim.width2()
        col, row = sim.profiles()
        H0 = sim.info().H0
    assert int(col.sum()) == int(row.sum()) == S1 - L * L * H0
