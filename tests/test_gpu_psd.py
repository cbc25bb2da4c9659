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
    (12288, 2, 0.75, 0.25, 3),  # slope planes; the second 256-word column block half idle
    (16384, 4, 1.0, 0.0, 4),    # two full column blocks
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


@pytest.mark.parametrize("kernel,p,q", [(4, 0.75, 0.25), (2, 1.0, 0.0)])
def test_profiles_against_bond_counts_and_heights(okz, kernel, p, q):
    """L = 2^15 (eight 256-word column blocks, many bands): every step of both
    profiles equals 2 n - L for the bond counts of the state, the profiles
    close periodically, col[0] is the sum of column 0's heights (built from
    its y-bonds, Eq. (3)) and sampled rows match the device heights."""
    L = 32768
    with okz.Simulation(L, p, q, seed=9, kernel=kernel) as sim:
        sim.sweep(6)
        col, row = sim.profiles()
        planes, H0, _ = sim.state()
        rows = {y: sim.heights(y, 1)[0].astype(np.int64) for y in (0, 1, 12345, L - 1)}
        col0_h = {y: int(sim.heights(y, 1)[0][0]) for y in (5, 20000)}
    bits = np.unpackbits(planes[0].view(np.uint8), axis=-1, bitorder="little")
    nX = bits.sum(axis=0, dtype=np.int64)
    del bits
    bits = np.unpackbits(planes[1].view(np.uint8), axis=-1, bitorder="little")
    nY = bits.sum(axis=1, dtype=np.int64)
    sy0 = 2 * bits[:, 0].astype(np.int64) - 1
    del bits
    assert np.array_equal(np.diff(col), 2 * nX[:-1] - L)
    assert np.array_equal(np.diff(row), 2 * nY[:-1] - L)
    assert col[-1] + 2 * nX[-1] - L == col[0] and row[-1] + 2 * nY[-1] - L == row[0]
    h0 = np.concatenate([[0], np.cumsum(sy0)[:-1]])  # h(0, y) - H0
    assert col[0] == h0.sum()
    for y, hy in col0_h.items():
        assert hy - H0 == h0[y]
    for y, hy in rows.items():
        assert row[y] == hy.sum() - L * H0


@pytest.mark.parametrize("L,kernel,p,q,n", [(8192, 4, 0.75, 0.25, 4), (16384, 4, 1.0, 0.0, 6)])
def test_psd_large_matches_oracle(okz, orc, L, kernel, p, q, n):
    """Lattices whose transforms go on past the shared-memory block (L = 2^13:
    a radix-2 stage and a radix-4 step; L = 2^14: two radix-4 steps)
    against the oracle's axis spectrum from its profile sums of the same
    state."""
    from oracle import psd
    with okz.Simulation(L, p, q, seed=5 * L + n, kernel=kernel) as sim:
        sim.sweep(n)
        S = sim.psd()
        h, H0 = _oracle_heights(orc, sim, L, p, q, 5 * L + n)
    col, row = psd.profile_sums(h, H0)
    del h
    ref = psd.psd_axes_from_profiles(col, row)
    assert S[0] == 0.0
    assert np.max(np.abs(S - ref)) <= 1e-12 * ref.sum()


@pytest.mark.parametrize("L", [32768, 131072])
def test_psd_parseval_and_sampled_modes(okz, L):
    """At L = 2^15 and 2^17 (the benchmark's size; radix-4 steps before the
    last) the spectrum satisfies Parseval's identity with the profiles,
    sum_k S = (L sum col^2 - (sum col)^2 + L sum row^2 - (sum row)^2) / (2 L^2),
    and sampled modes equal the explicit sums of Eq. (16) over the profiles."""
    with okz.Simulation(L, 1.0, 0.0, seed=21) as sim:
        sim.sweep(40)
        col, row = sim.profiles()
        S = sim.psd()
    c = col.astype(np.float64)
    r = row.astype(np.float64)
    tot = (L * np.sum(c * c) - np.sum(c) ** 2 + L * np.sum(r * r) - np.sum(r) ** 2) / (2.0 * L * L)
    assert S[0] == 0.0
    assert abs(S.sum() - tot) <= 1e-10 * tot
    x = np.arange(L)
    for k in (1, 2, 3, 7, L // 2 - 1, L // 2, L // 2 + 5, L - 1):
        e = np.exp(-2j * np.pi * ((k * x) % L) / L)
        Sk = (abs(np.dot(c, e)) ** 2 + abs(np.dot(r, e)) ** 2) / (2.0 * L * L)
        assert abs(S[k] - Sk) <= 1e-11 * tot, (k, S[k], Sk)
