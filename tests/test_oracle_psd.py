"""Pins of the power-spectrum oracle (Sec. III, Eqs. (15)-(16))."""
import cmath
import math

import numpy as np
import pytest

from oracle import psd


def _dft_by_hand(h):
    """Eq. (16) by its double sum, in plain Python complex arithmetic."""
    L = len(h)
    mean = sum(sum(r) for r in h) / (L * L)
    S = [[0.0] * L for _ in range(L)]
    for ky in range(L):
        for kx in range(L):
            acc = 0j
            for y in range(L):
                for x in range(L):
                    acc += (h[y][x] - mean) * cmath.exp(2j * math.pi * (kx * x + ky * y) / L)
            S[ky][kx] = abs(acc / L) ** 2
    return S


@pytest.mark.parametrize("L,seed", [(4, 1), (6, 2), (8, 3)])
def test_psd_matches_the_double_sum(L, seed):
    h = np.random.default_rng(seed).integers(-5, 6, size=(L, L))
    S = psd.psd_2d(h)
    ref = np.array(_dft_by_hand(h.tolist()))
    assert np.allclose(S, ref, rtol=1e-12, atol=1e-12)
    ax = psd.psd_axes(h)
    assert np.allclose(ax, 0.5 * (ref[0, :] + ref[:, 0]), rtol=1e-12, atol=1e-12)


def test_single_mode_closed_form():
    """h = cos(2 pi m x / L): |h(k)|^2 = L^2 / 4 at k = (+-m, 0), zero
    elsewhere, so the axis average is L^2 / 8 at k = m and L - m."""
    L, m = 32, 5
    x = np.arange(L)
    h = np.tile(np.cos(2 * np.pi * m * x / L), (L, 1))
    ax = psd.psd_axes(h)
    want = np.zeros(L)
    want[m] = want[L - m] = L * L / 8
    assert np.allclose(ax, want, atol=1e-9)
    hy = h.T.copy()  # the same mode along y gives the same axis average
    assert np.allclose(psd.psd_axes(hy), want, atol=1e-9)


def test_parseval_gives_the_width(orc):
    """sum over all k of S(k) = sum_chi (h - <h>)^2 = N W^2 (Eq. (4))."""
    sim = orc.Sim(64, 1.0, 0.0, 21)
    sim.sweep(40)
    h = sim.heights()
    N = 64 * 64
    assert psd.psd_2d(h).sum() == pytest.approx(N * sim.width2(), rel=1e-12)
    assert psd.psd_axes(h)[0] == pytest.approx(0.0, abs=1e-12)


def test_axis_cut_is_the_transform_of_the_profile_sums(orc):
    """S(k, 0) = |sum_x col[x] e^(i k x)|^2 / L^2 for k != 0, where col are
    the column sums (the mean only enters k = 0); likewise S(0, k) and the
    row sums. This is the reduction the device computes."""
    L = 96
    sim = orc.Sim(L, 0.75, 0.25, 22)
    sim.sweep(30)
    h = sim.heights()
    col, row = psd.profile_sums(h, sim.H0)
    assert col.sum() == row.sum() == int(h.sum()) - L * L * sim.H0
    S = psd.psd_2d(h)
    k = np.arange(L)
    E = np.exp(2j * np.pi * np.outer(k, np.arange(L)) / L)
    Sc = np.abs(E @ col.astype(float)) ** 2 / L ** 2
    Sr = np.abs(E @ row.astype(float)) ** 2 / L ** 2
    tol = 1e-12 * S.sum()
    assert np.allclose(S[0, 1:], Sc[1:], rtol=0, atol=tol)
    assert np.allclose(S[1:, 0], Sr[1:], rtol=0, atol=tol)
    # the oracle's large-lattice form agrees with the 2-D definition
    Sa = psd.psd_axes_from_profiles(col, row)
    assert Sa[0] == 0.0
    assert np.allclose(Sa, psd.psd_axes(h), rtol=0, atol=tol)


def test_profile_sums_by_hand():
    h = np.array([[1, 2, 3], [4, 5, 6], [7, 8, 10]])
    col, row = psd.profile_sums(h, 1)
    assert col.tolist() == [1 + 4 + 7 - 3, 2 + 5 + 8 - 3, 3 + 6 + 10 - 3]
    assert row.tolist() == [1 + 2 + 3 - 3, 4 + 5 + 6 - 3, 7 + 8 + 10 - 3]
