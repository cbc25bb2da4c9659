"""Oracle of the interface power spectrum (Kelling & Odor, Sec. III, Eqs. (15)-(16)).

TEST INFRASTRUCTURE, like the rest of this package: only tests/, the smoke
check and the benchmark's CPU legs use it; the CUDA library never imports it.

Definitions, written out on a height array h[y, x] of an L x L periodic
lattice (d = 2):

* Eq. (16): h(k) = L^(-d/2) sum_chi [h(chi) - <h>] exp(i k . chi), with
  k = 2 pi (kx, ky) / L. numpy's fft2 is the library step; its opposite sign
  convention gives h(-k), and |h(-k)| = |h(k)| for a real surface.
* Eq. (15): S(k) = <h(k) h(-k)> = |h(k)|^2 for one surface.
* "Averaged over the x and y directions" (Sec. III) is read as the mean of the
  two axis cuts: S_axes[k] = (S(k, 0) + S(0, k)) / 2 for k = 0 .. L-1, the
  index k standing for the wave number 2 pi k / L.

The column and row profile sums col[x] = sum_y (h[y, x] - c) and
row[y] = sum_x (h[y, x] - c) are plain sums of the array. On the k axes the
2-D transform reduces to the 1-D transforms of these sums (the mean only
enters k = 0), which gives the axis spectrum of large lattices without the
L x L transform.
"""
import numpy as np


def profile_sums(h, c=0):
    """(col, row) as int64: col[x] = sum_y (h[y, x] - c), row[y] = sum_x (h[y, x] - c)."""
    d = np.asarray(h, dtype=np.int64) - np.int64(c)
    return d.sum(axis=0), d.sum(axis=1)


def psd_2d(h):
    """S(k) of Eqs. (15)-(16) on the full L x L grid of wave vectors, indexed
    [ky, kx] (fp64)."""
    a = np.asarray(h, dtype=np.float64)
    L = a.shape[0]
    assert a.shape == (L, L)
    hk = np.fft.fft2(a - a.mean()) / L  # L^(-d/2) with d = 2
    return np.abs(hk) ** 2


def psd_axes(h):
    """S_axes[k] = (S(k, 0) + S(0, k)) / 2, k = 0 .. L-1."""
    S = psd_2d(h)
    return 0.5 * (S[0, :] + S[:, 0])


def psd_axes_from_profiles(col, row):
    """S_axes[k] from the profile sums: (|C(k)|^2 + |R(k)|^2) / (2 L^2) for
    k != 0, C and R the 1-D transforms of col and row (numpy's fft), and
    S_axes[0] = 0 (the mean is removed). Equal to psd_axes of the heights."""
    col = np.asarray(col, dtype=np.float64)
    row = np.asarray(row, dtype=np.float64)
    L = col.shape[0]
    S = (np.abs(np.fft.fft(col)) ** 2 + np.abs(np.fft.fft(row)) ** 2) / (2.0 * L * L)
    S[0] = 0.0
    return S
