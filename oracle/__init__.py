"""Plain CPU oracle of the octahedron-model sweep (Kelling & Odor, arXiv:1110.6745).

TEST INFRASTRUCTURE. Only tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU legs (CPU baseline, reference arm) may import this package. The product path (the CUDA library
under ``paper_1110_6745_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``okz_oracle.c``; this module only marshals numpy
arrays through ctypes and converts the oracle's one-byte-per-bond state into
the packed bit-plane layout of the C-ABI so that tests can compare the two.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    c = ctypes
    L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.orc_philox4x32_10.restype = None
    L.orc_thresholds.argtypes = [c.c_double, c.c_double, c.c_double, c.c_int,
                                 c.POINTER(c.c_int), c.POINTER(c.c_uint64),
                                 c.POINTER(c.c_uint64)]
    L.orc_thresholds.restype = c.c_int
    L.orc_rs_threshold.argtypes = [c.c_double]
    L.orc_rs_threshold.restype = c.c_uint64
    L.orc_site_uniform.argtypes = [c.c_uint64, c.c_int64, c.c_int64, c.c_int64,
                                   c.c_uint64, c.c_int]
    L.orc_site_uniform.restype = c.c_uint64
    L.orc_init_flat.argtypes = [c.c_int64, u8p, u8p]
    L.orc_init_flat.restype = None
    L.orc_halfsweep.argtypes = [c.c_int64, u8p, u8p, c.POINTER(c.c_int64),
                                c.c_uint64, c.c_uint64, c.c_int, c.c_int,
                                c.c_uint64, c.c_uint64]
    L.orc_halfsweep.restype = None
    L.orc_halfsweep_ordered.argtypes = [c.c_int64, u8p, u8p, c.POINTER(c.c_int64),
                                        c.c_uint64, c.c_uint64, c.c_int, c.c_int,
                                        c.c_uint64, c.c_uint64, i64p, c.c_int64]
    L.orc_halfsweep_ordered.restype = c.c_int
    L.orc_sweeps.argtypes = [c.c_int64, u8p, u8p, c.POINTER(c.c_int64), c.c_uint64,
                             c.c_uint64, c.c_int64, c.c_int, c.c_uint64, c.c_uint64]
    L.orc_sweeps.restype = None
    L.orc_sweeps_record.argtypes = [c.c_int64, u8p, u8p, c.POINTER(c.c_int64),
                                    c.c_uint64, c.c_uint64, c.c_int64, c.c_int,
                                    c.c_uint64, c.c_uint64, c.c_int64, u64p]
    L.orc_sweeps_record.restype = c.c_int
    L.orc_rs_sweeps.argtypes = [c.c_int64, u8p, u8p, c.POINTER(c.c_int64),
                                c.c_uint64, c.c_uint64, c.c_int64, c.c_uint64,
                                c.c_uint64]
    L.orc_rs_sweeps.restype = None
    L.orc_heights.argtypes = [c.c_int64, u8p, u8p, c.c_int64, i64p]
    L.orc_heights.restype = None
    L.orc_power_sums.argtypes = [c.c_int64, i64p, c.c_int64, i64p]
    L.orc_power_sums.restype = None
    L.orc_width2.argtypes = [c.c_int64, i64p, c.c_int64]
    L.orc_width2.restype = c.c_double
    L.orc_skew_kurt.argtypes = [c.c_int64, i64p, c.c_int64, f64p]
    L.orc_skew_kurt.restype = None
    L.orc_ddrs_sweeps.argtypes = [c.c_int64, c.c_int64, u8p, u8p, c.POINTER(c.c_int64),
                                  c.c_uint64, c.c_uint64, c.c_int64, c.c_uint64, c.c_uint64]
    L.orc_ddrs_sweeps.restype = c.c_int
    L.orc_window_init_flat.argtypes = [c.c_int64, c.c_int64, c.c_int64, c.c_int64, u8p,
                                       u8p]
    L.orc_window_init_flat.restype = None
    L.orc_window_sweeps.argtypes = [c.c_int64, c.c_int64, c.c_int64, c.c_int64, c.c_int64,
                                    u8p, u8p, c.c_uint64, c.c_uint64, c.c_int64, c.c_int,
                                    c.c_uint64, c.c_uint64]
    L.orc_window_sweeps.restype = None
    L.orc_height_packed.argtypes = [c.c_int64, u32p, u32p, c.c_int64, c.c_int64,
                                    c.c_int64]
    L.orc_height_packed.restype = c.c_int64
    L.orc_sample_times.argtypes = [c.c_uint64, c.c_int, u64p]
    L.orc_sample_times.restype = c.c_int
    _lib = L
    return L


def _i128(lo, hi):
    return (int(hi) << 64) | (int(lo) & 0xFFFFFFFFFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: ctr = 4 uint32, key = 2 uint32 -> 4 uint32."""
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def thresholds(p, q, s_sel=0.5, k_max=32):
    """(k, P, Q): acceptance precision and integer thresholds of the rule."""
    k = ctypes.c_int()
    P = ctypes.c_uint64()
    Q = ctypes.c_uint64()
    if lib().orc_thresholds(p, q, s_sel, k_max, ctypes.byref(k), ctypes.byref(P),
                            ctypes.byref(Q)) != 0:
        raise ValueError("parameters out of range")
    return k.value, P.value, Q.value


def rs_threshold(p):
    return int(lib().orc_rs_threshold(p))


def site_uniform(seed, L, x, y, t, k):
    return int(lib().orc_site_uniform(seed, L, x, y, t, k))


def sample_times(T, n):
    out = np.zeros(n + 1, np.uint64)
    if lib().orc_sample_times(T, n, out) != 0:
        raise ValueError("bad sample schedule (need 2 <= n <= T)")
    return [int(v) for v in out]


def window_flat_sweeps(L, x0, y0, w, h, p, q, seed, n, s_sel=0.5, k_max=32, t0=0):
    """n sweeps from the striped start on a w x h window at (x0, y0) of an L x L
    lattice. Returns (WX, WY) as (h, w) 0/1 arrays; only sites farther than
    2n + 1 from the window's edges are exact."""
    k, P, Q = thresholds(p, q, s_sel, k_max)
    WX = np.zeros((h, w), np.uint8)
    WY = np.zeros((h, w), np.uint8)
    lib().orc_window_init_flat(x0, y0, w, h, WX, WY)
    lib().orc_window_sweeps(L, x0, y0, w, h, WX, WY, seed, t0, n, k, P, Q)
    return WX, WY


def height_packed(L, Xw, Yw, H0, x, y):
    """h(x, y) by Eq. (3) directly from packed planes ((L, L/32) uint32 each)."""
    return int(lib().orc_height_packed(L, np.ascontiguousarray(Xw, np.uint32).ravel(),
                                       np.ascontiguousarray(Yw, np.uint32).ravel(),
                                       H0, x, y))


def pack_plane(bits):
    """(L, L) array of 0/1 bonds -> (L, L//32) uint32 words in the C-ABI layout:
    bit b of word w of row y holds the bond at x = 32*w + b."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    L = bits.shape[0]
    packed = np.packbits(bits, axis=1, bitorder="little")  # (L, L/8) bytes
    return packed.view("<u4").reshape(L, L // 32).copy()


def unpack_plane(words, L):
    """Inverse of pack_plane."""
    w = np.ascontiguousarray(np.asarray(words, dtype="<u4").reshape(L, L // 32))
    return np.unpackbits(w.view(np.uint8), axis=1, bitorder="little")[:, :L].copy()


class Sim:
    """A lattice held by the oracle: one byte per bond, exact integer sums."""

    def __init__(self, L, p, q, seed, s_sel=0.5, k_max=32):
        if L < 2 or L % 2:
            raise ValueError("L must be even and >= 2")
        self.L = int(L)
        self.p, self.q, self.seed = float(p), float(q), int(seed)
        self.s_sel, self.k_max = float(s_sel), int(k_max)
        self.k, self.P, self.Q = thresholds(p, q, s_sel, k_max)
        self.X = np.zeros((L, L), np.uint8)
        self.Y = np.zeros((L, L), np.uint8)
        lib().orc_init_flat(self.L, self.X, self.Y)
        self.H0 = 0
        self.t = 0

    @property
    def N(self):
        return self.L * self.L

    def halfsweep(self, s):
        H0 = ctypes.c_int64(self.H0)
        lib().orc_halfsweep(self.L, self.X, self.Y, ctypes.byref(H0), self.seed,
                            self.t, s, self.k, self.P, self.Q)
        self.H0 = H0.value

    def sweep(self, n=1):
        H0 = ctypes.c_int64(self.H0)
        lib().orc_sweeps(self.L, self.X, self.Y, ctypes.byref(H0), self.seed, self.t,
                         int(n), self.k, self.P, self.Q)
        self.H0 = H0.value
        self.t += int(n)

    def sweep_record(self, n, thin):
        """n sweeps of a lattice with L*L <= 32; state codes after every thin-th sweep."""
        codes = np.zeros(int(n) // int(thin), np.uint64)
        H0 = ctypes.c_int64(self.H0)
        if lib().orc_sweeps_record(self.L, self.X, self.Y, ctypes.byref(H0), self.seed,
                                   self.t, int(n), self.k, self.P, self.Q, int(thin),
                                   codes) != 0:
            raise ValueError("lattice too large to record")
        self.H0 = H0.value
        self.t += int(n)
        return codes

    def rs_sweep(self, n=1):
        """Random-sequential sweeps (p, q used directly; no selection factor)."""
        H0 = ctypes.c_int64(self.H0)
        lib().orc_rs_sweeps(self.L, self.X, self.Y, ctypes.byref(H0), self.seed,
                            self.t, int(n), rs_threshold(self.p), rs_threshold(self.q))
        self.H0 = H0.value
        self.t += int(n)

    def ddrs_sweep(self, n=1, C=32):
        """Domain-decomposed random-sequential sweeps (cells C x C, dead borders,
        random offsets; p, q used directly)."""
        H0 = ctypes.c_int64(self.H0)
        if lib().orc_ddrs_sweeps(self.L, C, self.X, self.Y, ctypes.byref(H0), self.seed,
                                 self.t, int(n), rs_threshold(self.p),
                                 rs_threshold(self.q)) != 0:
            raise ValueError("C must be a power of two >= 4 dividing L")
        self.H0 = H0.value
        self.t += int(n)

    def heights(self):
        h = np.zeros((self.L, self.L), np.int64)
        lib().orc_heights(self.L, self.X, self.Y, self.H0, h)
        return h

    def power_sums(self, c=None):
        """[S1, S2, S3, S4], S_n = sum (h - c)^n as Python ints (c = H0 by default)."""
        h = self.heights()
        raw = np.zeros(8, np.int64)
        lib().orc_power_sums(self.L, h, self.H0 if c is None else int(c), raw)
        return [_i128(raw[2 * n], raw[2 * n + 1]) for n in range(4)]

    def sums(self):
        """Absolute (S1, S2) = (sum h, sum h^2)."""
        S = self.power_sums(c=0)
        return S[0], S[1]

    def width2(self):
        return float(lib().orc_width2(self.L, self.heights(), self.H0))

    def skew_kurt(self):
        out = np.zeros(2, np.float64)
        lib().orc_skew_kurt(self.L, self.heights(), self.H0, out)
        return float(out[0]), float(out[1])

    def packed(self):
        """(X words, Y words) in the C-ABI bit-plane layout, each (L, L//32) uint32."""
        return pack_plane(self.X), pack_plane(self.Y)

    def load_packed(self, Xw, Yw, H0, t):
        self.X = unpack_plane(Xw, self.L)
        self.Y = unpack_plane(Yw, self.L)
        self.H0, self.t = int(H0), int(t)
