"""Python binding of the okz C-ABI (include/okz.h): argument marshalling only.

Every function here has the name of the C entry point it calls; all work runs
in the CUDA library ``_build/libokz.so`` (build it with
``python -c "import __graft_entry__ as g; g.build()"``). There is no CPU
fallback: when the library is missing, loading fails loudly.

PyTorch is optional plumbing: ``create_on_torch`` places a simulation in a
torch-allocated device buffer on torch's current stream.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libokz.so")

OKZ_OK, OKZ_EINVAL, OKZ_ENOMEM, OKZ_ECUDA, OKZ_ETIMEOUT, OKZ_EBUSY, OKZ_EOVERFLOW, \
    OKZ_EUNSUPPORTED = range(8)
OKZ_KERNEL_AUTO, OKZ_KERNEL_PLAIN, OKZ_KERNEL_STREAM = 0, 1, 2
OKZ_KERNEL_PARITY_PLAIN, OKZ_KERNEL_PARITY_STREAM, OKZ_KERNEL_PARITY_CTA = 3, 4, 5
STATUS_NAMES = {0: "OKZ_OK", 1: "OKZ_EINVAL", 2: "OKZ_ENOMEM", 3: "OKZ_ECUDA",
                4: "OKZ_ETIMEOUT", 5: "OKZ_EBUSY", 6: "OKZ_EOVERFLOW", 7: "OKZ_EUNSUPPORTED"}


class OkzError(RuntimeError):
    def __init__(self, status, func, msg):
        self.status = status
        super().__init__("%s failed: %s: %s" % (func, STATUS_NAMES.get(status, status), msg))


class okz_i128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_int64)]

    def value(self):
        return (int(self.hi) << 64) | int(self.lo)


class okz_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("p", ctypes.c_double), ("q", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("s_sel", ctypes.c_double),
                ("k_max", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("words_per_thread", ctypes.c_int32), ("sweeps_per_pass", ctypes.c_int32),
                ("band_rows", ctypes.c_int32)]


class okz_info(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("t", ctypes.c_uint64), ("H0", ctypes.c_int64),
                ("k", ctypes.c_int32), ("kernel", ctypes.c_int32), ("P", ctypes.c_uint64),
                ("Q", ctypes.c_uint64), ("device_bytes", ctypes.c_size_t),
                ("words_per_thread", ctypes.c_int32), ("sweeps_per_pass", ctypes.c_int32),
                ("graph_chunk", ctypes.c_int32), ("graph_replays", ctypes.c_uint64),
                ("band_rows", ctypes.c_int32)]


# C signatures: name -> (restype, argtypes)
_c = ctypes
_vp = _c.c_void_p
_SIGS = {
    "okz_params_init": (None, [_c.POINTER(okz_params)]),
    "okz_device_bytes": (_c.c_size_t, [_c.c_int64]),
    "okz_create": (_c.c_int, [_c.c_int64, _c.c_double, _c.c_double, _c.c_uint64,
                              _c.POINTER(_vp)]),
    "okz_create_ex": (_c.c_int, [_c.POINTER(okz_params), _vp, _c.c_size_t, _vp,
                                 _c.POINTER(_vp)]),
    "okz_sweep": (_c.c_int, [_vp, _c.c_int64]),
    "okz_sweep_rs": (_c.c_int, [_vp, _c.c_int64]),
    "okz_growth_series": (_c.c_int, [_vp, _c.c_int32, _vp, _vp, _vp, _vp, _vp]),
    "okz_stage_host": (_c.c_int, [_vp, _vp]),
    "okz_restore_staged": (_c.c_int, [_vp, _c.c_int64, _c.c_uint64]),
    "okz_width2": (_c.c_int, [_vp, _c.POINTER(okz_i128), _c.POINTER(okz_i128),
                              _c.POINTER(_c.c_double)]),
    "okz_moments": (_c.c_int, [_vp, _c.POINTER(okz_i128), _c.POINTER(_c.c_double),
                               _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)]),
    "okz_heights": (_c.c_int, [_vp, _c.c_int64, _c.c_int64, _vp, _c.c_int]),
    "okz_profiles": (_c.c_int, [_vp, _vp, _vp]),
    "okz_moments_enqueue": (_c.c_int, [_vp]),
    "okz_selftest_wait_timeout": (_c.c_int, [_vp]),
    "okz_alu_peak": (_c.c_int, [_vp, _c.c_int32, _c.POINTER(_c.c_double),
                                _c.POINTER(_c.c_double)]),
    "okz_tune_stream": (_c.c_int, [_c.POINTER(okz_params), _c.c_int32, _c.POINTER(_c.c_int32),
                                   _c.POINTER(_c.c_int32), _c.POINTER(_c.c_int32),
                                   _c.POINTER(_c.c_double)]),
    "okz_moments_fetch": (_c.c_int, [_vp, _c.POINTER(okz_i128), _c.POINTER(_c.c_double),
                               _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)]),
    "okz_psd": (_c.c_int, [_vp, _vp]),
    "okz_state": (_c.c_int, [_vp, _vp, _c.c_int, _c.POINTER(_c.c_int64),
                             _c.POINTER(_c.c_uint64)]),
    "okz_restore": (_c.c_int, [_vp, _vp, _c.c_int, _c.c_int64, _c.c_uint64]),
    "okz_get_info": (_c.c_int, [_vp, _c.POINTER(okz_info)]),
    "okz_synchronize": (_c.c_int, [_vp]),
    "okz_stream": (_vp, [_vp]),
    "okz_destroy": (_c.c_int, [_vp]),
    "okz_last_error": (_c.c_char_p, []),
    "okz_width2_noalloc": (_c.c_int, [_vp, _c.c_int64, _c.c_int64, _vp,
                                      _c.POINTER(okz_i128), _c.POINTER(okz_i128),
                                      _c.POINTER(_c.c_double)]),
    "okz_pool_create": (_c.c_int, [_c.c_size_t, _c.c_int32, _c.c_double, _c.c_int32, _vp,
                                   _c.POINTER(_vp)]),
    "okz_batch_create": (_c.c_int, [_c.c_int32, _vp, _vp, _vp, _vp, _c.POINTER(_vp)]),
    "okz_batch_add": (_c.c_int, [_vp, _c.c_int64, _c.c_double, _c.c_double, _c.c_uint64,
                                 _c.POINTER(_c.c_int32)]),
    "okz_batch_remove": (_c.c_int, [_vp, _c.c_int32]),
    "okz_batch_run": (_c.c_int, [_vp, _vp]),
    "okz_batch_sync": (_c.c_int, [_vp]),
    "okz_batch_stats": (_c.c_int, [_vp, _vp, _vp, _vp]),
    "okz_batch_sums": (_c.c_int, [_vp, _c.c_int32, _c.POINTER(okz_i128),
                                  _c.POINTER(_c.c_int64), _c.POINTER(_c.c_uint64)]),
    "okz_batch_measure": (_c.c_int, [_vp, _c.c_int32, _vp, _vp, _vp, _vp]),
    "okz_batch_state": (_c.c_int, [_vp, _c.c_int32, _vp, _c.POINTER(_c.c_int64),
                                   _c.POINTER(_c.c_uint64)]),
    "okz_batch_set_tiling": (_c.c_int, [_vp, _c.c_int32, _c.c_size_t]),
    "okz_batch_get_tiling": (_c.c_int, [_vp, _c.POINTER(_c.c_int32), _c.POINTER(_c.c_size_t),
                                        _c.POINTER(_c.c_int32)]),
    "okz_batch_autotune": (_c.c_int, [_vp, _c.c_int32]),
    "okz_batch_stream": (_vp, [_vp]),
    "okz_batch_destroy": (_c.c_int, [_vp]),
    "okz_thresholds": (_c.c_int, [_c.c_double, _c.c_double, _c.c_double, _c.c_int32,
                                  _c.POINTER(_c.c_int32), _c.POINTER(_c.c_uint64),
                                  _c.POINTER(_c.c_uint64)]),
}

_lib = None


def lib():
    """The loaded libokz.so. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libokz.so is missing (%s); build it with "
                               "__graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status, func):
    if status != OKZ_OK:
        raise OkzError(status, func, okz_last_error())


def okz_last_error():
    return lib().okz_last_error().decode()


def okz_params_init(L=0, p=1.0, q=0.0, seed=0, s_sel=0.5, k_max=32, kernel=OKZ_KERNEL_AUTO,
                    words_per_thread=0, sweeps_per_pass=0, band_rows=0):
    prm = okz_params()
    lib().okz_params_init(ctypes.byref(prm))
    prm.L, prm.p, prm.q, prm.seed = int(L), float(p), float(q), int(seed)
    prm.s_sel, prm.k_max, prm.kernel = float(s_sel), int(k_max), int(kernel)
    prm.words_per_thread, prm.sweeps_per_pass = int(words_per_thread), int(sweeps_per_pass)
    prm.band_rows = int(band_rows)
    return prm


def okz_device_bytes(L):
    return int(lib().okz_device_bytes(int(L)))


def okz_thresholds(p, q, s_sel=0.5, k_max=32):
    k, P, Q = ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().okz_thresholds(p, q, s_sel, k_max, ctypes.byref(k), ctypes.byref(P),
                                ctypes.byref(Q)), "okz_thresholds")
    return k.value, P.value, Q.value


def okz_create(L, p, q, seed):
    h = ctypes.c_void_p()
    _check(lib().okz_create(int(L), float(p), float(q), int(seed), ctypes.byref(h)),
           "okz_create")
    return h


def okz_create_ex(prm, dev_buf=None, nbytes=0, stream=None):
    h = ctypes.c_void_p()
    _check(lib().okz_create_ex(ctypes.byref(prm), dev_buf, int(nbytes), stream,
                               ctypes.byref(h)), "okz_create_ex")
    return h


def okz_sweep(h, n):
    _check(lib().okz_sweep(h, int(n)), "okz_sweep")


def okz_sweep_rs(h, n):
    _check(lib().okz_sweep_rs(h, int(n)), "okz_sweep_rs")


def okz_width2(h):
    """-> (S1, S2, W2) with S1 = sum h and S2 = sum h^2 as Python ints."""
    S1, S2, W2 = okz_i128(), okz_i128(), ctypes.c_double()
    _check(lib().okz_width2(h, ctypes.byref(S1), ctypes.byref(S2), ctypes.byref(W2)),
           "okz_width2")
    return S1.value(), S2.value(), W2.value


def okz_growth_series(h, times):
    """Sweeps to each sample time and takes the exact sums there in one call
    (one synchronisation) -> [(t, H0, S1, S2, W2)] with S1 = sum h and
    S2 = sum h^2 as Python ints."""
    times = np.ascontiguousarray(np.asarray(times, dtype=np.uint64))
    n = len(times)
    S1 = (okz_i128 * max(n, 1))()
    S2 = (okz_i128 * max(n, 1))()
    W2 = np.zeros(max(n, 1), np.float64)
    H0 = np.zeros(max(n, 1), np.int64)
    _check(lib().okz_growth_series(h, n, times.ctypes.data, ctypes.addressof(S1),
                                   ctypes.addressof(S2), W2.ctypes.data, H0.ctypes.data),
           "okz_growth_series")
    return [(int(times[i]), int(H0[i]), S1[i].value(), S2[i].value(), float(W2[i]))
            for i in range(n)]


def okz_selftest_wait_timeout(stream=None):
    """Runs the bounded-wait self-test; raises OkzError(OKZ_ETIMEOUT) when the
    wait gave up as intended, returns if it (wrongly) completed."""
    _check(lib().okz_selftest_wait_timeout(stream), "okz_selftest_wait_timeout")


def okz_alu_peak(stream=None, iters=20000):
    """Measured INT32 ALU-pipe rate of the current device -> (ops/s, best ms)."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().okz_alu_peak(stream, int(iters), ctypes.byref(ops), ctypes.byref(ms)),
           "okz_alu_peak")
    return ops.value, ms.value


def okz_tune_stream(L, p, q, s_sel=0.5, k_max=32, kernel=0, probe_sweeps=8):
    """Autotunes the stream kernels' (words per thread, sweeps per pass, band
    rows) for this workload; later Simulations with automatic tiling use the
    choice. -> (words_per_thread, sweeps_per_pass, band_rows, ms per sweep)."""
    prm = okz_params()
    lib().okz_params_init(ctypes.byref(prm))
    prm.L, prm.p, prm.q, prm.s_sel, prm.k_max, prm.kernel = int(L), float(p), float(q), \
        float(s_sel), int(k_max), int(kernel)
    w, f, b, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(lib().okz_tune_stream(ctypes.byref(prm), int(probe_sweeps), ctypes.byref(w),
                                 ctypes.byref(f), ctypes.byref(b), ctypes.byref(ms)),
           "okz_tune_stream")
    return w.value, f.value, b.value, ms.value


def okz_moments_enqueue(h):
    _check(lib().okz_moments_enqueue(h), "okz_moments_enqueue")


def okz_moments_fetch(h):
    """-> as okz_moments, for the sums enqueued by okz_moments_enqueue."""
    Sk = (okz_i128 * 4)()
    W2, sk, ku = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().okz_moments_fetch(h, Sk, ctypes.byref(W2), ctypes.byref(sk),
                                   ctypes.byref(ku)), "okz_moments_fetch")
    return [s.value() for s in Sk], W2.value, sk.value, ku.value


def okz_moments(h):
    """-> ([S1..S4] about H0, W2, skew, excess kurtosis)."""
    Sk = (okz_i128 * 4)()
    W2, sk, ku = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().okz_moments(h, Sk, ctypes.byref(W2), ctypes.byref(sk), ctypes.byref(ku)),
           "okz_moments")
    return [s.value() for s in Sk], W2.value, sk.value, ku.value


def okz_heights(h, y0, ny, L, out=None):
    """Heights of rows y0..y0+ny-1. out: None (returns a numpy int32 array), a
    numpy int32 array, or a CUDA torch int32 tensor (filled on the device)."""
    if out is None:
        out = np.empty((int(ny), int(L)), np.int32)
    is_dev = 0
    if isinstance(out, np.ndarray):
        assert out.dtype == np.int32 and out.flags.c_contiguous and out.size >= ny * L
        ptr = out.ctypes.data
    else:  # torch tensor on the device
        assert out.is_cuda and out.is_contiguous() and out.numel() >= ny * L
        ptr, is_dev = out.data_ptr(), 1
    _check(lib().okz_heights(h, int(y0), int(ny), ptr, is_dev), "okz_heights")
    return out


def okz_profiles(h, L):
    """-> (col, row): int64 numpy arrays of the column and row sums of h - H0."""
    col = np.empty(int(L), np.int64)
    row = np.empty(int(L), np.int64)
    _check(lib().okz_profiles(h, col.ctypes.data, row.ctypes.data), "okz_profiles")
    return col, row


def okz_psd(h, L):
    """-> S: float64 numpy array of the axis-averaged power spectrum, k = 0..L-1."""
    S = np.empty(int(L), np.float64)
    _check(lib().okz_psd(h, S.ctypes.data), "okz_psd")
    return S


def okz_state(h, L, out=None):
    """-> (planes, H0, t); planes is (2, L, L//32) uint32 (X plane, Y plane) or the
    given output (numpy array or CUDA torch tensor of 2*L*L/32 uint32/int32)."""
    if out is None:
        out = np.empty((2, int(L), int(L) // 32), np.uint32)
    is_dev = 0
    if isinstance(out, np.ndarray):
        assert out.nbytes >= 2 * L * L // 8 and out.flags.c_contiguous
        ptr = out.ctypes.data
    else:
        assert out.is_cuda and out.is_contiguous()
        ptr, is_dev = out.data_ptr(), 1
    H0, t = ctypes.c_int64(), ctypes.c_uint64()
    _check(lib().okz_state(h, ptr, is_dev, ctypes.byref(H0), ctypes.byref(t)), "okz_state")
    return out, H0.value, t.value


def okz_restore(h, planes, H0, t):
    if isinstance(planes, np.ndarray):
        planes = np.ascontiguousarray(planes, dtype=np.uint32)
        ptr, is_dev = planes.ctypes.data, 0
    else:
        assert planes.is_contiguous()
        ptr, is_dev = planes.data_ptr(), int(planes.is_cuda)
    _check(lib().okz_restore(h, ptr, is_dev, int(H0), int(t)), "okz_restore")


def okz_width2_noalloc(planes_dev_ptr, L, H0, stream=None):
    """Exact (S1, S2, W2) of caller-owned device planes (slope layout), for
    callers that cannot allocate device memory; uses a fixed scratch array
    shared by all calls (serialise calls that could overlap on the GPU)."""
    S1, S2, W2 = okz_i128(), okz_i128(), ctypes.c_double()
    _check(lib().okz_width2_noalloc(planes_dev_ptr, int(L), int(H0), stream, ctypes.byref(S1),
                                    ctypes.byref(S2), ctypes.byref(W2)), "okz_width2_noalloc")
    return S1.value(), S2.value(), W2.value


def okz_get_info(h):
    info = okz_info()
    _check(lib().okz_get_info(h, ctypes.byref(info)), "okz_get_info")
    return info


def okz_synchronize(h):
    _check(lib().okz_synchronize(h), "okz_synchronize")


def okz_stream(h):
    return lib().okz_stream(h)


def okz_destroy(h):
    _check(lib().okz_destroy(h), "okz_destroy")


class Simulation:
    """Owning wrapper: a simulation handle plus the torch buffer it may live in."""

    def __init__(self, L, p=1.0, q=0.0, seed=0, s_sel=0.5, k_max=32,
                 kernel=OKZ_KERNEL_AUTO, torch_buffer=False, stream=None,
                 words_per_thread=0, sweeps_per_pass=0, band_rows=0):
        self.L = int(L)
        self._buf = None
        prm = okz_params_init(L, p, q, seed, s_sel, k_max, kernel, words_per_thread,
                              sweeps_per_pass, band_rows)
        if torch_buffer:
            import torch
            nbytes = okz_device_bytes(L)
            self._buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._buf.data_ptr()
            aligned = (base + 255) & ~255
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
            self.h = okz_create_ex(prm, aligned, nbytes, stream)
        else:
            self.h = okz_create_ex(prm, None, 0, stream)

    def sweep(self, n=1):
        okz_sweep(self.h, n)

    def sweep_rs(self, n=1):
        okz_sweep_rs(self.h, n)

    def width2(self):
        return okz_width2(self.h)

    def moments(self):
        return okz_moments(self.h)

    def moments_enqueue(self):
        okz_moments_enqueue(self.h)

    def moments_fetch(self):
        return okz_moments_fetch(self.h)

    def heights(self, y0=0, ny=None, out=None):
        return okz_heights(self.h, y0, self.L - y0 if ny is None else ny, self.L, out)

    def profiles(self):
        return okz_profiles(self.h, self.L)

    def psd(self):
        return okz_psd(self.h, self.L)

    def state(self, out=None):
        return okz_state(self.h, self.L, out)

    def restore(self, planes, H0, t):
        okz_restore(self.h, planes, H0, t)

    def info(self):
        return okz_get_info(self.h)

    @property
    def wpt(self):
        return self.info().words_per_thread

    @property
    def fuse(self):
        return self.info().sweeps_per_pass

    @property
    def band_rows(self):
        return self.info().band_rows

    def synchronize(self):
        okz_synchronize(self.h)

    def stage_host(self, planes):
        """Starts the host-to-device copy of `planes` (a CPU tensor or array,
        slope-plane layout; kept alive here until the next stage_host)."""
        if isinstance(planes, np.ndarray):
            planes = np.ascontiguousarray(planes, dtype=np.uint32)
            ptr = planes.ctypes.data
        else:
            assert planes.is_contiguous() and not planes.is_cuda, "host planes expected"
            ptr = planes.data_ptr()
        self._staged_host = planes
        _check(lib().okz_stage_host(self.h, ptr), "okz_stage_host")

    def restore_staged(self, H0, t):
        _check(lib().okz_restore_staged(self.h, int(H0), int(t)), "okz_restore_staged")

    def growth_series(self, times):
        """[(t, H0, S1, S2, W2)] at every sample time, in one call."""
        return okz_growth_series(self.h, times)

    @property
    def stream(self):
        return okz_stream(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            okz_destroy(self.h)
            self.h = None
            self._buf = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Batched and pooled lattices
# ---------------------------------------------------------------------------
def okz_pool_create(arena_bytes, max_slots, s_sel=0.5, k_max=32, stream=None):
    h = ctypes.c_void_p()
    _check(lib().okz_pool_create(int(arena_bytes), int(max_slots), float(s_sel), int(k_max),
                                 stream, ctypes.byref(h)), "okz_pool_create")
    return h


def okz_batch_create(L, p, q, seed):
    n = len(L)
    La = np.ascontiguousarray(L, np.int64)
    pa = np.ascontiguousarray(p, np.float64)
    qa = np.ascontiguousarray(q, np.float64)
    sa = np.ascontiguousarray(seed, np.uint64)
    h = ctypes.c_void_p()
    _check(lib().okz_batch_create(n, La.ctypes.data, pa.ctypes.data, qa.ctypes.data,
                                  sa.ctypes.data, ctypes.byref(h)), "okz_batch_create")
    return h


def okz_batch_add(b, L, p, q, seed):
    slot = ctypes.c_int32()
    _check(lib().okz_batch_add(b, int(L), float(p), float(q), int(seed), ctypes.byref(slot)),
           "okz_batch_add")
    return slot.value


def okz_batch_remove(b, slot):
    _check(lib().okz_batch_remove(b, int(slot)), "okz_batch_remove")


def okz_batch_run(b, sweeps):
    sw = np.ascontiguousarray(sweeps, np.int64)
    _check(lib().okz_batch_run(b, sw.ctypes.data), "okz_batch_run")


def okz_batch_sync(b):
    _check(lib().okz_batch_sync(b), "okz_batch_sync")


def okz_batch_stats(b, max_slots):
    W2 = np.empty(max_slots, np.float64)
    sk = np.empty(max_slots, np.float64)
    ku = np.empty(max_slots, np.float64)
    _check(lib().okz_batch_stats(b, W2.ctypes.data, sk.ctypes.data, ku.ctypes.data),
           "okz_batch_stats")
    return W2, sk, ku


def okz_batch_sums(b, slot):
    Sk = (okz_i128 * 4)()
    H0, t = ctypes.c_int64(), ctypes.c_uint64()
    _check(lib().okz_batch_sums(b, int(slot), Sk, ctypes.byref(H0), ctypes.byref(t)),
           "okz_batch_sums")
    return [s.value() for s in Sk], H0.value, t.value


def okz_batch_measure(b, slots):
    """Exact sums of the listed slots in one launch -> [(Sk[4], H0, t)]."""
    n = len(slots)
    if n == 0:
        return []
    sl = np.ascontiguousarray(slots, np.int32)
    Sk = (okz_i128 * (4 * n))()
    H0 = np.empty(n, np.int64)
    t = np.empty(n, np.uint64)
    _check(lib().okz_batch_measure(b, n, sl.ctypes.data, Sk, H0.ctypes.data, t.ctypes.data),
           "okz_batch_measure")
    return [([Sk[4 * j + m].value() for m in range(4)], int(H0[j]), int(t[j])) for j in range(n)]


def okz_batch_state(b, slot, L):
    out = np.empty((2, int(L), int(L) // 32), np.uint32)
    H0, t = ctypes.c_int64(), ctypes.c_uint64()
    _check(lib().okz_batch_state(b, int(slot), out.ctypes.data, ctypes.byref(H0),
                                 ctypes.byref(t)), "okz_batch_state")
    return out, H0.value, t.value


def okz_batch_set_tiling(b, threads, smem_bytes):
    _check(lib().okz_batch_set_tiling(b, int(threads), int(smem_bytes)), "okz_batch_set_tiling")


def okz_batch_get_tiling(b):
    th, sm, gr = ctypes.c_int32(), ctypes.c_size_t(), ctypes.c_int32()
    _check(lib().okz_batch_get_tiling(b, ctypes.byref(th), ctypes.byref(sm), ctypes.byref(gr)),
           "okz_batch_get_tiling")
    return th.value, sm.value, gr.value


def okz_batch_autotune(b, probe_sweeps=8):
    _check(lib().okz_batch_autotune(b, int(probe_sweeps)), "okz_batch_autotune")


def okz_batch_stream(b):
    return lib().okz_batch_stream(b)


def okz_batch_destroy(b):
    _check(lib().okz_batch_destroy(b), "okz_batch_destroy")


class Batch:
    """Owning wrapper of an okz_batch slot table."""

    def __init__(self, L=None, p=None, q=None, seed=None, arena_bytes=None, max_slots=None,
                 s_sel=0.5, k_max=32, stream=None):
        if L is not None:
            self.h = okz_batch_create(L, p, q, seed)
            self.max_slots = len(L)
            self.L = {i: int(l) for i, l in enumerate(L)}
        else:
            self.h = okz_pool_create(arena_bytes, max_slots, s_sel, k_max, stream)
            self.max_slots = int(max_slots)
            self.L = {}

    def add(self, L, p, q, seed):
        slot = okz_batch_add(self.h, L, p, q, seed)
        self.L[slot] = int(L)
        return slot

    def remove(self, slot):
        okz_batch_remove(self.h, slot)
        self.L.pop(slot, None)

    def run(self, sweeps):
        if isinstance(sweeps, dict):
            arr = np.zeros(self.max_slots, np.int64)
            for k, v in sweeps.items():
                arr[k] = v
            sweeps = arr
        okz_batch_run(self.h, sweeps)

    def sync(self):
        okz_batch_sync(self.h)

    def stats(self):
        return okz_batch_stats(self.h, self.max_slots)

    def sums(self, slot):
        return okz_batch_sums(self.h, slot)

    def state(self, slot):
        return okz_batch_state(self.h, slot, self.L[slot])

    def measure(self, slots):
        return okz_batch_measure(self.h, list(slots))

    def set_tiling(self, threads, smem_bytes):
        okz_batch_set_tiling(self.h, threads, smem_bytes)

    def tiling(self):
        return okz_batch_get_tiling(self.h)

    def autotune(self, probe_sweeps=8):
        okz_batch_autotune(self.h, probe_sweeps)

    @property
    def stream(self):
        return okz_batch_stream(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            okz_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
