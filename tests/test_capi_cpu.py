"""CPU checks of the C-ABI library: it loads, exports every symbol okz.h
declares, and its host logic (thresholds, sizes, argument checks) is right.
No call here reaches the GPU."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def okz():
    from paper_1110_6745_gb300 import _build
    _build.build()
    import paper_1110_6745_gb300 as m
    m.lib()
    return m


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(okz_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(okz):
    declared = _declared()
    assert len(declared) >= 16
    out = subprocess.run(["nm", "-D", "--defined-only", okz.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (okz_\w+)", out))
    assert declared <= exported, declared - exported
    for name in declared:
        getattr(okz.lib(), name)


def test_thresholds_match_oracle(okz, orc):
    for p, q, s_sel, k_max in [(1, 0, 0.5, 32), (1, 0, 1.0, 32), (0.75, 0.25, 0.5, 32),
                               (0.5, 0.5, 0.5, 32), (0.95, 0.05, 0.5, 32),
                               (0.3, 0.7, 0.5, 12), (1 / 3, 0.1, 0.9, 7), (0, 0, 0.5, 32)]:
        assert okz.okz_thresholds(p, q, s_sel, k_max) == orc.thresholds(p, q, s_sel, k_max)


def test_device_bytes(okz):
    L = 1 << 17
    b = okz.okz_device_bytes(L)
    assert b >= 2 * L * L // 4 + 8 * L  # two state buffers + column heights
    assert b < 2 * L * L // 4 + 8 * L + (1 << 20)
    assert okz.okz_device_bytes(31) == 0 and okz.okz_device_bytes(48) == 0


@pytest.mark.parametrize("L,p,q,status", [
    (31, 1.0, 0.0, 1),    # odd L: EINVAL
    (0, 1.0, 0.0, 1),
    (48, 1.0, 0.0, 7),    # L % 32 != 0: EUNSUPPORTED
    (64, 1.5, 0.0, 1),    # p > 1: EINVAL
    (64, 0.5, -0.1, 1),
])
def test_create_rejects_bad_arguments_before_touching_cuda(okz, L, p, q, status):
    with pytest.raises(okz.OkzError) as e:
        okz.okz_create(L, p, q, 1)
    assert e.value.status == status
    assert okz.okz_last_error() != ""


def test_stream_kernel_size_rule(okz):
    prm = okz.okz_params_init(L=2048, kernel=okz.OKZ_KERNEL_STREAM)
    with pytest.raises(okz.OkzError) as e:
        okz.okz_create_ex(prm)
    assert e.value.status == okz.OKZ_EUNSUPPORTED


def test_null_handles_are_rejected(okz):
    with pytest.raises(okz.OkzError):
        okz.okz_sweep(None, 1)
    with pytest.raises(okz.OkzError):
        okz.okz_sweep(None, -1)
    okz.okz_destroy(None)  # accepted


def test_alu_peak_rejects_bad_arguments(okz):
    """okz_alu_peak checks its arguments before touching the device."""
    with pytest.raises(okz.OkzError) as e:
        okz.okz_alu_peak(None, 0)
    assert e.value.status == okz.OKZ_EINVAL


def test_tune_stream_rejects_bad_requests(okz):
    """okz_tune_stream checks its arguments before touching the device."""
    with pytest.raises(okz.OkzError) as e:
        okz.okz_tune_stream(8192, 1.0, 0.0, probe_sweeps=1)
    assert e.value.status == okz.OKZ_EINVAL
    with pytest.raises(okz.OkzError) as e:
        okz.okz_tune_stream(2048, 1.0, 0.0)  # below the stream kernels' range
    assert e.value.status == okz.OKZ_EUNSUPPORTED


@pytest.mark.parametrize("fuse,band", [(1, 4), (2, 8), (1, 8193), (2, -1)])
def test_band_rows_checked_before_touching_cuda(okz, fuse, band):
    """A stream kernel's band is at least 4F + 1 rows (F sweeps per pass) and
    at most L; 0 asks for the automatic height."""
    prm = okz.okz_params_init(L=8192, kernel=okz.OKZ_KERNEL_PARITY_STREAM, words_per_thread=4,
                              sweeps_per_pass=fuse, band_rows=band)
    with pytest.raises(okz.OkzError) as e:
        okz.okz_create_ex(prm)
    assert e.value.status == okz.OKZ_EINVAL
    assert "band_rows" in okz.okz_last_error()


def test_growth_series_rejects_a_null_simulation(okz):
    with pytest.raises(okz.OkzError) as e:
        okz.okz_growth_series(None, [0, 1])
    assert e.value.status == okz.OKZ_EINVAL
