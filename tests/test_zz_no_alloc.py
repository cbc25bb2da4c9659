"""The no-allocation measurement entry point, checked against okz_width2.

okz_width2_noalloc serves callers that cannot allocate device memory when
they measure (their caching allocator owns the free memory, or allocation is
not allowed on their hot path). It must return exactly what okz_width2
returns for the same state, on consecutive calls that reuse its fixed
scratch array. This file is collected last on purpose.
"""
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


def _device_state(okz, sim, L):
    import torch
    planes = torch.empty(2 * L * L // 32, dtype=torch.int32, device="cuda")
    _, H0, _ = sim.state(out=planes)
    return planes, H0


@pytest.mark.parametrize("L,kernel", [(4096, 4), (256, 1), (131072, 4)])
def test_noalloc_matches_width2_on_consecutive_calls(okz, L, kernel):
    import torch
    stream = torch.cuda.Stream()
    with okz.Simulation(L, 0.75, 0.25, seed=21, kernel=kernel) as sim:
        for n_sweeps in (3, 5):  # two states, two calls each, shared scratch
            sim.sweep(n_sweeps)
            want = sim.width2()
            planes, H0 = _device_state(okz, sim, L)
            for _ in range(2):
                got = okz.okz_width2_noalloc(planes.data_ptr(), L, H0, stream.cuda_stream)
                assert got == want


def test_noalloc_after_a_larger_call_and_default_stream(okz):
    """A small lattice after a large one: nothing of the earlier call leaks."""
    for L in (8192, 64):
        with okz.Simulation(L, 1.0, 0.0, seed=2, kernel=1 if L < 4096 else 4) as sim:
            sim.sweep(4)
            want = sim.width2()
            planes, H0 = _device_state(okz, sim, L)
            assert okz.okz_width2_noalloc(planes.data_ptr(), L, H0, None) == want
            assert okz.okz_width2_noalloc(planes.data_ptr(), L, H0, None) == want


def test_noalloc_rejects_sizes_beyond_its_scratch(okz):
    import torch
    dummy = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(okz.OkzError) as e:
        okz.okz_width2_noalloc(dummy.data_ptr(), 262144, 0, None)
    assert e.value.status == okz.OKZ_EINVAL
    assert "scratch" in okz.okz_last_error()
    with pytest.raises(okz.OkzError):
        okz.okz_width2_noalloc(dummy.data_ptr(), 100, 0, None)
    # an offset view of a tensor: not 16-byte aligned, refused before any launch
    with pytest.raises(okz.OkzError) as e:
        okz.okz_width2_noalloc(dummy.data_ptr() + 4, 32, 0, None)
    assert e.value.status == okz.OKZ_EINVAL
    assert "aligned" in okz.okz_last_error()
