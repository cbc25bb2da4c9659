"""Served requests: continuous batching gives every request the result it gets alone."""
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


def test_served_results_equal_alone(okz):
    """A burst of Poisson requests (all sizes 2^7..2^13, the three (p, q) classes)
    served with continuous batching, a small pool so that admission waits for
    slots and arena space, and a tick short enough that requests join while
    others run: every request's exact sums, H0 and W^2 equal its run alone."""
    from paper_1110_6745_gb300 import serve
    reqs = serve.poisson_requests(n=120, rate=400.0, seed=7, log_budget=(1.0, 2.3))
    srv = serve.Server(small_arena_bytes=3 << 20, max_slots=24, large_bytes=256 << 20,
                       max_large=3, tick_sweeps=16)
    res = srv.run(reqs)
    srv.close()
    assert len(res) == len(reqs)
    for r in reqs:
        got = res[r.rid]
        Sk, H0, W2 = serve.run_alone(r)
        assert (got.Sk, got.H0, got.W2) == (Sk, H0, W2), r
        assert got.latency >= 0 and got.finished >= got.admitted >= r.arrival - 1e-9
    # requests really shared the device: most were in flight together with another
    spans = sorted((res[r.rid].admitted, res[r.rid].finished) for r in reqs)
    overlapped = sum(1 for i, (a, f) in enumerate(spans)
                     if any(a2 < f and f2 > a for j, (a2, f2) in enumerate(spans) if j != i))
    assert overlapped > len(reqs) // 2


def test_admission_refuses_when_full(okz):
    with okz.Batch(arena_bytes=8192, max_slots=2) as b:
        b.add(128, 1.0, 0.0, 1)
        with pytest.raises(okz.OkzError) as e:
            b.add(256, 1.0, 0.0, 2)  # 8 KiB lattice does not fit the rest of the arena
        assert e.value.status == okz.OKZ_EBUSY
        b.add(64, 1.0, 0.0, 3)
        with pytest.raises(okz.OkzError) as e:
            b.add(64, 1.0, 0.0, 4)  # no slot
        assert e.value.status == okz.OKZ_EBUSY
