"""Failure detection on the GPU without a fault: a bounded device-side wait
that cannot complete must give up, report OKZ_ETIMEOUT and leave the context
usable."""
import time

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


def test_bounded_wait_times_out_and_the_context_survives(okz, orc):
    t0 = time.perf_counter()
    with pytest.raises(okz.OkzError) as e:
        okz.okz_selftest_wait_timeout()
    waited = time.perf_counter() - t0
    assert e.value.status == okz.OKZ_ETIMEOUT
    assert 1.5 < waited < 60, waited  # the library's limit is 2 s of %globaltimer
    # the same context still runs the hot path correctly
    ref = orc.Sim(4096, 1.0, 0.0, 9)
    ref.sweep(3)
    with okz.Simulation(4096, 1.0, 0.0, seed=9) as sim:
        sim.sweep(3)
        assert sim.width2()[2] == ref.width2()
