"""The measured INT32 ALU-pipe rate (okz_alu_peak), the roofline denominator
of the sweep kernels: it must lie near 64 lanes x SMs x the SM clock (the
ALU pipe of a GB300 SM sub-partition executes 16 lanes per clock), between
the rates at the lowest and the highest clock nvidia-smi reports."""
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


def test_alu_peak_is_physical(okz):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ops, ms = okz.okz_alu_peak(None, 20000)
    assert ms > 0.1
    # 64 thread-ops per SM per clock, the SM clock between 0.8 and 2.2 GHz
    assert 64 * sms * 0.8e9 < ops < 64 * sms * 2.2e9 * 1.05, ops
