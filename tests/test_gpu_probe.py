"""The pipe-rate probe (the measured denominator of the pair kernels'
roofline) returns plausible per-SM rates on the GPU."""
import pytest

from paper_2505_22797_gb300 import api

pytestmark = pytest.mark.gpu


def test_pipe_rates_plausible():
    fma, ms = api.mpi_probe_pipe_rate(api.PROBE_FMA, 8, 2048)
    assert ms > 0.0
    # FP32 FMA: at most 128 lanes per SM per clock, and far above the MUFU rate
    assert 32.0 <= fma <= 140.0
    for op in (api.PROBE_RSQRT, api.PROBE_EX2, api.PROBE_RCP):
        rate, _ = api.mpi_probe_pipe_rate(op, 8, 2048)
        assert 2.0 <= rate <= fma


def test_packed_fma_rate_plausible():
    # fma.rn.f32x2 counts two operations per instruction: the FP32 lanes it
    # keeps busy are bounded by the same 128 per SM per clock
    fma, _ = api.mpi_probe_pipe_rate(api.PROBE_FMA, 8, 2048)
    fma2, ms = api.mpi_probe_pipe_rate(api.PROBE_FMA2, 8, 2048)
    assert ms > 0.0
    assert 0.5 * fma <= fma2 <= 140.0
