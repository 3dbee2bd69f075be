"""Failure detection without a GPU fault.

A kernel waits, through the same bounded mbarrier wait the sweep kernels
use, on a barrier that nothing completes.  The wait gives up after about two
seconds, the kernel records the timeout in the handle's device error word
and returns; the host reads IDW_ERR_DEVICE_TIMEOUT and the context stays
usable for the next call.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as idw
    h = idw.Handle(0)
    idw.selftest_bounded_wait(handle=h)
    with pytest.raises(idw.IDWError) as e:
        idw.sync_status(handle=h)
    assert e.value.name == "IDW_ERR_DEVICE_TIMEOUT"
    # The error word was cleared and the context still computes.
    idw.sync_status(handle=h)
    d = torch.tensor([[0.0, 0.0, 1.0], [1.0, 0.0, 3.0]], device="cuda")
    q = torch.tensor([[0.5, 0.0]], device="cuda")
    z = idw.interpolate(d, q, 2.0, handle=h)
    assert abs(float(z[0]) - 2.0) < 1e-6
    h.close()


def test_pipe_rates_are_plausible():
    """The clock-counter probe behind the roofline's measured denominators:
    per SM per clock, FP32 FMA near 128 lanes (packed counted as two), MUFU
    reciprocal and log2 near 16, exp2 near 32 (twice rcp on this part), and
    FP64 FMA below 4."""
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as idw
    r = idw.measure_pipe_rates(0)
    assert 100 <= r["ffma"] <= 140, r
    assert 100 <= r["ffma2"] <= 140, r
    assert 12 <= r["mufu_rcp"] <= 20 and 12 <= r["mufu_lg2"] <= 20, r
    assert 24 <= r["mufu_ex2"] <= 40, r
    assert 0.5 <= r["dfma"] <= 4, r
