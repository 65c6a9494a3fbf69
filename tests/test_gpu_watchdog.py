"""Failure detection without a GPU fault: every wait inside the kernels is bounded. The probe
enqueues the same bounded mbarrier wait the coefficient kernel uses for its record copies, on a
barrier nothing arrives on; the wait must run out after its limit, set the device status word,
and leave the context usable (a following aggregation still matches the oracle)."""
import time

import numpy as np
import pytest

from gpu_helpers import check_against_oracle, oracle_case, run_path, torch_cuda

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    ctx = hgf.hgf_create(0)
    try:
        assert hgf.hgf_device_status(ctx, clear=True) == 0
        t0 = time.perf_counter()
        hgf.hgf_watchdog_probe(ctx, 20000)          # 20 ms
        status = hgf.hgf_device_status(ctx)          # waits for the device
        waited = time.perf_counter() - t0
        assert status == 1
        assert 0.015 <= waited < 5.0, waited
        assert hgf.hgf_device_status(ctx, clear=True) == 1
        assert hgf.hgf_device_status(ctx) == 0
        with pytest.raises(hgf.HGFError) as ei:
            hgf.hgf_watchdog_probe(ctx, 0)
        assert ei.value.status == hgf.HGF_EINVAL
        case, ref = oracle_case(120, 80, 5, 71, degree=2, r=9, eps=1e-4)
        q, labels, best = run_path(ctx, case.guidance, case.cost, "f32", 2, 9, 1e-4)
        check_against_oracle(q, labels, best, ref)
        assert hgf.hgf_device_status(ctx) == 0
    finally:
        hgf.hgf_destroy(ctx)
