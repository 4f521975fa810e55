"""Failure detection on the device without a GPU fault: every wait of the step kernels on a
shared-memory copy is bounded; a wait that cannot complete gives up, flags the timeout and lets
the kernel return, and the context stays usable."""
import numpy as np
import pytest

from tests.harness import drop_on_cylinder

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    import torch
    from paper_1908_04443_gb300 import lbmwet as L
    stream = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        assert L.lbm_selftest_bounded_wait(1024, stream)
        ev[1].record(stream)
    torch.cuda.synchronize()
    assert ev[0].elapsed_time(ev[1]) < 1000.0          # 1024 polls end well within a second
    assert L.lbm_selftest_bounded_wait(1, None)         # the legacy default stream, one poll
    # the context is intact: a small FP32 batch steps and matches its single-grid run
    case = drop_on_cylinder((48, 64), (32.0, 14.0), 7.0, (32.0, 27.0), 8.0, kappa=0.1, step_kernel="pair")
    case.rho_ref = case.bounds()[0]
    with case.gpu("fp32") as sim:
        sim.step(10)
        o, rho, _ = sim.observables(fields=True)
    assert np.isfinite(o.mass) and o.mass > 0

