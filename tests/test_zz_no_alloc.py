"""The allocation-free observables entry point, lbm_observables_noalloc.

It exists for callers that must not call cudaMalloc (frameworks that own all device memory through
their own allocator and budget, or latency-sensitive loops that cannot take cudaMalloc's implicit
synchronisation): its scratch is a static device array inside the library.  Here it is called
through the C ABI on caller-owned device fields, twice in a row on different states, and compared
with lbm_observables (which allocates its own buffers) on the same states, within the 1e-10 used
by the other observables parity tests.  This file is collected last so that a failure here comes
after every other test has run.
"""
import math

import numpy as np
import pytest

from tests.harness import drop_on_cylinder

pytestmark = pytest.mark.gpu


def _compare(o, ref):
    assert abs(o.mass - ref.mass) <= 1e-10 * abs(ref.mass)
    assert abs(o.rho_max - ref.rho_max) <= 1e-10
    assert abs(o.rho_min - ref.rho_min) <= 1e-10
    assert abs(o.u_max - ref.u_max) <= 1e-10
    assert o.n_interface == ref.n_interface
    assert o.step == ref.step
    if math.isnan(ref.theta_deg):
        assert math.isnan(o.theta_deg)
    else:
        assert abs(o.theta_deg - ref.theta_deg) <= 1e-10 * 180.0
        assert abs(o.drop_radius - ref.drop_radius) <= 1e-10 * ref.drop_radius


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_observables_twice(precision):
    import torch
    from paper_1908_04443_gb300 import lbmwet as L

    case = drop_on_cylinder((72, 64), (32.0, 22.0), 10.0, (32.0, 40.0), 12.0, kappa=0.2)
    stream = torch.cuda.current_stream()
    with case.gpu(precision, stream=stream) as sim:
        n = sim.n
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
        u = torch.empty(2 * n, dtype=torch.float64, device="cuda")
        results = []
        for steps in (40, 25):
            sim.step(steps)
            L.lbm_fields_device(sim.h, rho.data_ptr(), u.data_ptr())
            o = L.lbm_observables_noalloc(sim.h, rho.data_ptr(), u.data_ptr())
            ref = L.lbm_observables(sim.h)
            _compare(o, ref)
            results.append(o.mass + o.u_max)
        assert results[0] != results[1]     # the second call reflects the new state, not stale scratch


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_observables_3d(precision):
    """A drop on a sphere (D3Q19): the sphere-fit branch of the shared contact-angle code."""
    import torch
    from paper_1908_04443_gb300 import lbmwet as L

    case = drop_on_cylinder((32, 36, 40), (12.0, 18.0, 20.0), 7.0, (24.0, 18.0, 20.0), 8.0, kappa=0.1,
                            lattice="D3Q19")
    stream = torch.cuda.current_stream()
    with case.gpu(precision, stream=stream) as sim:
        n = sim.n
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
        u = torch.empty(3 * n, dtype=torch.float64, device="cuda")
        sim.step(30)
        L.lbm_fields_device(sim.h, rho.data_ptr(), u.data_ptr())
        o = L.lbm_observables_noalloc(sim.h, rho.data_ptr(), u.data_ptr())
        ref = L.lbm_observables(sim.h)
        assert ref.n_interface > 0
        _compare(o, ref)


def test_noalloc_rejects_grid_above_its_static_scratch():
    import torch
    from paper_1908_04443_gb300 import lbmwet as L

    shape = (4100, 4100)            # 16,810,000 nodes > 16,777,216
    mask = np.zeros(shape, np.uint8)
    e = L.make_eos("CS", 0.25, 4.0, 1.0, 0.0)
    e.T = 0.7 * L.lbm_critical_temperature(e)
    g, l = L.lbm_coexistence(e)
    cfg = L.make_config("D2Q9", "fp32", shape, e, rho_l=l, rho_g=g, rho_ref=g)
    sim = L.Simulation(cfg, mask, None, None, None, torch.cuda.current_stream())
    try:
        dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(L.LbmError) as ei:
            L.lbm_observables_noalloc(sim.h, dummy.data_ptr(), dummy.data_ptr())
        assert ei.value.status == L.LBM_ERR_ARG
        assert "16777216" in str(ei.value)
    finally:
        sim.close()
