"""The FP32 pair kernel (32 x 16 tiles, two nodes per thread, packed FP32x2 arithmetic) against
the FP64 oracle, one step from a common state, and against the scalar FP32 tile kernel.

One-step tolerance: the state is stored as FP32 deviations f_a - w_a rho_ref, so one step carries
their rounding (relative 6e-8 of the distributions) through the collision; 2e-6 of the largest
distribution bounds it with margin, as for the other FP32 kernels.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lbm
from tests.harness import Case, drop_on_cylinder

pytestmark = pytest.mark.gpu


def _one_step(case, steps_before=3):
    case.step_kernel = "pair"
    case.rho_ref = case.bounds()[0]
    geo, p, _ = case.oracle()
    with case.gpu("fp32") as sim:
        assert sim.step_kernel() == "pair"
        sim.step(steps_before)
        f0 = sim.get_state()
        sim.step(1)
        f1 = sim.get_state()
    ref = lbm.step(f0, geo, p)
    return f1, ref


@pytest.mark.parametrize("shape,center,R,dc,r", [
    ((100, 100), (50.0, 50.0), 20.0, (50.0, 95.0), 25.0),     # whole tiles, wrapping drop
    ((37, 53), (20.3, 17.1), 9.5, (21.0, 30.0), 10.0),         # ragged tiles in x and y
    ((8, 8), (3.0, 4.0), 1.5, (5.0, 4.0), 2.5),                # grid smaller than one tile
    ((5, 70), (30.0, 2.0), 1.0, (40.0, 2.0), 3.0),             # thin strip
    ((90, 200), (100.0, 40.0), 16.0, (100.0, 72.0), 17.0),     # interior tiles without wrap
    ((70, 130), (3.0, 35.0), 12.0, (3.0, 58.0), 12.0),         # body across the periodic x edge
])
def test_pair_one_step(shape, center, R, dc, r):
    f1, ref = _one_step(drop_on_cylinder(shape, center, R, dc, r, kappa=0.15))
    assert np.max(np.abs(f1 - ref)) <= 2e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("kw", [
    dict(kappa=-0.02),
    dict(wall="VD", rho_w_const=0.1),
    dict(wall="SF", Gw=-0.2),
    dict(wall="SF", Gw=0.3),
    dict(body_force=(1e-5, -3e-6, 0.0)),
    dict(eos_kind="PR", t_over_tc=0.86, sigma=0.11),
    dict(rates=dict(s_e=0.6, s_eps=1.5, s_q=1.2, s_nu=1.7)),
])
def test_pair_one_step_variants(kw):
    f1, ref = _one_step(drop_on_cylinder((48, 40), (20.0, 15.0), 7.0, (20.0, 28.0), 9.0, **kw), steps_before=2)
    assert np.max(np.abs(f1 - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_pair_per_wall_node_kappa_and_plates():
    base = drop_on_cylinder((40, 44), (22.0, 15.0), 8.0, (22.0, 28.0), 8.0)
    geo = lbm.Geometry(base.mask, "D2Q9")
    base.kappa = np.random.default_rng(3).uniform(-0.02, 0.4, len(geo.wall_flat))
    f1, ref = _one_step(base, steps_before=2)
    assert np.max(np.abs(f1 - ref)) <= 2e-6 * np.max(np.abs(ref))
    shape = (40, 100)
    mask = W.plates_mask(shape)
    g, l = Case("D2Q9", shape, mask, np.zeros(shape)).bounds()
    rho = W.tanh_drop_density(shape, (50.0, 20.0), 12.0, l, g) + W.density_noise(shape, 1e-6)
    plates = Case("D2Q9", shape, mask, np.where(mask != 0, g, rho), kappa=0.1)
    f1, ref = _one_step(plates)
    assert np.max(np.abs(f1 - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_pair_agrees_with_tile_kernel():
    """200 steps of a drop spreading on a cylinder: the pair and tile kernels differ only by the
    regrouping of FP32 operations."""
    states = {}
    for kernel in ("tile", "pair"):
        case = drop_on_cylinder((90, 200), (100.0, 40.0), 16.0, (100.0, 72.0), 17.0, kappa=0.15, step_kernel=kernel)
        case.rho_ref = case.bounds()[0]
        with case.gpu("fp32") as sim:
            sim.step(200)
            o, rho, _ = sim.observables(fields=True)
            states[kernel] = (o, rho)
    (ot, rt), (op, rp) = states["tile"], states["pair"]
    g, l = case.bounds()
    assert np.max(np.abs(rt - rp)) < 1e-4 * l
    assert abs(ot.mass / op.mass - 1) < 1e-6
    assert abs(ot.theta_deg - op.theta_deg) < 0.05


def test_pair_unstable_state_is_reported():
    from paper_1908_04443_gb300 import lbmwet as L
    case = drop_on_cylinder((16, 16), (8.0, 5.0), 2.0, (8.0, 10.0), 3.0, step_kernel="pair")
    case.rho_ref = case.bounds()[0]
    sim = case.gpu("fp32")
    sim.cfg.G = 1.0
    sim.close()
    sim = L.Simulation(sim.cfg, case.mask, case.rho0)
    with pytest.raises(L.LbmError) as ei:
        sim.step(2)
    assert ei.value.status == L.LBM_ERR_UNSTABLE
    sim.close()


def test_pair_rejected_for_fp64():
    from paper_1908_04443_gb300 import lbmwet as L
    case = drop_on_cylinder((16, 16), (8.0, 5.0), 2.0, (8.0, 10.0), 3.0, step_kernel="pair")
    with pytest.raises(L.LbmError) as ei:
        case.gpu("fp64")
    assert ei.value.status == L.LBM_ERR_ARG
