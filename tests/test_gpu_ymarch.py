"""The D2Q9 y-march step kernel (persistent CTAs walking runs of rows of 124-column blocks, planned
on the host) against the FP64 oracle and against the tile kernel.

Grids wider than one column block (ragged last block), a body that crosses the periodic x edge,
and grids with few rows; the planner cuts small grids into runs of 4 rows, so walls cross run
boundaries everywhere.  Both kernels evaluate every node with the same arithmetic in the same
order, so their states agree bit for bit.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lbm
from tests.harness import Case, drop_on_cylinder

pytestmark = pytest.mark.gpu


def _one_step(case, precision="fp64", steps_before=3):
    geo, p, _ = case.oracle()
    with case.gpu(precision) as sim:
        assert sim.step_kernel() == case.step_kernel
        sim.step(steps_before)
        f0 = sim.get_state()
        sim.step(1)
        f1 = sim.get_state()
    return f1, lbm.step(f0, geo, p)


WIDE = [
    ((200, 300), (150.0, 80.0), 30.0, (150.0, 125.0), 20.0),   # 3 column blocks, the last 52 wide
    ((130, 260), (5.0, 60.0), 25.0, (5.0, 100.0), 18.0),       # body across the periodic x edge
    ((9, 400), (100.0, 4.0), 2.0, (200.0, 4.0), 3.5),          # 9 rows
    ((60, 124), (62.0, 20.0), 10.0, (62.0, 40.0), 12.0),       # exactly one column block
]


@pytest.mark.parametrize("shape,center,R,dc,r", WIDE)
def test_ymarch_one_step_fp64(shape, center, R, dc, r):
    case = drop_on_cylinder(shape, center, R, dc, r, kappa=0.12, step_kernel="ymarch")
    f1, ref = _one_step(case)
    assert np.max(np.abs(f1 - ref)) < 1e-13


@pytest.mark.parametrize("kw", [dict(kappa=-0.03), dict(wall="VD", rho_w_const=0.15), dict(wall="SF", Gw=-0.2),
                                dict(eos_kind="PR", t_over_tc=0.86, sigma=0.11)])
def test_ymarch_one_step_variants(kw):
    case = drop_on_cylinder((140, 250), (125.0, 50.0), 20.0, (125.0, 85.0), 16.0, step_kernel="ymarch", **kw)
    f1, ref = _one_step(case, steps_before=2)
    assert np.max(np.abs(f1 - ref)) < 1e-13 * max(1.0, np.abs(ref).max())


def test_ymarch_plates_every_run_solid():
    """Solid rows at y = 0 and y = ny - 1: every run of a 40-row channel touches a wall."""
    shape = (40, 200)
    mask = W.plates_mask(shape)
    probe = Case("D2Q9", shape, mask, np.zeros(shape))
    g, l = probe.bounds()
    rho = W.tanh_drop_density(shape, (100.0, 20.0), 12.0, l, g) + W.density_noise(shape, 1e-6)
    rho = np.where(mask != 0, g, rho)
    case = Case("D2Q9", shape, mask, rho, kappa=0.1, step_kernel="ymarch")
    f1, ref = _one_step(case)
    assert np.max(np.abs(f1 - ref)) < 1e-13


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ymarch_equals_tile_kernel(precision):
    shape, center, R, dc, r = WIDE[0]
    states = {}
    for kernel in ("tile", "ymarch"):
        case = drop_on_cylinder(shape, center, R, dc, r, kappa=0.12, step_kernel=kernel)
        if precision == "fp32":
            case.rho_ref = case.bounds()[0]
        with case.gpu(precision) as sim:
            sim.step(21)
            states[kernel] = sim.get_state()
    assert np.array_equal(states["tile"], states["ymarch"])


def test_automatic_choice_and_record():
    from paper_1908_04443_gb300 import lbmwet as L
    small = drop_on_cylinder((100, 100), (50.0, 50.0), 20.0, (50.0, 95.0), 25.0)
    with small.gpu("fp32") as sim:
        assert sim.step_kernel() == "pair"
    with small.gpu("fp64") as sim:
        assert sim.step_kernel() == "tile"
    shape = (1024, 1024)
    big = drop_on_cylinder(shape, (512.0, 300.0), 100.0, (512.0, 470.0), 80.0, step_kernel="ymarch")
    with big.gpu("fp32") as sim:
        assert sim.step_kernel() == "ymarch"
        sim.step(2)
        L.lbm_record(sim.h, 4, 2)                # the adjoint's trajectory is stepped by the tile kernel
        assert sim.step_kernel() == "tile"
