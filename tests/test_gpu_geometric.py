"""The curved geometric-formulation scheme (Sec. III.A, Eqs. 10-15) in every D2Q9 step kernel
against the FP64 oracle: one step from a common state and short runs, FP64 (tile and y-march) to
1e-13, FP32 (tile, y-march and pair) to 2e-6 of the largest distribution as for the other wall
schemes; batches of instances with different prescribed angles equal the same grids stepped
alone; and the angles of drops on a cylinder follow the prescribed ones (Fig. 8)."""
import numpy as np
import pytest

from oracle import lbm
from tests.harness import drop_on_cylinder

pytestmark = pytest.mark.gpu

# (shape (ny, nx), cylinder centre, R, drop centre, r): whole tiles with a wrapping drop, ragged
# tiles in x and y, a body across the periodic x edge
GRIDS = [((100, 100), (50.0, 50.0), 20.0, (50.0, 95.0), 25.0),
         ((37, 53), (20.3, 17.1), 9.5, (21.0, 30.0), 10.0),
         ((70, 130), (3.0, 35.0), 12.0, (3.0, 58.0), 12.0)]


def _case(grid, theta_a, kernel):
    shape, c, R, dc, r = GRIDS[grid]
    case = drop_on_cylinder(shape, c, R, dc, r, wall="GF", theta_a=theta_a)
    case.step_kernel = kernel
    return case


def _one_step(case, precision, before=3):
    if precision == "fp32":
        case.rho_ref = case.bounds()[0]
    geo, p, _ = case.oracle()
    with case.gpu(precision) as sim:
        assert sim.step_kernel() == case.step_kernel
        sim.step(before)
        f0 = sim.get_state()
        sim.step(1)
        f1 = sim.get_state()
    return f1, lbm.step(f0, geo, p)


@pytest.mark.parametrize("kernel", ["tile", "ymarch"])
@pytest.mark.parametrize("theta_a", [30.0, 60.0, 90.0, 120.0, 150.0])
@pytest.mark.parametrize("grid", range(len(GRIDS)))
def test_gf_one_step_fp64(kernel, theta_a, grid):
    f1, ref = _one_step(_case(grid, theta_a, kernel), "fp64")
    assert np.max(np.abs(f1 - ref)) < 1e-13


@pytest.mark.parametrize("kernel", ["tile", "ymarch", "pair"])
@pytest.mark.parametrize("theta_a", [30.0, 60.0, 120.0, 150.0])
@pytest.mark.parametrize("grid", range(len(GRIDS)))
def test_gf_one_step_fp32(kernel, theta_a, grid):
    f1, ref = _one_step(_case(grid, theta_a, kernel), "fp32")
    assert np.max(np.abs(f1 - ref)) <= 2e-6 * np.max(np.abs(ref))


def _notch_case(theta_a, kernel):
    """A solid block with a notch and a post under it (concave corners: crossings with solid ends,
    unusable crossings and the Eq. 17 fallback all occur), a drop over the notch."""
    import workloads as W
    from tests.harness import Case
    base = drop_on_cylinder((40, 48), (24.0, 30.0), 5.0, (22.0, 24.0), 8.0)   # for the EOS and densities
    g, l = base.bounds()
    mask = np.zeros((40, 48), np.uint8)
    mask[5:20, 8:40] = 1
    mask[12:20, 18:26] = 0
    mask[20:30, 30:34] = 1
    rho = W.tanh_drop_density((40, 48), (22.0, 24.0), 8.0, l, g) + W.density_noise((40, 48), 1e-6, 99)
    rho = np.where(mask != 0, g, rho)
    return Case("D2Q9", (40, 48), mask, rho, wall="GF", theta_a=theta_a, step_kernel=kernel)


@pytest.mark.parametrize("precision,kernel", [("fp64", "tile"), ("fp64", "ymarch"), ("fp32", "pair")])
@pytest.mark.parametrize("theta_a", [20.0, 60.0, 170.0])
def test_gf_concave_corners(precision, kernel, theta_a):
    f1, ref = _one_step(_notch_case(theta_a, kernel), precision)
    if precision == "fp64":
        assert np.max(np.abs(f1 - ref)) < 1e-13
    else:
        assert np.max(np.abs(f1 - ref)) <= 2e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("kernel", ["tile", "ymarch"])
def test_gf_run_fp64(kernel):
    """40 steps from the initial state: the wall densities feed back through the whole run."""
    case = _case(1, 60.0, kernel)
    geo, p, f0 = case.oracle()
    ref = lbm.run(f0, geo, p, 40)
    with case.gpu("fp64") as sim:
        sim.step(40)
        f = sim.get_state()
    assert np.max(np.abs(f - ref)) < 1e-12


@pytest.mark.parametrize("precision,kernel", [("fp64", "tile"), ("fp64", "ymarch"), ("fp32", "ymarch"),
                                               ("fp32", "pair")])
def test_gf_batch_equals_single_runs(precision, kernel):
    from paper_1908_04443_gb300 import lbmwet as L
    cases = [_case(g, th, kernel) for g, th in ((0, 60.0), (1, 120.0), (2, 45.0), (1, 90.0))]
    sims = [cs.gpu(precision) for cs in cases]
    cfgs = [s.cfg for s in sims]
    for s in sims:
        s.close()
    b = L.lbm_batch_init(cfgs, [cs.mask for cs in cases], [cs.rho0 for cs in cases], [None] * len(cases))
    try:
        assert L.lbm_batch_step_kernel_used(b) == kernel
        L.lbm_batch_step(b, 21)
        for i, cs in enumerate(cases):
            fb = L.lbm_get_state(L.lbm_batch_handle(b, i), 9, cs.mask.size)
            with cs.gpu(precision) as sim:
                sim.step(21)
                fs = sim.get_state().reshape(-1)
            assert np.max(np.abs(fb - fs)) == 0.0
    finally:
        L.lbm_batch_destroy(b)


def test_gf_rejects_per_node_kappa_updates():
    from paper_1908_04443_gb300 import lbmwet as L
    case = _case(1, 60.0, "tile")
    with case.gpu("fp64") as sim:
        with pytest.raises(L.LbmError) as ei:
            L.lbm_set_kappa(sim.h, np.zeros(len(sim.wall_nodes())))
        assert ei.value.status == L.LBM_ERR_ARG


def test_fig8_cylinder_angles_follow_the_prescribed_ones():
    """Sec. IV.A geometry (300 x 350, PR at 0.86 Tc, cylinder R = 70 at (150, 130), drop r = 50 at
    (150, 230)) with the geometric formulation, FP32, 30,000 steps.  The paper reads 58, 88 and 121
    degrees for theta_a = 60, 90 and 120 (Fig. 8), spurious currents below 0.006 for this scheme
    (Fig. 10) and extreme densities at rho_l ~ 6.5 and rho_g ~ 0.38 (Fig. 11).  Measured here:
    62.4, 90.0 and 117.9 degrees, max |u| about 0.002."""
    thetas = []
    for theta_a in (60.0, 90.0, 120.0):
        case = drop_on_cylinder((350, 300), (150.0, 130.0), 70.0, (150.0, 230.0), 50.0, eos_kind="PR",
                                t_over_tc=0.86, sigma=0.11, wall="GF", theta_a=theta_a)
        case.rho_ref = case.bounds()[0]
        g, l = case.bounds()
        with case.gpu("fp32") as sim:
            sim.step(30000)
            o = sim.observables()[0]
        assert abs(o.theta_deg - theta_a) < 4.0
        assert o.u_max < 0.006
        assert abs(o.rho_max / l - 1) < 0.01 and abs(o.rho_min / g - 1) < 0.05
        thetas.append(o.theta_deg)
    assert thetas[0] < thetas[1] < thetas[2]
