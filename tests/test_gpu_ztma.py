"""The TMA-staged D3Q19 z-march (FP32, the default D3Q19 step) against the FP64 oracle.

Its columns are 32 x 8 cells over 32-plane chunks; chunks away from solids stage their pulls
through shared memory by TMA, and where a column's box crosses a periodic edge the out-of-range
columns and rows are loaded separately.  The grids below put boxed columns on every edge and
corner (x0 = 0 and x0 + 32 = nx, y0 = 0 and y0 + 8 = ny), mix them with chunks holding solids (the
z-pair march) and with ragged columns, and end in partial chunks.  One step from a common evolved
state is compared with the oracle (2e-6 of the largest distribution: FP32 rounding carried through
one collision), 60 steps are compared with the split FP32 density bounds, and the kernel is
checked to agree with the z-pair march and the scalar z-march run alone.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lbm, contact_angle as CA
from tests.fp32_bounds import split_errors
from tests.harness import Case, drop_on_cylinder

pytestmark = pytest.mark.gpu


def _sphere(shape, c, R, dc, r, **kw):
    case = drop_on_cylinder(shape, c, R, dc, r, lattice="D3Q19", **kw)
    case.rho_ref = case.bounds()[0]
    return case


# (nz, ny, nx), sphere centre (x, y, z), radius, drop centre, radius
GRIDS = {
    "edges": ((40, 24, 96), (48.0, 12.0, 14.0), 4.0, (48.0, 12.0, 24.0), 6.0),       # 3 x 3 columns, 2 chunks
    "ragged": ((37, 21, 100), (70.0, 10.0, 30.0), 3.5, (70.0, 10.0, 20.0), 5.0),     # ragged x and y columns
    "corner": ((33, 16, 64), (10.0, 3.0, 30.0), 2.5, (40.0, 8.0, 12.0), 5.0),        # every column on a corner
}


def _one_step(case, kernel, before=3):
    geo, p, f0 = case.oracle()
    case.step_kernel = kernel
    with case.gpu("fp32") as sim:
        assert sim.step_kernel() == kernel
        sim.step(before)
        s0 = sim.get_state()
        sim.step(1)
        s1 = sim.get_state()
    return s0, s1, lbm.step(s0, geo, p)


@pytest.mark.parametrize("grid", sorted(GRIDS))
@pytest.mark.parametrize("kw", [dict(kappa=0.2), dict(kappa=-0.03, body_force=(2e-6, -1e-6, 3e-6)),
                                dict(wall="SF", Gw=-0.2), dict(wall="VD", rho_w_const=0.1)])
def test_ztma_one_step(grid, kw):
    case = _sphere(*GRIDS[grid], **kw)
    s0, s1, ref = _one_step(case, "ztma")
    assert np.max(np.abs(s1 - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_ztma_all_fluid_flat_interface():
    """No solid anywhere: every column is boxed; a flat liquid slab normal to y crosses the columns'
    y edges and carries the largest density gradients through the wrapped rows."""
    shape = (36, 16, 64)
    g, l = Case("D3Q19", shape, np.zeros(shape, np.uint8), np.zeros(shape)).bounds()
    rho = W.slab_density(shape, 4, 12, l, g) + W.density_noise(shape, 1e-6)
    case = Case("D3Q19", shape, np.zeros(shape, np.uint8), rho, rho_ref=g)
    s0, s1, ref = _one_step(case, "ztma", before=5)
    assert np.max(np.abs(s1 - ref)) <= 2e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("grid", sorted(GRIDS))
def test_ztma_agrees_with_the_other_fp32_kernels(grid):
    """From the same state, one step of each FP32 D3Q19 kernel: the TMA z-march, the z-pair march and
    the scalar z-march agree to FP32 rounding (their operations are grouped differently)."""
    case = _sphere(*GRIDS[grid], kappa=0.15)
    out = {}
    for k in ("ztma", "pair", "tile"):
        out[k] = _one_step(case, k)
    ref = out["tile"][2]
    scale = np.max(np.abs(ref))
    for k in ("ztma", "pair"):
        assert np.max(np.abs(out[k][1] - out["tile"][1])) <= 2e-6 * scale, k


def test_ztma_60_steps_against_oracle():
    case = _sphere(*GRIDS["edges"], kappa=0.15)
    g, l = case.bounds()
    geo, p, f0 = case.oracle()
    o_ref, rho_ref, _ = lbm.observables(lbm.run(f0, geo, p, 60), geo, p)
    case.step_kernel = "ztma"
    with case.gpu("fp32") as sim:
        sim.step(60)
        o, rho, _ = sim.observables(fields=True)
    bulk, band, nb, ni = split_errors(rho, rho_ref, case.mask, l, g)
    print(f"ztma FP32 after 60 steps: bulk max |drho|/rho = {bulk:.3e} over {nb} nodes, "
          f"interface band max |drho|/rho_l = {band:.3e} over {ni} nodes")
    assert bulk <= 1e-4
    assert band <= 1e-4
    th, *_ = CA.contact_angle(rho_ref, case.mask, l, g, case.drop_hint, case.body[1], case.body[2])
    assert abs(o.theta_deg - th) < 0.5
    assert abs(o.mass / o_ref.mass - 1) < 1e-5


def test_ztma_kernel_selection():
    from paper_1908_04443_gb300 import lbmwet as L
    case = _sphere(*GRIDS["corner"], kappa=0.1)
    with case.gpu("fp32") as sim:
        assert sim.step_kernel() == "ztma"          # the FP32 default
    with case.gpu("fp64") as sim:
        assert sim.step_kernel() == "tile"          # FP64: the scalar z-march
    case.step_kernel = "ztma"
    with pytest.raises(L.LbmError):
        case.gpu("fp64")


def test_ztma_state_round_trip():
    """A state written from outside the step (set_state of a state read back, or a reloaded
    checkpoint) steps on exactly as the original."""
    from paper_1908_04443_gb300 import lbmwet as L
    case = _sphere(*GRIDS["edges"], kappa=0.1)
    case.step_kernel = "ztma"
    with case.gpu("fp32") as sim:
        sim.step(5)
        s5 = sim.get_state()
        blob = L.lbm_save_state(sim.h)
        sim.step(1)
        s6 = sim.get_state()
        sim.set_state(s5, step=5)
        sim.step(1)
        assert np.max(np.abs(sim.get_state() - s6)) <= 1e-6 * np.max(np.abs(s6))
        L.lbm_load_state(sim.h, blob)
        sim.step(1)
        assert np.array_equal(sim.get_state(), s6)


@pytest.mark.parametrize("plate", [(0, 2), (35, 37)])
def test_ztma_plate_band(plate):
    """A flat plate filling whole planes (at the bottom, so that its neighbourhood wraps to the top
    planes, or in the middle of the z-range) with a drop on it: every column's z-range is cut into a
    band on the path for planes near solids and bulk pieces on both sides of it, the last bulk piece
    shorter than the minimum and joined to its neighbour.  One step from a common state against the
    oracle covers every plane exactly once."""
    from oracle import eos as E
    shape = (70, 16, 64)                                   # (nz, ny, nx): 2 x 2 boxed columns
    eos = E.cs_config().at_reduced_temperature(0.7)
    g, l = E.maxwell(eos)
    mask = np.zeros(shape, np.uint8)
    mask[plate[0]:plate[1]] = 1
    dc = (32.0, 8.0, float(plate[1] + 5))
    rho = W.tanh_drop_density(shape, dc, 6.0, l, g) + W.density_noise(shape, 1e-6)
    rho = np.where(mask != 0, g, rho)
    case = Case("D3Q19", shape, mask, rho, kappa=0.1, drop_hint=dc, rho_ref=g)
    s0, s1, ref = _one_step(case, "ztma")
    assert np.max(np.abs(s1 - ref)) <= 2e-6 * np.max(np.abs(ref))
