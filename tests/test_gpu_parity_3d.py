"""D3Q19 parity of the CUDA path with the FP64 oracle: one step on ragged 3D grids (tiles of
32 x 4 x 4 do not divide them), 60 steps of a drop on a sphere in FP64 (1e-11) and FP32 deviation
storage (1e-4 relative at bulk nodes, 1e-4 of the liquid density in the interface band),
per-wall-node kappa, the constant virtual density, and the 3D observables (mass, extremes,
max |u|, sphere-fit contact angle)."""
import numpy as np
import pytest

from oracle import lbm, contact_angle as CA
from tests.fp32_bounds import split_errors
from tests.harness import drop_on_cylinder

pytestmark = pytest.mark.gpu


def sphere_case(shape=(22, 20, 26), c=(13.0, 10.0, 8.0), R=4.5, dc=(13.0, 10.0, 16.0), r=6.0, **kw):
    # shape is numpy (nz, ny, nx); centres are (x, y, z)
    return drop_on_cylinder(shape, c, R, dc, r, lattice="D3Q19", **kw)


def _one_step(case, precision="fp64", before=2):
    geo, p, f0 = case.oracle()
    with case.gpu(precision) as sim:
        sim.step(before)
        s0 = sim.get_state()
        sim.step(1)
        s1 = sim.get_state()
    return s1, lbm.step(s0, geo, p)


@pytest.mark.parametrize("kw", [dict(kappa=0.2), dict(kappa=-0.03), dict(wall="VD", rho_w_const=0.1),
                                dict(wall="SF", Gw=-0.2), dict(body_force=(2e-6, -1e-6, 3e-6))])
def test_one_step_d3q19_fp64(kw):
    s1, ref = _one_step(sphere_case(**kw))
    assert np.max(np.abs(s1 - ref)) < 1e-13


def test_one_step_d3q19_tiny_grid():
    s1, ref = _one_step(sphere_case(shape=(5, 6, 7), c=(3.0, 3.0, 2.0), R=1.0, dc=(3.0, 3.0, 3.5), r=1.5))
    assert np.max(np.abs(s1 - ref)) < 1e-13


def test_per_wall_node_kappa_3d():
    case = sphere_case()
    geo = lbm.Geometry(case.mask, "D3Q19")
    case.kappa = np.random.default_rng(9).uniform(-0.03, 0.3, len(geo.wall_flat))
    s1, ref = _one_step(case)
    assert np.max(np.abs(s1 - ref)) < 1e-13


def test_sphere_60_steps_fp64_and_fp32():
    case = sphere_case(kappa=0.15)
    g, l = case.bounds()
    geo, p, f0 = case.oracle()
    f = lbm.run(f0, geo, p, 60)
    o_ref, rho_ref, u_ref = lbm.observables(f, geo, p)
    fl = geo.fluid
    with case.gpu("fp64") as sim:
        sim.step(60)
        o, rho, u = sim.observables(fields=True)
    assert np.max(np.abs(rho[fl] - rho_ref[fl])) < 1e-11
    assert np.max(np.abs(u[:, fl] - u_ref[:, fl])) < 1e-11
    assert abs(o.mass / o_ref.mass - 1) < 1e-12
    assert abs(o.u_max - o_ref.u_max) < 1e-11
    th, c, r, npts = CA.contact_angle(rho_ref, case.mask, l, g, case.drop_hint, case.body[1], case.body[2])
    assert o.n_interface == npts
    assert abs(o.theta_deg - th) < 1e-6
    case.rho_ref = g
    with case.gpu("fp32") as sim:
        sim.step(60)
        o32, rho32, _ = sim.observables(fields=True)
    bulk, band, nb, ni = split_errors(rho32, rho_ref, case.mask, l, g)
    print(f"D3Q19 FP32 after 60 steps: bulk max |drho|/rho = {bulk:.3e} over {nb} nodes, "
          f"interface band max |drho|/rho_l = {band:.3e} over {ni} nodes")
    assert bulk <= 1e-4
    assert band <= 1e-4
    assert abs(o32.theta_deg - th) < 0.5


@pytest.mark.parametrize("shape,c,R,dc,r,kw", [
    ((22, 20, 26), (13.0, 10.0, 8.0), 4.5, (13.0, 10.0, 16.0), 6.0, dict(kappa=0.2)),
    ((21, 20, 26), (13.0, 10.0, 8.0), 4.5, (13.0, 10.0, 16.0), 6.0, dict(kappa=-0.03)),   # odd plane count
    ((70, 16, 40), (20.0, 8.0, 30.0), 5.0, (20.0, 8.0, 40.0), 6.0, dict(kappa=0.1)),      # 3 chunks, last of 6
    ((5, 6, 7), (3.0, 3.0, 2.0), 1.0, (3.0, 3.0, 3.5), 1.5, dict(kappa=0.2)),              # smaller than a column
    ((22, 20, 26), (13.0, 10.0, 8.0), 4.5, (13.0, 10.0, 16.0), 6.0, dict(wall="VD", rho_w_const=0.1)),
    ((22, 20, 26), (13.0, 10.0, 8.0), 4.5, (13.0, 10.0, 16.0), 6.0, dict(wall="SF", Gw=-0.2)),
    ((21, 20, 26), (13.0, 10.0, 8.0), 4.5, (13.0, 10.0, 16.0), 6.0, dict(wall="SF", Gw=0.3)),    # odd plane count
    ((22, 20, 26), (13.0, 10.0, 8.0), 4.5, (13.0, 10.0, 16.0), 6.0, dict(body_force=(2e-6, -1e-6, 3e-6))),
])
def test_one_step_d3q19_fp32(shape, c, R, dc, r, kw):
    """FP32 deviation storage (the z-pair march): one step against the oracle from a common state;
    2e-6 of the largest distribution bounds the FP32 rounding carried through one collision."""
    case = sphere_case(shape=shape, c=c, R=R, dc=dc, r=r, **kw)
    case.rho_ref = case.bounds()[0]
    s1, ref = _one_step(case, "fp32")
    assert np.max(np.abs(s1 - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_per_wall_node_kappa_3d_fp32():
    case = sphere_case()
    geo = lbm.Geometry(case.mask, "D3Q19")
    case.kappa = np.random.default_rng(9).uniform(-0.03, 0.3, len(geo.wall_flat))
    case.rho_ref = case.bounds()[0]
    s1, ref = _one_step(case, "fp32")
    assert np.max(np.abs(s1 - ref)) <= 2e-6 * np.max(np.abs(ref))
