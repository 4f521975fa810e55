"""Pins of the oracle's curved geometric-formulation scheme (Sec. III.A, Eqs. 10-15): the
isotropy of the Eq. 14 weights, the Eq. 13 normal on flat and curved walls, the mesh crossing of a
characteristic against an independent bisection, the flat-wall closed form (the scheme reduces to
the form of Eq. 9 on a linear density field), mirror symmetry of a symmetric drop, and the
prescribed angle reached by a drop on a flat wall (Fig. 8: theta close to theta_a)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import contact_angle as CA, eos as E, geometric as GF, lbm

CS07 = E.cs_config().at_reduced_temperature(0.7)
G07, L07 = E.maxwell(CS07)


def _moment(px, py):
    return sum(w * ex ** px * ey ** py for ex, ey, w in GF.eq14_stencil())


def test_eq14_weights_are_eighth_order_isotropic():
    """Sums of w e_x^i e_y^j over the 24 vectors equal those of an isotropic tensor up to rank 8
    (ratios 3:1 at rank 4, 15:3 at rank 6, 105:15:9 at rank 8), with sum w e_x^2 = 1: a wrong
    weight or a missing |e|^2 shell breaks one of them."""
    assert len(GF.eq14_stencil()) == 24
    assert _moment(2, 0) == pytest.approx(1.0, abs=1e-15)
    assert _moment(1, 1) == pytest.approx(0.0, abs=1e-15)
    assert _moment(4, 0) == pytest.approx(3 * _moment(2, 2), abs=1e-14)
    assert _moment(6, 0) == pytest.approx(5 * _moment(4, 2), abs=1e-14)
    assert _moment(4, 2) == pytest.approx(_moment(2, 4), abs=1e-14)
    c8 = _moment(4, 4) / 9
    assert _moment(8, 0) == pytest.approx(105 * c8, abs=1e-13)
    assert _moment(6, 2) == pytest.approx(15 * c8, abs=1e-13)


# (solid slab rows or columns, wall node P (x, y), outward normal)
FLAT = [("x", slice(0, 6), (5, 8), (1.0, 0.0)),
        ("x", slice(12, 18), (12, 8), (-1.0, 0.0)),
        ("y", slice(0, 6), (7, 5), (0.0, 1.0)),
        ("y", slice(10, 16), (7, 10), (0.0, -1.0))]


@pytest.mark.parametrize("axis,slab,P,want", FLAT)
def test_normal_of_flat_walls(axis, slab, P, want):
    """Eq. 13 next to a solid slab is the outward axis vector exactly."""
    solid = np.zeros((16, 18), bool)
    if axis == "x":
        solid[:, slab] = True
    else:
        solid[slab, :] = True
    assert GF.solid_normal(solid, *P) == pytest.approx(want, abs=1e-15)


def test_normal_of_a_diagonal_wall():
    """Next to the staircase half-plane x + y <= 20 the normal is (1, 1)/sqrt(2) exactly."""
    solid = np.fromfunction(lambda y, x: x + y <= 20, (40, 40))
    for x in range(4, 17):
        n = GF.solid_normal(solid, x, 20 - x)
        assert n == pytest.approx((math.sqrt(0.5), math.sqrt(0.5)), abs=1e-15)


def test_normal_of_a_cylinder():
    """Around a staircase disc of radius 30 the normals point outwards (within 20 degrees of the
    radius at every wall node, within 10 on average: the staircase bends them) and form a field
    with the disc's mirror symmetries (x -> 90 - x and x <-> y)."""
    shape, c, R = (91, 91), (45.0, 45.0), 30.0
    mask = W.ball_mask(shape, c, R)
    geo = lbm.Geometry(mask, "D2Q9")
    errs = []
    for g in geo.wall_flat:
        y, x = divmod(int(g), shape[1])
        n = GF.solid_normal(geo.solid, x, y)
        r = (x - c[0], y - c[1])
        cosang = (n[0] * r[0] + n[1] * r[1]) / math.hypot(*r)
        errs.append(math.degrees(math.acos(min(1.0, cosang))))
        m = GF.solid_normal(geo.solid, 90 - x, y)
        assert m == pytest.approx((-n[0], n[1]), abs=1e-15)
        t = GF.solid_normal(geo.solid, y, x)
        assert t == pytest.approx((n[1], n[0]), abs=1e-15)
    assert max(errs) < 20.0 and np.mean(errs) < 10.0


def _exit_point_by_bisection(d):
    lo, hi = 0.0, 4.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if max(abs(mid * d[0]), abs(mid * d[1])) < 1.0:
            lo = mid
        else:
            hi = mid
    return lo * d[0], lo * d[1]


def test_mesh_crossing_against_bisection():
    """The interpolation nodes of a crossing are lattice neighbours on the square's boundary, their
    weights are positive and sum to 1, and the weighted node position is the ray's exit point found
    by bisection."""
    rng = np.random.default_rng(3)
    angles = list(rng.uniform(0, 2 * math.pi, 400)) + [k * math.pi / 4 for k in range(8)]
    for a in angles:
        d = (math.cos(a), math.sin(a))
        ends = GF.mesh_crossing(d)
        assert 1 <= len(ends) <= 2
        assert sum(w for _, w in ends) == pytest.approx(1.0, abs=1e-15)
        for (ex, ey), w in ends:
            assert w > 0 and max(abs(ex), abs(ey)) == 1
        px = sum(w * ex for (ex, _), w in ends)
        py = sum(w * ey for (_, ey), w in ends)
        bx, by = _exit_point_by_bisection(d)
        assert (px, py) == pytest.approx((bx, by), abs=1e-12)


@pytest.mark.parametrize("theta_a", [60.0, 75.0, 90.0, 105.0, 120.0])
def test_flat_wall_reduces_to_the_eq9_form(theta_a):
    """On a flat wall with a linear density field rho = a + b x + c y in the fluid, the
    characteristics of P = (x, y_w) cross the first fluid row at x -+ tan(theta'), so Eq. 11 gives
    rho_P = rho(x, y_w + 1) + tan(pi/2 - theta_a) |b| - the discrete form of Eq. 9 (central
    difference of the first fluid row, normal offset of one node)."""
    ny, nx, thick = 14, 24, 4
    mask = W.flat_wall_mask((ny, nx), thick)
    geo = lbm.Geometry(mask, "D2Q9")
    a, b, c = 0.2, 0.013, -0.004
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    rho = np.where(mask == 0, a + b * xx + c * yy, 0.0)
    rho_ave = np.zeros(len(geo.wall_flat))
    rw = GF.wall_density(rho, geo, theta_a, rho_ave)
    tp = math.tan(math.pi / 2 - math.radians(theta_a))
    checked = 0
    for k, g in enumerate(geo.wall_flat):
        y, x = divmod(int(g), nx)
        if y != thick - 1 or not 2 <= x <= nx - 3:
            continue                                      # top of the slab, away from the x seam
        want = a + b * x + c * (y + 1) + tp * abs(b)
        assert rw[k] == pytest.approx(want, abs=1e-15)
        checked += 1
    assert checked == nx - 4


def test_gf_mirror_symmetry_and_mass():
    """A drop centred over a cylinder stays mirror-symmetric under the scheme (n_1 and n_2 of Eq. 15
    are mirror images, so a wrong rotation sign breaks the symmetry), and mass is conserved."""
    wl = W.c1_parity_cylinder()
    wl.noise = 0.0
    mask = wl.mask()
    geo = lbm.Geometry(mask, "D2Q9")
    p = lbm.Params("D2Q9", CS07, sigma=0.12, rho_l=L07, rho_g=G07, wall="GF", theta_a=60.0)
    f0 = lbm.init_state(wl.rho0(L07, G07), geo)
    f = lbm.run(f0, geo, p, 150)
    o, rho, u = lbm.observables(f, geo, p)
    mir = np.roll(rho[:, ::-1], 1, axis=1)
    assert np.max(np.abs(rho - mir)) < 1e-12
    assert abs(f.sum() / f0.sum() - 1) < 1e-12
    assert o.u_max > 1e-5


def test_no_normal_for_a_one_node_thick_plate():
    """Next to a solid line one node thick the Eq. 13 sum cancels (up to rounding): no normal, and
    the scheme refuses the geometry; a two-node plate has the outward normals."""
    solid = np.zeros((8, 10), bool)
    solid[4, :] = True
    assert GF.solid_normal(solid, 3, 4) is None
    geo = lbm.Geometry(solid.astype(np.uint8), "D2Q9")
    with pytest.raises(ValueError):
        GF.characteristics(geo, 60.0)
    solid[5, :] = True
    assert GF.solid_normal(solid, 3, 4) == pytest.approx((0.0, -1.0), abs=1e-15)
    assert GF.solid_normal(solid, 3, 5) == pytest.approx((0.0, 1.0), abs=1e-15)


def test_gf_rejects_three_dimensions():
    mask = np.zeros((5, 6, 7), np.uint8)
    mask[:, :2, :] = 1
    geo = lbm.Geometry(mask, "D3Q19")
    p = lbm.Params("D3Q19", CS07, sigma=0.12, rho_l=L07, rho_g=G07, wall="GF", theta_a=60.0)
    with pytest.raises(ValueError):
        lbm.step(lbm.init_state(np.full(mask.shape, G07), geo), geo, p)


def test_flat_wall_drop_takes_the_prescribed_angle():
    """Fig. 8: the geometric formulation makes the interface meet the wall at the prescribed angle
    (the paper reads 58, 88 and 121 degrees for 60, 90 and 120 on a cylinder).  A drop on a flat
    wall after 3000 steps: within 4 degrees of theta_a, in order."""
    shape, thick = (48, 80), 4
    mask = W.flat_wall_mask(shape, thick)
    geo = lbm.Geometry(mask, "D2Q9")
    thetas = []
    for theta_a in (60.0, 90.0, 120.0):
        rho0 = W.tanh_drop_density(shape, (40.0, thick + 4.0), 14.0, L07, G07)
        rho0 = np.where(mask != 0, G07, rho0)
        p = lbm.Params("D2Q9", CS07, sigma=0.12, rho_l=L07, rho_g=G07, wall="GF", theta_a=theta_a)
        f = lbm.run(lbm.init_state(rho0, geo), geo, p, 3000)
        o, rho, u = lbm.observables(f, geo, p)
        th = CA.contact_angle(rho, mask, L07, G07, (40.0, thick + 4.0), wall_y=thick - 0.5)[0]
        assert abs(th - theta_a) < 4.0
        thetas.append(th)
    assert thetas[0] < thetas[1] < thetas[2]
