"""Pins of the oracle's contact-angle measurement: the Kasa fit on exact points, the angle formula
against an independent construction from the two circles' intersection, and interface extraction
on a synthetic tanh drop (with periodic unwrapping)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import contact_angle as CA


@pytest.mark.parametrize("d", [2, 3])
def test_kasa_exact_points(d):
    rng = np.random.default_rng(1)
    c = rng.uniform(-5, 5, d)
    r = 7.25
    v = rng.normal(size=(200, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pts = c + r * v
    cf, rf = CA.kasa_fit(pts)
    assert np.allclose(cf, c, atol=1e-10)
    assert abs(rf - r) < 1e-10


@pytest.mark.parametrize("theta", [20.0, 60.0, 90.0, 125.0, 160.0])
def test_angle_on_body_against_intersection(theta):
    """Build a drop circle meeting a body circle (wall radius R + 1/2) at angle theta, locate an
    intersection point P by solving the two circle equations, and measure the angle between the
    outward normals there (0 for a wetting film, 180 for a touching ball)."""
    R = 20.0
    Rw = R + 0.5
    r = 13.0
    # place the drop centre on the +y axis at a distance chosen by the angle between normals
    t = math.radians(theta)
    dist = math.sqrt(Rw * Rw + r * r - 2 * Rw * r * math.cos(t))
    Cb = np.array([3.0, -2.0])
    Cd = Cb + np.array([0.0, dist])
    # circle intersection: P = Cb + a e_y + h e_x
    a = (Rw * Rw - r * r + dist * dist) / (2 * dist)
    h = math.sqrt(Rw * Rw - a * a)
    P = Cb + np.array([h, a])
    nb = (P - Cb) / Rw
    nd = (P - Cd) / r
    assert abs(np.linalg.norm(P - Cd) - r) < 1e-12
    ref = math.degrees(math.acos(float(np.clip(nb @ nd, -1, 1))))
    assert abs(CA.angle_on_body(Cd, r, Cb, R) - ref) < 1e-9
    assert abs(ref - theta) < 1e-9


def test_angle_on_plane():
    # centre at the wall: 90; centre r/2 above: 120; centre r/2 below: 60
    assert abs(CA.angle_on_plane((0, 10.0), 4.0, 10.0) - 90) < 1e-12
    assert abs(CA.angle_on_plane((0, 12.0), 4.0, 10.0) - 120) < 1e-12
    assert abs(CA.angle_on_plane((0, 8.0), 4.0, 10.0) - 60) < 1e-12


def test_interface_extraction_tanh_drop_periodic():
    """The mid-density contour of a tanh drop is the circle |x - c| = r; the drop straddles the
    periodic boundary, so the points must be unwrapped around the hint."""
    shape = (60, 70)
    c = (35.3, 55.6)
    r = 14.2
    rho = W.tanh_drop_density(shape, c, r, 0.4, 0.01, width=3.0)
    solid = np.zeros(shape, np.uint8)
    pts = CA.interface_points(rho, solid, 0.5 * (0.4 + 0.01), hint=(35.0, 55.0))
    assert len(pts) > 100
    cf, rf = CA.kasa_fit(pts)
    assert np.allclose(cf, c, atol=0.02)
    assert abs(rf - r) < 0.05


def test_interface_extraction_skips_near_wall():
    shape = (40, 40)
    rho = W.tanh_drop_density(shape, (20, 20), 8.0, 0.4, 0.01)
    solid = np.zeros(shape, np.uint8)
    solid[:, :3] = 1
    pts_all = CA.interface_points(rho, np.zeros(shape, np.uint8), 0.205, (20, 20))
    pts = CA.interface_points(rho, solid, 0.205, (20, 20))
    assert len(pts) == len(pts_all)         # the drop is far from the wall: nothing dropped
    solid2 = np.zeros(shape, np.uint8)
    solid2[:, :10] = 1                       # wall within 3 nodes of the drop's left side
    pts2 = CA.interface_points(rho, solid2, 0.205, (20, 20))
    assert len(pts2) < len(pts_all)
    assert np.all(pts2[:, 0] > 12.0)
