"""Contact angle of a drop on a cylinder, sphere or flat wall (oracle; test infrastructure).

The paper reads its angles off density contours (Figs. 4-8, 14) and states no measurement recipe,
so this follows the reading stated in the design notes:
  1. interface points: on every lattice link (+x, +y[, +z]) joining two fluid nodes whose
     densities straddle rho_mid = (rho_l + rho_g)/2, the point at linear interpolation;
     links with an end within 3 nodes (Euclidean) of a solid node are dropped;
     coordinates are unwrapped to the periodic image nearest a hint point;
  2. Kasa algebraic fit of a circle (2D) / sphere (3D) to the points (linear least squares);
  3. the angle through the liquid between the drop surface and a body of radius R_w = R + 1/2
     (the halfway wall): cos(theta) = (R_w^2 + r^2 - d^2) / (2 R_w r), d = |C_drop - C_body|;
     on a flat wall at height y_w: cos(theta) = -(y_c - y_w)/r.
"""
from __future__ import annotations

import itertools

import numpy as np

from .lbm import neighbour


def near_wall(solid: np.ndarray, radius: float = 3.0) -> np.ndarray:
    """Nodes within Euclidean distance `radius` of a solid node (periodic)."""
    d = solid.ndim
    r = int(np.floor(radius))
    out = np.zeros(solid.shape, dtype=bool)
    s = solid.astype(bool)
    for off in itertools.product(range(-r, r + 1), repeat=d):
        if sum(o * o for o in off) <= radius * radius:
            out |= neighbour(s, off)
    return out


def interface_points(rho: np.ndarray, solid: np.ndarray, rho_mid: float, hint, exclude=3.0):
    """Interface points (n, d) in unwrapped lattice coordinates (x, y[, z])."""
    shape = rho.shape
    d = rho.ndim
    fluid = ~solid.astype(bool)
    nw = near_wall(solid, exclude)
    coords = np.indices(shape, dtype=np.float64)[::-1]      # (x, y[, z])
    pts = []
    for axis in range(d):
        e = [0] * d
        e[axis] = 1
        rb = neighbour(rho, e)
        fb = neighbour(fluid, e)
        nb = neighbour(nw, e)
        ok = fluid & fb & ~nw & ~nb & ((rho - rho_mid) * (rb - rho_mid) < 0.0)
        t = (rho_mid - rho[ok]) / (rb[ok] - rho[ok])
        p = np.stack([c[ok] for c in coords], axis=1)
        p[:, axis] += t
        pts.append(p)
    pts = np.concatenate(pts, axis=0)
    sizes = np.array(shape[::-1], dtype=np.float64)
    hint = np.asarray(hint, dtype=np.float64)
    dd = pts - hint
    dd -= sizes * np.round(dd / sizes)
    return hint + dd


def kasa_fit(pts: np.ndarray):
    """Kasa fit: minimise sum (|x|^2 + D.x + F)^2 over (D, F); centre = -D/2, r^2 = |D|^2/4 - F."""
    n, d = pts.shape
    A = np.concatenate([pts, np.ones((n, 1))], axis=1)
    b = -np.sum(pts * pts, axis=1)
    sol, *_ = np.linalg.lstsq(A, b, rcond=None)
    D, F = sol[:d], sol[d]
    c = -D / 2.0
    r = float(np.sqrt(np.dot(c, c) - F))
    return c, r


def angle_on_body(center, r, body_center, body_radius):
    """Contact angle (degrees) of a drop circle/sphere (center, r) on a body of radius R
    (wall at R + 1/2), by the law of cosines in the triangle of the two centres and a contact point."""
    Rw = float(body_radius) + 0.5
    dist = float(np.linalg.norm(np.asarray(center) - np.asarray(body_center)))
    c = (Rw * Rw + r * r - dist * dist) / (2.0 * Rw * r)
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def angle_on_plane(center, r, wall_y):
    c = -(float(center[1]) - wall_y) / r
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def contact_angle(rho, solid, rho_l, rho_g, hint, body_center=None, body_radius=None, wall_y=None):
    pts = interface_points(rho, solid, 0.5 * (rho_l + rho_g), hint)
    c, r = kasa_fit(pts)
    if wall_y is not None:
        return angle_on_plane(c, r, wall_y), c, r, len(pts)
    return angle_on_body(c, r, body_center, body_radius), c, r, len(pts)
