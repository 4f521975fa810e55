"""Curved geometric-formulation contact-angle scheme, 2D (Sec. III.A, Eqs. 10-15) (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain float64 numpy and Python loops over the
wall nodes.

For a wall node P (a solid node with a fluid neighbour in the Eq. 5 stencil):
  1. the unit normal of the solid surface, Eq. 13, with the eighth-order isotropic weights of
     Eq. 14 over the 24 neighbours with |e|^2 in {1, 2, 4, 5, 8}, and the switch s = 1 on solid
     nodes (as in Eq. 8): n_s = -sum w s(P + e) e / |sum w s(P + e) e|;
  2. the two characteristic directions, Eq. 15: n_s rotated by +theta' and by -theta',
     theta' = pi/2 - theta_a;
  3. along each direction, the first point D where the line from P crosses a mesh line: the edge
     of the square of side 2 centred on P (readings below);
  4. the density at D by linear interpolation between the two lattice nodes of that mesh line on
     either side of D (the paper allows linear interpolation in place of the quadratic one);
  5. Eq. 11: rho_P = max(rho_D1, rho_D2) for theta_a <= 90 degrees, min(...) otherwise.

Readings (the paper defers the intersection cases to a reference that is not available):
  * D is the first crossing of the characteristic with a mesh line x = P_x +- 1 or y = P_y +- 1,
    i.e. with the boundary of the square [P_x - 1, P_x + 1] x [P_y - 1, P_y + 1]; its nodes are
    therefore neighbours of P in the D2Q9 stencil, like the nodes of Eq. 17.
  * A crossing within 1e-12 of a lattice node is taken at that node.
  * Only fluid nodes carry a density: when one of the two nodes of D's mesh segment is solid, rho_D
    is the other node's density; when both are solid, D is dropped from Eq. 11.  With both D
    dropped, rho_P is the mean of Eq. 17 over the fluid neighbours (phi = 1).
  * A wall node whose sum in Eq. 13 vanishes has no normal; the scheme is then undefined there and
    `characteristics` raises.  Every Eq. 14 weight is a multiple of 1/5040, so a nonzero component
    of the sum is at least 1/5040: a sum below 1e-9 (rounding of cancelling terms) counts as zero.
  * The densities are those of the same step (after streaming, before collision), as for Eq. 17.
"""
from __future__ import annotations

import math

import numpy as np

# Eq. 14: weights of the eighth-order isotropic discretisation, by |e|^2
EQ14_WEIGHTS = {1: 4.0 / 21.0, 2: 4.0 / 45.0, 4: 1.0 / 60.0, 5: 2.0 / 315.0, 8: 1.0 / 5040.0}

SNAP = 1e-12
NO_NORMAL = 1e-9


def eq14_stencil():
    """The 24 vectors e with |e|^2 in Eq. 14 and their weights, ex outer, ey inner, from -2 to 2."""
    out = []
    for ex in range(-2, 3):
        for ey in range(-2, 3):
            e2 = ex * ex + ey * ey
            if e2 in EQ14_WEIGHTS:
                out.append((ex, ey, EQ14_WEIGHTS[e2]))
    return out


def solid_normal(solid: np.ndarray, x: int, y: int):
    """Eq. 13 at node (x, y) of a periodic 2D solid mask (numpy shape (ny, nx)); None if the sum
    vanishes."""
    ny, nx = solid.shape
    gx = 0.0
    gy = 0.0
    for ex, ey, w in eq14_stencil():
        s = 1.0 if solid[(y + ey) % ny, (x + ex) % nx] else 0.0
        gx += w * s * ex
        gy += w * s * ey
    norm = math.hypot(gx, gy)
    if norm < NO_NORMAL:
        return None
    return -gx / norm, -gy / norm


def rotate(n, angle):
    """n rotated counter-clockwise by `angle` (the first line of Eq. 15 for +theta')."""
    c, s = math.cos(angle), math.sin(angle)
    return n[0] * c - n[1] * s, n[0] * s + n[1] * c


def mesh_crossing(d):
    """The point where the ray from the origin along the unit vector d leaves the square
    [-1, 1]^2, and the two lattice nodes of the mesh segment it lies on with their linear weights:
    [((dx, dy), w), ...] (one entry when the crossing is at a node)."""
    ax, ay = abs(d[0]), abs(d[1])
    if ax >= ay:
        # crosses the vertical mesh line x = sign(d_x) at y = d_y / |d_x|
        X = 1 if d[0] > 0 else -1
        yc = d[1] / ax
        y0 = math.floor(yc)
        lam = yc - y0
        ends = [((X, y0), 1.0 - lam), ((X, y0 + 1), lam)]
    else:
        Y = 1 if d[1] > 0 else -1
        xc = d[0] / ay
        x0 = math.floor(xc)
        lam = xc - x0
        ends = [((x0, Y), 1.0 - lam), ((x0 + 1, Y), lam)]
    out = []
    for node, w in ends:
        if w > 1.0 - SNAP:
            return [(node, 1.0)]
        if w >= SNAP:
            out.append((node, w))
    return out


def characteristics(geo, theta_a_deg: float):
    """For every wall node (in wall-node order): a list of the usable crossings D, each a list of
    (flat neighbour index, weight) over fluid nodes with weights summing to 1."""
    solid = geo.solid
    ny, nx = solid.shape
    tp = math.pi / 2.0 - math.radians(theta_a_deg)
    table = []
    for g in geo.wall_flat:
        y, x = divmod(int(g), nx)
        n = solid_normal(solid, x, y)
        if n is None:
            raise ValueError(f"wall node ({x}, {y}) has no normal (Eq. 13 sums to zero)")
        ds = []
        for d in (rotate(n, tp), rotate(n, -tp)):       # n_1 and n_2 of Eq. 15
            pts = []
            for (ex, ey), w in mesh_crossing(d):
                xx, yy = (x + ex) % nx, (y + ey) % ny
                if not solid[yy, xx]:
                    pts.append((yy * nx + xx, w))
            if pts:
                tot = sum(w for _, w in pts)
                ds.append([(i, w / tot) for i, w in pts])
        table.append(ds)
    return table


def wall_density(rho: np.ndarray, geo, theta_a_deg: float, rho_ave: np.ndarray) -> np.ndarray:
    """Eq. 11 at every wall node (wall-node order), from the same-step density field and the
    Eq. 17 mean rho_ave (used where no crossing is usable)."""
    key = ("gf", float(theta_a_deg))
    cache = geo.__dict__.setdefault("_gf_cache", {})
    if key not in cache:
        cache[key] = characteristics(geo, theta_a_deg)
    table = cache[key]
    flat = rho.reshape(-1)
    out = np.empty(len(table))
    for k, ds in enumerate(table):
        if not ds:
            out[k] = rho_ave[k]
            continue
        vals = [sum(w * flat[i] for i, w in pts) for pts in ds]
        out[k] = max(vals) if theta_a_deg <= 90.0 else min(vals)
    return out
