"""The FP32 density tolerance, applied per node where it is a statement about storage precision.

Deviation storage is held to 1e-4 relative in density.  In the bulk phases, away from the liquid-gas
interface and from walls, that bound is applied node by node: |rho_fp32 - rho_ref| <= 1e-4 rho_ref.
Inside the interface band (within `band` nodes, Euclidean, of the rho_mid = (rho_l + rho_g)/2
contour of the reference field, or of a solid node) the density changes by rho_l - rho_g over about
four nodes, so rounding that shifts the interface by a tiny fraction of a node changes the density
there by a large fraction of rho_l: that band is held to 1e-4 rho_l instead.  Both maxima are
returned (and printed by the tests) so that a run reports what it reached in each region.
"""
from __future__ import annotations

import itertools

import numpy as np


def _dilate(mask: np.ndarray, radius: float) -> np.ndarray:
    """Nodes within Euclidean distance `radius` of a node of `mask` (periodic)."""
    r = int(np.floor(radius))
    out = np.zeros(mask.shape, dtype=bool)
    axes = tuple(range(mask.ndim))
    for off in itertools.product(range(-r, r + 1), repeat=mask.ndim):
        if sum(o * o for o in off) <= radius * radius:
            out |= np.roll(mask, off, axis=axes)
    return out


def interface_band(rho_ref: np.ndarray, solid: np.ndarray, rho_l: float, rho_g: float, band: float = 3.0):
    """Boolean mask of fluid nodes within `band` of the rho_mid contour or of a solid node."""
    solid = solid.astype(bool)
    fluid = ~solid
    mid = 0.5 * (rho_l + rho_g)
    side = np.where(fluid, rho_ref > mid, False)
    cross = np.zeros(rho_ref.shape, dtype=bool)
    for ax in range(rho_ref.ndim):
        nb_side = np.roll(side, -1, axis=ax)
        nb_fluid = np.roll(fluid, -1, axis=ax)
        link = fluid & nb_fluid & (side != nb_side)
        cross |= link | np.roll(link, 1, axis=ax)
    return fluid & (_dilate(cross, band) | _dilate(solid, band))


def split_errors(rho: np.ndarray, rho_ref: np.ndarray, solid: np.ndarray, rho_l: float, rho_g: float,
                 band: float = 3.0):
    """(max relative error over bulk fluid nodes, max |error| / rho_l over the interface band,
    number of bulk nodes, number of band nodes)."""
    fluid = ~solid.astype(bool)
    b = interface_band(rho_ref, solid, rho_l, rho_g, band)
    bulk = fluid & ~b
    d = np.abs(rho - rho_ref)
    rel_bulk = float(np.max(d[bulk] / np.abs(rho_ref[bulk]))) if bulk.any() else 0.0
    band_l = float(np.max(d[b]) / rho_l) if b.any() else 0.0
    return rel_bulk, band_l, int(bulk.sum()), int(b.sum())
