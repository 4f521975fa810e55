"""Reference gradients of a density loss with respect to the per-wall-node wettability parameter
(oracle; test infrastructure).

The loss is L = sum over fluid nodes of (rho_T(x) - rho_target(x))^2, with rho_T the density of the
post-streaming state after n steps of `oracle.lbm.step` from f0, and the wall parameter kappa_j of
the improved virtual-density scheme (Eq. 16, unified form) given per wall node.  The gradient is
taken by central finite differences of the FP64 oracle, one wall node at a time:
  dL/dkappa_j ~ (L(kappa + h e_j) - L(kappa - h e_j)) / (2 h).
"""
from __future__ import annotations

import numpy as np

from . import lbm


def loss(f0, geo, p, kappa, n_steps, target):
    q = lbm.Params(**{**p.__dict__, "kappa": np.asarray(kappa, dtype=np.float64)})
    f = lbm.run(f0, geo, q, n_steps)
    rho = f.sum(axis=0)
    d = np.where(geo.fluid, rho - target, 0.0)
    return float(np.sum(d * d)), rho


def fd_gradient(f0, geo, p, kappa, n_steps, target, indices, h=1e-6):
    """Central differences of `loss` for the wall nodes listed in `indices` (positions in the
    wall-node order)."""
    kappa = np.asarray(kappa, dtype=np.float64)
    out = []
    for j in indices:
        kp = kappa.copy()
        km = kappa.copy()
        kp[j] += h
        km[j] -= h
        lp, _ = loss(f0, geo, p, kp, n_steps, target)
        lm, _ = loss(f0, geo, p, km, n_steps, target)
        out.append((lp - lm) / (2.0 * h))
    return np.asarray(out)
