"""Lattice tables of the oracle (test infrastructure; see the package docstring).

D2Q9: velocities, the transformation matrix M of the MRT collision (Eq. 2; the paper defers M,
Lambda and m^eq to its Ref. [34], so the standard Lallemand-Luo D2Q9 basis is used, with the moment
order (rho, e, eps, jx, qx, jy, qy, pxx, pxy) that matches Lambda in Sec. II.A and S in Eq. 7).

D3Q19: the paper defers the 3D model to its Refs. [32,33,39] (Sec. II.A, Sec. IV.C); the standard
d'Humieres D3Q19 basis with moment order
(rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz) is used.

Each row of M is written as the polynomial in the velocity components that defines it.
m^eq = M f^eq (Sec. II.A) with f^eq the second-order polynomial equilibrium, and the Guo source
G (whose moments S = M G are Eq. 7 without the sigma terms) is written in velocity space.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0   # lattice sound speed squared c_s^2 = c^2/3 with c = 1 (Sec. II.A)


class Lattice:
    """A DdQq lattice: velocities E (q, d), equilibrium weights W, force weights WF (Eq. 5), opposite
    index OPP, transformation matrix M (q, q) and its inverse."""

    def __init__(self, name, E, W, WF, M):
        self.name = name
        self.E = np.asarray(E, dtype=np.int64)
        self.q, self.d = self.E.shape
        self.W = np.asarray(W, dtype=np.float64)
        self.WF = np.asarray(WF, dtype=np.float64)
        self.M = np.asarray(M, dtype=np.float64)
        self.Minv = np.linalg.inv(self.M)
        opp = []
        for a in range(self.q):
            matches = [b for b in range(self.q) if np.all(self.E[b] == -self.E[a])]
            assert len(matches) == 1
            opp.append(matches[0])
        self.OPP = np.asarray(opp, dtype=np.int64)

    # f^eq_a = w_a rho [1 + e.u/cs2 + (e.u)^2/(2 cs2^2) - u.u/(2 cs2)]  (second-order polynomial)
    def feq(self, rho, u):
        """Equilibrium distributions, shape (q, *rho.shape). u has shape (d, *rho.shape)."""
        uu = sum(u[i] * u[i] for i in range(self.d))
        out = np.empty((self.q,) + rho.shape)
        for a in range(self.q):
            eu = sum(self.E[a, i] * u[i] for i in range(self.d))
            out[a] = self.W[a] * rho * (1.0 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2))
        return out

    # Guo forcing in velocity space: G_a = w_a [ (e_a - u)/cs2 + (e_a.u) e_a / cs2^2 ] . F
    def guo_source(self, u, F):
        out = np.empty((self.q,) + u.shape[1:])
        for a in range(self.q):
            eu = sum(self.E[a, i] * u[i] for i in range(self.d))
            acc = 0.0
            for i in range(self.d):
                acc = acc + ((self.E[a, i] - u[i]) / CS2 + eu * self.E[a, i] / (CS2 * CS2)) * F[i]
            out[a] = self.W[a] * acc
        return out


def _rows(E, polys):
    return [[p(*e) for e in E] for p in polys]


def _d2q9():
    # e0=(0,0); e1..e4 = (1,0),(0,1),(-1,0),(0,-1); e5..e8 = (1,1),(-1,1),(-1,-1),(1,-1)
    E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    # Eq. 5 weights: 1/3 for |e|^2 = 1, 1/12 for |e|^2 = 2 (w_0 unused)
    WF = [0.0] + [1 / 3] * 4 + [1 / 12] * 4
    n2 = lambda x, y: x * x + y * y
    polys = [
        lambda x, y: 1,                                          # rho
        lambda x, y: -4 + 3 * n2(x, y),                          # e
        lambda x, y: 4 - 21 * n2(x, y) / 2 + 9 * n2(x, y) ** 2 / 2,  # eps
        lambda x, y: x,                                          # jx
        lambda x, y: (-5 + 3 * n2(x, y)) * x,                    # qx
        lambda x, y: y,                                          # jy
        lambda x, y: (-5 + 3 * n2(x, y)) * y,                    # qy
        lambda x, y: x * x - y * y,                              # pxx
        lambda x, y: x * y,                                      # pxy
    ]
    return Lattice("D2Q9", E, W, WF, _rows(E, polys))


def _d3q19():
    E = [(0, 0, 0),
         (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
         (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
         (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
         (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
    W = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
    # force weights: 1/6 for |e|^2 = 1 and 1/12 for |e|^2 = 2, so that sum_a w_a e_ax^2 = 1 as in 2D
    WF = [0.0] + [1 / 6] * 6 + [1 / 12] * 12
    n2 = lambda x, y, z: x * x + y * y + z * z
    polys = [
        lambda x, y, z: 1,                                                   # rho
        lambda x, y, z: 19 * n2(x, y, z) - 30,                               # e
        lambda x, y, z: (21 * n2(x, y, z) ** 2 - 53 * n2(x, y, z) + 24) / 2,  # eps
        lambda x, y, z: x,                                                   # jx
        lambda x, y, z: (5 * n2(x, y, z) - 9) * x,                           # qx
        lambda x, y, z: y,                                                   # jy
        lambda x, y, z: (5 * n2(x, y, z) - 9) * y,                           # qy
        lambda x, y, z: z,                                                   # jz
        lambda x, y, z: (5 * n2(x, y, z) - 9) * z,                           # qz
        lambda x, y, z: 3 * x * x - n2(x, y, z),                             # 3pxx
        lambda x, y, z: (3 * n2(x, y, z) - 5) * (3 * x * x - n2(x, y, z)),   # 3pixx
        lambda x, y, z: y * y - z * z,                                       # pww
        lambda x, y, z: (3 * n2(x, y, z) - 5) * (y * y - z * z),             # piww
        lambda x, y, z: x * y,                                               # pxy
        lambda x, y, z: y * z,                                               # pyz
        lambda x, y, z: x * z,                                               # pxz
        lambda x, y, z: (y * y - z * z) * x,                                 # mx
        lambda x, y, z: (z * z - x * x) * y,                                 # my
        lambda x, y, z: (x * x - y * y) * z,                                 # mz
    ]
    return Lattice("D3Q19", E, W, WF, _rows(E, polys))


D2Q9 = _d2q9()
D3Q19 = _d3q19()


def lattice(name: str) -> Lattice:
    return {"D2Q9": D2Q9, "D3Q19": D3Q19}[name]
