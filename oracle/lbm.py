"""One time step of the pseudopotential MRT-LB method with contact-angle walls (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain float64 numpy, vectorised over nodes.

State: the post-streaming distributions f(x, t) at fluid nodes, shape (q, *shape) with numpy shape
(ny, nx) or (nz, ny, nx) (x fastest).  Entries at solid nodes are kept at zero and never used.

A step, in the paper's order:
  1. rho = sum_a f_a                                                    (Eq. 4)
  2. at wall nodes (solid nodes with a fluid neighbour in the Eq. 5 stencil) the virtual density:
     IVD  rho_w = phi rho_ave (phi >= 1) or rho_ave - drho (drho >= 0),
          rho_ave = sum_a w_a rho(x+e_a) s_w(x+e_a) / sum_a w_a s_w(x+e_a),   (Eqs. 16-17)
          limited to rho_g <= rho_w <= rho_l                             (Sec. III.B)
     VD   rho_w = constant (Sec. II.B)
     GF   (2D) rho_w = max or min of the densities where the two characteristic lines of the
          prescribed angle theta_a cross the mesh (Eqs. 10-15; `oracle.geometric`)
  3. psi from Eq. 6 at fluid nodes (rho) and at wall nodes (rho_w)
  4. F_m = -G psi(x) sum_a w_a psi(x + e_a) e_a at fluid nodes (Eq. 5);  F = F_m + F_body
     (SF scheme: F_ads = -G_w rho(x) sum_a w_a s(x + e_a) e_a is added, Eq. 8, with psi = 0 on solids)
  5. rho u = sum_a e_a f_a + F/2                                         (Eq. 4)
  6. m = M f,  m^eq = M f^eq,  S (Eq. 7),  m* = m - Lambda (m - m^eq) + (I - Lambda/2) S (Eq. 2),
     f* = M^-1 m*
  7. streaming f_a(x + e_a, t+1) = f*_a(x, t) (Eq. 3) with halfway bounce-back on links that end in
     a solid node (Fig. 3): such a population returns to x as f_abar(x, t+1) = f*_a(x, t).

The unified wettability parameter kappa (scalar or one value per wall node) stands for both IVD
branches: kappa >= 0 means phi = 1 + kappa, kappa < 0 means drho = -kappa (continuous at 0).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from . import geometric
from .eos import EOS, CS2
from .lattice import Lattice, lattice as get_lattice


@dataclasses.dataclass
class Params:
    lattice: str
    eos: EOS
    G: float = -1.0
    sigma: float = 0.0
    # MRT rates s = 1/tau; D3Q19 also uses s_pi (3pixx, piww) and s_m (mx, my, mz)
    s_rho: float = 1.0
    s_e: float = 0.8
    s_eps: float = 0.8
    s_j: float = 1.0
    s_q: float = 1.1
    s_nu: float = 1.0 / 0.95
    s_pi: float = 1.1
    s_m: float = 1.1
    rho_l: float = 1.0        # limiter bounds of Sec. III.B
    rho_g: float = 0.1
    body_force: tuple = (0.0, 0.0, 0.0)
    wall: str = "IVD"          # "IVD", "VD", "SF" or "GF"
    kappa: object = 0.0        # IVD: scalar or array (one per wall node, in wall-node order)
    rho_w_const: float = 1.0   # VD
    Gw: float = 0.0            # SF
    theta_a: float = 90.0      # GF: prescribed contact angle (degrees)

    @property
    def lat(self) -> Lattice:
        return get_lattice(self.lattice)

    def rates(self) -> np.ndarray:
        """Diagonal of Lambda in the moment order of `lattice`."""
        if self.lattice == "D2Q9":
            # Lambda = diag(1/tau_rho, 1/tau_e, 1/tau_eps, 1/tau_j, 1/tau_q, 1/tau_j, 1/tau_q, 1/tau_nu, 1/tau_nu)
            return np.array([self.s_rho, self.s_e, self.s_eps, self.s_j, self.s_q, self.s_j, self.s_q,
                             self.s_nu, self.s_nu])
        return np.array([self.s_rho, self.s_e, self.s_eps,
                         self.s_j, self.s_q, self.s_j, self.s_q, self.s_j, self.s_q,
                         self.s_nu, self.s_pi, self.s_nu, self.s_pi,
                         self.s_nu, self.s_nu, self.s_nu,
                         self.s_m, self.s_m, self.s_m])


def neighbour(a: np.ndarray, e) -> np.ndarray:
    """a(x + e) on the periodic lattice (e given as (ex, ey[, ez]); arrays are x-fastest)."""
    axes = tuple(range(a.ndim - 1, -1, -1))[: len(e)]   # x is the last numpy axis
    return np.roll(a, shift=tuple(-int(c) for c in e), axis=axes)


class Geometry:
    """Solid mask s(x) (1 solid, 0 fluid), fluid mask s_w = 1 - s (Eq. 17), and the wall nodes:
    solid nodes with at least one fluid neighbour in the Eq. 5 stencil, ordered by linear index."""

    def __init__(self, solid_mask: np.ndarray, lattice_name: str):
        lat = get_lattice(lattice_name)
        self.lat = lat
        self.shape = solid_mask.shape
        self.solid = solid_mask.astype(bool)
        self.fluid = ~self.solid
        touch = np.zeros(self.shape, dtype=bool)
        for a in range(1, lat.q):
            touch |= neighbour(self.fluid, lat.E[a])
        self.wall = self.solid & touch
        self.wall_flat = np.flatnonzero(self.wall.ravel())   # wall-node order = ascending linear index


def ivd_virtual_density(rho_ave, kappa, rho_g, rho_l):
    """Eq. 16 with the limiter of Sec. III.B, in the unified kappa form:
    kappa >= 0: rho_w = (1 + kappa) rho_ave  (phi = 1 + kappa >= 1, decreases theta)
    kappa <  0: rho_w = rho_ave - (-kappa)   (drho = -kappa > 0, increases theta)
    then rho_g <= rho_w <= rho_l."""
    rho_ave = np.asarray(rho_ave, dtype=np.float64)
    kappa = np.broadcast_to(np.asarray(kappa, dtype=np.float64), rho_ave.shape)
    rw = np.where(kappa >= 0.0, (1.0 + kappa) * rho_ave, rho_ave + kappa)
    rw = np.where(rw > rho_l, rho_l, rw)
    rw = np.where(rw < rho_g, rho_g, rw)
    return rw


def psi_of(eos: EOS, rho, G):
    """Eq. 6; a non-positive square-root argument is an error of the model state."""
    arg = 2.0 * (eos.pressure(rho) - rho * CS2) / G
    if np.any(~(arg > 0.0)):
        raise FloatingPointError("psi: non-positive square-root argument in Eq. 6")
    return np.sqrt(arg)


def wall_density(rho, geo: Geometry, p: Params):
    """Virtual density at the wall nodes (array over the grid, meaningful only at wall nodes)."""
    lat = geo.lat
    rw = np.zeros(geo.shape)
    if p.wall == "VD":
        rw[geo.wall] = p.rho_w_const
        return rw
    num = np.zeros(geo.shape)
    den = np.zeros(geo.shape)
    sw = geo.fluid.astype(np.float64)
    rho_f = np.where(geo.fluid, rho, 0.0)
    for a in range(1, lat.q):
        num += lat.WF[a] * neighbour(rho_f, lat.E[a]) * neighbour(sw, lat.E[a])
        den += lat.WF[a] * neighbour(sw, lat.E[a])
    rho_ave = num[geo.wall] / den[geo.wall]
    if p.wall == "GF":
        if lat.d != 2:
            raise ValueError("the geometric-formulation scheme is two-dimensional (Sec. III.A)")
        rw[geo.wall] = geometric.wall_density(rho_f, geo, p.theta_a, rho_ave)
        return rw
    kappa = p.kappa
    if np.ndim(kappa) > 0:
        kappa = np.asarray(kappa, dtype=np.float64)
        assert kappa.shape == (len(geo.wall_flat),)
        # geo.wall is iterated in C order by boolean indexing = ascending linear index
    rw[geo.wall] = ivd_virtual_density(rho_ave, kappa, p.rho_g, p.rho_l)
    return rw


def macroscopic(f, geo: Geometry, p: Params):
    """rho, psi field, F_m, F and u at the current post-streaming state (steps 1-5)."""
    lat = geo.lat
    rho = f.sum(axis=0)
    rho = np.where(geo.fluid, rho, 0.0)
    if p.wall == "SF":
        psi = np.zeros(geo.shape)
        psi[geo.fluid] = psi_of(p.eos, rho[geo.fluid], p.G)
    else:
        rw = wall_density(rho, geo, p)
        psi = np.zeros(geo.shape)
        psi[geo.fluid] = psi_of(p.eos, rho[geo.fluid], p.G)
        psi[geo.wall] = psi_of(p.eos, rw[geo.wall], p.G)
    Fm = np.zeros((lat.d,) + geo.shape)
    for a in range(1, lat.q):
        pn = neighbour(psi, lat.E[a])
        for i in range(lat.d):
            Fm[i] += lat.WF[a] * pn * lat.E[a, i]
    Fm = -p.G * psi * Fm
    F = Fm.copy()
    if p.wall == "SF":
        s = geo.solid.astype(np.float64)
        Fads = np.zeros_like(F)
        for a in range(1, lat.q):
            sn = neighbour(s, lat.E[a])
            for i in range(lat.d):
                Fads[i] += lat.WF[a] * sn * lat.E[a, i]
        F = F + (-p.Gw * rho) * Fads
    for i in range(lat.d):
        F[i] = F[i] + p.body_force[i]
    F = np.where(geo.fluid, F, 0.0)
    Fm = np.where(geo.fluid, Fm, 0.0)
    mom = np.zeros((lat.d,) + geo.shape)
    for a in range(lat.q):
        for i in range(lat.d):
            if lat.E[a, i] != 0:
                mom[i] += lat.E[a, i] * f[a]
    safe = np.where(geo.fluid, rho, 1.0)
    u = np.where(geo.fluid, (mom + 0.5 * F) / safe, 0.0)
    return rho, psi, Fm, F, u


def source_moments(p: Params, u, F, Fm, psi):
    """S in moment space.  D2Q9: Eq. 7 as printed (reading its tau_varsigma as tau_eps).
    D3Q19: S = M G (Guo source) plus the consistency terms on e and eps, scaled so that the
    isotropic pressure-tensor correction per dimension equals the one of Eq. 7 in 2D."""
    lat = p.lat
    tau_e, tau_eps = 1.0 / p.s_e, 1.0 / p.s_eps
    fm2 = sum(Fm[i] * Fm[i] for i in range(lat.d))
    psi_safe = np.where(psi > 0, psi, 1.0)
    X = p.sigma * fm2 / (psi_safe ** 2)
    uF = sum(u[i] * F[i] for i in range(lat.d))
    if p.lattice == "D2Q9":
        ux, uy = u
        Fx, Fy = F
        S = np.stack([
            np.zeros_like(ux),
            6.0 * uF + 12.0 * X / (tau_e - 0.5),
            -6.0 * uF - 12.0 * X / (tau_eps - 0.5),
            Fx,
            -Fx,
            Fy,
            -Fy,
            2.0 * (ux * Fx - uy * Fy),
            ux * Fy + uy * Fx,
        ])
        return S
    G = lat.guo_source(u, F)
    S = np.einsum("ab,b...->a...", lat.M, G)
    S[1] = S[1] + 114.0 * X / (tau_e - 0.5)
    S[2] = S[2] - 33.0 * X / (tau_eps - 0.5)
    return S


def collide(f, geo: Geometry, p: Params):
    """Steps 1-6: returns f* (post-collision, before streaming) and the macroscopic fields."""
    lat = geo.lat
    rho, psi, Fm, F, u = macroscopic(f, geo, p)
    q = lat.q
    shape = geo.shape
    m = (lat.M @ f.reshape(q, -1)).reshape((q,) + shape)
    rho_s = np.where(geo.fluid, rho, 1.0)
    meq = (lat.M @ lat.feq(rho_s, u).reshape(q, -1)).reshape((q,) + shape)
    S = source_moments(p, u, F, Fm, psi)
    lam = p.rates().reshape((q,) + (1,) * len(shape))
    mstar = m - lam * (m - meq) + (1.0 - lam / 2.0) * S
    fstar = (lat.Minv @ mstar.reshape(q, -1)).reshape((q,) + shape)
    fstar = np.where(geo.fluid[None], fstar, 0.0)
    return fstar, (rho, psi, Fm, F, u)


def stream(fstar, geo: Geometry):
    """Step 7: f_a(x + e_a) = f*_a(x) (Eq. 3) with halfway bounce-back: a population whose target
    x + e_a is solid comes back to x in the opposite direction (Fig. 3).  Written as its pull form
    f_a(x) = f*_a(x - e_a) if x - e_a is fluid, else f*_abar(x)."""
    lat = geo.lat
    fnew = np.zeros_like(fstar)
    for a in range(lat.q):
        src_fluid = neighbour(geo.fluid, -lat.E[a])
        pulled = neighbour(fstar[a], -lat.E[a])
        bounced = fstar[lat.OPP[a]]
        fnew[a] = np.where(src_fluid, pulled, bounced)
    fnew = np.where(geo.fluid[None], fnew, 0.0)
    return fnew


def step(f, geo: Geometry, p: Params):
    fstar, _ = collide(f, geo, p)
    return stream(fstar, geo)


def init_state(rho0, geo: Geometry, u0=None):
    """f = f^eq(rho0, u0) at fluid nodes (u0 = 0 if not given)."""
    lat = geo.lat
    if u0 is None:
        u0 = np.zeros((lat.d,) + geo.shape)
    rho_s = np.where(geo.fluid, rho0, 1.0)
    f = lat.feq(rho_s, u0)
    return np.where(geo.fluid[None], f, 0.0)


def run(f, geo: Geometry, p: Params, n: int):
    for _ in range(n):
        f = step(f, geo, p)
    return f


@dataclasses.dataclass
class Observables:
    mass: float
    rho_max: float
    rho_min: float
    u_max: float


def observables(f, geo: Geometry, p: Params):
    """Total fluid mass, fluid density extremes (Fig. 11) and the maximum spurious current |u|
    (Fig. 10) of the state f; returns (Observables, rho, u)."""
    rho, psi, Fm, F, u = macroscopic(f, geo, p)
    umag = np.sqrt(sum(u[i] ** 2 for i in range(geo.lat.d)))
    o = Observables(mass=float(rho[geo.fluid].sum()),
                    rho_max=float(rho[geo.fluid].max()),
                    rho_min=float(rho[geo.fluid].min()),
                    u_max=float(umag[geo.fluid].max()))
    return o, rho, u
