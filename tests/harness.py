"""Test harness: one case description -> identical inputs for the oracle and for the CUDA path.

The oracle side gets oracle.lbm.Params; the CUDA side gets an lbm_config through the binding.
Both receive the same mask, initial density, limiter bounds (from the oracle's Maxwell
construction) and parameters; nothing computed by one side is fed to the other except where a
test explicitly takes a GPU state as the common starting point of one oracle step.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

import workloads as W
from oracle import eos as E, lbm


@dataclasses.dataclass
class Case:
    lattice: str
    shape: tuple
    mask: np.ndarray
    rho0: np.ndarray
    eos_kind: str = "CS"
    t_over_tc: float = 0.7
    sigma: float = 0.12
    kappa: object = 0.0
    wall: str = "IVD"
    rho_w_const: float = 0.2
    Gw: float = 0.0
    theta_a: float = 90.0
    body_force: tuple = (0.0, 0.0, 0.0)
    u0: Optional[np.ndarray] = None
    rates: dict = dataclasses.field(default_factory=dict)
    body: Optional[tuple] = None
    drop_hint: tuple = (0.0, 0.0, 0.0)
    rho_ref: float = 0.0
    step_kernel: str = "auto"

    def oracle_eos(self):
        base = E.cs_config() if self.eos_kind == "CS" else E.pr_paper()
        return base.at_reduced_temperature(self.t_over_tc)

    def bounds(self):
        return E.maxwell(self.oracle_eos())

    def oracle(self):
        g, l = self.bounds()
        p = lbm.Params(self.lattice, self.oracle_eos(), sigma=self.sigma, rho_l=l, rho_g=g, kappa=self.kappa,
                       wall=self.wall, rho_w_const=self.rho_w_const, Gw=self.Gw, theta_a=self.theta_a,
                       body_force=self.body_force, **self.rates)
        geo = lbm.Geometry(self.mask, self.lattice)
        f0 = lbm.init_state(self.rho0, geo, self.u0)
        return geo, p, f0

    def gpu(self, precision="fp64", stream=None):
        from paper_1908_04443_gb300 import lbmwet as L
        oe = self.oracle_eos()
        e = L.make_eos(self.eos_kind, oe.a, oe.b, oe.R, oe.T, oe.omega)
        g, l = self.bounds()
        kappa_scalar = float(self.kappa) if np.ndim(self.kappa) == 0 else 0.0
        cfg = L.make_config(self.lattice, precision, self.shape, e, sigma=self.sigma, rho_l=l, rho_g=g,
                            kappa=kappa_scalar, wall=self.wall, rho_w_const=self.rho_w_const, Gw=self.Gw,
                            theta_a=self.theta_a,
                            body_force=self.body_force, body=self.body, drop_hint=self.drop_hint,
                            rho_ref=self.rho_ref, step_kernel=self.step_kernel, **self.rates)
        kpw = None if np.ndim(self.kappa) == 0 else np.asarray(self.kappa, dtype=np.float64)
        u0 = None if self.u0 is None else self.u0.reshape(-1)
        return L.Simulation(cfg, self.mask, self.rho0, u0, kpw, stream)


def c1_case(noise=True) -> Case:
    wl = W.c1_parity_cylinder()
    if not noise:
        wl.noise = 0.0
    eos = E.cs_config().at_reduced_temperature(wl.t_over_tc)
    g, l = E.maxwell(eos)
    return Case("D2Q9", wl.shape, wl.mask(), wl.rho0(l, g), kappa=wl.kappa,
                body=("ball", wl.body_center, wl.body_radius), drop_hint=wl.drop_center)


def drop_on_cylinder(shape, center, R, dcenter, r, kappa=0.1, eos_kind="CS", t_over_tc=0.7, seed=1234,
                     lattice="D2Q9", **kw) -> Case:
    base = E.cs_config() if eos_kind == "CS" else E.pr_paper()
    eos = base.at_reduced_temperature(t_over_tc)
    g, l = E.maxwell(eos)
    mask = W.ball_mask(shape, center, R)
    rho = W.tanh_drop_density(shape, dcenter, r, l, g) + W.density_noise(shape, 1e-6, seed)
    rho = np.where(mask != 0, g, rho)
    return Case(lattice, shape, mask, rho, eos_kind=eos_kind, t_over_tc=t_over_tc, kappa=kappa,
                body=("ball", center, R), drop_hint=dcenter, **kw)
