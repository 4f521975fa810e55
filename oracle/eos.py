"""Equations of state, pseudopotential and coexistence densities (oracle; test infrastructure).

* Peng-Robinson, Eq. 18 (Sec. IV.A):
    p = rho R T/(1 - b rho) - a phi(T) rho^2/(1 + 2 b rho - b^2 rho^2),
    phi(T) = [1 + (0.37464 + 1.54226 w - 0.26992 w^2)(1 - sqrt(T/Tc))]^2,
    a = 0.45724 R^2 Tc^2/pc, b = 0.0778 R Tc/pc, so Tc = 0.0778 a / (0.45724 b R).
* Carnahan-Starling (the equation of state of the benchmark configurations; the paper cites its
  Ref. [35] for alternative equations of state):
    p = rho R T (1 + eta + eta^2 - eta^3)/(1 - eta)^3 - a rho^2,  eta = b rho / 4.
* Pseudopotential, Eq. 6:  psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2)), with c = 1, c_s^2 = 1/3.
* Coexistence densities by the Maxwell equal-area rule on the p-v plane (v = 1/rho), which the
  paper uses as the target of thermodynamic consistency (Sec. II.A; rho_g ~ 0.38, rho_l ~ 6.5
  for PR at 0.86 Tc, Sec. IV.A).  Solved with scipy root brackets and adaptive quadrature.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import integrate, optimize

CS2 = 1.0 / 3.0


@dataclasses.dataclass
class EOS:
    kind: str            # "PR" or "CS"
    a: float
    b: float
    R: float = 1.0
    T: float = 0.0       # absolute temperature (set from T/Tc with `at_reduced_temperature`)
    omega: float = 0.344  # PR acentric factor (Sec. IV.A)

    def tc(self) -> float:
        """Critical temperature: PR from its definitions of a and b (Eq. 18); C-S from the
        numerical critical point (dp/drho = d2p/drho2 = 0)."""
        if self.kind == "PR":
            return 0.0778 * self.a / (0.45724 * self.b * self.R)
        return critical_point(self)[0]

    def at_reduced_temperature(self, t_over_tc: float) -> "EOS":
        return dataclasses.replace(self, T=t_over_tc * self.tc())

    def pressure(self, rho, T=None):
        T = self.T if T is None else T
        rho = np.asarray(rho, dtype=np.float64)
        if self.kind == "PR":
            tc = self.tc()
            kappa = 0.37464 + 1.54226 * self.omega - 0.26992 * self.omega ** 2
            phi_t = (1.0 + kappa * (1.0 - math.sqrt(T / tc))) ** 2
            return (rho * self.R * T / (1.0 - self.b * rho)
                    - self.a * phi_t * rho ** 2 / (1.0 + 2.0 * self.b * rho - self.b ** 2 * rho ** 2))
        eta = self.b * rho / 4.0
        return (rho * self.R * T * (1.0 + eta + eta ** 2 - eta ** 3) / (1.0 - eta) ** 3
                - self.a * rho ** 2)


def pr_paper() -> EOS:
    """Peng-Robinson constants a = 2/49, b = 2/21, R = 1 (the paper prints only the formulas)."""
    return EOS("PR", a=2.0 / 49.0, b=2.0 / 21.0, R=1.0)


def cs_config() -> EOS:
    """Carnahan-Starling constants a = 0.25, b = 4, R = 1 of the benchmark configurations."""
    return EOS("CS", a=0.25, b=4.0, R=1.0)


def psi_squared_arg(eos: EOS, rho, G=-1.0):
    """The argument of the square root in Eq. 6: 2 (p_EOS - rho c_s^2) / (G c^2)."""
    return 2.0 * (eos.pressure(rho) - np.asarray(rho) * CS2) / G


def psi(eos: EOS, rho, G=-1.0):
    """Eq. 6.  Raises if the square-root argument is not positive (the model then has no psi)."""
    arg = psi_squared_arg(eos, rho, G)
    if np.any(~(arg > 0.0)):
        raise FloatingPointError("psi: non-positive square-root argument in Eq. 6")
    return np.sqrt(arg)


def _dp(eos, rho, T, h=1e-6):
    return (eos.pressure(rho + h, T) - eos.pressure(rho - h, T)) / (2 * h)


def _max_density(eos) -> float:
    # PR: 1 - b rho > 0; C-S: eta < 1.
    return (1.0 / eos.b) if eos.kind == "PR" else (4.0 / eos.b)


def critical_point(eos: EOS):
    """(Tc, rho_c) where dp/drho and d2p/drho2 vanish, found numerically."""
    rmax = _max_density(eos)

    def dp(rho, T):
        return float(_dp(eos, rho, T))

    def min_dp(T):
        res = optimize.minimize_scalar(lambda r: dp(r, T), bounds=(1e-6 * rmax, 0.9 * rmax),
                                       method="bounded", options={"xatol": 1e-14})
        return res.fun, res.x

    # dp/drho minimum over rho is zero at the critical temperature
    lo, hi = 1e-8, 1.0
    while min_dp(hi)[0] < 0:
        hi *= 2
    tc = optimize.brentq(lambda T: min_dp(T)[0], lo, hi, xtol=1e-15, rtol=1e-14)
    return tc, min_dp(tc)[1]


def spinodals(eos: EOS):
    """The two densities where dp/drho = 0 at the EOS temperature (below Tc)."""
    rmax = _max_density(eos)
    T = eos.T
    res = optimize.minimize_scalar(lambda r: float(_dp(eos, r, T)), bounds=(1e-6 * rmax, 0.9 * rmax),
                                   method="bounded", options={"xatol": 1e-14})
    rm = res.x
    if res.fun >= 0:
        raise ValueError("temperature is not below the critical temperature")
    f = lambda r: float(_dp(eos, r, T))
    lo = 1e-9
    r1 = optimize.brentq(f, lo, rm, xtol=1e-15)
    hi = rm
    while f(hi) < 0:
        hi = hi + 0.5 * (0.999 * rmax - hi)
    r2 = optimize.brentq(f, rm, hi, xtol=1e-15)
    return r1, r2


def maxwell(eos: EOS):
    """Coexistence densities (rho_g, rho_l) by the equal-area rule:
    p(rho_g) = p(rho_l) = p*, and  integral_{v_l}^{v_g} p dv = p* (v_g - v_l),  v = 1/rho."""
    r1, r2 = spinodals(eos)
    p = lambda r: float(eos.pressure(r))
    pmin, pmax = p(r2), p(r1)       # local min (liquid spinodal) and local max (gas spinodal)
    rmax = _max_density(eos)

    def roots(ps):
        lo_r = 1e-3 * ps / (eos.R * eos.T)   # p ~ rho R T at low density, so p(lo_r) < ps
        rg = optimize.brentq(lambda r: p(r) - ps, lo_r, r1, xtol=1e-300, rtol=1e-15)
        hi = r2
        while p(hi) - ps < 0:
            hi = hi + 0.5 * (0.999999 * rmax - hi)
        rl = optimize.brentq(lambda r: p(r) - ps, r2, hi, xtol=1e-300, rtol=1e-15)
        return rg, rl

    def area(ps):
        rg, rl = roots(ps)
        # integral over v of p, with v = 1/rho: int_{rl}^{rg} p(rho) * (-1/rho^2) d rho ... as v grows
        val, _ = integrate.quad(lambda r: (p(r) - ps) / (r * r), rg, rl, epsabs=1e-15, epsrel=1e-13,
                                limit=400)
        return val

    lo = max(pmin, 1e-14) + 1e-13 * abs(pmax)
    hi = pmax - 1e-13 * abs(pmax)
    ps = optimize.brentq(area, lo, hi, xtol=1e-18, rtol=1e-15)
    return roots(ps)


# Closed-form chemical potentials mu = df/drho of the Helmholtz free-energy density f(rho) whose
# pressure p = rho mu - f is the EOS; used only to pin `maxwell` (mu_g = mu_l at coexistence).
def chemical_potential(eos: EOS, rho):
    rho = np.asarray(rho, dtype=np.float64)
    R, T = eos.R, eos.T
    if eos.kind == "CS":
        eta = eos.b * rho / 4.0
        g = (4 * eta - 3 * eta ** 2) / (1 - eta) ** 2
        dg = (4 - 2 * eta) / (1 - eta) ** 3
        return R * T * (np.log(rho) + g + eta * dg) - 2 * eos.a * rho
    tc = eos.tc()
    kappa = 0.37464 + 1.54226 * eos.omega - 0.26992 * eos.omega ** 2
    aphi = eos.a * (1.0 + kappa * (1.0 - math.sqrt(T / tc))) ** 2
    b = eos.b
    s2 = math.sqrt(2.0)
    # f = rho R T [ln(rho/(1-b rho)) - 1] - aphi/(2 sqrt2 b) rho ln[(1+(1+s2) b rho)/(1+(1-s2) b rho)]
    L = np.log((1 + (1 + s2) * b * rho) / (1 + (1 - s2) * b * rho))
    dL = (1 + s2) * b / (1 + (1 + s2) * b * rho) - (1 - s2) * b / (1 + (1 - s2) * b * rho)
    ideal = R * T * (np.log(rho / (1 - b * rho)) - 1) + R * T * (1 + b * rho / (1 - b * rho))
    attr = -aphi / (2 * s2 * b) * (L + rho * dL)
    return ideal + attr
