"""Pins of the oracle's equation of state, pseudopotential and coexistence solver, and of the
improved virtual-density rule (Eqs. 16-17) against the paper's worked example."""
import math

import numpy as np
import pytest

from oracle import eos as E, lbm


def test_pr_critical_temperature_from_definitions():
    # a = 0.45724 R^2 Tc^2/pc and b = 0.0778 R Tc/pc (Eq. 18) with a = 2/49, b = 2/21, R = 1
    pr = E.pr_paper()
    tc = pr.tc()
    pc = 0.0778 * pr.R * tc / pr.b
    assert abs(0.45724 * pr.R ** 2 * tc ** 2 / pc - pr.a) < 1e-15
    # the numerical critical point of the PR curve lies within the rounding of 0.45724/0.0778
    tcn, rcn = E.critical_point(pr)
    assert abs(tcn / tc - 1) < 2e-4


def test_cs_critical_point_closed_form():
    # Carnahan-Starling: Tc = 0.3773 a/(b R) and eta_c = 0.1304 (literature closed forms)
    cs = E.cs_config()
    tc, rc = E.critical_point(cs)
    assert abs(tc / (0.3773 * cs.a / (cs.b * cs.R)) - 1) < 1e-4
    assert abs(cs.b * rc / 4 - 0.1304) < 2e-4


def test_pr_coexistence_matches_paper():
    # Sec. IV.A: T = 0.86 Tc gives rho_g ~ 0.38 and rho_l ~ 6.5
    pr = E.pr_paper().at_reduced_temperature(0.86)
    g, l = E.maxwell(pr)
    assert round(g, 2) == 0.38
    assert round(l, 1) == 6.5


@pytest.mark.parametrize("eos,tr", [(E.pr_paper(), 0.86), (E.cs_config(), 0.7), (E.cs_config(), 0.6)])
def test_maxwell_equal_chemical_potential(eos, tr):
    """Coexistence means equal pressure and equal chemical potential; mu comes from the closed-form
    free energy, independent of the equal-area quadrature used by `maxwell`."""
    e = eos.at_reduced_temperature(tr)
    g, l = E.maxwell(e)
    assert g < l
    assert abs(float(e.pressure(g) - e.pressure(l))) < 1e-14 * max(1.0, abs(float(e.pressure(g))))
    assert abs(float(E.chemical_potential(e, g) - E.chemical_potential(e, l))) < 1e-11
    # and the chemical potential is the derivative of the free energy whose Legendre transform is p
    r = np.linspace(0.05 * g + 0.01 * l, 0.9 * l, 7)
    h = 1e-6
    # d(p)/d(rho) = rho d(mu)/d(rho) (Gibbs-Duhem at fixed T)
    dp = (e.pressure(r + h) - e.pressure(r - h)) / (2 * h)
    dmu = (E.chemical_potential(e, r + h) - E.chemical_potential(e, r - h)) / (2 * h)
    assert np.allclose(dp, r * dmu, rtol=1e-6, atol=1e-10)


def test_psi_definition_and_domain():
    # Eq. 6 with G = -1, c = 1: psi^2 = 2 (rho/3 - p)
    cs = E.cs_config().at_reduced_temperature(0.7)
    rho = np.array([0.01, 0.1, 0.3])
    assert np.allclose(E.psi(cs, rho) ** 2, 2 * (rho / 3 - cs.pressure(rho)), rtol=1e-14)
    # G > 0 makes the argument negative: an error, never a silent clamp
    with pytest.raises(FloatingPointError):
        E.psi(cs, rho, G=+1.0)


# ---- Eqs. 16-17 and the limiter: the worked example of Sec. III.B (rho_g = 0.5, rho_l = 10) ----

def test_ivd_worked_example_phi_branch():
    g, l = 0.5, 10.0
    # rho_ave = 5 and phi = 1.1 raise the virtual density from 5 to 5.5
    assert math.isclose(float(lbm.ivd_virtual_density(5.0, 0.1, g, l)), 5.5, rel_tol=1e-15)
    # the minimum virtual density of the phi branch is phi * rho_g = 0.55 (not 1.0 as rho_ave + 0.5)
    assert math.isclose(float(lbm.ivd_virtual_density(0.5, 0.1, g, l)), 0.55, rel_tol=1e-15)
    # values above rho_l are set to rho_l
    assert float(lbm.ivd_virtual_density(9.5, 0.1, g, l)) == 10.0


def test_ivd_worked_example_drho_branch():
    g, l = 0.5, 10.0
    # rho_ave - drho: the maximum virtual density is rho_l - drho = 9.5 (rho_l/phi would give 9.09)
    assert float(lbm.ivd_virtual_density(10.0, -0.5, g, l)) == 9.5
    # values below rho_g are set to rho_g
    assert float(lbm.ivd_virtual_density(0.7, -0.5, g, l)) == 0.5
    # the standard case phi = 1 / drho = 0 is rho_w = rho_ave
    assert float(lbm.ivd_virtual_density(3.3, 0.0, g, l)) == 3.3
    assert float(lbm.ivd_virtual_density(3.3, -0.0, g, l)) == 3.3


def test_ivd_rho_ave_weights():
    """Eq. 17 on a hand-made 2D configuration: a wall node with fluid neighbours of known density."""
    mask = np.zeros((5, 5), np.uint8)
    mask[2, 2] = 1                       # one solid node at (2,2); all neighbours fluid
    mask[2, 3] = 1                       # ... except its +x neighbour
    geo = lbm.Geometry(mask, "D2Q9")
    rho = np.zeros((5, 5))
    rho[2, 1] = 1.0   # -x neighbour (w = 1/3)
    rho[3, 2] = 2.0   # +y neighbour (w = 1/3)
    rho[1, 2] = 4.0   # -y neighbour (w = 1/3)
    rho[3, 3] = 8.0   # (+1,+1) (w = 1/12)
    p = lbm.Params("D2Q9", E.cs_config(), rho_g=0.0, rho_l=100.0, kappa=0.0)
    rw = lbm.wall_density(rho, geo, p)
    # fluid neighbours of (2,2): -x, +y, -y (w 1/3 each) and all four diagonals (w 1/12 each)
    num = (1.0 + 2.0 + 4.0) / 3 + 8.0 / 12
    den = 3 / 3 + 4 / 12
    assert math.isclose(rw[2, 2], num / den, rel_tol=1e-15)
    assert geo.wall[2, 2] and geo.wall[2, 3] and not geo.wall[0, 0]
