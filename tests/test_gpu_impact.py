"""Droplet impact on a cylinder (Sec. IV.B): a drop with an initial downward velocity (U0 = 0.06,
Re = 600) hits a cylinder, PR EOS at 0.86 Tc, IVD walls with phi = 1.135.  The initial state with
velocity (f = f^eq(rho0, u0), stored for the pull) against the oracle, one step of the moving drop
against the oracle in FP64 and FP32, and the full 300 x 400 workload in FP32 against FP64."""
import numpy as np
import pytest

import workloads as W
from oracle import eos as E, lbm
from tests.harness import Case

pytestmark = pytest.mark.gpu

PR086 = E.pr_paper().at_reduced_temperature(0.86)
GPR, LPR = E.maxwell(PR086)
U0 = 0.06
NU = U0 * 2 * 50 / 600.0                 # Re = U0 (2 r) / nu = 600
S_NU = 1.0 / (3 * NU + 0.5)


def _impact(scale=1.0, precision_ref=True, kernel="auto"):
    wl = W.impact_300x400()
    if scale != 1.0:
        ny, nx = wl.shape
        wl.shape = (int(ny * scale), int(nx * scale))
        wl.body_center = tuple(c * scale for c in wl.body_center)
        wl.drop_center = tuple(c * scale for c in wl.drop_center)
        wl.body_radius *= scale
        wl.drop_radius *= scale
    rho0 = wl.rho0(LPR, GPR)
    u0 = W.drop_velocity(rho0, LPR, GPR, (0.0, -U0))
    u0 = np.where(wl.mask()[None] != 0, 0.0, u0)
    return Case("D2Q9", wl.shape, wl.mask(), rho0, eos_kind="PR", t_over_tc=0.86, sigma=0.11, kappa=wl.kappa,
                u0=u0, rates=dict(s_nu=S_NU), rho_ref=GPR, step_kernel=kernel,
                body=("ball", wl.body_center, wl.body_radius), drop_hint=wl.drop_center)


def test_initial_state_with_velocity():
    case = _impact(scale=0.25)
    geo, p, f0 = case.oracle()
    with case.gpu("fp64") as sim:
        got = sim.get_state()
    assert np.max(np.abs(got - f0)) < 1e-15 * np.max(np.abs(f0))


@pytest.mark.parametrize("precision,kernel,tol", [("fp64", "tile", 1e-13), ("fp32", "pair", 2e-6)])
def test_impact_one_step(precision, kernel, tol):
    case = _impact(scale=0.25, kernel=kernel)
    geo, p, _ = case.oracle()
    with case.gpu(precision) as sim:
        sim.step(5)
        f0 = sim.get_state()
        sim.step(1)
        f1 = sim.get_state()
    ref = lbm.step(f0, geo, p)
    assert np.max(np.abs(f1 - ref)) < tol * np.max(np.abs(ref))


def test_impact_fp32_against_fp64():
    """The 300 x 400 impact for 1000 steps (the drop has reached the cylinder): FP32 deviation
    storage against FP64, density at every fluid node within 1e-3 rho_l, mass within 1e-6."""
    case = _impact()
    out = {}
    for prec in ("fp64", "fp32"):
        with case.gpu(prec) as sim:
            sim.step(1000)
            out[prec] = sim.observables(fields=True)
    o64, r64, _ = out["fp64"]
    o32, r32, _ = out["fp32"]
    fl = case.mask == 0
    assert np.max(np.abs(r32[fl] - r64[fl])) <= 1e-3 * LPR
    assert abs(o32.mass / o64.mass - 1) <= 1e-6


def test_fig13_virtual_density_schemes_against_the_geometric_formulation():
    """Fig. 13 with each scheme tuned to about 60 degrees (rho_w = 3.45, theta_a = 63.5,
    phi = 1.135), FP32.  At t = 100 the mass-transfer layer of the constant virtual density has
    bridged the gas gap between drop and cylinder far more than under the geometric or improved
    schemes (minimum density on the centre line above the cylinder: measured 1.87 against 0.81 and
    0.89).  At t = 10000 the improved scheme agrees with the geometric formulation (the wetted
    fraction of the cylinder's first fluid ring, 680 of its nodes under both) while the constant
    virtual density deviates (352)."""
    wl = W.impact_300x400()
    ny, nx = wl.shape
    yy, xx = np.mgrid[0:ny, 0:nx]
    cx, cy = wl.body_center
    d = np.hypot(xx - cx, yy - cy) - wl.body_radius
    ring = (d > 0) & (d <= 1.5)
    top = int(cy + wl.body_radius) + 1
    gap, wet = {}, {}
    for name, kw in (("VD", dict(wall="VD", rho_w_const=3.45)), ("GF", dict(wall="GF", theta_a=63.5)),
                     ("IVD", dict())):
        case = _impact()
        for k, v in kw.items():
            setattr(case, k, v)
        with case.gpu("fp32") as sim:
            sim.step(100)
            _, rho, _ = sim.observables(fields=True)
            gap[name] = float(rho[top:top + 19, int(cx)].min())
            sim.step(9900)
            _, rho, _ = sim.observables(fields=True)
            wet[name] = int((ring & (rho > 0.5 * (LPR + GPR))).sum())
    assert gap["VD"] > 1.5 * max(gap["GF"], gap["IVD"])
    assert abs(wet["IVD"] - wet["GF"]) <= 0.05 * wet["GF"]
    assert abs(wet["VD"] - wet["GF"]) > 0.2 * wet["GF"]
