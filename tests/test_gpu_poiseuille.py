"""The Poiseuille channel of Sec. IV.B on the GPU: a liquid-filled channel between two plates driven
by a body force.  With the IVD scheme and phi >= 1 the wall density equals the liquid density
(after the limiter), so F_m = 0 and the steady flow is the parabola u = F_b/(2 mu) y'(L - y') with
the walls halfway between nodes; with the 'magic' rate product 3/16 of the MRT rates the lattice
solution is exact (in D3Q19 both odd moment families, q and m, take the magic rate), so the relative error E_r = sum |u - u_a| / sum |u_a| of Sec. IV.B measures the
arithmetic alone (the oracle's own pin reaches E_r < 1e-6 after the same 4000 steps).  D2Q9 (tile, y-march and pair kernels) and D3Q19 (z-march and z-pair march),
FP64 and FP32; plus the workload against the oracle stepped alongside.
"""
import numpy as np
import pytest

import workloads as W
from oracle import eos as E, lbm
from tests.harness import Case

pytestmark = pytest.mark.gpu

PR086 = E.pr_paper().at_reduced_temperature(0.86)
GPR, LPR = E.maxwell(PR086)
NU = 1.0 / 6.0
S_NU = 1.0 / (3 * NU + 0.5)
S_Q = 8 * (2 - S_NU) / (8 - S_NU)       # Lambda_nu Lambda_q = 3/16
FB = 1e-5


def _channel(shape, step_kernel="auto"):
    mask = W.plates_mask(shape)
    rho0 = np.full(shape, LPR)
    return Case("D2Q9" if len(shape) == 2 else "D3Q19", shape, mask, rho0, eos_kind="PR", t_over_tc=0.86,
                sigma=0.11, kappa=0.2, body_force=(FB, 0.0, 0.0), rho_ref=LPR,
                rates=dict(s_nu=S_NU, s_q=S_Q, s_m=S_Q), step_kernel=step_kernel)


def _e_r(u, ny):
    """E_r of Sec. IV.B over the fluid rows, x velocity against the parabola."""
    lw = ny - 2.0
    y = np.arange(ny) - 0.5
    ua = FB / (2 * LPR * NU) * y * (lw - y)
    ux = u[0]
    ux = ux.reshape(-1, ny, ux.shape[-1])[:, 1:-1, :]          # (z or 1, fluid rows, x)
    ua = ua[1:-1][None, :, None]
    return np.sum(np.abs(ux - ua)) / np.sum(np.abs(np.broadcast_to(ua, ux.shape)))


@pytest.mark.parametrize("shape,precision,kernel,tol", [
    ((18, 48), "fp64", "tile", 1e-6),
    ((18, 48), "fp64", "ymarch", 1e-6),
    ((18, 48), "fp32", "pair", 1e-4),
    ((6, 18, 8), "fp64", "auto", 1e-6),      # z-march
    ((6, 18, 8), "fp32", "auto", 1e-4),      # z-pair march
])
def test_poiseuille_closed_form(shape, precision, kernel, tol):
    case = _channel(shape, kernel)
    with case.gpu(precision) as sim:
        sim.step(4000)
        o, rho, u = sim.observables(fields=True)
    assert _e_r(u, shape[-2]) < tol
    fl = case.mask == 0
    assert np.max(np.abs(rho[fl] - LPR)) < 1e-6 * LPR


def test_poiseuille_against_oracle():
    """The channel's first 300 steps on the GPU (FP64) and in the oracle agree to round-off."""
    case = _channel((18, 40))
    geo, p, f0 = case.oracle()
    ref = lbm.run(f0, geo, p, 300)
    with case.gpu("fp64") as sim:
        sim.step(300)
        got = sim.get_state()
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
