"""Pins of the oracle's reference gradient (central finite differences of the FP64 oracle's density
loss with respect to per-wall-node kappa): step-size convergence, the identity between the sum of
the per-node derivatives and the derivative for a uniform shift of kappa, and a zero gradient when
no step is taken."""
import numpy as np

from oracle import gradient as GR, lbm
from tests.harness import drop_on_cylinder


def _setup(n_wall_frac=1.0):
    case = drop_on_cylinder((24, 26), (13.0, 8.0), 4.0, (13.0, 15.0), 5.0, kappa=0.1)
    geo, p, f0 = case.oracle()
    nw = len(geo.wall_flat)
    rng = np.random.default_rng(2)
    kappa = rng.uniform(0.05, 0.25, nw)
    target = f0.sum(0) * (1 + 0.01 * rng.uniform(-1, 1, geo.shape))
    return geo, p, f0, kappa, target


def test_fd_step_convergence():
    geo, p, f0, kappa, target = _setup()
    idx = [0, 5, 11]
    g1 = GR.fd_gradient(f0, geo, p, kappa, 6, target, idx, h=1e-5)
    g2 = GR.fd_gradient(f0, geo, p, kappa, 6, target, idx, h=2e-5)
    assert np.max(np.abs(g1)) > 0
    assert np.allclose(g1, g2, rtol=1e-6, atol=1e-9 * np.max(np.abs(g1)))


def test_fd_sum_equals_uniform_shift():
    geo, p, f0, kappa, target = _setup()
    nw = len(kappa)
    g = GR.fd_gradient(f0, geo, p, kappa, 5, target, range(nw), h=1e-5)
    h = 1e-5
    lp, _ = GR.loss(f0, geo, p, kappa + h, 5, target)
    lm, _ = GR.loss(f0, geo, p, kappa - h, 5, target)
    assert abs(g.sum() - (lp - lm) / (2 * h)) < 1e-6 * np.sum(np.abs(g))


def test_no_step_no_gradient():
    geo, p, f0, kappa, target = _setup()
    g = GR.fd_gradient(f0, geo, p, kappa, 0, target, [0, 3], h=1e-5)
    assert np.all(g == 0.0)
