"""The D2Q9 discrete adjoint through the C ABI (lbm_record + lbm_adjoint): dL/dkappa per wall node for
L = sum (rho_T - rho_target)^2, against central finite differences of the FP64 oracle at every wall
node (FP64: 1e-6 of the largest derivative; FP32 deviation storage: 2e-3), independence of the
checkpoint interval, and the torch.autograd.Function wrapper."""
import numpy as np
import pytest

from oracle import gradient as GR, lbm
from tests.harness import drop_on_cylinder

pytestmark = pytest.mark.gpu

N_STEPS = 24


def _problem():
    case = drop_on_cylinder((40, 44), (22.0, 14.0), 7.0, (22.0, 25.0), 8.0, kappa=0.1)
    geo, p, f0 = case.oracle()
    nw = len(geo.wall_flat)
    rng = np.random.default_rng(11)
    kappa = rng.uniform(0.02, 0.3, nw)
    kappa_target = kappa + 0.08 * rng.uniform(-1, 1, nw)
    _, rho_target = GR.loss(f0, geo, p, kappa_target, N_STEPS, np.zeros(geo.shape))
    return case, geo, p, f0, kappa, rho_target


def _gpu_gradient(case, kappa, target, precision, ckpt):
    import torch
    from paper_1908_04443_gb300 import lbmwet as L
    case.kappa = kappa
    if precision == "fp32":
        case.rho_ref = case.bounds()[0]
    with case.gpu(precision, stream=torch.cuda.current_stream()) as sim:
        L.lbm_record(sim.h, N_STEPS, ckpt)
        rho = torch.zeros(sim.n, dtype=torch.float64, device="cuda")
        L.lbm_fields_device(sim.h, rho.data_ptr(), None)
        fluid = torch.as_tensor((case.mask.reshape(-1) == 0), device="cuda")
        tgt = torch.as_tensor(target.reshape(-1), device="cuda")
        drho = torch.where(fluid, 2.0 * (rho - tgt), torch.zeros_like(rho))
        g = L.lbm_adjoint(sim.h, drho.data_ptr(), len(kappa))
        loss = float(torch.sum(torch.where(fluid, (rho - tgt) ** 2, torch.zeros_like(rho))).item())
    return g, loss


def test_adjoint_fp64_matches_oracle_fd_every_wall_node():
    case, geo, p, f0, kappa, target = _problem()
    g_gpu, loss_gpu = _gpu_gradient(case, kappa, target, "fp64", ckpt=7)
    loss_ref, _ = GR.loss(f0, geo, p, kappa, N_STEPS, target)
    assert abs(loss_gpu - loss_ref) <= 1e-10 * abs(loss_ref)
    g_fd = GR.fd_gradient(f0, geo, p, kappa, N_STEPS, target, range(len(kappa)), h=1e-5)
    scale = np.max(np.abs(g_fd))
    assert scale > 0
    assert np.max(np.abs(g_gpu - g_fd)) <= 1e-6 * scale


def test_adjoint_checkpoint_interval_does_not_matter():
    case, geo, p, f0, kappa, target = _problem()
    g1, _ = _gpu_gradient(case, kappa, target, "fp64", ckpt=1)
    g2, _ = _gpu_gradient(case, kappa, target, "fp64", ckpt=5)
    g3, _ = _gpu_gradient(case, kappa, target, "fp64", ckpt=100)
    scale = np.max(np.abs(g1))
    assert np.max(np.abs(g1 - g2)) <= 1e-13 * scale
    assert np.max(np.abs(g1 - g3)) <= 1e-13 * scale


def test_adjoint_fp32_deviation_storage():
    case, geo, p, f0, kappa, target = _problem()
    g32, _ = _gpu_gradient(case, kappa, target, "fp32", ckpt=7)
    g_fd = GR.fd_gradient(f0, geo, p, kappa, N_STEPS, target, range(len(kappa)), h=1e-5)
    scale = np.max(np.abs(g_fd))
    assert np.max(np.abs(g32 - g_fd)) <= 2e-3 * scale


def test_adjoint_requires_the_recorded_state():
    import torch
    from paper_1908_04443_gb300 import lbmwet as L
    case, geo, p, f0, kappa, target = _problem()
    case.kappa = kappa
    with case.gpu("fp64") as sim:
        L.lbm_record(sim.h, 5, 2)
        sim.step(1)                      # the state moved on: the recording no longer applies
        d = torch.zeros(sim.n, dtype=torch.float64, device="cuda")
        with pytest.raises(L.LbmError) as ei:
            L.lbm_adjoint(sim.h, d.data_ptr(), len(kappa))
        assert ei.value.status == L.LBM_ERR_STATE


def test_autograd_function():
    import torch
    from paper_1908_04443_gb300.autograd import DensityFromWettability
    case, geo, p, f0, kappa, target = _problem()
    case.kappa = kappa
    with case.gpu("fp64") as sim:
        initial = sim.get_state()
        k = torch.tensor(kappa, dtype=torch.float64, device="cuda", requires_grad=True)
        rho = DensityFromWettability.apply(k, sim, initial, N_STEPS, 6)
        fluid = torch.as_tensor(case.mask == 0, device="cuda")
        tgt = torch.as_tensor(target, device="cuda")
        loss = torch.sum(torch.where(fluid, (rho - tgt) ** 2, torch.zeros_like(rho)))
        loss.backward()
    g_fd = GR.fd_gradient(f0, geo, p, kappa, N_STEPS, target, range(0, len(kappa), 7), h=1e-5)
    g = k.grad.cpu().numpy()[::7]
    assert np.max(np.abs(g - g_fd)) <= 1e-6 * np.max(np.abs(g_fd))
