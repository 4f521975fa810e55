"""torch.autograd.Function over the lbmwet adjoint: the density field after n steps as a function of
the per-wall-node wettability parameter kappa (Eq. 16 in the unified form).

Forward: set kappa, reset the state to `initial` (post-streaming distributions), run n steps with
checkpoints (lbm_record) and return rho_T on the device.  Backward: dL/drho_T from autograd goes to
lbm_adjoint, which returns dL/dkappa.  All arithmetic runs in liblbmwet.so; this module moves
tensors and pointers.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbmwet as L


class DensityFromWettability(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa: torch.Tensor, sim: "L.Simulation", initial: np.ndarray, n_steps: int,
                ckpt_every: int):
        L.lbm_set_kappa(sim.h, kappa.detach().double().cpu().numpy())
        sim.set_state(initial, step=0)
        L.lbm_record(sim.h, n_steps, ckpt_every)
        rho = torch.empty(sim.n, dtype=torch.float64, device="cuda")
        L.lbm_fields_device(sim.h, rho.data_ptr(), None)
        ctx.sim = sim
        ctx.n_wall = kappa.numel()
        ctx.kappa_device = kappa.device
        return rho.view(sim.shape)

    @staticmethod
    def backward(ctx, grad_rho: torch.Tensor):
        g = grad_rho.detach().to(dtype=torch.float64, device="cuda").contiguous().view(-1)
        dk = L.lbm_adjoint(ctx.sim.h, g.data_ptr(), ctx.n_wall)
        return torch.as_tensor(dk, device=ctx.kappa_device), None, None, None, None
