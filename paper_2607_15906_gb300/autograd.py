"""torch.autograd.Function for E(theta) of a fixed ansatz.

Forward and backward both come from one adjoint sweep on the GPU
(gocp_energy_grad): the forward pass keeps dE/dtheta for the backward pass,
which scales it by the incoming gradient.  theta may live on the CPU or on
the problem's GPU; the result is a 0-d float64 tensor on theta's device.
"""

from __future__ import annotations

import numpy as np
import torch


class AnsatzEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, problem, ops, ws=None):
        th = theta.detach()
        if th.is_cuda:
            dev = th.device
            ops_t = torch.as_tensor(np.asarray(ops, np.int32), device=dev)
            e = torch.zeros(1, dtype=torch.float64, device=dev)
            de = torch.zeros(max(int(ops_t.numel()), 1), dtype=torch.float64, device=dev)
            problem.energy_grad(ops_t, th.to(torch.float64).contiguous(), ws=ws, out_e=e, out_de=de)
            ctx.save_for_backward(de[: ops_t.numel()])
            return e[0]
        e, de = problem.energy_grad(np.asarray(ops, np.int32), th.double().numpy(), ws=ws)
        ctx.save_for_backward(torch.from_numpy(de))
        return torch.tensor(e, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        (de,) = ctx.saved_tensors
        return grad_out * de.to(grad_out.device), None, None, None


def ansatz_energy(theta, problem, ops, ws=None):
    return AnsatzEnergy.apply(theta, problem, ops, ws)
