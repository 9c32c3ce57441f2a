"""Differentiable VGICP factors: a torch.autograd.Function over se(3) increments.

For a set of factors (target map, source cloud, base pose T0_p) the forward
pass evaluates err_p(xi_p) = e^M at T_p = T0_p Exp(xi_p) (arXiv 2202.00242
Eq. 2) on the GPU.  The backward pass calls the library's gradient kernel at
the same poses, which emits d err / d delta for the right perturbation
T_p Exp(delta): 2 J^T W d (W held, ``exact=False``) or the exact derivative that
also differentiates W (``exact=True``), maps it to xi with the SE(3) right
Jacobian, d err / d xi = J_r(xi)^T d err / d delta, and scales it by the
incoming gradient.  The poses T0_p Exp(xi_p) and J_r are composed on the device
in binary64 (vgicp_plan_evaluate), so a forward and backward pass with xi on
the GPU runs without host round trips.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


class FactorSet:
    """Factors sharing one differentiable pose increment each.  The work list is
    planned once (an ``api.Plan``); ``rebase`` moves the base poses."""

    def __init__(self, maps, sources, pairs, base_poses, neighbours=1, exact=False, tile=0):
        self.maps = list(maps)
        self.sources = list(sources)
        self.pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        self.neighbours = neighbours
        self.exact = exact
        self.plan = api.Plan(self.maps, self.sources, self.pairs, neighbours=neighbours, tile=tile)
        self.device = self.plan.device
        self.rebase(base_poses)

    def rebase(self, base_poses):
        """New base poses T0 (host (P, 4, 4) or a CUDA float64 tensor)."""
        b = torch.as_tensor(np.asarray(base_poses, dtype=np.float64)
                            if not isinstance(base_poses, torch.Tensor) else base_poses)
        self.base = b.to(device=self.device, dtype=torch.float64).reshape(-1, 4, 4).contiguous()
        if self.base.shape[0] != self.pairs.shape[0]:
            raise ValueError("one base pose per pair")

    def poses(self, xi) -> np.ndarray:
        """Host binary64 T0_p Exp(xi_p) (for inspection; the passes compose on the device)."""
        x = np.asarray(xi.detach().cpu() if isinstance(xi, torch.Tensor) else xi, np.float64)
        base = self.base.cpu().numpy()
        return np.stack([api.pose_mul(base[p], api.se3_exp(x[p])) for p in range(base.shape[0])])

    def cost(self, xi) -> torch.Tensor:
        return VGICPCost.apply(xi, self)


class VGICPCost(torch.autograd.Function):
    """err (P,) = VGICPCost.apply(xi (P, 6) float64, factor_set)."""

    @staticmethod
    def forward(ctx, xi: torch.Tensor, fs: FactorSet):
        x = xi.detach().to(device=fs.device, dtype=torch.float64).contiguous()
        out, _ = fs.plan.evaluate(fs.base, x, mode=api.COST)
        ctx.fs = fs
        ctx.x = x
        ctx.xi_device = xi.device
        return out[:, 6].to(device=xi.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        fs = ctx.fs
        mode = api.EXACT_GRADIENT if fs.exact else api.GRADIENT
        g = grad_out.detach().to(device=fs.device, dtype=torch.float64).contiguous()
        out, _ = fs.plan.evaluate(fs.base, ctx.x, mode=mode, grad_scale=g)
        return out[:, :6].to(ctx.xi_device), None
