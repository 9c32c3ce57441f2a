"""Differentiable VGICP factors: a torch.autograd.Function over se(3) increments.

For a set of factors (target map, source cloud, base pose T0_p) the forward
pass evaluates err_p(xi_p) = e^M at T_p = T0_p Exp(xi_p) (arXiv 2202.00242
Eq. 2) on the GPU.  The backward pass calls the library's gradient kernel at
the same poses, which emits d err / d delta for the right perturbation
T_p Exp(delta): 2 J^T W d (W held, ``exact=False``) or the exact derivative that
also differentiates W (``exact=True``), and maps it to xi with the SE(3) right
Jacobian (binary64, host): d err / d xi = J_r(xi)^T d err / d delta.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


class FactorSet:
    """Factors sharing one differentiable pose increment each."""

    def __init__(self, maps, sources, pairs, base_poses, neighbours=1, exact=False):
        self.maps = list(maps)
        self.sources = list(sources)
        self.pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        self.base = np.ascontiguousarray(np.asarray(base_poses, dtype=np.float64)).reshape(-1, 4, 4)
        self.neighbours = neighbours
        self.exact = exact

    def poses(self, xi: np.ndarray) -> np.ndarray:
        return np.stack([api.pose_mul(self.base[p], api.se3_exp(xi[p]))
                         for p in range(self.base.shape[0])])

    def cost(self, xi) -> torch.Tensor:
        return VGICPCost.apply(xi, self)


class VGICPCost(torch.autograd.Function):
    """err (P,) = VGICPCost.apply(xi (P, 6) float64, factor_set)."""

    @staticmethod
    def forward(ctx, xi: torch.Tensor, fs: FactorSet):
        x = xi.detach().cpu().numpy().astype(np.float64)
        poses = fs.poses(x)
        _, err, _ = api.evaluate_batched(fs.maps, fs.sources, fs.pairs, poses, mode=api.COST,
                                         neighbours=fs.neighbours)
        ctx.fs = fs
        ctx.x = x
        ctx.poses = poses
        ctx.xi_device = xi.device
        return err.to(device=xi.device, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        fs = ctx.fs
        mode = api.EXACT_GRADIENT if fs.exact else api.GRADIENT
        g, _, _ = api.evaluate_batched(fs.maps, fs.sources, fs.pairs, ctx.poses, mode=mode,
                                       neighbours=fs.neighbours)
        g = g.cpu().numpy()
        Jr = np.stack([api.se3_right_jacobian(ctx.x[p]) for p in range(ctx.x.shape[0])])
        gx = np.einsum("pij,pi->pj", Jr, g)  # J_r^T g
        w = grad_out.detach().cpu().numpy().astype(np.float64)[:, None]
        return torch.from_numpy(w * gx).to(ctx.xi_device), None
