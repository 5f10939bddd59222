"""torch.autograd wrapper: homogenised stress of an SVK cell as a
differentiable function of its per-voxel shear and bulk moduli.

forward solves the cell (Newton-CG through the C ABI) for the macroscopic
deformation; backward is one adjoint CG solve with the same operator
followed by the per-voxel sensitivity kernel (rve_adjoint_grad), which
gives both gradients from the same adjoint field.
"""
from __future__ import annotations

import numpy as np
import torch

from .rve import RVE


class HomogenizedStress(torch.autograd.Function):
    """P-bar(mu, K) for a fixed macroscopic F-bar (K: tensor of the same
    shape as mu, or a scalar / array treated as constant)."""

    @staticmethod
    def forward(ctx, mu, K, Fbar, increments=1, tol_newton=1e-5, tol_cg=1e-8,
                precision="fp64", adjoint_tol=1e-10, cg_atol=0.0):
        mu_np = mu.detach().cpu().numpy().astype(np.float64)
        K_np = (K.detach().cpu().numpy() if isinstance(K, torch.Tensor)
                else np.broadcast_to(np.asarray(K, np.float64), mu_np.shape))
        shape = mu_np.shape
        r = RVE(shape, voxel_params=np.stack([np.broadcast_to(K_np, shape), mu_np]),
                precision=precision, cg_atol=cg_atol)
        Fbar = np.asarray(Fbar, dtype=np.float64)
        eye = np.eye(3)
        for k in range(1, increments + 1):
            r.set_macro_F(eye + (k / increments) * (Fbar - eye))
            r.solve_increment(tol_newton, tol_cg)
        ctx.rve = r
        ctx.adjoint_tol = adjoint_tol
        ctx.device = mu.device
        ctx.K_is_tensor = isinstance(K, torch.Tensor)
        return torch.from_numpy(r.homogenized_P()).to(mu.device)

    @staticmethod
    def backward(ctx, grad_P):
        W = grad_P.detach().cpu().numpy().astype(np.float64)
        gK, gmu, _ = ctx.rve.adjoint_grad(W, ctx.adjoint_tol)
        ctx.rve.close()
        dK = torch.from_numpy(gK).to(ctx.device) if ctx.K_is_tensor else None
        return (torch.from_numpy(gmu).to(ctx.device), dK) + (None,) * 7


def homogenized_stress(mu, K, Fbar, **kw):
    """Differentiable P-bar (3x3 float64) of an SVK cell with per-voxel shear
    moduli `mu` ([nx, ny, nz] tensor) and bulk moduli `K`."""
    args = [kw.pop(k, d) for k, d in (("increments", 1), ("tol_newton", 1e-5),
                                       ("tol_cg", 1e-8), ("precision", "fp64"),
                                       ("adjoint_tol", 1e-10), ("cg_atol", 0.0))]
    if kw:
        raise TypeError(f"unknown arguments {sorted(kw)}")
    return HomogenizedStress.apply(mu, K, Fbar, *args)
