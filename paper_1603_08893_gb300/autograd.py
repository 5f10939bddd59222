"""torch.autograd wrappers: homogenised stress of an SVK cell as a
differentiable function of its per-voxel shear and bulk moduli, and of a J2
cell after a path of increments from the virgin state as a function of its
per-voxel K, mu, tau_y0 and H.

forward solves the cell (Newton-CG through the C ABI) for the macroscopic
deformation; backward is one adjoint CG solve with the same operator
followed by the per-voxel sensitivity kernel (rve_adjoint_grad /
rve_adjoint_grad_params), which gives every gradient from the same adjoint
field.  For CUDA inputs the per-voxel parameters go to rve_create as a
device array (converted on the device) and the gradients are written by the
library straight into CUDA tensors (grads_on_device = 1): only P-bar and
dJ/dP-bar (9 values each) cross to the host.
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
        shape = tuple(mu.shape)
        if mu.is_cuda:
            # parameters stay on the device: the library converts them there
            m = mu.detach().to(torch.float64)
            k = (K.detach().to(device=mu.device, dtype=torch.float64) if isinstance(K, torch.Tensor)
                 else torch.as_tensor(np.asarray(K, np.float64), device=mu.device))
            vp = torch.stack([k.expand(shape), m]).contiguous()
        else:
            mu_np = mu.detach().numpy().astype(np.float64)
            K_np = (K.detach().numpy() if isinstance(K, torch.Tensor)
                    else np.asarray(K, np.float64))
            vp = np.stack([np.broadcast_to(K_np, shape), mu_np])
        r = RVE(shape, voxel_params=vp, precision=precision, cg_atol=cg_atol)
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
        W = grad_P.detach().cpu().numpy().astype(np.float64)  # 9 values
        dev = ctx.device.type == "cuda"
        gK, gmu, _ = ctx.rve.adjoint_grad(W, ctx.adjoint_tol, device=dev)
        ctx.rve.close()
        wrap = (lambda g: g) if dev else (lambda g: torch.from_numpy(g))
        dK = wrap(gK) if ctx.K_is_tensor else None
        return (wrap(gmu), dK) + (None,) * 7


def homogenized_stress(mu, K, Fbar, **kw):
    """Differentiable P-bar (3x3 float64) of an SVK cell with per-voxel shear
    moduli `mu` ([nx, ny, nz] tensor) and bulk moduli `K`."""
    args = [kw.pop(k, d) for k, d in (("increments", 1), ("tol_newton", 1e-5),
                                       ("tol_cg", 1e-8), ("precision", "fp64"),
                                       ("adjoint_tol", 1e-10), ("cg_atol", 0.0))]
    if kw:
        raise TypeError(f"unknown arguments {sorted(kw)}")
    return HomogenizedStress.apply(mu, K, Fbar, *args)


class J2HomogenizedStress(torch.autograd.Function):
    """P-bar(K, mu, tau_y0, H) of a J2 cell after increments from the virgin
    state to the F-bar of each (Fbar: one 3x3 tensor, or a sequence of them
    for a path).  One increment: backward by rve_adjoint_grad_params; a path
    (float64 handles): recorded with rve_tape and differentiated through the
    history by rve_adjoint_grad_path.  Each parameter is a tensor of the
    cell's shape (or a scalar)."""

    @staticmethod
    def forward(ctx, K, mu, ty0, H, Fbar, tol_newton=1e-5, tol_cg=1e-8, precision="fp64",
                adjoint_tol=1e-10, cg_atol=0.0):
        ref = next(t for t in (K, mu, ty0, H) if isinstance(t, torch.Tensor) and t.dim() == 3)
        shape = tuple(ref.shape)
        if ref.is_cuda:
            vals = [(t.detach().to(device=ref.device, dtype=torch.float64) if isinstance(t, torch.Tensor)
                     else torch.as_tensor(np.asarray(t, np.float64), device=ref.device)).expand(shape)
                    for t in (K, mu, ty0, H)]
            vp = torch.stack(vals).contiguous()
        else:
            vp = np.stack([np.broadcast_to((t.detach().numpy() if isinstance(t, torch.Tensor)
                                            else np.asarray(t)).astype(np.float64), shape)
                           for t in (K, mu, ty0, H)])
        r = RVE(shape, model="j2", voxel_params=vp, precision=precision, cg_atol=cg_atol)
        ramp = np.asarray(Fbar, dtype=np.float64).reshape(-1, 3, 3)
        ctx.path = len(ramp) > 1
        if ctx.path:
            r.tape(True)
        for Fb in ramp:
            r.set_macro_F(Fb)
            r.solve_increment(tol_newton, tol_cg)
        ctx.rve = r
        ctx.adjoint_tol = adjoint_tol
        ctx.device = ref.device
        ctx.is_tensor = [isinstance(t, torch.Tensor) for t in (K, mu, ty0, H)]
        return torch.from_numpy(r.homogenized_P()).to(ref.device)

    @staticmethod
    def backward(ctx, grad_P):
        W = grad_P.detach().cpu().numpy().astype(np.float64)  # 9 values
        dev = ctx.device.type == "cuda"
        if ctx.path:
            g, _ = ctx.rve.adjoint_grad_path(W, ctx.adjoint_tol, device=dev)
        else:
            g, _ = ctx.rve.adjoint_grad_params(W, ctx.adjoint_tol, device=dev)
        ctx.rve.close()
        wrap = (lambda a: a) if dev else (lambda a: torch.from_numpy(np.ascontiguousarray(a)))
        out = [wrap(g[k]) if ctx.is_tensor[k] else None for k in range(4)]
        return tuple(out) + (None,) * 6


def j2_homogenized_stress(K, mu, tau_y0, H, Fbar, **kw):
    """Differentiable P-bar (3x3 float64) of a J2 cell with per-voxel
    parameters after the increments to `Fbar` (a 3x3 F-bar, or a sequence
    of them) from the virgin state."""
    args = [kw.pop(k, d) for k, d in (("tol_newton", 1e-5), ("tol_cg", 1e-8),
                                       ("precision", "fp64"), ("adjoint_tol", 1e-10),
                                       ("cg_atol", 0.0))]
    if kw:
        raise TypeError(f"unknown arguments {sorted(kw)}")
    return J2HomogenizedStress.apply(K, mu, tau_y0, H, Fbar, *args)
