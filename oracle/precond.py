"""Reference-medium preconditioned conjugate gradients (TEST INFRASTRUCTURE,
see the package docstring).

Not in the paper: it solves Eq. iter:system by plain CG and notes (Sec. 5.5)
that CG slows down as the phase contrast grows.  Reading used here:

* The preconditioner is M = G : K0 : G for a homogeneous isotropic reference
  medium K0 : A = lam0 tr(A) I + mu0 (A + A^T), symmetric positive definite
  on the compatible fields (the range of G), where the projected system
  lives.  Its pseudo-inverse applied after G, Gamma0 = M^+ G, is diagonal in
  Fourier space: per frequency the 9x9 matrix pinv(G-hat K0 G-hat) G-hat,
  zero at q = 0 and at Nyquist frequencies like G-hat (Appendix C).
* lam0 and mu0 are the voxel averages of the elastic Lame parameters; the
  iterates do not depend on a common scale of K0, only on lam0 / mu0.
* CG is the textbook preconditioned recurrence (z = Gamma0 r); it stops at
  sqrt(r.z) <= max(eta sqrt(r0.z0), atol), the M^-1-norm of the residual in
  place of the 2-norm of reading 3.
"""
from __future__ import annotations

import numpy as np

from . import fourier
from .solver import SolverError, vdot


def reference_medium(lam, mu):
    """(lam0, mu0) = voxel averages of the Lame parameters."""
    return float(np.mean(lam)), float(np.mean(mu))


def k0_matrix(lam0, mu0):
    """K0 as a 9x9 matrix on components 3i+j: (K0 : A)_ij."""
    K = np.zeros((9, 9))
    for i in range(3):
        for j in range(3):
            if i == j:
                for k in range(3):
                    K[3 * i + j, 3 * k + k] += lam0
            K[3 * i + j, 3 * i + j] += mu0
            K[3 * i + j, 3 * j + i] += mu0
    return K


def gamma0_hat(grid_shape, lam0, mu0):
    """Gamma0-hat per frequency, [9, 9, nx, ny, nz]: pinv(G K0 G) G with the
    81-component G-hat of Eq. G written as a 9x9 matrix."""
    G4 = fourier.ghat4(grid_shape)                   # [3,3,3,3,*grid], C_ij = G_ijlm A_ml
    Gm = np.einsum("ijlm...->ij" "ml...", G4).reshape((9, 9) + tuple(grid_shape))
    K0 = k0_matrix(lam0, mu0)
    out = np.zeros_like(Gm)
    for idx in np.ndindex(*grid_shape):
        g = Gm[(slice(None), slice(None)) + idx]
        if not g.any():
            continue
        out[(slice(None), slice(None)) + idx] = np.linalg.pinv(g @ K0 @ g, rcond=1e-12) @ g
    return out


def gamma0(B, lam0, mu0, ghat=None):
    """Gamma0 : B for a real field [3, 3, *grid]."""
    grid = B.shape[-3:]
    if ghat is None:
        ghat = gamma0_hat(grid, lam0, mu0)
    Bh = fourier.dft3(np.asarray(B, dtype=np.float64)).reshape((9,) + tuple(grid))
    Ch = np.einsum("ab...,b...->a...", ghat, Bh).reshape((3, 3) + tuple(grid))
    return np.real(fourier.dft3(Ch, inverse=True))


def pcg(apply_A, b, apply_Minv, tol, maxiter=10_000, atol=0.0):
    """Textbook preconditioned CG from x0 = 0.  Returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_Minv(r)
    rz = vdot(r, z)
    if rz <= 0.0:
        return x, 0
    stop = max(tol * np.sqrt(rz), atol)
    p = z.copy()
    for k in range(1, maxiter + 1):
        Ap = apply_A(p)
        pAp = vdot(p, Ap)
        if pAp == 0.0 or not np.isfinite(pAp):
            raise SolverError("PCG breakdown: p.Ap = 0 or not finite")
        alpha = rz / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        z = apply_Minv(r)
        rz_new = vdot(r, z)
        if np.sqrt(max(rz_new, 0.0)) <= stop:
            return x, k
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise SolverError("PCG did not converge")


def linear_solver(grid_shape, lam0, mu0, tol, atol=0.0):
    """``linear_solver(K4, b)`` for ``solver.solve_increment``: PCG with the
    reference-medium preconditioner."""
    from .solver import tangent_operator
    gh = gamma0_hat(tuple(grid_shape), lam0, mu0)

    def solve(K4, b):
        return pcg(tangent_operator(K4), b, lambda r: gamma0(r, lam0, mu0, gh), tol, atol=atol)
    return solve
