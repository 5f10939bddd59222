"""Gradient of a homogenised-stress functional with respect to per-voxel
shear and bulk moduli, Saint Venant-Kirchhoff (Sec. 4), by one adjoint solve.

Not in the paper; derived from its equilibrium equations.  With
F = Fbar + w (w compatible, zero mean) the converged state satisfies
R(w, mu) = G : P(Fbar + w, mu) = 0 (Eq. weak:discr:FFT).  For
J = W : P-bar = (1/n) sum_v W_ab P_ab(F_v, mu_v):

  dJ/dmu_k = (1/n) W : (dP/dmu)_k + <dJ/dF, dw/dmu_k>,
  dw/dmu_k = -A^-1 G : (dP/dmu_k e_k),   A = G K G on compatible fields.

K (the matrix of Eq. iter:varP, dP_ab = D_ab,cd dF_cd) is symmetric for a
hyper-elastic material, so dJ/dF = (1/n) D W and the adjoint field solves
A lambda = G : (K : W) / n -- the same CG system as the Newton steps.  Then

  dJ/dmu_k = (1/n) W : (dP/dmu)_k - lambda_k : (dP/dmu)_k,
  (dP/dmu)_k = F_k . (2 dev E_k)   (S = lambda tr(E) I + 2 mu E with
                                    lambda = K - 2 mu/3, K fixed),
and in the same way, with the same lambda, for the bulk moduli
  (dP/dK)_k = F_k . (tr(E_k) I)    (mu fixed).
"""
import numpy as np

from . import fourier, solver, svk, tensor as t


def dP_dmu(F):
    """(dP/dmu) = F . (2 dev E) at fixed bulk modulus, [3,3,*grid]."""
    E = svk.green_lagrange(F)
    I = t.EYE.reshape((3, 3) + (1,) * (F.ndim - 2))
    devE = E - np.trace(E) / 3.0 * I
    return t.dot_2_2(F, 2.0 * devE)


def dP_dK(F):
    """(dP/dK) = F . (tr(E) I) at fixed shear modulus, [3,3,*grid]."""
    E = svk.green_lagrange(F)
    I = t.EYE.reshape((3, 3) + (1,) * (F.ndim - 2))
    return t.dot_2_2(F, np.trace(E) * I)


def adjoint_field(problem, W, tol_cg=1e-12, cg_atol=0.0):
    """lambda solving G K G lambda = G (K : W) / n at the converged state."""
    W = np.asarray(W, dtype=np.float64)
    grid = problem.shape
    n = int(np.prod(grid))
    _, K4 = problem.constitutive(problem.F)
    op = solver.tangent_operator(K4)
    b = fourier.G(svk.tangent_apply(K4, t.uniform(W, grid)) / n)
    lam, _, _ = solver.cg(op, b, tol_cg, atol=cg_atol)
    return lam


def grad_params(problem, W, tol_cg=1e-12, cg_atol=0.0):
    """(dJ/dK, dJ/dmu) per voxel for J = W : P-bar, from one adjoint field."""
    W = np.asarray(W, dtype=np.float64)
    n = problem.F[0, 0].size
    lam = adjoint_field(problem, W, tol_cg, cg_atol)
    out = []
    for d in (dP_dK(problem.F), dP_dmu(problem.F)):
        out.append(np.einsum("ab,ab...->...", W, d) / n - np.einsum("ab...,ab...->...", lam, d))
    return tuple(out)


def grad_mu(problem, W, tol_cg=1e-12, cg_atol=0.0):
    """dJ/dmu per voxel for J = W : P-bar at the problem's converged state."""
    W = np.asarray(W, dtype=np.float64)
    grid = problem.shape
    n = int(np.prod(grid))
    _, K4 = problem.constitutive(problem.F)
    op = solver.tangent_operator(K4)
    g = svk.tangent_apply(K4, t.uniform(W, grid)) / n        # dJ/dF = (1/n) D W
    b = fourier.G(g)
    lam, _, _ = solver.cg(op, b, tol_cg, atol=cg_atol)
    d = dP_dmu(problem.F)
    explicit = np.einsum("ab,ab...->...", W, d) / n
    return explicit - np.einsum("ab...,ab...->...", lam, d)


def localization(problem, W, tol_cg=1e-12, cg_atol=0.0):
    """Microscopic response L = W + dF to a unit macroscopic perturbation W
    (the predictor system of Eq. bc:lin with dFbar = W); gives the same
    gradient through dJ/dmu_k = (1/n) L_k : (dP/dmu)_k."""
    W = np.asarray(W, dtype=np.float64)
    grid = problem.shape
    _, K4 = problem.constitutive(problem.F)
    op = solver.tangent_operator(K4)
    U = t.uniform(W, grid)
    dF, _, _ = solver.cg(op, -op(U), tol_cg, atol=cg_atol)
    return U + dF
