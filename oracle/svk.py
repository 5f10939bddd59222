"""Saint Venant-Kirchhoff hyper-elasticity in the reference configuration.

Sec. 4.2-4.3: S = C : E (Eq. elas:S), C = lambda I(x)I + 2 mu I4s
(Eq. elas:C), E = (F^T.F - I)/2, P = F.S (Eq. elas:S-P), and the consistent
tangent K = S.I4 + I4rt : (F.C.F^T) : I4rt (Eq. elas:K), defined through
delta P^T = K : delta F^T (Eq. iter:varP).

Materials are given by bulk modulus K and shear modulus mu (the parameters of
the paper's example), so lambda = K - 2 mu / 3.  K and mu are scalars or
grids ``[nx, ny, nz]``.
"""
import numpy as np

from . import tensor as t


def lame_lambda(K, mu):
    return np.asarray(K) - 2.0 * np.asarray(mu) / 3.0


def stiffness(K, mu):
    """C = lambda I (x) I + 2 mu I4s (Eq. elas:C); broadcasts over grids."""
    lam = lame_lambda(K, mu)
    II = t.dyad_2_2(t.EYE, t.EYE)
    I4s = t.identity4_sym()
    lam = np.asarray(lam)
    mu = np.asarray(mu)
    return (II.reshape(II.shape + (1,) * lam.ndim) * lam
            + 2.0 * I4s.reshape(I4s.shape + (1,) * mu.ndim) * mu)


def green_lagrange(F):
    """E = (F^T . F - I) / 2."""
    I = t.EYE.reshape((3, 3) + (1,) * (F.ndim - 2))
    return 0.5 * (t.dot_2_2(t.T2(F), F) - I)


def second_pk(F, K, mu):
    """S = C : E (Eq. elas:S) written with lambda and mu:
    S = lambda tr(E) I + 2 mu E (C is minor-symmetric, E symmetric)."""
    E = green_lagrange(F)
    lam = lame_lambda(K, mu)
    I = t.EYE.reshape((3, 3) + (1,) * (F.ndim - 2))
    return lam * np.trace(E) * I + 2.0 * mu * E


def stress(F, K, mu):
    """First Piola-Kirchhoff stress P = F . S (Eq. elas:S-P)."""
    return t.dot_2_2(F, second_pk(F, K, mu))


def constitutive(F, K, mu):
    """Return (P, K4) for a grid of deformation gradients ``[3,3,*grid]``.

    K4 follows Eq. elas:K literally: S.I4 + I4rt : (F.C.F^T) : I4rt, with
    (F.C.F^T)_ijkl = F_ia C_ajkb F_lb.
    """
    C4 = stiffness(K, mu)
    E = green_lagrange(F)
    S = t.ddot_4_2(C4, E)                      # Eq. elas:S
    P = t.dot_2_2(F, S)                        # Eq. elas:S-P
    FC = t.dot_2_4(F, C4)                      # F . C
    FCFt = t.dot_4_2(FC, t.T2(F))              # (F . C) . F^T
    I4 = t.identity4()
    I4rt = t.identity4_rt()
    K4 = t.dot_2_4(S, I4) + t.ddot_4_4(t.ddot_4_4(I4rt, FCFt), I4rt)
    return P, K4


def energy(F, K, mu):
    """Strain energy density W = lambda/2 tr(E)^2 + mu E:E, whose derivative
    dW/dF is P (used as an independent check of P and of P-bar)."""
    E = green_lagrange(F)
    lam = lame_lambda(K, mu)
    trE = np.trace(E)
    return 0.5 * lam * trE * trE + mu * np.einsum("ij...,ij...->...", E, E)


def tangent_apply(K4, dF):
    """(K : dF) in the convention of Eq. iter:varP: delta P^T = K : delta F^T,
    i.e. delta P_ji = K_ijkl delta F_kl.  Returns delta P ``[3,3,*grid]``."""
    return np.einsum("ijkl...,kl...->ji...", K4, dF)
