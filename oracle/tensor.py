"""Tensor algebra on voxel grids, following the nomenclature of Appendix A.

Tensors are stored component-first: a second-order field is ``[3, 3, *grid]``
and a fourth-order field ``[3, 3, 3, 3, *grid]``.  Constant tensors (no grid
axes) broadcast against grid tensors.

Appendix A conventions used throughout:
  (A . B)_ik   = A_ij B_jk                     single contraction
  (A : B)      = A_ij B_ji                     double contraction (scalar)
  (A4 : B)_ij  = A_ijkl B_lk
  (A4 : B4)_ijmn = A_ijkl B_lkmn
  (A . B4)_ikmn = A_ij B_jkmn
  (A4 . B)_ijkm = A_ijkl B_lm
  (A x B)_ijkl = A_ij B_kl                      dyadic product
  I4_ijkl = d_il d_jk,  I4rt_ijkl = d_ik d_jl,  I4s = (I4 + I4rt)/2
"""
import numpy as np

EYE = np.eye(3)


def T2(A):
    """Transpose of a second-order tensor: C_ji = A_ij."""
    return np.swapaxes(A, 0, 1)


def dot_2_2(A, B):
    """C_ik = A_ij B_jk."""
    return np.einsum("ij...,jk...->ik...", A, B)


def ddot_4_2(A, B):
    """C_ij = A_ijkl B_lk."""
    return np.einsum("ijkl...,lk...->ij...", A, B)


def ddot_4_4(A, B):
    """C_ijmn = A_ijkl B_lkmn."""
    return np.einsum("ijkl...,lkmn...->ijmn...", A, B)


def dot_2_4(A, B):
    """C_ikmn = A_ij B_jkmn."""
    return np.einsum("ij...,jkmn...->ikmn...", A, B)


def dot_4_2(A, B):
    """C_ijkm = A_ijkl B_lm."""
    return np.einsum("ijkl...,lm...->ijkm...", A, B)


def dyad_2_2(A, B):
    """C_ijkl = A_ij B_kl."""
    return np.einsum("ij...,kl...->ijkl...", A, B)


def identity4():
    """Fourth-order identity: I4_ijkl = d_il d_jk (so that I4 : A = A)."""
    return np.einsum("il,jk->ijkl", EYE, EYE)


def identity4_rt():
    """Right-transposed identity: I4rt_ijkl = d_ik d_jl (I4rt : A = A^T)."""
    return np.einsum("ik,jl->ijkl", EYE, EYE)


def identity4_sym():
    """Symmetrisation tensor (I4 + I4rt)/2."""
    return 0.5 * (identity4() + identity4_rt())


def grid_mean(A):
    """Volume average over the trailing three grid axes (trapezoidal rule,
    Sec. 2.5: every node carries the same weight)."""
    return A.mean(axis=(-3, -2, -1))


def uniform(A, grid_shape):
    """Broadcast a constant tensor onto a grid (a copy)."""
    A = np.asarray(A, dtype=np.float64)
    return np.broadcast_to(A.reshape(A.shape + (1, 1, 1)),
                           A.shape + tuple(grid_shape)).copy()
