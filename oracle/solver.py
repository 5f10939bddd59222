"""Conjugate gradients, Newton iterations and the incremental loop.

Follows Sec. 2.6 (Eq. iter:F, iter:varP, iter:system), Sec. 3.1 (boundary
condition predictor, Eq. bc:lin), Algorithm 1 and the order of operations of
the paper's printed example (Appendix B).  Readings:

* CG (the paper calls scipy's ``cg`` with ``tol``): x0 = 0, stop as soon as
  ||r_k||_2 <= max(eta_CG ||b||_2, atol); if ||b|| = 0 return x = 0 without
  iterating.  The iteration count is the number of operator applications.  As in the
  library routine the paper calls, the sign of p.Ap is not tested: the
  consistent tangent of the J2 model (Sec. 5) with low hardening can be
  mildly indefinite on some compatible directions (geometric stress terms of
  the size of the plastic modulus), where CG still converges; only an exact
  zero or a non-finite p.Ap stops it.
  ``atol`` defaults to 0 (the paper's purely relative test).  It exists for
  tightly converged reference runs: once Newton has converged far, ||b|| is
  so small that the FP64 round-off of G:P (about 1e-16 ||P||) is no longer
  negligible relative to it, and a purely relative test can never be met.
* Convergence test of Algorithm 1: its printed ">" is read as "<" (the
  listing breaks when ||dF||/||F|| < eta_NW and i > 0).  ||.|| is the
  Frobenius norm over all 9n entries and ||F|| is taken once per increment,
  right after the macroscopic increment is added.
* The predictor tangent is the one of the last converged state.
* P-bar is the voxel average of P (the average over Omega_0, Sec. 3.1).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fourier, tensor as t


class SolverError(RuntimeError):
    pass


def norm(A):
    return float(np.sqrt(np.sum(np.asarray(A) ** 2)))


def vdot(A, B):
    return float(np.sum(np.asarray(A) * np.asarray(B)))


def cg(apply_A, b, tol, maxiter=10_000, atol=0.0):
    """Plain conjugate gradients on a symmetric operator restricted to the
    range of G (Sec. 2.6).  Returns (x, iterations, residual history)."""
    x = np.zeros_like(b)
    bnorm = norm(b)
    hist = []
    if bnorm == 0.0:
        return x, 0, hist
    r = b.copy()
    p = r.copy()
    rr = vdot(r, r)
    for k in range(1, maxiter + 1):
        Ap = apply_A(p)
        pAp = vdot(p, Ap)
        if pAp == 0.0 or not np.isfinite(pAp):
            raise SolverError("CG breakdown: p.Ap = 0 or not finite")
        alpha = rr / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = vdot(r, r)
        hist.append(np.sqrt(rr_new) / bnorm)
        if np.sqrt(rr_new) <= max(tol * bnorm, atol):
            return x, k, hist
        beta = rr_new / rr
        rr = rr_new
        p = r + beta * p
    raise SolverError("CG did not converge")


def tangent_operator(K4):
    """v -> G : (K : v) with the tangent convention of Eq. iter:varP."""
    from .svk import tangent_apply

    def op(v):
        return fourier.G(tangent_apply(K4, v))
    return op


@dataclasses.dataclass
class IncrementStats:
    newton_iters: int = 0
    cg_iters: list = dataclasses.field(default_factory=list)
    rel_update: list = dataclasses.field(default_factory=list)
    residual: list = dataclasses.field(default_factory=list)


def solve_increment(F0, Fbar, constitutive, tol_newton=1e-5, tol_cg=1e-8,
                    max_newton=50, max_cg=10_000, linear_solver=None,
                    cg_atol=0.0):
    """One load increment (Algorithm 1, inner loop).

    ``constitutive(F) -> (P, K4)`` evaluates the material at F with the
    committed history.  ``linear_solver(K4, b)`` may replace CG (used to
    cross-check CG with a dense direct solve); it returns (x, iterations).

    Returns (F, P, K4, stats).
    """
    grid = F0.shape[-3:]
    st = IncrementStats()
    P, K4 = constitutive(F0)                      # tangent at F_(0)
    dFbar = t.uniform(np.asarray(Fbar) - t.grid_mean(F0), grid)

    def solve(K4, b):
        if linear_solver is not None:
            return linear_solver(K4, b)
        x, k, _ = cg(tangent_operator(K4), b, tol_cg, max_cg, cg_atol)
        return x, k

    b = -tangent_operator(K4)(dFbar)              # Eq. bc:lin right-hand side
    F = F0 + dFbar
    Fn = norm(F)
    i = 0
    while True:
        dF, k = solve(K4, b)                      # Eq. iter:system / bc:lin
        st.cg_iters.append(k)
        F = F + dF                                # Eq. iter:F
        P, K4 = constitutive(F)
        b = -fourier.G(P)                         # residual -G:P
        st.residual.append(norm(b))
        rel = norm(dF) / Fn
        st.rel_update.append(rel)
        st.newton_iters = i + 1
        if not np.isfinite(rel):
            raise SolverError("non-finite Newton update")
        if rel < tol_newton and i > 0:
            break
        # divergence: an update larger than half of F, or updates that grew
        # in two consecutive equilibrium iterations
        e = st.rel_update
        if rel > 0.5 or (i >= 3 and e[-1] > e[-2] > e[-3]):
            raise SolverError("Newton diverged")
        i += 1
        if i >= max_newton:
            raise SolverError("Newton did not converge")
    return F, P, K4, st


def homogenized(P):
    """P-bar = <P> (voxel average)."""
    return t.grid_mean(P)


class SVKProblem:
    """A periodic cell of Saint Venant-Kirchhoff material (Sec. 4)."""

    def __init__(self, shape, K, mu):
        self.shape = tuple(shape)
        self.K = np.broadcast_to(np.asarray(K, dtype=np.float64), self.shape)
        self.mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), self.shape)
        self.F = t.uniform(np.eye(3), self.shape)  # F_(0) = I
        self.P = np.zeros((3, 3) + self.shape)
        self.stats = []

    @classmethod
    def from_phase(cls, phase, phase_params):
        params = np.asarray(phase_params, dtype=np.float64)
        return cls(phase.shape, params[phase, 0], params[phase, 1])

    def constitutive(self, F):
        from . import svk
        return svk.constitutive(F, self.K, self.mu)

    def increment(self, Fbar, tol_newton=1e-5, tol_cg=1e-8, **kw):
        F, P, _, st = solve_increment(self.F, Fbar, self.constitutive,
                                      tol_newton, tol_cg, **kw)
        self.F, self.P = F, P                     # store converged state
        self.stats.append(st)
        return st

    def homogenized_P(self):
        return homogenized(self.P)


class J2Problem:
    """A periodic cell of finite-strain J2 material (Sec. 5) with history."""

    def __init__(self, shape, K, mu, ty0, H):
        from . import j2
        self.shape = tuple(shape)
        self.mat = j2.J2Material(self.shape, K, mu, ty0, H)
        self.F = t.uniform(np.eye(3), self.shape)
        self.P = np.zeros((3, 3) + self.shape)
        self.stats = []

    @classmethod
    def from_phase(cls, phase, phase_params):
        p = np.asarray(phase_params, dtype=np.float64)
        return cls(phase.shape, p[phase, 0], p[phase, 1], p[phase, 2], p[phase, 3])

    def constitutive(self, F):
        return self.mat.constitutive(F)

    def increment(self, Fbar, tol_newton=1e-5, tol_cg=1e-8, **kw):
        F, P, _, st = solve_increment(self.F, Fbar, self.constitutive,
                                      tol_newton, tol_cg, **kw)
        # the last constitutive call was at the converged F: store its
        # history (Algorithm 1, "store history variables")
        self.mat.commit()
        self.F, self.P = F, P
        self.stats.append(st)
        return st

    def homogenized_P(self):
        return homogenized(self.P)


def solve_step(problem, Fbar, tol_newton=1e-5, tol_cg=1e-8, max_cuts=8, **kw):
    """Load step to the absolute Fbar along the straight path from the last
    committed macroscopic deformation; a failed increment is rolled back and
    retried with half the step, and after a success the step doubles again
    (up to the remainder).  Not in the paper (its examples use fixed small
    increments); the J2 switch of Sec. 5.3 makes full Newton steps diverge
    when an increment crosses the yield point by far.  Returns
    (increments solved, halvings)."""
    F0 = t.grid_mean(problem.F)
    target = np.asarray(Fbar, dtype=np.float64)
    done, step, cuts, sub = 0.0, 1.0, 0, 0
    while done < 1.0:
        to = min(1.0, done + step)
        Fb = target if to >= 1.0 else F0 + to * (target - F0)
        saved = (problem.F, problem.P, getattr(problem, "mat", None) and
                 (problem.mat.Cpi.copy(), problem.mat.ep.copy()))
        try:
            problem.increment(Fb, tol_newton, tol_cg, **kw)
        except SolverError:
            problem.F, problem.P = saved[0], saved[1]
            if saved[2]:
                problem.mat.Cpi, problem.mat.ep = saved[2]
            cuts += 1
            if cuts > max_cuts:
                raise
            step *= 0.5
            continue
        done = to
        sub += 1
        step = min(2.0 * step, 1.0)
    return sub, cuts
