"""Mixed macroscopic control: some components of P-bar prescribed, the others
of F-bar (TEST INFRASTRUCTURE, see the package docstring).

Not in the paper: Sec. 3.1 prescribes the full F-bar and leaves the general
case to the literature.  Reading used here:

* A mask selects the stress-controlled components c = 3i+j: P-bar_c is
  prescribed and F-bar_c is unknown; every other component has F-bar_c
  prescribed.  The state sought is the equilibrium G:P(F) = 0 of one
  increment from the committed state (history frozen there, as in
  Algorithm 1) with <F>_c = F-bar_c on the strain-controlled components and
  <P>_c = P*_c on the stress-controlled ones.
* It is reached by Newton on the free macroscopic components.  Every iterate
  is an ordinary increment (Sec. 3.1 predictor, Algorithm 1) to the current
  F-bar.  The Jacobian is the homogenised tangent: differentiating
  G:P(F-bar + F~) = 0 with respect to F-bar_b gives G:K:(E_b + dF_b) = 0,
  i.e. the predictor system Eq. bc:lin with dF-bar = E_b (E_b the uniform
  unit tensor of component b), and
      dP-bar_a / dF-bar_b = < K : (E_b + dF_b) >_a.
* The free components start from their committed values; the iteration
  stops when ||P-bar_S - P*_S|| <= tol_stress ||P-bar|| (Frobenius norms),
  checked after each increment.
"""
from __future__ import annotations

import numpy as np

from . import fourier, solver, tensor as t
from .svk import tangent_apply


def unit_field(c, grid):
    """Uniform field whose component c = 3i+j is 1, all others 0."""
    E = np.zeros(9)
    E[c] = 1.0
    return t.uniform(E.reshape(3, 3), grid)


def homogenized_tangent(K4, cols, tol_cg=1e-12, cg_atol=0.0):
    """Columns b in ``cols`` of dP-bar/dF-bar at an equilibrium state with
    tangent K4: [9][len(cols)], row a = component 3i+j of P-bar.  One solve
    of Eq. bc:lin per column (right-hand side -G:K:E_b)."""
    grid = K4.shape[-3:]
    op = solver.tangent_operator(K4)
    C = np.zeros((9, len(cols)))
    for k, b in enumerate(cols):
        E = unit_field(b, grid)
        x, _, _ = solver.cg(op, -op(E), tol_cg, atol=cg_atol)
        C[:, k] = t.grid_mean(tangent_apply(K4, E + x)).reshape(9)
    return C


def _commit(problem, F, P):
    mat = getattr(problem, "mat", None)
    if mat is not None:
        mat.commit()   # history of the last constitutive call (at F)
    problem.F, problem.P = F, P


def solve_mixed(problem, Fbar, Pbar, mask, tol_stress=1e-10, tol_newton=1e-5,
                tol_cg=1e-8, max_macro=30, tangent_tol_cg=1e-12, **kw):
    """One increment under mixed control from the committed state of
    ``problem`` (an SVKProblem or J2Problem); commits the converged state.
    Returns (F-bar reached, macro iterations, increment stats list)."""
    mask = np.asarray(mask, dtype=bool).reshape(9)
    S = np.flatnonzero(mask)
    Fb = np.asarray(Fbar, dtype=np.float64).reshape(9).copy()
    Pt = np.asarray(Pbar, dtype=np.float64).reshape(9)
    Fb[S] = t.grid_mean(problem.F).reshape(9)[S]
    F = problem.F
    stats = []
    for m in range(1, max_macro + 1):
        F, P, K4, st = solver.solve_increment(F, Fb.reshape(3, 3), problem.constitutive,
                                              tol_newton, tol_cg, **kw)
        stats.append(st)
        Pb = t.grid_mean(P).reshape(9)
        R = Pb[S] - Pt[S]
        if len(S) == 0 or solver.norm(R) <= tol_stress * solver.norm(Pb):
            _commit(problem, F, P)
            return Fb.reshape(3, 3), m, stats
        C = homogenized_tangent(K4, S, tangent_tol_cg, kw.get("cg_atol", 0.0))
        Fb[S] -= np.linalg.solve(C[S, :], R)
    raise solver.SolverError("mixed control: macroscopic Newton did not converge")


def solve_mixed_path(problem, Fbar, Pbar, mask, fractions, **kw):
    """Increments of ``solve_mixed`` along the straight path from the
    committed (F-bar, P-bar) to (Fbar, Pbar) on the controlled components,
    ending at each of ``fractions`` (increasing, the last one 1)."""
    mask = np.asarray(mask, dtype=bool).reshape(9)
    F0 = t.grid_mean(problem.F).reshape(9)
    P0 = t.grid_mean(problem.P).reshape(9)
    F1 = np.asarray(Fbar, dtype=np.float64).reshape(9)
    P1 = np.asarray(Pbar, dtype=np.float64).reshape(9)
    out = None
    for s in fractions:
        Fb = F1 if s >= 1.0 else F0 + s * (F1 - F0)
        Pb = P1 if s >= 1.0 else P0 + s * (P1 - P0)
        out = solve_mixed(problem, Fb, Pb, mask, **kw)
    return out
