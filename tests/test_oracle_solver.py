"""Pins of the oracle's CG / Newton solver (CPU only).

Independent references: a dense direct solve of the projected linear system,
the closed-form laminate solution (Kabel-type layered cell, Sec. 4.1
footnote), exact preservation of a homogeneous state (Sec. 3.1),
Hill-Mandel energy consistency, P-bar as derivative of the mean energy,
quadratic Newton convergence, and the paper's printed iteration count of its
worked example (Sec. 4.4).
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import fourier, solver, svk, tensor as t

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# absolute CG floor for tightly converged runs (FP64 round-off of G:P)
TIGHT_ATOL = 1e-13


def _problem(shape, seed, contrast=10.0, frac=0.4):
    rng = np.random.default_rng(seed)
    ph = (rng.uniform(size=shape) < frac).astype(np.uint8)
    return solver.SVKProblem.from_phase(ph, synth.two_phase_params(contrast))


def _dense_solver(shape):
    n = int(np.prod(shape))

    def lin(K4, b):
        op = solver.tangent_operator(K4)
        M = np.zeros((9 * n, 9 * n))
        Gm = np.zeros((9 * n, 9 * n))
        for k in range(9 * n):
            e = np.zeros(9 * n)
            e[k] = 1.0
            E = e.reshape((3, 3) + shape)
            M[:, k] = op(E).reshape(-1)
            Gm[:, k] = fourier.G(E).reshape(-1)
        A = M @ Gm + (np.eye(9 * n) - Gm)
        x = np.linalg.solve(A, b.reshape(-1))
        return x.reshape(b.shape), 0
    return lin


def test_cg_matches_dense_direct_solve():
    shape = (5, 5, 5)
    prob = _problem(shape, 1)
    rng = np.random.default_rng(2)
    F = synth.random_F(shape, rng, 0.05)
    _, K4 = prob.constitutive(F)
    b = fourier.G(rng.standard_normal((3, 3) + shape))
    x_cg, k, _ = solver.cg(solver.tangent_operator(K4), b, 1e-14)
    x_d, _ = _dense_solver(shape)(K4, b)
    assert k > 5
    assert np.abs(x_cg - x_d).max() < 1e-11 * np.abs(x_d).max()


def test_newton_cg_matches_newton_dense():
    shape = (5, 3, 5)
    Fbar = synth.simple_shear(0.3)
    p1 = _problem(shape, 3)
    p2 = _problem(shape, 3)
    p1.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=TIGHT_ATOL)
    p2.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=TIGHT_ATOL,
                 linear_solver=_dense_solver(shape))
    assert np.abs(p1.F - p2.F).max() < 1e-11
    assert np.abs(p1.P - p2.P).max() < 1e-11 * np.abs(p2.P).max()


def test_homogeneous_material_gives_uniform_F():
    shape = (7, 5, 3)
    prob = solver.SVKProblem(shape, 0.833, 0.386)
    Fbar = np.eye(3) + 0.1 * np.random.default_rng(4).uniform(-1, 1, (3, 3))
    st = prob.increment(Fbar)
    # the predictor alone lands on F = F-bar; the residuals are round-off
    assert st.newton_iters == 2
    assert max(st.residual) < 1e-14
    assert np.abs(prob.F - t.uniform(Fbar, shape)).max() < 1e-14
    assert np.allclose(prob.homogenized_P(), svk.stress(Fbar, 0.833, 0.386),
                       rtol=1e-14, atol=1e-16)


def _laminate_exact(Fbar, n, f1, mat1, mat0):
    """Solve (P1(F1) - P0(F0)) . n = 0 with F1 = Fbar + f0 a(x)n,
    F0 = Fbar - f1 a(x)n, for the vector a (3 equations)."""
    f0 = 1.0 - f1

    def res(a):
        F1 = Fbar + f0 * np.outer(a, n)
        F0 = Fbar - f1 * np.outer(a, n)
        return (svk.stress(F1, *mat1) - svk.stress(F0, *mat0)) @ n

    a = np.zeros(3)
    for _ in range(50):
        r = res(a)
        if np.abs(r).max() < 1e-15:
            break
        J = np.zeros((3, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-7
            J[:, k] = (res(a + e) - res(a - e)) / 2e-7
        a = a - np.linalg.solve(J, r)
    F1 = Fbar + f0 * np.outer(a, n)
    F0 = Fbar - f1 * np.outer(a, n)
    return F1, F0


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_laminate_closed_form(axis):
    shape = [5, 5, 5]
    shape[axis] = 9
    shape = tuple(shape)
    ph = synth.laminate(shape, axis, fraction=4 / 9)
    params = synth.two_phase_params(5.0)
    prob = solver.SVKProblem.from_phase(ph, params)
    Fbar = np.eye(3) + np.array([[0.05, 0.2, -0.03],
                                 [0.01, -0.04, 0.1],
                                 [0.02, 0.03, 0.06]])
    prob.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=TIGHT_ATOL)
    n = np.zeros(3)
    n[axis] = 1.0
    f1 = ph.mean()
    F1, F0 = _laminate_exact(Fbar, n, f1, tuple(params[1]), tuple(params[0]))
    exact = np.where(ph[None, None] == 1, F1[:, :, None, None, None],
                     F0[:, :, None, None, None])
    assert np.abs(prob.F - exact).max() < 1e-10


def test_hill_mandel_and_mean_deformation():
    shape = (7, 7, 7)
    prob = _problem(shape, 7, contrast=8.0)
    Fbar = np.eye(3) + np.array([[0.1, 0.05, 0], [0, -0.02, 0.03], [0.04, 0, 0.0]])
    prob.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=TIGHT_ATOL)
    assert np.abs(t.grid_mean(prob.F) - Fbar).max() < 1e-14
    lhs = np.mean(np.einsum("ij...,ij...->...", prob.P, prob.F))
    Pbar = prob.homogenized_P()
    rhs = np.sum(Pbar * Fbar)
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)


def test_homogenized_stress_is_derivative_of_mean_energy():
    shape = (5, 5, 5)
    base = np.eye(3) + np.array([[0.05, 0.1, 0], [0, 0.02, 0], [0, 0, -0.03]])
    prob = _problem(shape, 9, contrast=6.0)
    prob.increment(base, tol_newton=1e-10, tol_cg=1e-12, cg_atol=TIGHT_ATOL)
    Pbar = prob.homogenized_P()
    h = 1e-5
    for (a, b) in [(0, 1), (2, 2), (1, 0)]:
        vals = []
        for s in (+1, -1):
            q = _problem(shape, 9, contrast=6.0)
            Fb = base.copy()
            Fb[a, b] += s * h
            q.increment(Fb, tol_newton=1e-10, tol_cg=1e-12, cg_atol=TIGHT_ATOL)
            vals.append(np.mean(svk.energy(q.F, q.K, q.mu)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - Pbar[a, b]) < 1e-7 * np.abs(Pbar).max()


def test_newton_converges_quadratically():
    prob = solver.SVKProblem.from_phase(synth.cube_inclusion(11, 4),
                                        synth.two_phase_params(10.0))
    st = prob.increment(synth.simple_shear(0.6), tol_newton=1e-10, tol_cg=1e-12, cg_atol=TIGHT_ATOL)
    e = st.rel_update
    pairs = [(e[k], e[k + 1]) for k in range(len(e) - 1) if 1e-9 < e[k] < 1e-2]
    assert pairs, e
    for ek, ek1 in pairs:
        assert ek1 < 50.0 * ek * ek


def test_paper_example_iteration_count():
    """Sec. 4.4: the printed example converges in five Newton iterations."""
    g = json.load(open(os.path.join(GOLDEN, "paper_e1.json")))
    n = g["grid"]
    prob = solver.SVKProblem.from_phase(synth.cube_inclusion(n, 9),
                                        synth.two_phase_params(10.0))
    st = prob.increment(synth.simple_shear(g["gamma"]), tol_newton=1e-5,
                        tol_cg=1e-8)
    assert abs(st.newton_iters - g["newton_iterations"]) <= g["newton_iterations_tolerance"]
    # the prescribed macroscopic deformation is held exactly (Eq. mean:zero)
    assert np.abs(t.grid_mean(prob.F) - synth.simple_shear(1.0)).max() < 1e-13


# ---- even grids (Appendix C: Nyquist frequencies of G-hat zeroed) ----

def test_even_grid_newton_cg_matches_newton_dense():
    shape = (4, 3, 4)
    Fbar = synth.simple_shear(0.2)
    p1 = _problem(shape, 5)
    p2 = _problem(shape, 5)
    p1.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=TIGHT_ATOL)
    p2.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=TIGHT_ATOL,
                 linear_solver=_dense_solver(shape))
    assert np.abs(p1.F - p2.F).max() < 1e-11
    # F stays compatible: no Nyquist content in its fluctuation
    Fh = np.fft.fftn(p1.F - t.uniform(Fbar, shape), axes=(-3, -2, -1))
    assert np.abs(Fh[:, :, fourier.nyquist_mask(shape)]).max() < 1e-12


def test_even_grid_laminate_closed_form():
    """Layers of even thickness on an even grid: the exact piecewise-constant
    solution has no Nyquist content, so the Appendix C projection reproduces
    it exactly."""
    shape = (8, 4, 6)
    ph = synth.laminate(shape, 0, fraction=0.5)
    params = synth.two_phase_params(5.0)
    prob = solver.SVKProblem.from_phase(ph, params)
    Fbar = np.eye(3) + np.array([[0.05, 0.2, -0.03], [0.01, -0.04, 0.1], [0.02, 0.03, 0.06]])
    prob.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=TIGHT_ATOL)
    F1, F0 = _laminate_exact(Fbar, np.eye(3)[0], ph.mean(), tuple(params[1]), tuple(params[0]))
    exact = np.where(ph[None, None] == 1, F1[:, :, None, None, None], F0[:, :, None, None, None])
    assert np.abs(prob.F - exact).max() < 1e-10
