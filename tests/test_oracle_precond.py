"""Pins of the oracle's reference-medium preconditioned CG (CPU only).

Independent references: the closed-form inverse of the isotropic acoustic
tensor (per frequency, Gamma0-hat B = (N0^-1 B xi / |xi|^2) (x) xi with
N0 = mu0 I + (lam0 + mu0) n (x) n); Gamma0 inverting K0 on compatible
fields; convergence in one iteration when the tangent is the reference
medium itself; a dense direct solve of the projected system; Newton with
PCG against Newton with plain CG.
"""
import numpy as np
import pytest

import synth
from oracle import fourier, precond, solver, svk, tensor as t


def test_gamma0_matches_acoustic_tensor_closed_form():
    grid = (5, 6, 7)   # even axis: Nyquist frequencies are zero like G-hat
    lam0, mu0 = 0.6, 0.4
    gh = precond.gamma0_hat(grid, lam0, mu0)
    xi = fourier.scaled_frequencies(grid)
    n2 = (xi * xi).sum(0)
    keep = (n2 > 0) & ~fourier.nyquist_mask(grid)
    c = (lam0 + mu0) / (lam0 + 2 * mu0)
    for idx in np.ndindex(*grid):
        G = gh[(slice(None), slice(None)) + idx]
        if not keep[idx]:
            assert not G.any()
            continue
        q = xi[(slice(None),) + idx]
        nn = np.outer(q, q) / n2[idx]
        Ninv = (np.eye(3) - c * nn) / mu0
        ref = np.einsum("ik,l,j->ijkl", Ninv, q, q).reshape(9, 9) / n2[idx]
        assert np.abs(G - ref).max() < 1e-12 * np.abs(ref).max()


def test_gamma0_inverts_the_reference_medium_on_compatible_fields():
    grid = (7, 5, 9)
    lam0, mu0 = 1.3, 0.7
    A = fourier.G(np.random.default_rng(1).standard_normal((3, 3) + grid))
    K0 = precond.k0_matrix(lam0, mu0)
    KA = np.einsum("ab,b...->a...", K0, A.reshape((9,) + grid)).reshape((3, 3) + grid)
    assert np.abs(precond.gamma0(KA, lam0, mu0) - A).max() < 1e-12 * np.abs(A).max()


def _two_phase(shape, seed, contrast):
    rng = np.random.default_rng(seed)
    ph = (rng.uniform(size=shape) < 0.4).astype(np.uint8)
    params = synth.two_phase_params(contrast)
    prob = solver.SVKProblem.from_phase(ph, params)
    lam = svk.lame_lambda(prob.K, prob.mu)
    return prob, precond.reference_medium(lam, prob.mu)


def test_pcg_converges_in_one_iteration_on_the_reference_medium():
    grid = (5, 7, 3)
    K, mu = 0.833, 0.386
    prob = solver.SVKProblem(grid, K, mu)
    _, K4 = prob.constitutive(t.uniform(np.eye(3), grid))   # tangent at F = I is K0
    lam0 = svk.lame_lambda(K, mu)
    b = fourier.G(np.random.default_rng(2).standard_normal((3, 3) + grid))
    op = solver.tangent_operator(K4)
    x, k = precond.pcg(op, b, lambda r: precond.gamma0(r, lam0, mu), 1e-12)
    assert k == 1
    assert np.abs(op(x) - b).max() < 1e-13 * np.abs(b).max()


def test_pcg_matches_dense_direct_solve():
    grid = (5, 5, 5)
    prob, (lam0, mu0) = _two_phase(grid, 3, 20.0)
    rng = np.random.default_rng(4)
    _, K4 = prob.constitutive(synth.random_F(grid, rng, 0.05))
    b = fourier.G(rng.standard_normal((3, 3) + grid))
    n = int(np.prod(grid))
    op = solver.tangent_operator(K4)
    M = np.zeros((9 * n, 9 * n))
    Gm = np.zeros((9 * n, 9 * n))
    for k in range(9 * n):
        e = np.zeros(9 * n)
        e[k] = 1.0
        E = e.reshape((3, 3) + grid)
        M[:, k] = op(E).reshape(-1)
        Gm[:, k] = fourier.G(E).reshape(-1)
    x_d = np.linalg.solve(M @ Gm + (np.eye(9 * n) - Gm), b.reshape(-1)).reshape(b.shape)
    gh = precond.gamma0_hat(grid, lam0, mu0)
    x, k = precond.pcg(op, b, lambda r: precond.gamma0(r, lam0, mu0, gh), 1e-14)
    assert k > 3
    assert np.abs(x - x_d).max() < 1e-11 * np.abs(x_d).max()


def test_newton_with_pcg_matches_newton_with_cg_and_needs_fewer_iterations():
    grid = (9, 7, 11)
    p1, (lam0, mu0) = _two_phase(grid, 5, 100.0)
    p2, _ = _two_phase(grid, 5, 100.0)
    Fbar = synth.simple_shear(0.05)
    st1 = p1.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=1e-13)
    st2 = p2.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12,
                       linear_solver=precond.linear_solver(grid, lam0, mu0, 1e-12, 1e-14))
    assert np.abs(p1.F - p2.F).max() < 1e-11
    assert np.abs(p1.P - p2.P).max() < 1e-11 * np.abs(p1.P).max()
    assert sum(st2.cg_iters) < 0.8 * sum(st1.cg_iters)
