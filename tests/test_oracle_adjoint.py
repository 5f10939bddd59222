"""Pins of the oracle's adjoint gradient dJ/dmu (CPU only).

Against central finite differences of the converged P-bar with respect to
single-voxel shear moduli, the independent forward (localisation) formula,
and the envelope identity for the mean strain energy,
dW-bar/dmu_k = (1/n) devE_k : devE_k at fixed F-bar (the fluctuation
derivative vanishes at equilibrium).
"""
import numpy as np
import pytest

import synth
from oracle import adjoint, solver, svk, tensor as t

TIGHT = dict(tol_newton=1e-11, tol_cg=1e-13, cg_atol=1e-14)


def _problem(shape, mu, K=0.833):
    return solver.SVKProblem(shape, np.full(shape, K), mu)


@pytest.fixture(scope="module")
def state():
    shape = (5, 7, 5)
    rng = np.random.default_rng(3)
    mu = synth.lognormal_mu(shape, rng)
    Fbar = synth.simple_shear(0.05)
    p = _problem(shape, mu)
    p.increment(Fbar, **TIGHT)
    return shape, mu, Fbar, p, rng


@pytest.mark.parametrize("W", [np.eye(3)[[0]].T @ np.eye(3)[[1]],  # P-bar_xy
                               np.diag([1.0, 0.5, -0.3])])
def test_gradient_matches_finite_differences(state, W):
    shape, mu, Fbar, p, rng = state
    g = adjoint.grad_mu(p, W, tol_cg=1e-13, cg_atol=1e-15)
    n = mu.size
    for flat in rng.choice(n, 5, replace=False):
        idx = np.unravel_index(flat, shape)
        h = 1e-4 * mu[idx]
        vals = []
        for s in (+1, -1):
            m2 = mu.copy()
            m2[idx] += s * h
            q = _problem(shape, m2)
            q.increment(Fbar, **TIGHT)
            vals.append(np.sum(W * q.homogenized_P()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g[idx] - fd) < 1e-6 * np.abs(g).max()


def test_adjoint_equals_localization_formula(state):
    shape, mu, Fbar, p, _ = state
    W = np.zeros((3, 3))
    W[0, 1] = 1.0
    g = adjoint.grad_mu(p, W, tol_cg=1e-13, cg_atol=1e-15)
    L = adjoint.localization(p, W, tol_cg=1e-13, cg_atol=1e-15)
    d = adjoint.dP_dmu(p.F)
    g2 = np.einsum("ab...,ab...->...", L, d) / mu.size
    assert np.abs(g - g2).max() < 1e-10 * np.abs(g).max()


def test_envelope_identity_for_mean_energy(state):
    shape, mu, Fbar, p, rng = state
    E = svk.green_lagrange(p.F)
    devE = E - np.trace(E) / 3.0 * t.EYE.reshape(3, 3, 1, 1, 1)
    expected = np.einsum("ab...,ab...->...", devE, devE) / mu.size
    for flat in rng.choice(mu.size, 3, replace=False):
        idx = np.unravel_index(flat, shape)
        h = 1e-4 * mu[idx]
        vals = []
        for s in (+1, -1):
            m2 = mu.copy()
            m2[idx] += s * h
            q = _problem(shape, m2)
            q.increment(Fbar, **TIGHT)
            vals.append(np.mean(svk.energy(q.F, q.K, q.mu)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - expected[idx]) < 1e-6 * np.abs(expected).max()


def _problem_K(shape, mu, K):
    return solver.SVKProblem(shape, K, mu)


def test_bulk_gradient_matches_finite_differences(state):
    shape, mu, Fbar, p, rng = state
    W = np.diag([1.0, 0.5, -0.3])
    W[0, 1] = 0.7
    gK, gmu = adjoint.grad_params(p, W, tol_cg=1e-13, cg_atol=1e-15)
    assert np.abs(gmu - adjoint.grad_mu(p, W, tol_cg=1e-13, cg_atol=1e-15)).max() < 1e-12 * np.abs(gmu).max()
    K = np.full(shape, 0.833)
    for flat in rng.choice(mu.size, 4, replace=False):
        idx = np.unravel_index(flat, shape)
        h = 1e-4 * K[idx]
        vals = []
        for s in (+1, -1):
            K2 = K.copy()
            K2[idx] += s * h
            q = _problem_K(shape, mu, K2)
            q.increment(Fbar, **TIGHT)
            vals.append(np.sum(W * q.homogenized_P()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(gK[idx] - fd) < 1e-6 * np.abs(gK).max()


def test_bulk_envelope_identity(state):
    """dW-bar/dK_k = (1/n) (tr E_k)^2 / 2 at fixed F-bar (W = K tr^2(E)/2 + ...)."""
    shape, mu, Fbar, p, rng = state
    E = svk.green_lagrange(p.F)
    expected = 0.5 * np.trace(E) ** 2 / mu.size
    K = np.full(shape, 0.833)
    for flat in rng.choice(mu.size, 3, replace=False):
        idx = np.unravel_index(flat, shape)
        h = 1e-3 * K[idx]
        vals = []
        for s in (+1, -1):
            K2 = K.copy()
            K2[idx] += s * h
            q = _problem_K(shape, mu, K2)
            q.increment(Fbar, **TIGHT)
            vals.append(np.mean(svk.energy(q.F, q.K, q.mu)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - expected[idx]) < 1e-6 * np.abs(expected).max() + 1e-14
