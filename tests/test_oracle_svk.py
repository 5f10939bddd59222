"""Pins of the oracle's Saint Venant-Kirchhoff model (CPU only).

Checks against what the mathematics fixes independently of the formulas
being tested: the tangent is the derivative of P (central differences), P is
the derivative of the strain energy, objectivity, the major symmetry that a
hyper-elastic tangent must have, and the small-strain limit (linear
isotropic elasticity).
"""
import numpy as np
import pytest

import synth
from oracle import svk, tensor as t


@pytest.fixture
def state():
    rng = np.random.default_rng(11)
    shape = (3, 5, 7)
    F = synth.random_F(shape, rng, 0.3)
    K = rng.uniform(0.5, 3.0, shape)
    mu = rng.uniform(0.2, 1.5, shape)
    return F, K, mu, rng


def test_tangent_is_derivative_of_stress(state):
    F, K, mu, rng = state
    _, K4 = svk.constitutive(F, K, mu)
    for _ in range(3):
        dF = rng.standard_normal(F.shape)
        h = 1e-6
        fd = (svk.stress(F + h * dF, K, mu) - svk.stress(F - h * dF, K, mu)) / (2 * h)
        got = svk.tangent_apply(K4, dF)
        assert np.abs(got - fd).max() < 1e-8 * np.abs(fd).max()


def test_stress_is_derivative_of_energy(state):
    F, K, mu, _ = state
    P = svk.stress(F, K, mu)
    h = 1e-6
    for i in range(3):
        for j in range(3):
            Fp, Fm = F.copy(), F.copy()
            Fp[i, j] += h
            Fm[i, j] -= h
            fd = (svk.energy(Fp, K, mu) - svk.energy(Fm, K, mu)) / (2 * h)
            assert np.abs(fd - P[i, j]).max() < 1e-8 * np.abs(P).max()


def test_constitutive_stress_matches_direct_formula(state):
    F, K, mu, _ = state
    P, _ = svk.constitutive(F, K, mu)
    assert np.abs(P - svk.stress(F, K, mu)).max() < 1e-14 * np.abs(P).max()


def test_tangent_major_symmetry(state):
    F, K, mu, _ = state
    _, K4 = svk.constitutive(F, K, mu)
    # K_ijkl = K_lkji (fourth-order transpose of Appendix A)
    K4T = np.einsum("ijkl...->lkji...", K4)
    assert np.abs(K4 - K4T).max() < 1e-13 * np.abs(K4).max()


def test_objectivity(state):
    F, K, mu, rng = state
    # random rotation
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    RF = np.einsum("ij,jk...->ik...", Q, F)
    P = svk.stress(F, K, mu)
    P_rot = svk.stress(RF, K, mu)
    assert np.abs(P_rot - np.einsum("ij,jk...->ik...", Q, P)).max() < 1e-13


def test_small_strain_limit_is_linear_elasticity():
    K, mu = 1.7, 0.6
    lam = K - 2 * mu / 3
    rng = np.random.default_rng(5)
    H = rng.standard_normal((3, 3))
    for eps in (1e-3, 1e-4):
        F = np.eye(3) + eps * H
        P = svk.stress(F, K, mu)
        e = 0.5 * (H + H.T) * eps
        lin = lam * np.trace(e) * np.eye(3) + 2 * mu * e
        # the error is second order in eps
        assert np.abs(P - lin).max() < 10 * eps ** 2 * (abs(lam) + mu) * np.abs(H).max() ** 2
    # no stress in the reference state
    assert np.abs(svk.stress(np.eye(3), K, mu)).max() == 0.0
    # at F = I the tangent reduces to the isotropic stiffness
    _, K4 = svk.constitutive(np.eye(3), K, mu)
    dP = svk.tangent_apply(K4, H)
    e = 0.5 * (H + H.T)
    assert np.allclose(dP, lam * np.trace(e) * np.eye(3) + 2 * mu * e, atol=1e-14)
