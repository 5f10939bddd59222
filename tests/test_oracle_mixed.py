"""Pins of the oracle's mixed stress / deformation control (CPU only).

Independent references: the closed-form uniaxial-stress response of a
homogeneous Saint Venant-Kirchhoff cell (Poisson contraction of the Green
strain) and of a homogeneous J2 cell loaded from the virgin state (1-D
linear hardening in logarithmic strain); the layered cell under mixed
control solved as a small dense system (traction continuity across the
layers plus the prescribed mean stress); the homogenised tangent against
central differences of P-bar over fully solved increments; and the
reduction to an ordinary increment when nothing is stress-controlled.
"""
import numpy as np
import pytest

import synth
from oracle import mixed, solver, svk, tensor as t

TIGHT = dict(tol_newton=1e-11, tol_cg=1e-12, cg_atol=1e-13)


def test_uniaxial_stress_svk_homogeneous_closed_form():
    K, mu = 0.833, 0.386
    shape = (3, 5, 3)
    prob = solver.SVKProblem(shape, K, mu)
    l1 = 1.06
    Fbar = np.eye(3)
    Fbar[0, 0] = l1
    Fb, m, _ = mixed.solve_mixed(prob, Fbar, np.zeros((3, 3)), synth.uniaxial_stress_mask(),
                                 tol_stress=1e-13, **TIGHT)
    lam = K - 2.0 * mu / 3.0
    nu = lam / (2.0 * (lam + mu))                 # Poisson ratio of the Green strain
    Ey = mu * (3.0 * lam + 2.0 * mu) / (lam + mu)
    e1 = 0.5 * (l1 * l1 - 1.0)
    l2 = np.sqrt(1.0 - 2.0 * nu * e1)
    exact = np.diag([l1, l2, l2])
    assert m >= 2
    assert np.abs(Fb - exact).max() < 1e-12
    assert np.abs(prob.F - t.uniform(exact, shape)).max() < 1e-12
    Pb = prob.homogenized_P()
    assert abs(Pb[0, 0] - l1 * Ey * e1) < 1e-12
    assert np.abs(Pb.reshape(9)[synth.uniaxial_stress_mask()]).max() < 1e-13


def test_uniaxial_stress_j2_homogeneous_closed_form():
    """One plastic increment from the virgin state under uniaxial Kirchhoff
    stress: principal axes fixed, so the radial return in logarithmic strain
    is exact and reduces to 1-D linear hardening."""
    K, mu, ty0, H = 1.0 / 1.2, 1.0 / 2.6, 0.003, 0.01
    shape = (3, 3, 3)
    prob = solver.J2Problem(shape, K, mu, ty0, H)
    e1 = 0.02
    Fbar = np.eye(3)
    Fbar[0, 0] = np.exp(e1)
    Fb, _, _ = mixed.solve_mixed(prob, Fbar, np.zeros((3, 3)), synth.uniaxial_stress_mask(),
                                 tol_stress=1e-13, **TIGHT)
    Ey = 9.0 * K * mu / (3.0 * K + mu)
    nu = (3.0 * K - 2.0 * mu) / (2.0 * (3.0 * K + mu))
    assert Ey * e1 > ty0                          # the increment yields
    sig = (ty0 + H * e1) / (1.0 + H / Ey)         # axial Kirchhoff stress
    ep = e1 - sig / Ey
    e2 = -nu * sig / Ey - 0.5 * ep                # lateral logarithmic strain
    exact = np.diag([np.exp(e1), np.exp(e2), np.exp(e2)])
    assert np.abs(Fb - exact).max() < 1e-12
    Pb = prob.homogenized_P()
    assert abs(Pb[0, 0] - sig / np.exp(e1)) < 1e-12   # P = tau F^-T
    assert np.allclose(prob.mat.ep, ep, rtol=0, atol=1e-12)


def _laminate_mixed_exact(Fbar, Pt, mask, nrm, f1, mat1, mat0):
    """Unknowns: the jump vector a and the free F-bar components; equations:
    (P1 - P0) . n = 0 and (f1 P1 + f0 P0)_S = P*_S, with
    F1 = F-bar + f0 a (x) n, F0 = F-bar - f1 a (x) n."""
    f0 = 1.0 - f1
    S = np.flatnonzero(mask)

    def unpack(u):
        Fb = np.asarray(Fbar, dtype=np.float64).reshape(9).copy()
        Fb[S] = u[3:]
        Fb = Fb.reshape(3, 3)
        a = u[:3]
        return Fb + f0 * np.outer(a, nrm), Fb - f1 * np.outer(a, nrm)

    def res(u):
        F1, F0 = unpack(u)
        P1, P0 = svk.stress(F1, *mat1), svk.stress(F0, *mat0)
        return np.concatenate([(P1 - P0) @ nrm, (f1 * P1 + f0 * P0).reshape(9)[S] - Pt[S]])

    u = np.concatenate([np.zeros(3), np.asarray(Fbar, dtype=np.float64).reshape(9)[S]])
    for _ in range(60):
        r = res(u)
        if np.abs(r).max() < 1e-15:
            break
        J = np.zeros((len(u), len(u)))
        for k in range(len(u)):
            e = np.zeros(len(u))
            e[k] = 1e-7
            J[:, k] = (res(u + e) - res(u - e)) / 2e-7
        u = u - np.linalg.solve(J, r)
    return unpack(u)


@pytest.mark.parametrize("axis", [0, 1])
def test_laminate_mixed_closed_form(axis):
    shape = [5, 5, 5]
    shape[axis] = 9
    shape = tuple(shape)
    ph = synth.laminate(shape, axis, fraction=4 / 9)
    params = synth.two_phase_params(5.0)
    prob = solver.SVKProblem.from_phase(ph, params)
    mask = synth.uniaxial_stress_mask()
    Fbar = np.eye(3)
    Fbar[0, 0] = 1.04
    Fbar[1, 0] = 0.01
    Pt = np.zeros(9)
    Pt[4] = 0.002            # some lateral tension besides the free components
    mixed.solve_mixed(prob, Fbar, Pt, mask, tol_stress=1e-13, **TIGHT)
    nrm = np.eye(3)[axis]
    F1, F0 = _laminate_mixed_exact(Fbar, Pt, mask, nrm, ph.mean(), tuple(params[1]),
                                   tuple(params[0]))
    exact = np.where(ph[None, None] == 1, F1[:, :, None, None, None],
                     F0[:, :, None, None, None])
    assert np.abs(prob.F - exact).max() < 1e-10
    assert np.abs(prob.homogenized_P().reshape(9)[mask] - Pt[mask]).max() < 1e-12


def test_homogenized_tangent_matches_finite_differences():
    shape = (5, 5, 5)
    rng = np.random.default_rng(7)
    ph = (rng.uniform(size=shape) < 0.4).astype(np.uint8)
    params = synth.two_phase_params(10.0)
    base = solver.SVKProblem.from_phase(ph, params)
    F0 = synth.simple_shear(0.1)
    F0[0, 0] += 0.03
    base.increment(F0, **TIGHT)
    _, K4 = base.constitutive(base.F)
    cols = [0, 1, 5, 7]
    C = mixed.homogenized_tangent(K4, cols, 1e-13, 1e-14)
    h = 1e-5
    for k, b in enumerate(cols):
        Pb = []
        for s in (1.0, -1.0):
            p = solver.SVKProblem.from_phase(ph, params)
            p.F = base.F.copy()
            E = np.zeros(9)
            E[b] = s * h
            p.increment(F0 + E.reshape(3, 3), **TIGHT)
            Pb.append(p.homogenized_P().reshape(9))
        fd = (Pb[0] - Pb[1]) / (2 * h)
        assert np.abs(C[:, k] - fd).max() < 1e-7 * np.abs(C).max()


def test_no_stress_control_is_an_ordinary_increment():
    shape = (5, 3, 5)
    rng = np.random.default_rng(3)
    ph = (rng.uniform(size=shape) < 0.4).astype(np.uint8)
    params = synth.two_phase_params(10.0)
    p1 = solver.SVKProblem.from_phase(ph, params)
    p2 = solver.SVKProblem.from_phase(ph, params)
    Fbar = synth.simple_shear(0.2)
    p1.increment(Fbar, **TIGHT)
    Fb, m, _ = mixed.solve_mixed(p2, Fbar, np.ones((3, 3)), np.zeros(9, dtype=bool), **TIGHT)
    assert m == 1
    assert np.array_equal(p1.F, p2.F)
    assert np.array_equal(Fb, Fbar)
