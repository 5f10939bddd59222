"""Pins of the oracle's adjoint gradients (CPU only).

Against central finite differences of the converged P-bar with respect to
single-voxel shear moduli, the independent forward (localisation) formula,
and the envelope identity for the mean strain energy,
dW-bar/dmu_k = (1/n) devE_k : devE_k at fixed F-bar (the fluctuation
derivative vanishes at equilibrium).  J2: the stress derivatives with
respect to K, mu, tau_y0, H against central differences of the return map
(from a plastic committed history, elastic and plastic branches); the
adjoint gradient summed over a phase against central differences of P-bar
over re-solved increments from the virgin state; Euler's identity for a
stress homogeneous of degree one in the parameters.
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


# ---------------------------------------------------------------------------
# J2: derivative at fixed start-of-increment history
# ---------------------------------------------------------------------------
J2_PARAMS = np.array([[1 / 1.2, 1 / 2.6, 0.003, 0.01], [1 / 1.2, 1 / 2.6, 0.006, 0.01]])


def test_j2_stress_parameter_derivatives_match_finite_differences():
    from oracle import j2
    rng = np.random.default_rng(11)
    m = 64
    K = np.full(m, 1 / 1.2)
    mu = np.full(m, 1 / 2.6)
    ty0 = rng.uniform(0.002, 0.006, m)
    H = rng.uniform(0.005, 0.05, m)
    # a committed history from an earlier plastic step, then a further step
    F0 = np.moveaxis(synth.random_F((m,), rng, 0.01), -1, 0)
    st0 = j2.return_map(F0, np.broadcast_to(np.eye(3), (m, 3, 3)).copy(), np.zeros(m), K, mu,
                        ty0, H)
    Cpi, ep = st0["Cpi_new"], st0["ep_new"]
    # partly unloading (elastic), partly loading further (plastic)
    sc = rng.uniform(0.5, 1.5, m)[:, None, None]
    F = np.eye(3) + sc * (F0 - np.eye(3)) + np.moveaxis(rng.uniform(-1e-3, 1e-3, (3, 3, m)), -1, 0)
    d = adjoint.j2_dP_dparams(F, Cpi, ep, K, mu, ty0, H)
    st = j2.return_map(F, Cpi, ep, K, mu, ty0, H)
    assert 0.2 < st["plastic"].mean() < 1.0 and ep.max() > 0.0
    args = [K, mu, ty0, H]
    for k in range(4):
        h = 1e-6 * args[k]
        a_p = [a.copy() for a in args]
        a_m = [a.copy() for a in args]
        a_p[k] = args[k] + h
        a_m[k] = args[k] - h
        fd = (j2.return_map(F, Cpi, ep, *a_p)["P"] - j2.return_map(F, Cpi, ep, *a_m)["P"]) \
            / (2 * h)[:, None, None]
        assert np.abs(d[k] - fd).max() < 1e-6 * np.abs(fd).max() + 1e-12, k


def _j2_cell():
    rng = np.random.default_rng(13)
    shape = (7, 5, 9)
    ph = (rng.uniform(size=shape) < 0.5).astype(np.uint8)
    return shape, ph


def _j2_Pbar(shape, ph, params, Fbar):
    prob = solver.J2Problem.from_phase(ph, params)
    prob.increment(Fbar, **TIGHT)
    return prob


def test_j2_adjoint_gradient_matches_phase_finite_differences_and_euler():
    shape, ph = _j2_cell()
    # shear with some stretch: simple shear alone is isochoric and, with the
    # phases' equal elastic moduli, leaves dJ/dK at round-off level
    Fbar = synth.simple_shear(0.006) + np.diag([0.003, 0.0, 0.0])
    W = np.zeros((3, 3))
    W[0, 1] = 1.0
    prob = _j2_Pbar(shape, ph, J2_PARAMS, Fbar)
    n = ph.size
    assert prob.mat.ep.max() > 1e-4
    p = J2_PARAMS[ph.reshape(-1)]
    g = adjoint.j2_grad_params(prob.F, np.broadcast_to(np.eye(3), (n, 3, 3)).copy(), np.zeros(n),
                               p[:, 0], p[:, 1], p[:, 2], p[:, 3], W, 1e-13, 1e-15)
    J = float(np.sum(W * prob.homogenized_P()))
    # Euler: P-bar is homogeneous of degree one in (K, mu, tau_y0, H)
    euler = sum(float(np.sum(p[:, k] * g[k].reshape(-1))) for k in range(4))
    assert abs(euler - J) < 1e-9 * abs(J)
    for phase in (0, 1):
        for k in range(4):
            h = 1e-6 * J2_PARAMS[phase, k]
            Jpm = []
            for sgn in (1.0, -1.0):
                q = J2_PARAMS.copy()
                q[phase, k] += sgn * h
                Jpm.append(float(np.sum(W * _j2_Pbar(shape, ph, q, Fbar).homogenized_P())))
            fd = (Jpm[0] - Jpm[1]) / (2 * h)
            adj = float(g[k][ph == phase].sum())
            assert abs(adj - fd) < 1e-5 * max(abs(fd), 1e-3 * abs(J) / J2_PARAMS[phase, k]), \
                (phase, k, adj, fd)


def _j2_path(shape, ph, params, ramp):
    prob = solver.J2Problem.from_phase(ph, params)
    states = []
    for Fb in ramp:
        Cpi0, ep0 = prob.mat.Cpi.copy(), prob.mat.ep.copy()
        prob.increment(Fb, **TIGHT)
        states.append((prob.F.copy(), Cpi0, ep0))
    return prob, states


def test_j2_path_adjoint_matches_finite_differences_over_the_path():
    shape, ph = _j2_cell()
    # loading, reversal and reloading: the history of earlier increments
    # shapes the last one (the reverse sweep through dH/dh is exercised)
    ramp = [synth.simple_shear(g) + np.diag([g / 2, 0.0, 0.0]) for g in (0.004, 0.008, -0.002, 0.006)]
    W = np.zeros((3, 3))
    W[0, 1] = 1.0
    prob, states = _j2_path(shape, ph, J2_PARAMS, ramp)
    n = ph.size
    p = J2_PARAMS[ph.reshape(-1)]
    assert prob.mat.ep.max() > 1e-3
    g = adjoint.j2_path_grad_params(states, p[:, 0], p[:, 1], p[:, 2], p[:, 3], W, 1e-13, 1e-15)
    # one increment: the fixed-history gradient
    g1 = adjoint.j2_path_grad_params(states[:1], p[:, 0], p[:, 1], p[:, 2], p[:, 3], W,
                                     1e-13, 1e-15)
    F1, C0, e0 = states[0]
    ref1 = adjoint.j2_grad_params(F1, C0, e0, p[:, 0], p[:, 1], p[:, 2], p[:, 3], W, 1e-13, 1e-15)
    assert np.abs(g1 - ref1).max() < 1e-8 * np.abs(ref1).max()
    J = float(np.sum(W * prob.homogenized_P()))
    for phase in (0, 1):
        for k in range(4):
            h = 1e-6 * J2_PARAMS[phase, k]
            Jpm = []
            for sgn in (1.0, -1.0):
                q = J2_PARAMS.copy()
                q[phase, k] += sgn * h
                Jpm.append(float(np.sum(W * _j2_path(shape, ph, q, ramp)[0].homogenized_P())))
            fd = (Jpm[0] - Jpm[1]) / (2 * h)
            adj = float(g[k][ph == phase].sum())
            # floor: the finite difference of J (converged to ~1e-11) over a
            # 1e-6 step resolves p dJ/dp to ~1e-7 |J|
            assert abs(adj - fd) < 1e-5 * max(abs(fd), 1e-2 * abs(J) / J2_PARAMS[phase, k]), \
                (phase, k, adj, fd)
    # the history matters: the last-increment derivative alone misses it
    F3, C2, e2 = states[-1]
    last = adjoint.j2_grad_params(F3, C2, e2, p[:, 0], p[:, 1], p[:, 2], p[:, 3], W, 1e-13,
                                  1e-15)
    assert abs(float(last[2][ph == 0].sum()) - float(g[2][ph == 0].sum())) > \
        1e-3 * abs(float(g[2][ph == 0].sum()))


def test_j2_return_map_closed_form_derivatives():
    """The return map linearised step by step (Daleckii-Krein for ln and
    exp, radial return, pull-backs) against central differences, and its F
    derivative against the consistent tangent."""
    from oracle import j2
    rng = np.random.default_rng(11)
    m = 64
    K, mu = np.full(m, 1 / 1.2), np.full(m, 1 / 2.6)
    ty0, H = rng.uniform(0.002, 0.006, m), rng.uniform(0.005, 0.05, m)
    F0 = np.moveaxis(synth.random_F((m,), rng, 0.01), -1, 0)
    st0 = j2.return_map(F0, np.broadcast_to(np.eye(3), (m, 3, 3)).copy(), np.zeros(m), K, mu,
                        ty0, H)
    Cpi, ep = st0["Cpi_new"], st0["ep_new"]
    sc = rng.uniform(0.5, 1.5, m)[:, None, None]
    F = np.eye(3) + sc * (F0 - np.eye(3)) + np.moveaxis(rng.uniform(-1e-3, 1e-3, (3, 3, m)), -1, 0)
    closed = adjoint.j2_local_jacobians_closed(F, Cpi, ep, K, mu, ty0, H)
    fd = adjoint.j2_local_jacobians(F, Cpi, ep, K, mu, ty0, H, step=1e-6)
    for a, b in zip(closed, fd):
        assert np.abs(a - b).max() < 1e-6 * np.abs(b).max()
    st = j2.return_map(F, Cpi, ep, K, mu, ty0, H)
    K4 = j2.tangent(F, Cpi, K, mu, H, st)
    assert 0.2 < st["plastic"].mean() < 1.0
    for a in range(9):
        dF = np.zeros((m, 3, 3))
        dF[:, a // 3, a % 3] = 1.0
        dP, _ = adjoint.j2_return_map_directional(F, Cpi, ep, K, mu, ty0, H, dF=dF)
        ref = np.swapaxes(K4[:, :, :, a // 3, a % 3], -1, -2)   # K_ijkl = dP_ji/dF_kl
        assert np.abs(dP - ref).max() < 1e-13 * np.abs(ref).max()


def test_j2_parameter_derivatives_two_derivations_agree():
    """dP/d(K, mu, tau_y0, H) from the principal-basis formulas and from the
    step-by-step linearisation of the return map."""
    from oracle import j2
    rng = np.random.default_rng(5)
    m = 48
    K, mu = np.full(m, 1 / 1.2), np.full(m, 1 / 2.6)
    ty0, H = rng.uniform(0.002, 0.006, m), rng.uniform(0.005, 0.05, m)
    F0 = np.moveaxis(synth.random_F((m,), rng, 0.012), -1, 0)
    st0 = j2.return_map(F0, np.broadcast_to(np.eye(3), (m, 3, 3)).copy(), np.zeros(m), K, mu,
                        ty0, H)
    F = F0 + np.moveaxis(rng.uniform(-2e-3, 2e-3, (3, 3, m)), -1, 0)
    a = adjoint.j2_dP_dparams(F, st0["Cpi_new"], st0["ep_new"], K, mu, ty0, H)
    for t in range(4):
        d = np.zeros((4, m))
        d[t] = 1.0
        dP, _ = adjoint.j2_return_map_directional(F, st0["Cpi_new"], st0["ep_new"], K, mu, ty0, H,
                                                  dprm=d)
        assert np.abs(dP - a[t]).max() < 1e-12 * max(np.abs(a[t]).max(), 1e-30), t


@pytest.mark.parametrize("F0", [np.eye(3), np.diag([1.01, 1.0, 1.0]), np.diag([1.02, 0.99, 0.99])])
def test_j2_closed_form_derivatives_at_repeated_eigenvalues(F0):
    """Repeated eigenvalues of be (the virgin state, uniaxial stretches):
    the divided differences take their limits and still equal central
    differences."""
    m = 2
    K, mu = np.full(m, 1 / 1.2), np.full(m, 1 / 2.6)
    ty0, H = np.array([0.003, 0.001]), np.full(m, 0.01)
    F = np.broadcast_to(F0, (m, 3, 3)).copy()
    Cpi = np.broadcast_to(np.eye(3), (m, 3, 3)).copy()
    ep = np.zeros(m)
    closed = adjoint.j2_local_jacobians_closed(F, Cpi, ep, K, mu, ty0, H)
    fd = adjoint.j2_local_jacobians(F, Cpi, ep, K, mu, ty0, H, step=1e-6)
    for a, b in zip(closed, fd):
        assert np.abs(a - b).max() < 1e-6 * max(np.abs(b).max(), 1.0)
