"""Pins of the oracle's finite-strain J2 model (CPU only).

Independent of the formulas under test: the tangent equals central finite
differences of the stress (history frozen); below yield the model is Hencky
hyper-elasticity (tau = K tr(e) I + 2 mu dev(e), e = ln(F F^T)/2, with the
matrix logarithm taken by an independent route); on proportional paths
with fixed principal axes it reduces to the textbook small-strain J2 radial
return in logarithmic strains (closed form for linear hardening); plastic
flow is isochoric (det Cp = 1); the updated stress lies on the yield
surface; objectivity.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import j2

K, MU, TY0, H = 1.0 / 1.2, 1.0 / 2.6, 0.003, 0.01


def _vox(n, val):
    return np.full(n, val, dtype=np.float64)


def _material(n, ty0=TY0, h=H):
    return _vox(n, K), _vox(n, MU), _vox(n, ty0), _vox(n, h)


def _stress(F, Cpi, ep):
    k, m, t0, hh = _material(F.shape[0])
    return j2.return_map(F, Cpi, ep, k, m, t0, hh)


def _random_F(n, amp, rng):
    F = np.eye(3) + amp * rng.uniform(-1, 1, size=(n, 3, 3))
    return F


@pytest.mark.parametrize("amp", [1e-4, 0.02, 0.3])
def test_tangent_is_derivative_of_stress(amp):
    rng = np.random.default_rng(1)
    n = 40
    F = _random_F(n, amp, rng)
    Cpi = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
    # some voxels with a non-trivial committed history
    Fp = _random_F(n, 0.05, rng)
    Fp /= np.cbrt(np.linalg.det(Fp))[:, None, None]
    Fpi = np.linalg.inv(Fp)
    Cpi[n // 2:] = (Fpi @ np.swapaxes(Fpi, -1, -2))[n // 2:]
    ep = rng.uniform(0, 0.02, n)
    k, m, t0, hh = _material(n)
    st = j2.return_map(F, Cpi, ep, k, m, t0, hh)
    K4 = j2.tangent(F, Cpi, k, m, hh, st)
    h = 1e-7
    for _ in range(3):
        dF = rng.standard_normal((n, 3, 3))
        Pp = j2.return_map(F + h * dF, Cpi, ep, k, m, t0, hh)["P"]
        Pm = j2.return_map(F - h * dF, Cpi, ep, k, m, t0, hh)["P"]
        fd = (Pp - Pm) / (2 * h)
        got = np.swapaxes(np.einsum("nijkl,nkl->nij", K4, dF), -1, -2)
        assert np.abs(got - fd).max() < 2e-6 * np.abs(fd).max()
    if amp > 0.01:
        assert st["plastic"].any()


def test_tangent_at_identity_is_linear_elasticity():
    n = 2
    F = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
    Cpi = F.copy()
    st = _stress(F, Cpi, np.zeros(n))
    K4 = j2.tangent(F, Cpi, _vox(n, K), _vox(n, MU), _vox(n, H), st)
    Hm = np.random.default_rng(2).standard_normal((3, 3))
    dP = np.einsum("ijkl,kl->ji", K4[0], Hm)
    e = 0.5 * (Hm + Hm.T)
    lin = (K - 2 * MU / 3) * np.trace(e) * np.eye(3) + 2 * MU * e
    assert np.abs(dP - lin).max() < 1e-12


def test_elastic_range_is_hencky():
    rng = np.random.default_rng(3)
    n = 20
    F = _random_F(n, 0.0008, rng)
    Cpi = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
    st = _stress(F, Cpi, np.zeros(n))
    assert not st["plastic"].any()
    for v in range(n):
        e = 0.5 * scipy.linalg.logm(F[v] @ F[v].T).real
        tau = K * np.trace(e) * np.eye(3) + 2 * MU * (e - np.trace(e) / 3 * np.eye(3))
        assert np.abs(st["tau"][v] - tau).max() < 1e-12
        assert np.abs(st["P"][v] - tau @ np.linalg.inv(F[v]).T).max() < 1e-12


def _closed_form_pure_shear(a):
    """Small-strain J2 radial return in log strain for e = diag(a, -a, 0)."""
    ed = np.array([a, -a, 0.0])
    nrm = np.linalg.norm(ed)
    teq_tr = 2 * MU * np.sqrt(1.5) * nrm
    if teq_tr <= TY0:
        ep, s = 0.0, 2 * MU * ed
    else:
        ep = (teq_tr - TY0) / (3 * MU + H)
        teq = TY0 + H * ep
        s = teq * np.sqrt(2.0 / 3.0) * ed / nrm
    return ep, s  # tau = s (no volume change)


def test_proportional_path_matches_small_strain_closed_form():
    n = 1
    Cpi = np.eye(3)[None].copy()
    ep = np.zeros(1)
    k, m, t0, hh = _material(n)
    for step in range(1, 9):
        a = 0.0015 * step  # crosses yield around step 2
        F = np.diag([np.exp(a), np.exp(-a), 1.0])[None]
        st = j2.return_map(F, Cpi, ep, k, m, t0, hh)
        ep_ref, s_ref = _closed_form_pure_shear(a)
        assert abs(st["ep_new"][0] - ep_ref) < 1e-13
        assert np.abs(np.diag(st["tau"][0]) - s_ref).max() < 1e-13
        Cpi, ep = st["Cpi_new"], st["ep_new"]


def test_plastic_flow_isochoric_and_consistent():
    rng = np.random.default_rng(4)
    n = 30
    F = _random_F(n, 0.2, rng)
    Cpi = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
    st = _stress(F, Cpi, np.zeros(n))
    pl = st["plastic"]
    assert pl.sum() > 10
    assert np.abs(np.linalg.det(st["Cpi_new"]) - 1.0).max() < 1e-12
    tau = st["tau"]
    dev = tau - np.trace(tau, axis1=-2, axis2=-1)[:, None, None] * np.eye(3) / 3
    teq = np.sqrt(1.5 * (dev * dev).sum((-2, -1)))
    assert np.abs(teq[pl] - (TY0 + H * st["ep_new"][pl])).max() < 1e-13


def test_objectivity_and_tangent_symmetry():
    rng = np.random.default_rng(5)
    n = 10
    F = _random_F(n, 0.2, rng)
    Cpi = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    P = _stress(F, Cpi, np.zeros(n))["P"]
    PQ = _stress(Q @ F, Cpi, np.zeros(n))["P"]
    assert np.abs(PQ - Q @ P).max() < 1e-13
    k, m, t0, hh = _material(n)
    st = j2.return_map(F, Cpi, np.zeros(n), k, m, t0, hh)
    K4 = j2.tangent(F, Cpi, k, m, hh, st)
    K4T = np.einsum("nijkl->nlkji", K4)
    # the return map derives from an incremental potential: major symmetry
    assert np.abs(K4 - K4T).max() < 1e-10 * np.abs(K4).max()


def test_two_newton_iterations_per_increment_in_the_plastic_regime():
    """Sec. 5.5: about two Newton iterations per increment once the cell
    deforms plastically (more only around the yield point): the predictor
    tangent at a state on the yield surface is the elasto-plastic one.
    Pure shear diag(l, 1/l, 1) in steps of 0.2/250 on a two-phase Voronoi
    cell with the contrast chi = 2 of the example."""
    import synth
    from oracle import solver
    ph, _ = synth.voronoi(9, 8, np.random.default_rng(2))
    K, mu = 1 / 1.2, 1 / 2.6
    params = np.array([[K, mu, 0.003, 0.01], [K, mu, 0.006, 0.02]])
    prob = solver.J2Problem.from_phase(ph, params)
    counts = []
    for k in range(50):
        lam = 1.0 + 0.2 * (k + 1) / 250
        counts.append(prob.increment(np.diag([lam, 1 / lam, 1.0]), 1e-5, 1e-8).newton_iters)
    assert prob.mat.ep.max() > 0.01 and (prob.mat.ep > 0).mean() > 0.5
    assert max(counts[:15]) >= 3                 # around the yield point
    assert np.mean(counts[-10:]) <= 2.3          # plastic regime
