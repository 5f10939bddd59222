"""GPU adjoint gradient of the homogenised stress with respect to per-voxel
shear moduli (SVK), through the C ABI and torch.autograd; J2 gradients with
respect to K, mu, tau_y0, H at the history of the last increment's start.

Checks: against the oracle's adjoint gradient (1e-9), against central finite
differences of GPU solves at 64 random voxels of a 31^3 lognormal cell
(1e-5 relative per entry, with an absolute floor of 1e-8 of the largest
entry for the round-off of the difference quotient), mixed vs float64.
"""
import numpy as np
import pytest

import synth
from oracle import adjoint as oadj
from oracle import solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1603_08893_gb300 import RVE  # noqa: E402
from paper_1603_08893_gb300.autograd import homogenized_stress  # noqa: E402

TIGHT = dict(tol_newton=1e-11, tol_cg=1e-13)
WXY = np.zeros((3, 3))
WXY[0, 1] = 1.0


def _cell(n, seed=4):
    rng = np.random.default_rng(seed)
    mu = synth.lognormal_mu((n, n, n), rng)
    return mu, np.full(mu.shape, synth.K_SOFT), rng


def _solve(mu, K, Fbar, precision="fp64"):
    r = RVE(mu.shape, voxel_params=np.stack([K, mu]), precision=precision, cg_atol=1e-14)
    r.set_macro_F(Fbar)
    r.solve_increment(**TIGHT)
    return r


def test_adjoint_matches_oracle():
    mu, K, _ = _cell(9)
    Fbar = synth.simple_shear(0.05)
    prob = solver.SVKProblem(mu.shape, K, mu)
    prob.increment(Fbar, cg_atol=1e-14, **TIGHT)
    W = np.array([[0.3, 1.0, 0.0], [0.2, -0.5, 0.1], [0.0, 0.4, 0.7]])
    g_ref = oadj.grad_mu(prob, W, tol_cg=1e-13, cg_atol=1e-16)
    r = _solve(mu, K, Fbar)
    g, its = r.adjoint_grad_mu(W, tol_cg=1e-13)
    assert its > 5
    assert np.abs(g - g_ref).max() < 1e-9 * np.abs(g_ref).max()
    r.close()


def test_adjoint_matches_finite_differences_31():
    mu, K, rng = _cell(31)
    Fbar = synth.simple_shear(0.05)
    r = _solve(mu, K, Fbar)
    g, _ = r.adjoint_grad_mu(WXY, tol_cg=1e-12)
    r.close()
    gmax = np.abs(g).max()
    for flat in rng.choice(mu.size, 64, replace=False):
        idx = np.unravel_index(flat, mu.shape)
        h = 1e-4 * mu[idx]
        vals = []
        for s in (+1, -1):
            m2 = mu.copy()
            m2[idx] += s * h
            q = _solve(m2, K, Fbar)
            vals.append(q.homogenized_P()[0, 1])
            q.close()
        fd = (vals[0] - vals[1]) / (2 * h)
        # per entry: the difference quotient carries O((h/mu)^2) = 1e-8
        # truncation and ~1e-17 / (2h) round-off of the two P-bar values
        assert abs(g[idx] - fd) <= 1e-5 * abs(fd) + 1e-8 * gmax, (idx, g[idx], fd)


def test_mixed_adjoint_matches_fp64():
    mu, K, _ = _cell(15)
    Fbar = synth.simple_shear(0.05)
    a = _solve(mu, K, Fbar, "fp64")
    b = _solve(mu, K, Fbar, "mixed")
    ga, _ = a.adjoint_grad_mu(WXY, tol_cg=1e-11)
    gb, _ = b.adjoint_grad_mu(WXY, tol_cg=1e-11)
    assert np.abs(ga - gb).max() < 1e-8 * np.abs(ga).max()
    a.close()
    b.close()


def test_autograd_function():
    mu, K, _ = _cell(9)
    mu_t = torch.tensor(mu, dtype=torch.float64, device="cuda", requires_grad=True)
    Pbar = homogenized_stress(mu_t, K, synth.simple_shear(0.05), tol_newton=1e-11,
                              tol_cg=1e-13, cg_atol=1e-14, adjoint_tol=1e-13)
    J = (Pbar * torch.tensor(WXY, device="cuda")).sum()
    (g,) = torch.autograd.grad(J, mu_t)
    r = _solve(mu, K, synth.simple_shear(0.05))
    g_ref, _ = r.adjoint_grad_mu(WXY, tol_cg=1e-13)
    r.close()
    assert g.shape == mu_t.shape
    assert np.abs(g.cpu().numpy() - g_ref).max() < 1e-10 * np.abs(g_ref).max()


def test_bulk_gradient_matches_oracle_and_fd():
    """dJ/dK from the same adjoint field: against the oracle (1e-9) and
    central finite differences of GPU solves at 8 voxels of a 15^3 cell."""
    mu, K, rng = _cell(9)
    Fbar = synth.simple_shear(0.05) + np.diag([0.01, -0.005, 0.0])
    prob = solver.SVKProblem(mu.shape, K, mu)
    prob.increment(Fbar, cg_atol=1e-14, **TIGHT)
    W = np.array([[0.3, 1.0, 0.0], [0.2, -0.5, 0.1], [0.0, 0.4, 0.7]])
    gK_ref, gmu_ref = oadj.grad_params(prob, W, tol_cg=1e-13, cg_atol=1e-16)
    r = _solve(mu, K, Fbar)
    gK, gmu, _ = r.adjoint_grad(W, tol_cg=1e-13)
    r.close()
    assert np.abs(gK - gK_ref).max() < 1e-9 * np.abs(gK_ref).max()
    assert np.abs(gmu - gmu_ref).max() < 1e-9 * np.abs(gmu_ref).max()
    mu, K, rng = _cell(15)
    r = _solve(mu, K, Fbar)
    gK, _, _ = r.adjoint_grad(WXY, tol_cg=1e-12)
    r.close()
    for flat in rng.choice(mu.size, 8, replace=False):
        idx = np.unravel_index(flat, mu.shape)
        h = 1e-4 * K[idx]
        vals = []
        for s in (+1, -1):
            K2 = K.copy()
            K2[idx] += s * h
            q = _solve(mu, K2, Fbar)
            vals.append(q.homogenized_P()[0, 1])
            q.close()
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(gK[idx] - fd) <= 1e-5 * abs(fd) + 1e-8 * np.abs(gK).max(), (idx, gK[idx], fd)


def test_autograd_bulk_and_shear():
    mu, K, _ = _cell(9)
    mu_t = torch.tensor(mu, dtype=torch.float64, device="cuda", requires_grad=True)
    K_t = torch.tensor(K, dtype=torch.float64, device="cuda", requires_grad=True)
    Pbar = homogenized_stress(mu_t, K_t, synth.simple_shear(0.05), tol_newton=1e-11,
                              tol_cg=1e-13, cg_atol=1e-14, adjoint_tol=1e-13)
    J = (Pbar * torch.tensor(WXY, device="cuda")).sum()
    gmu, gK = torch.autograd.grad(J, (mu_t, K_t))
    r = _solve(mu, K, synth.simple_shear(0.05))
    gK_ref, gmu_ref, _ = r.adjoint_grad(WXY, tol_cg=1e-13)
    r.close()
    assert np.abs(gmu.cpu().numpy() - gmu_ref).max() < 1e-10 * np.abs(gmu_ref).max()
    assert np.abs(gK.cpu().numpy() - gK_ref).max() < 1e-10 * np.abs(gK_ref).max()


# ---------------------------------------------------------------------------
# J2: gradient with respect to K, mu, tau_y0, H at the history of the last
# increment's start (rve_adjoint_grad_params)
# ---------------------------------------------------------------------------
J2_PARAMS = np.array([[1 / 1.2, 1 / 2.6, 0.003, 0.01], [1 / 1.2, 1 / 2.6, 0.006, 0.01]])


def _j2_cell():
    rng = np.random.default_rng(13)
    shape = (7, 5, 9)
    return shape, (rng.uniform(size=shape) < 0.5).astype(np.uint8)


def _j2_oracle_grad(prob_F, Cpi, ep, ph):
    p = J2_PARAMS[ph.reshape(-1)]
    return oadj.j2_grad_params(prob_F, Cpi, ep, p[:, 0], p[:, 1], p[:, 2], p[:, 3], WXY,
                               1e-13, 1e-15)


def test_j2_adjoint_matches_oracle_over_two_increments():
    """Increment 1 from the virgin state (exact derivative), increment 2 with
    the history committed by increment 1 held fixed."""
    shape, ph = _j2_cell()
    n = ph.size
    prob = solver.J2Problem.from_phase(ph, J2_PARAMS)
    r = RVE(shape, model="j2", phase=ph, phase_params=J2_PARAMS, precision="fp64",
            cg_atol=1e-14)
    # shear with some stretch (simple shear alone is isochoric and, with equal
    # elastic phases, leaves dJ/dK at round-off level)
    for k, Fb in enumerate((synth.simple_shear(0.004) + np.diag([0.002, 0, 0]),
                            synth.simple_shear(0.008) + np.diag([0.004, 0, 0]))):
        Cpi0, ep0 = prob.mat.Cpi.copy(), prob.mat.ep.copy()
        prob.increment(Fb, tol_newton=1e-11, tol_cg=1e-13, cg_atol=1e-14)
        r.set_macro_F(Fb)
        r.solve_increment(**TIGHT)
        ref = _j2_oracle_grad(prob.F, Cpi0, ep0, ph)
        got, _ = r.adjoint_grad_params(WXY, tol_cg=1e-13)
        # compared as parameter x derivative (the units of J)
        th = np.moveaxis(J2_PARAMS[ph], -1, 0)
        scale = np.abs(th * ref).max()
        for q in range(4):
            assert np.abs(th[q] * (got[q] - ref[q])).max() < 1e-9 * scale, (k, q)
        gK, gmu = r.adjoint_grad(WXY, tol_cg=1e-13)[:2]
        assert np.array_equal(gK, got[0]) and np.array_equal(gmu, got[1])
    assert prob.mat.ep.max() > 1e-4
    # Euler's identity holds for the first increment only (virgin history)
    r.close()


def test_j2_adjoint_euler_identity_and_mixed():
    shape, ph = _j2_cell()
    Fb = synth.simple_shear(0.006) + np.diag([0.003, 0, 0])
    p = J2_PARAMS[ph]
    out = {}
    for prec in ("fp64", "mixed"):
        r = RVE(shape, model="j2", phase=ph, phase_params=J2_PARAMS, precision=prec,
                cg_atol=1e-14)
        r.set_macro_F(Fb)
        r.solve_increment(**TIGHT)
        g, _ = r.adjoint_grad_params(WXY, tol_cg=1e-12)
        J = float(r.homogenized_P()[0, 1])
        euler = float(sum(np.sum(p[..., k] * g[k]) for k in range(4)))
        out[prec] = (g, J, euler)
        r.close()
    g64, J, euler = out["fp64"]
    assert abs(euler - J) < 1e-9 * abs(J)
    gmx = out["mixed"][0]
    th = np.moveaxis(p, -1, 0)
    scale = np.abs(th * g64).max()
    for q in range(4):
        assert np.abs(th[q] * (gmx[q] - g64[q])).max() < 1e-4 * scale


def test_j2_autograd_one_increment():
    from paper_1603_08893_gb300.autograd import j2_homogenized_stress
    shape, ph = _j2_cell()
    p = J2_PARAMS[ph]
    ts = [torch.tensor(np.ascontiguousarray(p[..., k]), dtype=torch.float64, requires_grad=True)
          for k in range(4)]
    Fb = synth.simple_shear(0.006) + np.diag([0.003, 0, 0])
    Pbar = j2_homogenized_stress(*ts, Fb, tol_newton=1e-11, tol_cg=1e-13, cg_atol=1e-14,
                                 adjoint_tol=1e-13)
    J = Pbar[0, 1]
    grads = torch.autograd.grad(J, ts)
    r = RVE(shape, model="j2", phase=ph, phase_params=J2_PARAMS, precision="fp64",
            cg_atol=1e-14)
    r.set_macro_F(Fb)
    r.solve_increment(**TIGHT)
    ref, _ = r.adjoint_grad_params(WXY, tol_cg=1e-13)
    r.close()
    scale = max(float(np.abs(p[..., k] * ref[k]).max()) for k in range(4))
    for k in range(4):
        assert np.abs(p[..., k] * (grads[k].numpy() - ref[k])).max() < 1e-9 * scale
    euler = float(sum((t.detach() * g).sum() for t, g in zip(ts, grads)))
    Jv = float(J.detach())
    assert abs(euler - Jv) < 1e-9 * abs(Jv)


def test_svk_adjoint_grad_params_equals_adjoint_grad():
    mu, K, _ = _cell(9)
    r = _solve(mu, K, synth.simple_shear(0.05))
    g, _ = r.adjoint_grad_params(WXY, tol_cg=1e-12)
    gK, gmu, _ = r.adjoint_grad(WXY, tol_cg=1e-12)
    assert g.shape == (2,) + mu.shape
    assert np.array_equal(g[0], gK) and np.array_equal(g[1], gmu)
    r.close()


def test_j2_path_adjoint_matches_oracle():
    """Through the history of a loading-reversal-reloading path (reverse
    sweep over the taped increments, the return map's derivatives in closed
    form) against the oracle's reverse sweep, to 1e-9 of the largest
    parameter-weighted gradient entry."""
    shape, ph = _j2_cell()
    ramp = [synth.simple_shear(g) + np.diag([g / 2, 0.0, 0.0]) for g in (0.004, 0.008, -0.002, 0.006)]
    prob = solver.J2Problem.from_phase(ph, J2_PARAMS)
    states = []
    r = RVE(shape, model="j2", phase=ph, phase_params=J2_PARAMS, precision="fp64",
            cg_atol=1e-14)
    r.tape(True)
    for k, Fb in enumerate(ramp):
        Cpi0, ep0 = prob.mat.Cpi.copy(), prob.mat.ep.copy()
        prob.increment(Fb, tol_newton=1e-11, tol_cg=1e-13, cg_atol=1e-14)
        states.append((prob.F.copy(), Cpi0, ep0))
        r.set_macro_F(Fb)
        r.solve_increment(**TIGHT)
        if k == 0:
            # one increment: the fixed-history derivative in closed form
            g1, _ = r.adjoint_grad_path(WXY, tol_cg=1e-13)
            ref1, _ = r.adjoint_grad_params(WXY, tol_cg=1e-13)
            th = np.moveaxis(J2_PARAMS[ph], -1, 0)
            assert np.abs(th * (g1 - ref1)).max() < 1e-9 * np.abs(th * ref1).max()
    assert r.tape_length() == len(ramp)
    before = (r.get_F(), r.get_P(), r.get_history(), r.get_K4())
    g, _ = r.adjoint_grad_path(WXY, tol_cg=1e-13)
    after = (r.get_F(), r.get_P(), r.get_history(), r.get_K4())
    assert all(np.array_equal(x, y) for x, y in zip(before, after))   # state untouched
    p = J2_PARAMS[ph.reshape(-1)]
    ref = oadj.j2_path_grad_params(states, p[:, 0], p[:, 1], p[:, 2], p[:, 3], WXY, 1e-13, 1e-15)
    th = np.moveaxis(J2_PARAMS[ph], -1, 0)
    scale = np.abs(th * ref).max()
    err = [float(np.abs(th[q] * (g[q] - ref[q])).max() / scale) for q in range(4)]
    print("path adjoint vs oracle (units of the largest th * dJ/dth):", err)
    assert max(err) < 1e-9, err
    r.set_F(r.get_F())          # a new path starts: the tape is cleared
    assert r.tape_length() == 0
    r.close()


def test_j2_autograd_along_a_path():
    from paper_1603_08893_gb300.autograd import j2_homogenized_stress
    shape, ph = _j2_cell()
    p = J2_PARAMS[ph]
    ts = [torch.tensor(np.ascontiguousarray(p[..., k]), dtype=torch.float64, requires_grad=True)
          for k in range(4)]
    ramp = np.stack([synth.simple_shear(g) + np.diag([g / 2, 0.0, 0.0])
                     for g in (0.004, 0.008, -0.002, 0.006)])
    Pbar = j2_homogenized_stress(*ts, ramp, tol_newton=1e-11, tol_cg=1e-13, cg_atol=1e-14,
                                 adjoint_tol=1e-13)
    grads = torch.autograd.grad(Pbar[0, 1], ts)
    r = RVE(shape, model="j2", phase=ph, phase_params=J2_PARAMS, precision="fp64",
            cg_atol=1e-14)
    r.tape(True)
    for Fb in ramp:
        r.set_macro_F(Fb)
        r.solve_increment(**TIGHT)
    ref, _ = r.adjoint_grad_path(WXY, tol_cg=1e-13)
    r.close()
    th = np.moveaxis(p, -1, 0)
    scale = np.abs(th * ref).max()
    for k in range(4):
        assert np.abs(th[k] * (grads[k].numpy() - ref[k])).max() < 1e-9 * scale


def test_device_voxel_params_match_host():
    """Per-voxel parameters handed over in device memory (converted by a
    kernel, no copy through the host) give the handle that host arrays give:
    the same solve bit for bit, the same reference medium for the
    preconditioned CG; the J2 parameter set likewise."""
    mu, K, _ = _cell(15)
    vp = np.stack([K, mu])
    Fbar = synth.simple_shear(0.05)
    out = []
    for src in (vp, torch.from_numpy(vp).cuda()):
        for precond in ("none", "reference"):
            r = RVE(mu.shape, voxel_params=src, precision="mixed", precond=precond)
            r.set_macro_F(Fbar)
            r.solve_increment()
            out.append(r.get_F())
            r.close()
    assert np.array_equal(out[0], out[2])
    assert np.abs(out[1] - out[3]).max() < 1e-12
    p = J2_PARAMS[_j2_cell()[1]]
    vj = np.moveaxis(p, -1, 0).copy()
    res = []
    for src in (vj, torch.from_numpy(vj).cuda()):
        r = RVE(vj.shape[1:], model="j2", voxel_params=src, precision="fp64")
        r.set_macro_F(synth.simple_shear(0.006))
        r.solve_increment()
        res.append((r.get_F(), r.get_history()))
        r.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
