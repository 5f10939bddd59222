"""GPU parity of mixed macroscopic stress / deformation control
(rve_solve_mixed) against the FP64 oracle's ``mixed.solve_mixed``.

The state sought is defined by its equations (equilibrium, prescribed F-bar
and P-bar components); the library and the oracle take different Newton
paths on the free components (Broyden updates of the homogenised tangent on
the device, exact tangents in the oracle), so both are converged tightly
(stress residual 1e-12 of ||P-bar||, eta_NW = 1e-10, eta_CG = 1e-12) and
compared at the float64 bar of 1e-10 (SVK) / 1e-9 (J2); the mixed-precision
path's P-bar at 1e-8 and its fields at 1e-7.
"""
import numpy as np
import pytest

import synth
from oracle import mixed, solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1603_08893_gb300 import RVE  # noqa: E402

J2_PARAMS = np.array([[1 / 1.2, 1 / 2.6, 0.003, 0.01], [1 / 1.2, 1 / 2.6, 0.006, 0.01]])
TIGHT = dict(tol_newton=1e-10, tol_cg=1e-12)
MASK = synth.uniaxial_stress_mask()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(b).max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_svk_homogeneous_uniaxial_stress_closed_form(precision):
    K, mu = 0.833, 0.386
    shape = (5, 7, 5)
    r = RVE(shape, phase=np.zeros(shape, np.uint8), phase_params=np.array([[K, mu]]),
            precision=precision, cg_atol=1e-13)
    l1 = 1.06
    Fb = np.eye(3)
    Fb[0, 0] = l1
    st = r.solve_mixed(Fb, np.zeros(9), MASK, tol_stress=1e-12, **TIGHT)
    lam = K - 2 * mu / 3
    nu = lam / (2 * (lam + mu))
    Ey = mu * (3 * lam + 2 * mu) / (lam + mu)
    e1 = 0.5 * (l1 * l1 - 1)
    l2 = np.sqrt(1 - 2 * nu * e1)
    assert st["macro_iters"] >= 2 and st["tangent_solves"] >= 5
    assert np.abs(r.macro_F() - np.diag([l1, l2, l2])).max() < 1e-12
    Pb = r.homogenized_P()
    assert abs(Pb[0, 0] - l1 * Ey * e1) < 1e-12
    assert np.abs(Pb.reshape(9)[MASK]).max() < 1e-13
    r.close()


@pytest.fixture(scope="module")
def svk_oracle():
    rng = np.random.default_rng(11)
    shape = (9, 11, 13)
    ph = (rng.uniform(size=shape) < 0.35).astype(np.uint8)
    params = synth.two_phase_params(10.0)
    prob = solver.SVKProblem.from_phase(ph, params)
    Fb = np.eye(3)
    Fb[0, 0] = 1.05
    Fb[1, 0] = 0.01
    Pt = np.zeros(9)
    Pt[4] = 0.001
    Fsol, _, _ = mixed.solve_mixed(prob, Fb, Pt, MASK, tol_stress=1e-12, cg_atol=1e-13, **TIGHT)
    return ph, params, Fb, Pt, Fsol, prob.F.copy(), prob.P.copy()


@pytest.mark.parametrize("tangent", ["recompute", "sym45", "full81"])
def test_svk_mixed_control_fp64_matches_oracle(svk_oracle, tangent):
    ph, params, Fb, Pt, Fsol, F_ref, P_ref = svk_oracle
    r = RVE(ph.shape, phase=ph, phase_params=params, precision="fp64", tangent=tangent,
            cg_atol=1e-13)
    st = r.solve_mixed(Fb, Pt, MASK, tol_stress=1e-12, **TIGHT)
    assert st["substeps"] == 1 and st["cuts"] == 0
    assert np.abs(r.macro_F() - Fsol).max() < 1e-11
    assert rel(r.get_F(), F_ref) < 1e-10
    assert rel(r.get_P(), P_ref) < 1e-10
    Pb = r.homogenized_P().reshape(9)
    assert np.abs(Pb[MASK] - Pt[MASK]).max() < 1e-12 * np.linalg.norm(Pb)
    r.close()


def test_svk_mixed_control_mixed_precision_matches_oracle(svk_oracle):
    ph, params, Fb, Pt, Fsol, F_ref, P_ref = svk_oracle
    r = RVE(ph.shape, phase=ph, phase_params=params, precision="mixed", cg_atol=1e-13)
    r.solve_mixed(Fb, Pt, MASK, tol_stress=1e-12, **TIGHT)
    assert maxrel(r.homogenized_P(), P_ref.mean(axis=(2, 3, 4))) < 1e-8
    assert rel(r.get_F(), F_ref) < 1e-7
    assert rel(r.get_P(), P_ref) < 1e-7
    r.close()


def test_j2_mixed_control_matches_oracle():
    """One plastic increment from the virgin state (no history ambiguity)."""
    ph, _ = synth.voronoi(9, 8, np.random.default_rng(2))
    Fb = np.eye(3)
    Fb[0, 0] = np.exp(0.006)
    prob = solver.J2Problem.from_phase(ph, J2_PARAMS)
    Fsol, _, _ = mixed.solve_mixed(prob, Fb, np.zeros(9), MASK, tol_stress=1e-12,
                                   cg_atol=1e-12, **TIGHT)
    assert prob.mat.ep.max() > 1e-3
    for prec in ("fp64", "mixed"):
        r = RVE(ph.shape, model="j2", phase=ph, phase_params=J2_PARAMS, precision=prec,
                cg_atol=1e-12)
        r.solve_mixed(Fb, np.zeros(9), MASK, tol_stress=1e-12, **TIGHT)
        if prec == "fp64":
            assert np.abs(r.macro_F() - Fsol).max() < 1e-10
            assert rel(r.get_F(), prob.F) < 1e-9
            assert rel(r.get_P(), prob.P) < 1e-9
            ep = r.get_history()[6].reshape(-1)
            assert np.abs(ep - prob.mat.ep).max() < 1e-9 * prob.mat.ep.max()
        else:
            assert maxrel(r.homogenized_P(), prob.P.mean(axis=(2, 3, 4))) < 1e-8
        r.close()


def test_j2_mixed_control_substeps_replayed_by_oracle():
    """A step that needs halving: the oracle replays the library's reported
    sub-increments (the path matters for plasticity) and must land on the
    same state."""
    ph, _ = synth.voronoi(7, 6, np.random.default_rng(5))
    Fb = np.eye(3)
    Fb[0, 0] = np.exp(0.03)
    r = RVE(ph.shape, model="j2", phase=ph, phase_params=J2_PARAMS, precision="fp64",
            max_cg=3000, cg_atol=1e-12)
    st = r.solve_mixed(Fb, np.zeros(9), MASK, tol_stress=1e-12, max_cuts=8, **TIGHT)
    assert st["substep_to"][-1] == 1.0 and st["substeps"] == len(st["substep_to"])
    prob = solver.J2Problem.from_phase(ph, J2_PARAMS)
    mixed.solve_mixed_path(prob, Fb, np.zeros(9), MASK, st["substep_to"], tol_stress=1e-12,
                           cg_atol=1e-12, **TIGHT)
    assert rel(r.get_F(), prob.F) < 1e-9
    assert rel(r.get_P(), prob.P) < 1e-9
    r.close()


def test_no_stress_control_equals_increment():
    rng = np.random.default_rng(3)
    shape = (7, 5, 9)
    ph = (rng.uniform(size=shape) < 0.4).astype(np.uint8)
    params = synth.two_phase_params(10.0)
    Fb = synth.simple_shear(0.1)
    a = RVE(shape, phase=ph, phase_params=params, precision="fp64")
    b = RVE(shape, phase=ph, phase_params=params, precision="fp64")
    a.set_macro_F(Fb)
    a.solve_increment()
    st = b.solve_mixed(Fb, np.full(9, np.nan), np.zeros(9, dtype=bool))
    assert st["macro_iters"] == 1 and st["tangent_solves"] == 0
    assert np.array_equal(a.get_F(), b.get_F())
    assert np.array_equal(b.macro_F(), Fb)
    a.close()
    b.close()


def test_singular_stress_control_fails_and_rolls_back():
    """All nine components stress-controlled at zero stress from F = I: the
    rotations are free (K : skew = 0), the homogenised tangent is singular."""
    rng = np.random.default_rng(4)
    shape = (5, 5, 7)
    ph = (rng.uniform(size=shape) < 0.4).astype(np.uint8)
    r = RVE(shape, phase=ph, phase_params=synth.two_phase_params(5.0), precision="fp64")
    P = np.zeros(9)
    P[0] = 0.01
    st = r.solve_mixed(np.eye(3), P, np.ones(9, dtype=bool), check=False)
    assert st["status"] == -1
    eye = np.broadcast_to(np.eye(3)[:, :, None, None, None], (3, 3) + shape)
    assert np.array_equal(r.get_F(), eye)
    assert np.array_equal(r.macro_F(), np.eye(3))
    r.close()


def test_invalid_mixed_control_arguments():
    shape = (5, 5, 5)
    r = RVE(shape, phase=np.zeros(shape, np.uint8), phase_params=[[0.833, 0.386]])
    Fb = np.eye(3)
    st = r.solve_mixed(Fb, np.zeros(9), MASK, tol_stress=0.0, check=False)
    assert st["status"] == -1
    P = np.zeros(9)
    P[4] = np.nan                      # a prescribed stress component
    st = r.solve_mixed(Fb, P, MASK, check=False)
    assert st["status"] == -1
    F = np.eye(3)
    F[1, 1] = np.nan                   # a free component: ignored
    st = r.solve_mixed(F, np.zeros(9), MASK, tol_stress=1e-10)
    assert st["status"] == 0 and np.isfinite(r.macro_F()).all()
    r.close()


def test_mixed_control_with_preconditioned_cg(svk_oracle):
    _, params, Fb, Pt, _, _, _ = svk_oracle
    shape = (15, 11, 13)   # x length with a four-step kernel (preconditioned x pass)
    rng = np.random.default_rng(11)
    ph = (rng.uniform(size=shape) < 0.35).astype(np.uint8)
    prob = solver.SVKProblem.from_phase(ph, params)
    Fs, _, _ = mixed.solve_mixed(prob, Fb, Pt, MASK, tol_stress=1e-12, cg_atol=1e-13, **TIGHT)
    r = RVE(shape, phase=ph, phase_params=params, precision="mixed", precond="reference",
            cg_atol=1e-13)
    r.solve_mixed(Fb, Pt, MASK, tol_stress=1e-12, **TIGHT)
    assert np.abs(r.macro_F() - Fs).max() < 1e-8
    assert maxrel(r.homogenized_P(), prob.homogenized_P()) < 1e-8
    assert rel(r.get_F(), prob.F) < 1e-7
    r.close()
