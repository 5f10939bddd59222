"""GPU parity of the reference-medium preconditioned CG
(rve_options.precond = RVE_PRECOND_REFERENCE, float32 CG of the mixed path)
against the FP64 oracle.

Preconditioning changes the CG iterates and their stopping norm, not the
Newton fixed point: converged states are compared with the oracle's (plain
or preconditioned -- its two Newton solutions agree to 1e-11) at the mixed
path's bar (P-bar 1e-8, fields 1e-7), and the iteration counts against the
unpreconditioned float32 CG.
"""
import numpy as np
import pytest

import synth
from oracle import precond as opre
from oracle import solver, svk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1603_08893_gb300 import RVE, RVEBatch, RVEError  # noqa: E402

J2_PARAMS = np.array([[1 / 1.2, 1 / 2.6, 0.003, 0.01], [1 / 1.2, 1 / 2.6, 0.006, 0.01]])
TIGHT = dict(tol_newton=1e-10, tol_cg=1e-12)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(b).max())


@pytest.mark.parametrize("shape", [(15, 9, 11), (21, 16, 13), (27, 7, 10), (45, 6, 5)])
@pytest.mark.parametrize("tangent", ["recompute", "sym45"])
def test_preconditioned_newton_matches_oracle(shape, tangent):
    rng = np.random.default_rng(sum(shape))
    ph = (rng.uniform(size=shape) < 0.35).astype(np.uint8)
    params = synth.two_phase_params(30.0)
    Fbar = synth.simple_shear(0.04)
    Fbar[0, 0] += 0.01
    prob = solver.SVKProblem.from_phase(ph, params)
    lam0, mu0 = opre.reference_medium(svk.lame_lambda(prob.K, prob.mu), prob.mu)
    prob.increment(Fbar, linear_solver=opre.linear_solver(shape, lam0, mu0, 1e-12, 1e-14), **TIGHT)
    r = RVE(shape, phase=ph, phase_params=params, precision="mixed", tangent=tangent,
            precond="reference", cg_atol=1e-13)
    r.set_macro_F(Fbar)
    r.solve_increment(**TIGHT)
    assert maxrel(r.homogenized_P(), prob.homogenized_P()) < 1e-8
    assert rel(r.get_F(), prob.F) < 1e-7
    assert rel(r.get_P(), prob.P) < 1e-7
    r.close()


def test_fewer_cg_iterations_at_high_contrast():
    ph, _ = synth.spheres(45, 0.3, 4.0, 10.0, np.random.default_rng(1))
    params = synth.two_phase_params(100.0)
    Fbar = synth.uniaxial(0.01)
    out = {}
    for pc in ("none", "reference"):
        r = RVE(ph.shape, phase=ph, phase_params=params, precision="mixed", precond=pc)
        r.set_macro_F(Fbar)
        st = r.solve_increment(1e-5, 1e-8)
        out[pc] = (st["cg_iters_total"], r.homogenized_P())
        r.close()
    assert out["reference"][0] < 0.75 * out["none"][0]
    assert maxrel(out["reference"][1], out["none"][1]) < 1e-8


def test_preconditioned_j2_schedule_matches_oracle():
    ph, _ = synth.voronoi(15, 8, np.random.default_rng(2))
    prob = solver.J2Problem.from_phase(ph, J2_PARAMS)
    sched = synth.ramp(synth.simple_shear(0.008), 4)
    r = RVE(ph.shape, model="j2", phase=ph, phase_params=J2_PARAMS, precision="mixed",
            precond="reference", cg_atol=1e-12)
    for Fb in sched:
        prob.increment(Fb, cg_atol=1e-12, **TIGHT)
        r.set_macro_F(Fb)
        r.solve_increment(**TIGHT)
        assert maxrel(r.homogenized_P(), prob.homogenized_P()) < 1e-8
    assert prob.mat.ep.max() > 1e-4
    r.close()


def test_preconditioned_adjoint_gradient_matches_plain():
    rng = np.random.default_rng(6)
    shape = (15, 15, 15)
    ph = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    params = synth.two_phase_params(10.0)
    W = np.zeros((3, 3))
    W[0, 1] = 1.0
    g = {}
    for pc in ("none", "reference"):
        r = RVE(shape, phase=ph, phase_params=params, precision="mixed", precond=pc)
        r.set_macro_F(synth.simple_shear(0.05))
        r.solve_increment(1e-10, 1e-12)
        g[pc], _ = r.adjoint_grad_mu(W, tol_cg=1e-10)
        r.close()
    assert maxrel(g["reference"], g["none"]) < 1e-6


def test_preconditioned_batch_equals_individual_solves():
    rng = np.random.default_rng(9)
    cells = []
    for n in (15, 21, 27, 15):
        ph, _ = synth.spheres(n, 0.3, 4.0, 10.0, rng)
        cells.append(((n, n, n), ph, synth.two_phase_params(rng.uniform(2, 20)),
                      np.eye(3) + rng.uniform(-0.02, 0.02, (3, 3))))
    b = RVEBatch([c[0] for c in cells], [c[1] for c in cells], [c[2] for c in cells],
                 precision="mixed", precond="reference")
    st = b.solve(np.stack([c[3] for c in cells]))
    assert all(s["status"] == 0 for s in st)
    for i, (shape, ph, params, Fbar) in enumerate(cells):
        r = RVE(shape, phase=ph, phase_params=params, precision="mixed", precond="reference")
        r.set_macro_F(Fbar)
        s1 = r.solve_increment()
        assert s1["cg_iters_total"] == st[i]["cg_iters_total"]
        assert np.array_equal(r.get_F(), b.get_F(i))
        r.close()
    b.close()


def test_preconditioned_checkpoint_resume_is_bit_identical(tmp_path):
    rng = np.random.default_rng(21)
    shape = (15, 11, 13)
    ph = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    r = RVE(shape, phase=ph, phase_params=synth.two_phase_params(10.0), precision="mixed",
            precond="reference")
    sched = synth.ramp(synth.simple_shear(0.08), 4)
    for Fb in sched[:2]:
        r.set_macro_F(Fb)
        r.solve_increment(1e-6, 1e-9)
    path = str(tmp_path / "cell.ckpt")
    r.save(path)
    q = RVE.load(path)
    for Fb in sched[2:]:
        for c in (r, q):
            c.set_macro_F(Fb)
            c.solve_increment(1e-6, 1e-9)
    assert np.array_equal(r.get_F(), q.get_F())
    r.close()
    q.close()


def test_unsupported_combinations_are_refused():
    ph = np.zeros((9, 15, 15), np.uint8)
    with pytest.raises(RVEError) as e:   # no four-step kernel for x = 9
        RVE(ph.shape, phase=ph, phase_params=[[1.0, 0.5]], precision="mixed", precond="reference")
    assert e.value.code == -10
    ph = np.zeros((15, 15, 15), np.uint8)
    with pytest.raises(RVEError) as e:   # float64 CG
        RVE(ph.shape, phase=ph, phase_params=[[1.0, 0.5]], precision="fp64", precond="reference")
    assert e.value.code == -10
