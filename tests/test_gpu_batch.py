"""Batched cells of uneven size (one CUDA graph per group of CG iterations):
each cell's result equals the same cell solved on its own (bit for bit -- the
same kernels on the same data in the same order), and one cell is checked
against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1603_08893_gb300 import RVE, RVEBatch  # noqa: E402


def _cells(count, seed=3, sizes=(9, 15, 21)):
    rng = np.random.default_rng(seed)
    cells = []
    for _ in range(count):
        n = int(rng.choice(sizes))
        ph, _ = synth.spheres(n, rng.uniform(0.1, 0.4), 4.0, 10.0, rng)
        params = synth.two_phase_params(rng.uniform(2.0, 100.0))
        Fbar = np.eye(3) + rng.uniform(-0.05, 0.05, size=(3, 3))
        cells.append(((n, n, n), ph, params, Fbar))
    return cells


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_individual_solves(prec):
    cells = _cells(12)
    batch = RVEBatch([c[0] for c in cells], [c[1] for c in cells], [c[2] for c in cells],
                     precision=prec)
    st = batch.solve(np.stack([c[3] for c in cells]))
    assert all(s["status"] == 0 for s in st)
    Pb = batch.homogenized_P()
    for i, (shape, ph, params, Fbar) in enumerate(cells):
        r = RVE(shape, phase=ph, phase_params=params, precision=prec)
        r.set_macro_F(Fbar)
        s1 = r.solve_increment()
        assert s1["cg_iters_total"] == st[i]["cg_iters_total"]
        assert np.array_equal(r.get_F(), batch.get_F(i))
        assert np.array_equal(r.homogenized_P(), Pb[i])
        r.close()
    batch.close()


def test_batch_cell_matches_oracle():
    cells = _cells(5, seed=8)
    batch = RVEBatch([c[0] for c in cells], [c[1] for c in cells], [c[2] for c in cells])
    batch.solve(np.stack([c[3] for c in cells]))
    shape, ph, params, Fbar = cells[2]
    prob = solver.SVKProblem.from_phase(ph, params)
    prob.increment(Fbar)
    F = batch.get_F(2)
    assert np.linalg.norm(F - prob.F) / np.linalg.norm(prob.F) < 1e-10
    batch.close()


def test_j2_batch_commits_history_like_individual_solves():
    """J2 cells: the batch commits each cell's history as a single cell does
    (two increments, the second starting from the first's plastic state),
    bit for bit, in the batched passes and in the graph branches."""
    params = np.array([[1 / 1.2, 1 / 2.6, 0.003, 0.01], [1 / 1.2, 1 / 2.6, 0.006, 0.01]])
    cells = []
    # 15^3 and 21^3 cells run the batched passes (stored SYM45 tangent),
    # the 9^3 cells are graph branches
    for n, seed in ((9, 1), (15, 2), (9, 3), (21, 4), (15, 5)):
        ph, _ = synth.voronoi(n, 6, np.random.default_rng(seed))
        cells.append(((n, n, n), ph))
    b = RVEBatch([c[0] for c in cells], [c[1] for c in cells], [params] * len(cells),
                 model="j2", precision="mixed")
    singles = [RVE(c[0], model="j2", phase=c[1], phase_params=params, precision="mixed")
               for c in cells]
    for gamma in (0.004, 0.008):
        Fb = synth.simple_shear(gamma)
        st = b.solve(np.stack([Fb] * len(cells)))
        assert all(s["status"] == 0 for s in st)
        for i, r in enumerate(singles):
            r.set_macro_F(Fb)
            r.solve_increment()
            assert np.array_equal(r.get_F(), b.get_F(i))
    from paper_1603_08893_gb300 import rve as api
    for i, r in enumerate(singles):
        hb = api.rve_get_history(api.lib.rve_batch_cell(b.h, i), r.n)
        assert np.array_equal(r.get_history().reshape(-1), hb)
        assert r.get_history().reshape(7, -1)[6].max() > 0.0
        r.close()
    b.close()


def test_mixed_batch_runs_one_launch_per_pass():
    """Cells whose axes all have batched four-step kernels run each pass of
    the float32 CG iteration for the whole batch in one launch: the batch
    launches far fewer kernels than the same cells solved one by one, with
    bit-identical results."""
    cells = _cells(10, seed=5, sizes=(15, 21, 27))
    batch = RVEBatch([c[0] for c in cells], [c[1] for c in cells], [c[2] for c in cells],
                     precision="mixed")
    st = batch.solve(np.stack([c[3] for c in cells]))
    assert all(s["status"] == 0 for s in st)
    singles = 0
    for i, (shape, ph, params, Fbar) in enumerate(cells):
        r = RVE(shape, phase=ph, phase_params=params, precision="mixed")
        r.set_macro_F(Fbar)
        r.solve_increment()
        singles += r.launch_count()
        assert np.array_equal(r.get_F(), batch.get_F(i))
        r.close()
    assert batch.launch_count() < 0.5 * singles
    batch.close()


def test_autotuned_mixed_batch_matches_oracle():
    """An autotuned mixed batch (each cell's kernel variants timed and chosen,
    tile heights included; cells on the four-step lengths run the batched
    passes whatever tile heights they chose) reaches the oracle's converged
    state for every cell: P-bar 1e-8, F 1e-7 (tight oracle, float32 CG inside
    the float64 Newton refinement)."""
    cells = _cells(4, seed=9, sizes=(15, 21))
    batch = RVEBatch([c[0] for c in cells], [c[1] for c in cells], [c[2] for c in cells],
                     precision="mixed", autotune=True)
    st = batch.solve(np.stack([c[3] for c in cells]), tol_newton=1e-10, tol_cg=1e-8)
    assert all(s["status"] == 0 for s in st)
    Pb = batch.homogenized_P()
    for i, (shape, ph, params, Fbar) in enumerate(cells):
        prob = solver.SVKProblem.from_phase(ph, params)
        prob.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=1e-13)
        ref = prob.homogenized_P()
        assert np.abs(Pb[i] - ref).max() < 1e-8 * np.abs(ref).max(), i
        F = batch.get_F(i)
        assert np.linalg.norm(F - prob.F) / np.linalg.norm(prob.F) < 1e-7, i
    batch.close()
