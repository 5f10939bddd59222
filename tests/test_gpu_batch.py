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
