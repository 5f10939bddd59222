"""The batch workload (256 SVK cells, one increment each from F = I to a
random F-bar = I + H, H_ij uniform in +-0.05) has cells that the GPU reports
as failed (Newton divergence or det F <= 0), in float32/float64 mixed
precision and in plain float64, with up to 10 halvings of the load step.
This checks the smallest of them (cell 159: 21^3, contrast 40.6, det F-bar
0.93) with the FP64 oracle under the same load-step cutting: the oracle's
Newton-CG fails on it too, so the failure belongs to the Saint
Venant-Kirchhoff cell under that compression, not to the GPU path."""
import numpy as np
import pytest

import synth
from oracle import solver


@pytest.mark.slow
def test_oracle_also_fails_on_the_smallest_failing_batch_cell():
    cells = synth.config_batch()
    c = cells[159]
    assert c["shape"] == (21, 21, 21)
    assert np.linalg.det(c["Fbar"]) < 1.0  # a compression
    prob = solver.SVKProblem.from_phase(c["phase"], c["phase_params"])
    with pytest.raises(solver.SolverError):
        solver.solve_step(prob, c["Fbar"], 1e-5, 1e-8, max_cuts=4, max_cg=20000)
