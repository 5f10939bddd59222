"""Checkpoint / resume: a cell saved after some increments and loaded into a
new handle continues bit-identically to the saved one (deterministic
reductions, material restored in its internal form)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1603_08893_gb300 import RVE  # noqa: E402

J2_PARAMS = np.array([[1 / 1.2, 1 / 2.6, 0.003, 0.01], [1 / 1.2, 1 / 2.6, 0.006, 0.01]])


def _cell(model, prec):
    if model == "svk":
        rng = np.random.default_rng(21)
        shape = (9, 11, 13)
        ph = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
        r = RVE(shape, phase=ph, phase_params=synth.two_phase_params(10.0), precision=prec)
        sched = synth.ramp(synth.simple_shear(0.08), 4)
    else:
        ph, _ = synth.voronoi(9, 8, np.random.default_rng(2))
        r = RVE(ph.shape, model="j2", phase=ph, phase_params=J2_PARAMS, precision=prec)
        sched = synth.ramp(synth.simple_shear(0.008), 4)
    return r, sched


@pytest.mark.parametrize("model,prec", [("svk", "fp64"), ("svk", "mixed"), ("j2", "mixed"),
                                        ("j2", "fp64")])
def test_resume_is_bit_identical(tmp_path, model, prec):
    r, sched = _cell(model, prec)
    for Fb in sched[:2]:
        r.set_macro_F(Fb)
        r.solve_increment(1e-6, 1e-9)
    path = str(tmp_path / "cell.ckpt")
    r.save(path)
    q = RVE.load(path)
    assert q.shape == r.shape
    for Fb in sched[2:]:
        for c in (r, q):
            c.set_macro_F(Fb)
            c.solve_increment(1e-6, 1e-9)
    assert np.array_equal(r.get_F(), q.get_F())
    assert np.array_equal(r.get_P(), q.get_P())
    assert np.array_equal(r.homogenized_P(), q.homogenized_P())
    if model == "j2":
        assert np.array_equal(r.get_history(), q.get_history())
    r.close()
    q.close()
