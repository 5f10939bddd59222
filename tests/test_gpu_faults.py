"""Failure detection, injected from the host (no kernel is made to fault,
trap or hang): non-finite fields and macroscopic loads, iteration caps, a
workspace that is too small.  Every failed increment leaves the last
committed state in place."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1603_08893_gb300 import RVE, RVEError  # noqa: E402
from paper_1603_08893_gb300 import _lib  # noqa: E402

SHAPE = (9, 11, 13)


def _cell(**opt):
    rng = np.random.default_rng(31)
    ph = (rng.uniform(size=SHAPE) < 0.3).astype(np.uint8)
    return RVE(SHAPE, phase=ph, phase_params=synth.two_phase_params(20.0), **opt)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nonfinite_field_is_detected(prec):
    r = _cell(precision=prec)
    F = np.broadcast_to(np.eye(3)[:, :, None, None, None], (3, 3) + SHAPE).copy()
    F[0, 1, 4, 5, 6] = np.nan
    # the constitutive update of the new field reports it
    with pytest.raises(RVEError) as e:
        r.set_F(F)
    assert e.value.code == -7
    r.close()


def test_nonfinite_macro_load_is_rejected():
    r = _cell()
    bad = synth.simple_shear(0.01)
    bad[1, 2] = np.inf
    with pytest.raises(RVEError) as e:
        r.set_macro_F(bad)
    assert e.value.code == -1
    r.close()


@pytest.mark.parametrize("opt,code", [(dict(max_cg=3), -4), (dict(max_newton=1), -6)])
def test_iteration_caps_roll_back(opt, code):
    r = _cell(**opt)
    F0 = r.get_F()
    r.set_macro_F(synth.simple_shear(0.05))
    st = r.solve_increment(check=False)
    assert st["status"] == code
    assert np.array_equal(r.get_F(), F0)
    r.close()


def test_workspace_too_small_is_reported():
    o = _lib.rve_options()
    _lib.lib.rve_default_options(ctypes.byref(o))
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    o.workspace = ctypes.c_void_p(ws.data_ptr())
    o.workspace_bytes = 1024
    ph = np.zeros(SHAPE, np.uint8)
    pp = np.array([[1.0, 0.5]])
    h = ctypes.c_void_p()
    code = _lib.lib.rve_create(ctypes.byref(h), *SHAPE, 0, 1, ph.ctypes.data_as(ctypes.c_void_p),
                               pp.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(o))
    assert code == -3 and not h.value


def test_device_wait_timeout_is_reported_and_rolled_back():
    """The last pass of the fused float32 CG iteration waits, bounded, on its
    own TMA copies.  With the poll count set to 0 every first wait gives up
    at once (the block then waits, bounded, for its copies to land, so
    nothing faults and nothing hangs): the increment ends with
    RVE_ERR_TIMEOUT and the committed state stays in place; with the default
    poll count restored the same increment solves to the result of a handle
    that never timed out."""
    from paper_1603_08893_gb300 import rve_set_wait_polls

    shape = (45, 45, 45)  # four-step lengths: the TMA-staged last z pass
    rng = np.random.default_rng(32)
    ph = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    kw = dict(phase=ph, phase_params=synth.two_phase_params(20.0), precision="mixed")
    steps = [synth.simple_shear(0.01), synth.simple_shear(0.02)]
    r = RVE(shape, **kw)
    r.set_macro_F(steps[0])
    r.solve_increment()
    F1 = r.get_F()
    rve_set_wait_polls(r.h, 0)
    r.set_macro_F(steps[1])
    st = r.solve_increment(check=False)
    assert st["status"] == _lib.RVE_ERR_TIMEOUT
    assert np.array_equal(r.get_F(), F1)
    rve_set_wait_polls(r.h, 1 << 20)
    st = r.solve_increment(check=False)
    assert st["status"] == 0
    ref = RVE(shape, **kw)
    for Fb in steps:
        ref.set_macro_F(Fb)
        ref.solve_increment()
    assert np.array_equal(r.get_F(), ref.get_F())
    r.close()
    ref.close()
