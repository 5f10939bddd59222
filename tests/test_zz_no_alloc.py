"""The allocation-free projection entry point (rve_project_noalloc).

Some callers of this library cannot allocate device memory: plugins whose
host program owns every device allocation, and real-time paths that must
not allocate (an allocation can synchronise the device).  For them the
library keeps the projection's scratch in a fixed device array.  These tests
call that entry point through the C ABI twice in a row and check each
result against the FP64 oracle's G (Eq. G / Eq. G_red, Appendix C on even
axes) and against the regular rve_project entry point, with the tolerance
used for the projection elsewhere in the tests (1e-12 of the largest
entry); they also check the in-place form (out = A), that the calls leave
the device's free memory unchanged, the size limits and the binding's
argument checks.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from oracle import fourier

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1603_08893_gb300 import RVE, rve_project_noalloc  # noqa: E402
from paper_1603_08893_gb300._lib import RVE_ERR_INVALID, RVE_ERR_NOMEM, lib  # noqa: E402

TOL = 1e-12


def _maxrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _call(shape, A, out, stream):
    return lib.rve_project_noalloc(shape[0], shape[1], shape[2],
                                   ctypes.c_void_p(A.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("shape", [(31, 31, 31), (15, 21, 9), (45, 45, 45), (16, 10, 12)])
def test_noalloc_projection_matches_oracle_and_rve_project(shape):
    rng = np.random.default_rng(11)
    ref_handle = RVE(shape, phase=np.zeros(shape, np.uint8), phase_params=[[1.0, 0.5]])
    stream = torch.cuda.current_stream()
    out = torch.empty((3, 3) + shape, dtype=torch.float64, device="cuda")
    for call in range(2):
        # a different field each call: nothing of the previous call's
        # contents of the shared scratch may leak into the result
        A = rng.standard_normal((3, 3) + shape)
        At = torch.from_numpy(A).cuda()
        assert _call(shape, At, out, stream) == 0
        stream.synchronize()
        got = out.cpu().numpy()
        assert _maxrel(got, fourier.G(A)) < TOL, call
        assert _maxrel(got, ref_handle.project(A)) < TOL, call
    ref_handle.close()


def test_noalloc_in_place_and_no_device_allocation():
    shape = (27, 21, 15)
    rng = np.random.default_rng(12)
    stream = torch.cuda.current_stream()
    A = rng.standard_normal((3, 3) + shape)
    buf = torch.from_numpy(A).cuda()
    assert _call(shape, buf, buf, stream) == 0  # first call: per-device set-up
    stream.synchronize()
    assert _maxrel(buf.cpu().numpy(), fourier.G(A)) < TOL
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for call in range(2):
        B = rng.standard_normal((3, 3) + shape)
        buf.copy_(torch.from_numpy(B))
        assert _call(shape, buf, buf, stream) == 0  # out = A
        stream.synchronize()
        assert _maxrel(buf.cpu().numpy(), fourier.G(B)) < TOL, call
        assert torch.cuda.mem_get_info()[0] == free0, call
        assert torch.cuda.memory_allocated() == alloc0, call


def test_noalloc_rejects_grids_beyond_its_scratch():
    shape = (63, 63, 63)  # half spectrum of 9 components > 16 MiB
    A = torch.zeros((3, 3) + shape, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    assert _call(shape, A, A, stream) == RVE_ERR_NOMEM
    assert _call((0, 5, 5), A, A, stream) == RVE_ERR_INVALID
    assert _call((5, 5, 4096), A, A, stream) == RVE_ERR_INVALID
    code = lib.rve_project_noalloc(5, 5, 5, None, ctypes.c_void_p(A.data_ptr()), None)
    assert code == RVE_ERR_INVALID


def test_noalloc_binding_checks_its_arguments():
    shape = (9, 9, 9)
    good = torch.zeros((3, 3) + shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        rve_project_noalloc(shape, good.float(), good)
    with pytest.raises(ValueError):
        rve_project_noalloc(shape, good[..., :8], good)
    with pytest.raises(ValueError):
        rve_project_noalloc(shape, good.transpose(2, 4), good)
    with pytest.raises(ValueError):
        rve_project_noalloc(shape, good.cpu(), good)
    rng = np.random.default_rng(13)
    A = rng.standard_normal((3, 3) + shape)
    out = torch.empty_like(good)
    rve_project_noalloc(shape, torch.from_numpy(A).cuda(), out)
    torch.cuda.current_stream().synchronize()
    assert _maxrel(out.cpu().numpy(), fourier.G(A)) < TOL
