"""The allocation-free projection entry point (rve_project_noalloc).

Some callers of this library cannot allocate device memory -- code that
runs while a CUDA graph is being captured, plugins whose host program owns
every device allocation, real-time paths that must not allocate.  For them
the library keeps the projection's scratch in a fixed device array.  This
test calls that entry point through the C ABI twice in a row and checks each
result against the regular rve_project entry point, with the tolerance used
for the projection elsewhere in the tests (1e-12 of the largest entry).
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1603_08893_gb300 import RVE  # noqa: E402
from paper_1603_08893_gb300._lib import RVE_ERR_NOMEM, lib  # noqa: E402


def _maxrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("shape", [(31, 31, 31), (15, 21, 9), (45, 45, 45)])
def test_noalloc_projection_matches_rve_project(shape):
    rng = np.random.default_rng(11)
    ref_handle = RVE(shape, phase=np.zeros(shape, np.uint8), phase_params=[[1.0, 0.5]])
    stream = torch.cuda.current_stream()
    out = torch.empty((3, 3) + shape, dtype=torch.float64, device="cuda")
    for call in range(2):
        # a different field each call: nothing of the previous call's
        # contents of the shared scratch may leak into the result
        A = rng.standard_normal((3, 3) + shape)
        ref = ref_handle.project(A)
        At = torch.from_numpy(A).cuda()
        code = lib.rve_project_noalloc(shape[0], shape[1], shape[2],
                                       ctypes.c_void_p(At.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream))
        assert code == 0
        stream.synchronize()
        assert _maxrel(out.cpu().numpy(), ref) < 1e-12
    ref_handle.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    shape = (63, 63, 63)  # half spectrum of 9 components > 16 MiB
    A = torch.zeros((3, 3) + shape, dtype=torch.float64, device="cuda")
    code = lib.rve_project_noalloc(63, 63, 63, ctypes.c_void_p(A.data_ptr()),
                                   ctypes.c_void_p(A.data_ptr()), None)
    assert code == RVE_ERR_NOMEM
    code = lib.rve_project_noalloc(0, 5, 5, ctypes.c_void_p(A.data_ptr()),
                                   ctypes.c_void_p(A.data_ptr()), None)
    assert code == -1
