"""The C-ABI library builds, loads without a GPU and exports every function
that include/*.h declares (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(hdr).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(rve_[A-Za-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1603_08893_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_1603_08893_gb300 import _lib
    assert _declared() <= set(_lib._SIGS), _declared() - set(_lib._SIGS)


def test_options_and_status_without_gpu(lib):
    from paper_1603_08893_gb300 import _lib
    o = _lib.rve_options()
    _lib.lib.rve_default_options(ctypes.byref(o))
    assert o.max_newton == 50 and o.max_cg == 10000 and o.precision == 0
    assert _lib.lib.rve_status_string(-5).decode().startswith("CG breakdown")
    n = ctypes.c_size_t(0)
    # even sizes are accepted (Appendix C); non-positive sizes are not
    assert _lib.lib.rve_workspace_size(4, 5, 5, 0, ctypes.byref(o), ctypes.byref(n)) == 0
    assert _lib.lib.rve_workspace_size(0, 5, 5, 0, ctypes.byref(o), ctypes.byref(n)) == -1
    assert _lib.lib.rve_workspace_size(125, 125, 125, 0, ctypes.byref(o), ctypes.byref(n)) == 0
    assert n.value > 9 * 125 ** 3 * 8 * 4
    o.precision = 1
    m = ctypes.c_size_t(0)
    assert _lib.lib.rve_workspace_size(125, 125, 125, 0, ctypes.byref(o), ctypes.byref(m)) == 0
    assert 0 < m.value < 2 * n.value


def test_load_rejects_malformed_checkpoint(lib, tmp_path):
    import ctypes
    from paper_1603_08893_gb300 import _lib
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"not a checkpoint" * 4)
    h = ctypes.c_void_p()
    assert _lib.lib.rve_load(ctypes.byref(h), str(bad).encode(), None) == -1
    assert _lib.lib.rve_load(ctypes.byref(h), str(tmp_path / "missing").encode(), None) == -1
