"""Python binding of the C ABI (same function names as ``include/rve.h``).

Only argument marshalling happens here.  Tensor fields are exchanged as
float64 arrays shaped ``[3, 3, nx, ny, nz]`` (numpy on the host, or torch
CUDA tensors on the device), which is exactly the C layout ``[9][n]``.
Device memory for a handle is taken from PyTorch's allocator and handed to
the library as its workspace.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _lib
from ._lib import lib

try:
    import torch
except Exception:  # pragma: no cover
    torch = None

_MODELS = {"svk": _lib.RVE_SVK, "j2": _lib.RVE_J2}
_PREC = {"fp64": _lib.RVE_FP64, "mixed": _lib.RVE_MIXED}
_TAN = {"auto": _lib.RVE_TAN_AUTO, "full81": _lib.RVE_TAN_FULL81,
        "recompute": _lib.RVE_TAN_RECOMPUTE, "sym45": _lib.RVE_TAN_SYM45}


class RVEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code}: "
                         f"{lib.rve_status_string(code).decode()})")
        self.code = code


def _check(code, h=None, what=""):
    if code != 0:
        msg = lib.rve_last_error(h).decode() if h else what
        raise RVEError(code, msg or what)


def _is_torch_cuda(a):
    return torch is not None and isinstance(a, torch.Tensor) and a.is_cuda


def _in_ptr(a, n):
    """(pointer, on_device, keepalive) of a float64 [9][n] input."""
    if _is_torch_cuda(a):
        t = a.detach().to(torch.float64).contiguous()
        if t.numel() != 9 * n:
            raise ValueError("expected 9*n values")
        return C.c_void_p(t.data_ptr()), 1, t
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if arr.size != 9 * n:
        raise ValueError("expected 9*n values")
    return arr.ctypes.data_as(C.c_void_p), 0, arr


def _options(precision="fp64", tangent="auto", max_newton=50, max_cg=10000,
             cg_tol_floor=1e-5, cg_atol=0.0, mixed_refine=0, residual="floatfloat",
             autotune=False, precond="none", stream=None):
    o = _lib.rve_options()
    lib.rve_default_options(C.byref(o))
    o.precision = _PREC[precision]
    o.tangent = _TAN[tangent]
    o.max_newton = int(max_newton)
    o.max_cg = int(max_cg)
    o.cg_tol_floor = float(cg_tol_floor)
    o.cg_atol = float(cg_atol)
    o.mixed_refine = int(mixed_refine)
    o.residual = {"floatfloat": 0, "fp64": 1}[residual]
    o.autotune = 1 if autotune else 0
    o.precond = {"none": 0, "reference": 1}[precond]
    if stream is None and torch is not None and torch.cuda.is_available():
        stream = torch.cuda.current_stream().cuda_stream
    o.stream = C.c_void_p(int(stream)) if stream else None
    return o


def rve_workspace_size(shape, model="svk", **opt):
    nbytes = C.c_size_t(0)
    o = _options(**opt)
    _check(lib.rve_workspace_size(int(shape[0]), int(shape[1]), int(shape[2]),
                                  _MODELS[model], C.byref(o), C.byref(nbytes)),
           what="rve_workspace_size")
    return int(nbytes.value)


def rve_create(shape, model="svk", phase=None, phase_params=None,
               voxel_params=None, torch_workspace=True, **opt):
    """Returns (handle, keepalive) -- keepalive owns the device workspace."""
    nx, ny, nz = (int(s) for s in shape)
    o = _options(**opt)
    keep = []
    if torch_workspace and torch is not None and torch.cuda.is_available():
        nbytes = rve_workspace_size(shape, model, **opt)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        keep.append(ws)
        o.workspace = C.c_void_p(ws.data_ptr())
        o.workspace_bytes = nbytes
    h = C.c_void_p()
    ph = pp = vp = None
    nphase = 0
    if phase is not None:
        ph = np.ascontiguousarray(phase, dtype=np.uint8)
        pp = np.ascontiguousarray(phase_params, dtype=np.float64)
        nphase = pp.shape[0]
        keep += [ph, pp]
    vptr = None
    if voxel_params is not None and _is_torch_cuda(voxel_params):
        # device tensor: the library converts it on the device
        t = voxel_params.detach().to(torch.float64).contiguous()
        if t.numel() != (4 if model == "j2" else 2) * nx * ny * nz:
            raise ValueError("voxel_params must hold nparam * n values")
        keep.append(t)
        vptr = C.c_void_p(t.data_ptr())
    elif voxel_params is not None:
        vp = np.ascontiguousarray(voxel_params, dtype=np.float64)
        keep.append(vp)
        vptr = vp.ctypes.data_as(C.c_void_p)
    ptr = (lambda a: a.ctypes.data_as(C.c_void_p) if a is not None else None)
    code = lib.rve_create(C.byref(h), nx, ny, nz, _MODELS[model], nphase,
                          ptr(ph), ptr(pp), vptr, C.byref(o))
    _check(code, what="rve_create failed")
    return h, keep


def rve_destroy(h):
    lib.rve_destroy(h)


def rve_set_macro_F(h, Fbar):
    F = np.ascontiguousarray(Fbar, dtype=np.float64).reshape(9)
    _check(lib.rve_set_macro_F(h, F.ctypes.data_as(C.c_void_p)), h)


def rve_solve_increment(h, tol_newton=1e-5, tol_cg=1e-8, check=True):
    st = _lib.rve_stats()
    code = lib.rve_solve_increment(h, float(tol_newton), float(tol_cg), C.byref(st))
    k = min(st.newton_iters, _lib.RVE_MAX_NEWTON_LOG)
    out = dict(status=code, newton_iters=st.newton_iters,
               cg_iters_total=st.cg_iters_total,
               cg_iters=list(st.cg_iters[:k]),
               rel_update=list(st.rel_update[:k]),
               residual=list(st.residual[:k]),
               elapsed_ms=st.elapsed_ms)
    if check:
        _check(code, h)
    return out


def rve_solve_step(h, Fbar, tol_newton=1e-5, tol_cg=1e-8, max_cuts=8, check=True):
    """Load step to Fbar with automatic halving of failed increments."""
    F = np.ascontiguousarray(Fbar, dtype=np.float64).reshape(9)
    st = _lib.rve_stats()
    code = lib.rve_solve_step(h, F.ctypes.data_as(C.c_void_p), float(tol_newton),
                              float(tol_cg), int(max_cuts), C.byref(st))
    out = dict(status=code, newton_iters=st.newton_iters,
               cg_iters_total=st.cg_iters_total, substeps=st.substeps,
               cuts=st.cuts, elapsed_ms=st.elapsed_ms,
               substep_to=list(st.substep_to[:min(st.substeps, _lib.RVE_MAX_NEWTON_LOG)]))
    if check:
        _check(code, h)
    return out


def rve_solve_mixed(h, Fbar, Pbar, mask, tol_stress=1e-8, tol_newton=1e-5, tol_cg=1e-8,
                    max_cuts=0, check=True):
    """Load step under mixed control: mask[c] (c = 3i+j) true prescribes
    P-bar_ij = Pbar[c] and frees F-bar_ij, false prescribes F-bar_ij = Fbar[c]."""
    F = np.ascontiguousarray(Fbar, dtype=np.float64).reshape(9)
    P = np.ascontiguousarray(Pbar, dtype=np.float64).reshape(9)
    M = np.ascontiguousarray(np.asarray(mask).reshape(9) != 0, dtype=np.int32)
    st = _lib.rve_stats()
    code = lib.rve_solve_mixed(h, F.ctypes.data_as(C.c_void_p), P.ctypes.data_as(C.c_void_p),
                               M.ctypes.data_as(C.c_void_p), float(tol_stress),
                               float(tol_newton), float(tol_cg), int(max_cuts), C.byref(st))
    out = dict(status=code, newton_iters=st.newton_iters,
               cg_iters_total=st.cg_iters_total, substeps=st.substeps,
               cuts=st.cuts, elapsed_ms=st.elapsed_ms, macro_iters=st.macro_iters,
               tangent_solves=st.tangent_solves,
               substep_to=list(st.substep_to[:min(st.substeps, _lib.RVE_MAX_NEWTON_LOG)]))
    if check:
        _check(code, h)
    return out


def rve_macro_F(h):
    """F-bar of the last committed state, 3x3."""
    F = np.empty(9, dtype=np.float64)
    _check(lib.rve_macro_F(h, F.ctypes.data_as(C.c_void_p)), h)
    return F.reshape(3, 3)


def _get(fn, h, ncomp, n, out):
    if out is not None and _is_torch_cuda(out):
        if out.dtype != torch.float64 or not out.is_contiguous() or out.numel() != ncomp * n:
            raise ValueError("out must be a contiguous float64 CUDA tensor")
        _check(fn(h, C.c_void_p(out.data_ptr()), 1), h)
        return out
    if out is None:
        out = np.empty(ncomp * n, dtype=np.float64)
    _check(fn(h, out.ctypes.data_as(C.c_void_p), 0), h)
    return out


def rve_get_F(h, n, out=None):
    return _get(lib.rve_get_F, h, 9, n, out)


def rve_get_P(h, n, out=None):
    return _get(lib.rve_get_P, h, 9, n, out)


def rve_get_K4(h, n, out=None):
    return _get(lib.rve_get_K4, h, 81, n, out)


def rve_get_history(h, n, out=None):
    if out is None:
        out = np.empty(7 * n, dtype=np.float64)
    _check(lib.rve_get_history(h, out.ctypes.data_as(C.c_void_p), 0), h)
    return out


def rve_adjoint_grad_mu(h, W, n, tol_cg=1e-12, out=None):
    """dJ/dmu per voxel for J = W : P-bar; returns (grad, cg_iterations)."""
    Wc = np.ascontiguousarray(W, dtype=np.float64).reshape(9)
    its = C.c_int(0)
    if out is not None and _is_torch_cuda(out):
        _check(lib.rve_adjoint_grad_mu(h, Wc.ctypes.data_as(C.c_void_p), float(tol_cg),
                                       C.c_void_p(out.data_ptr()), 1, C.byref(its)), h)
        return out, its.value
    g = np.empty(n, dtype=np.float64)
    _check(lib.rve_adjoint_grad_mu(h, Wc.ctypes.data_as(C.c_void_p), float(tol_cg),
                                   g.ctypes.data_as(C.c_void_p), 0, C.byref(its)), h)
    return g, its.value


def _grad_buffer(count, device):
    """(buffer, pointer, on_device): a float64 CUDA tensor written by the
    library in place (device=True), else a host array."""
    if device:
        t = torch.empty(count, dtype=torch.float64, device="cuda")
        return t, C.c_void_p(t.data_ptr()), 1
    a = np.empty(count, dtype=np.float64)
    return a, a.ctypes.data_as(C.c_void_p), 0


def rve_adjoint_grad(h, W, n, tol_cg=1e-12, device=False):
    """(dJ/dK, dJ/dmu) per voxel for J = W : P-bar from one adjoint solve;
    returns (grad_K, grad_mu, cg_iterations).  device=True: the gradients
    are CUDA tensors written by the library directly (no host copy)."""
    Wc = np.ascontiguousarray(W, dtype=np.float64).reshape(9)
    its = C.c_int(0)
    gK, pK, dev = _grad_buffer(n, device)
    gm, pm, _ = _grad_buffer(n, device)
    _check(lib.rve_adjoint_grad(h, Wc.ctypes.data_as(C.c_void_p), float(tol_cg), pK, pm, dev,
                                C.byref(its)), h)
    return gK, gm, its.value


def rve_adjoint_grad_params(h, W, n, nparam, tol_cg=1e-12, device=False):
    """dJ/d(parameters) per voxel, [nparam, n], for J = W : P-bar (SVK: K, mu;
    J2: K, mu, tau_y0, H at the history of the last increment's start), and
    the CG iterations (device=True: a CUDA tensor written directly)."""
    Wc = np.ascontiguousarray(W, dtype=np.float64).reshape(9)
    its = C.c_int(0)
    g, pg, dev = _grad_buffer(nparam * n, device)
    _check(lib.rve_adjoint_grad_params(h, Wc.ctypes.data_as(C.c_void_p), float(tol_cg), pg, dev,
                                       C.byref(its)), h)
    return g.reshape(nparam, n), its.value


def rve_homogenized_P(h):
    P = np.empty(9, dtype=np.float64)
    _check(lib.rve_homogenized_P(h, P.ctypes.data_as(C.c_void_p)), h)
    return P.reshape(3, 3)


def rve_set_F(h, F, n):
    p, dev, keep = _in_ptr(F, n)
    _check(lib.rve_set_F(h, p, dev), h)


def _unary(fn, h, A, n, out):
    p, dev, keep = _in_ptr(A, n)
    if dev:
        res = out if out is not None else torch.empty_like(keep)
        _check(fn(h, p, C.c_void_p(res.data_ptr()), 1), h)
        return res
    res = np.empty(9 * n, dtype=np.float64)
    _check(fn(h, p, res.ctypes.data_as(C.c_void_p), 0), h)
    return res


def rve_apply_operator(h, dF, n, out=None):
    return _unary(lib.rve_apply_operator, h, dF, n, out)


def rve_project(h, A, n, out=None):
    return _unary(lib.rve_project, h, A, n, out)


def rve_project_noalloc(shape, A, out, stream=None):
    """out = G : A (float64) without a handle and without any device
    allocation, for callers that cannot allocate device memory (the scratch
    lives in a fixed array inside the library).  A and out are contiguous
    float64 CUDA tensors of 9*nx*ny*nz values on the current device (out may
    be A).  Enqueues on `stream` (default: torch's current stream); raises
    RVEError on a non-zero status."""
    nx, ny, nz = (int(s) for s in shape)
    if not (_is_torch_cuda(A) and _is_torch_cuda(out)):
        raise ValueError("A and out must be CUDA tensors")
    dev = torch.cuda.current_device()
    for name, t in (("A", A), ("out", out)):
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() != 9 * nx * ny * nz:
            raise ValueError(f"{name} must hold 9*nx*ny*nz values")
        if t.device.index != dev:
            raise ValueError(f"{name} must be on the current device")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    code = lib.rve_project_noalloc(nx, ny, nz, C.c_void_p(A.data_ptr()),
                                   C.c_void_p(out.data_ptr()),
                                   C.c_void_p(int(stream)) if stream else None)
    _check(code, None, "rve_project_noalloc")


def rve_launch_count(h):
    c = C.c_longlong(0)
    _check(lib.rve_launch_count(h, C.byref(c)), h)
    return int(c.value)


def rve_save(h, path):
    """Checkpoint of the converged state of a handle."""
    _check(lib.rve_save(h, os.fsencode(path)), h)


def rve_load(path, stream=None):
    """Handle created from a checkpoint file (library-allocated memory)."""
    o = _options(stream=stream)
    h = C.c_void_p()
    _check(lib.rve_load(C.byref(h), os.fsencode(path), C.byref(o)), what=f"rve_load {path}")
    return h


TUNING_KNOBS = ("four_step_z", "z_blocks_per_sm", "four_step_y", "four_step_x",
                "composite_radices", "staged_z", "autotuned", "x_tile_half", "y_tile_half")


def rve_tuning(h):
    """Kernel variants in use (set by the autotuner or the defaults)."""
    k = (C.c_int * 9)()
    _check(lib.rve_tuning(h, k), h)
    return dict(zip(TUNING_KNOBS, (int(v) for v in k)))


def rve_set_tuning(h, **knobs):
    """Sets kernel variants by name (TUNING_KNOBS; the others keep their
    current values)."""
    cur = rve_tuning(h)
    cur.update(knobs)
    k = (C.c_int * 9)(*[int(cur[name]) for name in TUNING_KNOBS])
    _check(lib.rve_set_tuning(h, k), h)


def rve_kernel_timing(h, family, enable=True):
    _check(lib.rve_kernel_timing(h, int(family), int(bool(enable))), h)


def rve_set_wait_polls(h, polls):
    """Failure-test setting: polls of a bounded device wait before it gives
    up and the call reports RVE_ERR_TIMEOUT (default 1 << 20)."""
    _check(lib.rve_set_wait_polls(h, int(polls)), h)


def rve_kernel_time(h):
    ms = C.c_double(0)
    cnt = C.c_longlong(0)
    _check(lib.rve_kernel_time(h, C.byref(ms), C.byref(cnt)), h)
    return float(ms.value), int(cnt.value)


KERNEL_FAMILIES = ("zfwd", "fft_y_fwd", "fft_x_proj", "fft_y_inv", "zinv", "cg_update")


class RVE:
    """A periodic cell solved on the current CUDA device."""

    def __init__(self, shape, phase=None, phase_params=None, voxel_params=None,
                 model="svk", **opt):
        self.shape = tuple(int(s) for s in shape)
        self.n = int(np.prod(self.shape))
        self.h, self._keep = rve_create(self.shape, model, phase, phase_params,
                                        voxel_params, **opt)

    def close(self):
        h = getattr(self, "h", None)
        if h:
            rve_destroy(h)
            self.h = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape9(self, a):
        return a.reshape((3, 3) + self.shape)

    def set_macro_F(self, Fbar):
        rve_set_macro_F(self.h, Fbar)

    def solve_increment(self, tol_newton=1e-5, tol_cg=1e-8, check=True):
        return rve_solve_increment(self.h, tol_newton, tol_cg, check)

    def solve_step(self, Fbar, tol_newton=1e-5, tol_cg=1e-8, max_cuts=8, check=True):
        return rve_solve_step(self.h, Fbar, tol_newton, tol_cg, max_cuts, check)

    def solve_mixed(self, Fbar, Pbar, mask, tol_stress=1e-8, tol_newton=1e-5, tol_cg=1e-8,
                    max_cuts=0, check=True):
        return rve_solve_mixed(self.h, Fbar, Pbar, mask, tol_stress, tol_newton, tol_cg,
                               max_cuts, check)

    def macro_F(self):
        return rve_macro_F(self.h)

    def get_F(self, out=None):
        return self._shape9(rve_get_F(self.h, self.n, out))

    def get_P(self, out=None):
        return self._shape9(rve_get_P(self.h, self.n, out))

    def get_K4(self, out=None):
        return rve_get_K4(self.h, self.n, out).reshape((3, 3, 3, 3) + self.shape)

    def homogenized_P(self):
        return rve_homogenized_P(self.h)

    def adjoint_grad_mu(self, W, tol_cg=1e-12):
        """Gradient of W : P-bar with respect to per-voxel shear moduli, [*shape]."""
        g, its = rve_adjoint_grad_mu(self.h, W, self.n, tol_cg)
        return g.reshape(self.shape), its

    def adjoint_grad(self, W, tol_cg=1e-12, device=False):
        """(dJ/dK, dJ/dmu), each [*shape], for J = W : P-bar, and the CG
        iterations (device=True: CUDA tensors)."""
        gK, gm, its = rve_adjoint_grad(self.h, W, self.n, tol_cg, device)
        return gK.reshape(self.shape), gm.reshape(self.shape), its

    def adjoint_grad_params(self, W, tol_cg=1e-12, device=False):
        """dJ/d(K, mu[, tau_y0, H]) per voxel, [nparam, *shape], and the CG
        iterations (device=True: a CUDA tensor)."""
        nparam = 4 if lib.rve_model(self.h) == _MODELS["j2"] else 2
        g, its = rve_adjoint_grad_params(self.h, W, self.n, nparam, tol_cg, device)
        return g.reshape((nparam,) + self.shape), its

    def tape(self, enable=True):
        """J2: record (or stop recording) the path for adjoint_grad_path."""
        _check(lib.rve_tape(self.h, 1 if enable else 0), self.h)

    def tape_length(self):
        return int(lib.rve_tape_length(self.h))

    def adjoint_grad_path(self, W, tol_cg=1e-12, device=False):
        """J2: dJ/d(K, mu, tau_y0, H) per voxel, [4, *shape], for J = W : P-bar
        after the taped path (through the history), and the CG iterations
        (device=True: a CUDA tensor)."""
        Wc = np.ascontiguousarray(W, dtype=np.float64).reshape(9)
        its = C.c_int(0)
        g, pg, dev = _grad_buffer(4 * self.n, device)
        _check(lib.rve_adjoint_grad_path(self.h, Wc.ctypes.data_as(C.c_void_p), float(tol_cg),
                                         pg, dev, C.byref(its)), self.h)
        return g.reshape((4,) + self.shape), its.value

    def get_history(self):
        """J2: committed (Cp^-1 [6 symmetric components], eps_p) per voxel, [7, *shape]."""
        return rve_get_history(self.h, self.n).reshape((7,) + self.shape)

    def set_F(self, F):
        rve_set_F(self.h, F, self.n)

    def apply_operator(self, dF, out=None):
        return self._shape9(rve_apply_operator(self.h, dF, self.n, out))

    def project(self, A, out=None):
        return self._shape9(rve_project(self.h, A, self.n, out))

    def launch_count(self):
        return rve_launch_count(self.h)

    def tuning(self):
        return rve_tuning(self.h)

    def set_tuning(self, **knobs):
        rve_set_tuning(self.h, **knobs)

    def save(self, path):
        rve_save(self.h, path)

    @classmethod
    def load(cls, path, stream=None):
        """A cell resumed from a checkpoint written by save()."""
        self = cls.__new__(cls)
        self.h = rve_load(path, stream)
        dims = (C.c_int * 3)()
        _check(lib.rve_grid(self.h, dims), self.h)
        self.shape = tuple(int(d) for d in dims)
        self.n = int(np.prod(self.shape))
        self._keep = []
        return self


class RVEBatch:
    """Many independent cells of uneven size solved together (one CUDA graph
    per group of CG iterations, Newton steps in lockstep)."""

    def __init__(self, shapes, phases, phase_params, model="svk", **opt):
        n = len(shapes)
        self.shapes = [tuple(int(s) for s in sh) for sh in shapes]
        dims = np.ascontiguousarray(self.shapes, dtype=np.int32).reshape(-1)
        self._keep = [np.ascontiguousarray(ph, dtype=np.uint8) for ph in phases]
        self._keep += [np.ascontiguousarray(pp, dtype=np.float64) for pp in phase_params]
        nph = np.array([np.asarray(pp).shape[0] for pp in phase_params], dtype=np.int32)
        pptr = (C.c_void_p * n)(*[a.ctypes.data for a in self._keep[:n]])
        qptr = (C.c_void_p * n)(*[a.ctypes.data for a in self._keep[n:]])
        o = _options(**opt)
        h = C.c_void_p()
        code = lib.rve_batch_create(C.byref(h), n, dims.ctypes.data_as(C.c_void_p),
                                    _MODELS[model], nph.ctypes.data_as(C.c_void_p),
                                    C.cast(pptr, C.c_void_p), C.cast(qptr, C.c_void_p),
                                    C.byref(o))
        _check(code, what="rve_batch_create failed")
        self.h = h
        self.n = n
        self._dims = dims

    def close(self):
        h = getattr(self, "h", None)
        if h:
            lib.rve_batch_destroy(h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, Fbars, tol_newton=1e-5, tol_cg=1e-8, check=True, max_cuts=0):
        """One increment per cell (max_cuts > 0: with per-cell increment cutting)."""
        F = np.ascontiguousarray(Fbars, dtype=np.float64).reshape(self.n, 9)
        st = (_lib.rve_stats * self.n)()
        code = lib.rve_batch_solve_step(self.h, F.ctypes.data_as(C.c_void_p), float(tol_newton),
                                        float(tol_cg), int(max_cuts), C.cast(st, C.c_void_p))
        out = [dict(status=s.status, newton_iters=s.newton_iters,
                    cg_iters_total=s.cg_iters_total, elapsed_ms=s.elapsed_ms,
                    substeps=s.substeps, cuts=s.cuts) for s in st]
        if check and code != 0:
            raise RVEError(code, lib.rve_batch_last_error(self.h).decode())
        return out

    def homogenized_P(self):
        P = np.empty((self.n, 9), dtype=np.float64)
        _check(lib.rve_batch_homogenized_P(self.h, P.ctypes.data_as(C.c_void_p)),
               what="rve_batch_homogenized_P")
        return P.reshape(self.n, 3, 3)

    def get_F(self, i):
        h = lib.rve_batch_cell(self.h, int(i))
        n = int(np.prod(self.shapes[i]))
        return rve_get_F(h, n).reshape((3, 3) + self.shapes[i])

    def get_P(self, i):
        h = lib.rve_batch_cell(self.h, int(i))
        n = int(np.prod(self.shapes[i]))
        return rve_get_P(h, n).reshape((3, 3) + self.shapes[i])

    def launch_count(self):
        c = C.c_longlong(0)
        _check(lib.rve_batch_launch_count(self.h, C.byref(c)), what="launch count")
        return int(c.value)
