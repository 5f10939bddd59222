"""GB300-native finite-strain FFT homogenisation (de Geus et al., CMAME 2017).

The matrix-free Newton-CG solver of the paper -- projected tangent operator
G:(K:dF) with hand-written odd-length FFT passes, CG, constitutive update --
runs in CUDA kernels compiled for sm_103a into ``_build/librve.so`` and is
called through its C ABI (``include/rve.h``).  ``rve`` mirrors the C names;
:class:`RVE` is a convenience wrapper.  PyTorch is used only for device
memory and streams.

The compiled library is loaded on first use of a solver name (so that
``paper_1603_08893_gb300.build`` can run before it exists).
"""
_EXPORTS = ("RVE", "RVEBatch", "RVEError", "rve_adjoint_grad", "rve_adjoint_grad_mu", "rve_adjoint_grad_params", "rve_apply_operator", "rve_create", "rve_destroy",
            "rve_get_F", "rve_get_K4", "rve_get_P", "rve_get_history", "rve_homogenized_P",
            "rve_kernel_time", "rve_kernel_timing", "rve_set_wait_polls", "rve_launch_count", "rve_tuning", "rve_set_tuning", "rve_save", "rve_load",
            "rve_project", "rve_project_noalloc", "rve_set_F", "rve_set_macro_F", "rve_solve_increment", "rve_solve_step",
            "rve_solve_mixed", "rve_macro_F",
            "rve_workspace_size", "KERNEL_FAMILIES")

__all__ = list(_EXPORTS)


def __getattr__(name):
    if name in _EXPORTS:
        from . import rve
        return getattr(rve, name)
    raise AttributeError(name)
