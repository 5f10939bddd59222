"""FP64 CPU oracle for the finite-strain FFT Newton-CG method (de Geus et al.).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call
or link anything from this directory; only the test-suite, the smoke check
and the benchmark's CPU-baseline arm use it.  It shares no code with the CUDA
path: the only common module is ``synth`` (seeded inputs, no method
arithmetic).

Plain numpy in float64, written from the paper's equations:

* ``tensor``     -- tensor products of the nomenclature table (Appendix A).
* ``fourier``    -- DFT (naive matrices or numpy.fft), the projection operator
                    G-hat of Eq. G / Eq. G_red, and G:A (Eq. weak:discr:FFT).
* ``svk``        -- Saint Venant-Kirchhoff stress and tangent (Sec. 4.2-4.3).
* ``j2``         -- finite-strain J2 plasticity with logarithmic elastic
                    strain and return mapping (Sec. 5.2-5.4).
* ``solver``     -- conjugate gradients, Newton iterations with the boundary
                    condition predictor (Sec. 3.1, Algorithm 1), incremental
                    loop, homogenised stress.
* ``adjoint``    -- gradient of the homogenised stress w.r.t. per-voxel shear
                    moduli (not in the paper; derived from the same
                    equilibrium equations).

Every function states the passage it follows.  Functions whose parity is not
pinned by an independent check say "parity unpinned" in their docstring.
"""
