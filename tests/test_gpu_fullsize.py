"""Parity at the benchmark workloads' full sizes, in the launch configuration
bench.py times: on outputs the oracle computes voxel by voxel and on
properties that hold at any size (a full oracle solve of these grids is
hours of CPU time).

* 125^3 spheres, mixed path (fused float32 CG iteration on the four-step
  kernels, float-float residual): the converged increment has <F> = F-bar,
  F compatible and in equilibrium by the oracle's own float64 G (numpy FFT
  backend), the GPU's stress equals the oracle's constitutive response at
  sampled voxels, its reported residual ||G:P|| equals the oracle's, and
  P-bar is the average of the oracle's stress.
* 243^3 lognormal shear modulus (adjoint workload): P-bar is homogeneous of
  degree one in the moduli (equilibrium is unchanged when all moduli scale),
  so sum_v (mu_v dJ/dmu_v + K_v dJ/dK_v) = J for J = W : P-bar (Euler).
* 315^3 J2 constitutive update (the size of the J2 workload): P at sampled
  voxels against the oracle's return map from the virgin state.
"""
import os

import numpy as np
import pytest

import synth
from oracle import fourier, j2 as oj2, svk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1603_08893_gb300 import RVE  # noqa: E402


def _norm(A):
    return float(np.sqrt(np.sum(A * A)))


def test_spheres125_increment_at_full_size():
    cfg = synth.config_spheres()
    shape = cfg["shape"]
    params = cfg["phase_params"]
    ph = cfg["phase"]
    r = RVE(shape, phase=ph, phase_params=params, precision="mixed")
    Fb = cfg["schedule"][0]
    r.set_macro_F(Fb)
    st = r.solve_increment(1e-8, cfg["tol_cg"])
    F = r.get_F()
    P = r.get_P()
    Pbar = r.homogenized_P()
    r.close()
    assert np.abs(F.mean(axis=(2, 3, 4)) - Fb).max() < 1e-12
    K, mu = params[ph, 0], params[ph, 1]
    idx = np.random.default_rng(0).choice(int(np.prod(shape)), 400, replace=False)
    Fs = F.reshape(3, 3, -1)[:, :, idx]
    Ps = svk.stress(Fs, K.reshape(-1)[idx], mu.reshape(-1)[idx])
    assert np.abs(P.reshape(3, 3, -1)[:, :, idx] - Ps).max() < 1e-13 * np.abs(Ps).max()
    old = fourier.get_backend()
    try:
        fourier.set_backend("scipy", workers=os.cpu_count() or 1)
    except RuntimeError:
        fourier.set_backend("numpy")
    try:
        W = F - Fb[:, :, None, None, None]
        assert _norm(fourier.G(W) - W) < 1e-10 * _norm(W)     # compatible
        res = _norm(fourier.G(P))
    finally:
        fourier.set_backend(old["name"], old["workers"])
    assert res < 1e-8 * _norm(P)                              # equilibrium
    assert abs(res - st["residual"][-1]) < 1e-12 * _norm(P)   # the GPU's float64 residual
    assert np.abs(Pbar - P.mean(axis=(2, 3, 4))).max() < 1e-13


def test_lognormal243_adjoint_euler_identity():
    cfg = synth.config_lognormal()
    shape = cfg["shape"]
    vp = cfg["voxel_params"]
    r = RVE(shape, voxel_params=vp, precision="mixed")
    r.set_macro_F(cfg["schedule"][0])
    r.solve_increment(1e-10, cfg["tol_cg"])
    W = np.zeros((3, 3))
    W[0, 1] = 1.0
    gK, gmu, _ = r.adjoint_grad(W, tol_cg=1e-10)
    J = float(np.sum(W * r.homogenized_P()))
    r.close()
    lhs = float(np.sum(vp[0] * gK) + np.sum(vp[1] * gmu))
    assert abs(lhs - J) < 1e-6 * abs(J)


def test_j2_315_constitutive_sampled():
    n = 315
    shape = (n, n, n)
    rng = np.random.default_rng(5)
    ph = (rng.uniform(size=shape) < 0.5).astype(np.uint8)
    params = np.array([[1 / 1.2, 1 / 2.6, 0.003, 0.01], [1 / 1.2, 1 / 2.6, 0.006, 0.01]])
    F = synth.random_F(shape, rng, 0.01)
    r = RVE(shape, model="j2", phase=ph, phase_params=params, precision="mixed")
    r.set_F(F)
    P = r.get_P()
    r.close()
    idx = rng.choice(n ** 3, 500, replace=False)
    Fv = np.moveaxis(F.reshape(3, 3, -1)[:, :, idx], -1, 0)
    p = params[ph.reshape(-1)[idx]]
    m = len(idx)
    st = oj2.return_map(Fv, np.broadcast_to(np.eye(3), (m, 3, 3)).copy(), np.zeros(m),
                        p[:, 0], p[:, 1], p[:, 2], p[:, 3])
    got = np.moveaxis(P.reshape(3, 3, -1)[:, :, idx], -1, 0)
    assert st["plastic"].mean() > 0.2   # the sample reaches the plastic branch
    assert np.abs(got - st["P"]).max() < 1e-12 * np.abs(st["P"]).max()
