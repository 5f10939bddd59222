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
* One application of the tangent operator G:(K:dF) on the whole 125^3
  sphere cell (SVK, float32 and float64 paths) and on the whole 315^3
  Voronoi cell (J2, float32 with the stored tangent) against the oracle's
  G(K:dF) at every voxel (scipy.fft backend on all host cores).  The J2 cell
  takes its deformation from a table of 2048 random F (amplitude 0.004,
  plastic at about half of the (F, phase) pairs) by a random index map, so that the
  oracle's return map runs once per (F, phase) pair, not per voxel.
* 243^3 lognormal cell: the adjoint gradient dP-bar_xy/dmu_k equals the
  forward (localisation) formula (1/n) (F.2devE)_k : L_k with
  L = dF/dF-bar_xy, because P-bar = dW-bar/dF-bar and dW-bar/dmu_k =
  (1/n) devE_k:devE_k for the hyperelastic SVK law; L by central
  differences of two solves at F-bar +- h e_x(x)e_y.
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class _ScipyBackend:
    """The oracle's scipy.fft backend on all host cores for a block."""

    def __enter__(self):
        self.old = fourier.get_backend()
        try:
            fourier.set_backend("scipy", workers=os.cpu_count() or 1)
        except RuntimeError:
            fourier.set_backend("numpy")

    def __exit__(self, *exc):
        fourier.set_backend(self.old["name"], self.old["workers"])


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
    # the oracle's stress evaluated in extended precision: in float64 its
    # F^T F - I loses about log10(1/|E|) digits at these strains (7e-14 of
    # the largest stress at 1e-3), more than the bar below
    ld = np.longdouble
    Ps = svk.stress(Fs.astype(ld), K.reshape(-1)[idx].astype(ld), mu.reshape(-1)[idx].astype(ld))
    assert float(np.abs(P.reshape(3, 3, -1)[:, :, idx] - Ps).max()) < 1e-13 * float(np.abs(Ps).max())
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


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_spheres125_operator_at_full_size(precision):
    cfg = synth.config_spheres()
    shape, params, ph = cfg["shape"], cfg["phase_params"], cfg["phase"]
    rng = np.random.default_rng(21)
    F = synth.random_F(shape, rng, 0.1)
    dF = rng.standard_normal((3, 3) + shape)
    r = RVE(shape, phase=ph, phase_params=params, precision=precision)
    r.set_F(F)
    got = r.apply_operator(dF)
    r.close()
    _, K4 = svk.constitutive(F, params[ph, 0], params[ph, 1])
    with _ScipyBackend():
        ref = fourier.G(svk.tangent_apply(K4, dF))
    del K4
    if precision == "mixed":
        assert _rel(got, ref) < 5e-6
    else:
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_voronoi315_j2_operator_at_full_size():
    cfg = synth.config_voronoi_j2()
    shape, params, ph = cfg["shape"], cfg["phase_params"], cfg["phase"]
    n = int(np.prod(shape))
    rng = np.random.default_rng(22)
    S = 2048
    Ftab = synth.random_F((S, 1, 1), rng, 0.004).reshape(3, 3, S)
    idx = rng.integers(0, S, size=n)
    # the oracle's return map and tangent once per (F, phase) pair
    pp = np.concatenate([np.repeat(params[:1], S, 0), np.repeat(params[1:], S, 0)])
    mat = oj2.J2Material((2 * S, 1, 1), *(pp[:, k].reshape(2 * S, 1, 1) for k in range(4)))
    Fpair = np.concatenate([Ftab, Ftab], axis=-1)[:, :, :, None, None]
    _, K4tab = mat.constitutive(Fpair)
    K4tab = K4tab.reshape(3, 3, 3, 3, 2 * S)
    plastic = np.mean(mat._trial[1] > 0)
    assert 0.3 < plastic < 0.7  # elastic and elasto-plastic tangents both present
    combo = idx + S * ph.reshape(-1).astype(np.int64)
    F = np.ascontiguousarray(Ftab[:, :, idx]).reshape((3, 3) + shape)
    dF = rng.standard_normal((3, 3) + shape)
    r = RVE(shape, model="j2", phase=ph, phase_params=params, precision="mixed")
    r.set_F(F)
    got = r.apply_operator(dF)
    r.close()
    del F
    KdF = np.empty((3, 3, n))
    dFv = dF.reshape(3, 3, n)
    for a in range(0, n, 1 << 20):
        b = min(n, a + (1 << 20))
        KdF[:, :, a:b] = svk.tangent_apply(K4tab[..., combo[a:b]], dFv[:, :, a:b])
    del dF, dFv
    with _ScipyBackend():
        ref = fourier.G(KdF.reshape((3, 3) + shape))
    assert _rel(got, ref) < 5e-6


def test_lognormal243_adjoint_equals_forward_formula():
    cfg = synth.config_lognormal()
    shape = cfg["shape"]
    vp = cfg["voxel_params"]
    n = int(np.prod(shape))
    Fb = cfg["schedule"][0]
    E = np.zeros((3, 3))
    E[0, 1] = 1.0
    h = 1e-4

    def solve(Fbar, grad=False):
        r = RVE(shape, voxel_params=vp, precision="mixed")
        r.set_macro_F(Fbar)
        r.solve_increment(1e-10, cfg["tol_cg"])
        F = r.get_F().reshape(3, 3, n)
        g = r.adjoint_grad(E, tol_cg=1e-10)[1].reshape(-1) if grad else None
        r.close()
        return F, g

    F, g = solve(Fb, grad=True)
    L = solve(Fb + h * E)[0]
    L -= solve(Fb - h * E)[0]
    L /= 2 * h
    # (dP/dmu)_k = F_k . 2 dev(E_k), E = (F^T F - I)/2, at fixed K
    C = np.einsum("kiv,kjv->ijv", F, F)
    Eg = 0.5 * (C - np.eye(3)[:, :, None])
    dev = Eg - (np.trace(Eg) / 3.0)[None, None, :] * np.eye(3)[:, :, None]
    dPdmu = 2.0 * np.einsum("ikv,kjv->ijv", F, dev)
    g_fwd = np.einsum("ijv,ijv->v", dPdmu, L) / n
    gmax = np.abs(g_fwd).max()
    err = np.abs(g - g_fwd)
    print("adjoint vs forward formula at 243^3: max rel per entry",
          float((err / (np.abs(g_fwd) + 1e-300)).max()), "max abs / gmax", float(err.max() / gmax))
    assert np.all(err <= 1e-5 * np.abs(g_fwd) + 1e-7 * gmax)
