"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances: float64 path 1e-12 for single operator applications and 1e-10
(relative 2-norm over the field) for full solves; mixed path (float32 CG
operator) 5e-6 relative for one operator application -- float32 round-off
accumulated over three DFT passes of length <= 63 -- and P-bar 1e-8 /
fields 1e-7 for converged solves.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import fourier, solver, svk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1603_08893_gb300 import RVE, RVEError  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SHAPES = [(1, 1, 1), (3, 5, 7), (5, 1, 3), (9, 11, 13), (15, 15, 15),
          (21, 27, 33), (31, 31, 31), (45, 45, 45), (63, 63, 63), (27, 3, 125),
          (81, 75, 7), (105, 9, 5), (7, 5, 225),
          # even sizes (Appendix C: G-hat zeroed at Nyquist frequencies)
          (4, 6, 8), (16, 16, 16), (15, 16, 17), (2, 3, 4), (10, 12, 14)]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def _random_problem(shape, seed, prec="fp64", tangent="auto", amp=0.15):
    rng = np.random.default_rng(seed)
    phase = (rng.uniform(size=shape) < 0.35).astype(np.uint8)
    params = synth.two_phase_params(7.0)
    r = RVE(shape, phase=phase, phase_params=params, precision=prec, tangent=tangent)
    F = synth.random_F(shape, rng, amp)
    r.set_F(F)
    K = params[phase, 0]
    mu = params[phase, 1]
    return r, F, K, mu, rng


@pytest.mark.parametrize("shape", SHAPES)
def test_projection_matches_oracle(shape):
    rng = np.random.default_rng(sum(shape))
    r = RVE(shape, phase=np.zeros(shape, np.uint8), phase_params=[[1.0, 0.5]])
    A = rng.standard_normal((3, 3) + shape)
    got = r.project(A)
    ref = fourier.G(A)
    if np.abs(ref).max() == 0:
        assert np.abs(got).max() < 1e-14
    else:
        assert maxrel(got, ref) < 1e-12
    # device-resident input and output
    At = torch.from_numpy(A).cuda()
    got_d = r.project(At).cpu().numpy()
    assert np.array_equal(got_d, got)
    r.close()


# x and y lengths with four-step float-float passes (several tiles, ragged
# last kz tile, even z lengths for the Nyquist planes)
FF_FOURSTEP_SHAPES = [(125, 125, 6), (125, 15, 125), (243, 243, 3), (315, 21, 4),
                      (15, 315, 2), (63, 45, 9), (33, 27, 20)]


@pytest.mark.parametrize("shape", SHAPES + FF_FOURSTEP_SHAPES)
def test_floatfloat_projection_matches_oracle(shape):
    """G:A in the float-float arithmetic of the mixed path (hi + lo float
    pairs, rounding ~2^-47 relative to the operands per operation): the
    transform's error stays at the float64 bar of this test family."""
    rng = np.random.default_rng(sum(shape) + 1)
    r = RVE(shape, phase=np.zeros(shape, np.uint8), phase_params=[[1.0, 0.5]],
            precision="mixed", residual="floatfloat")
    A = rng.standard_normal((3, 3) + shape)
    got = r.project(A)
    ref = fourier.G(A)
    if np.abs(ref).max() == 0:
        assert np.abs(got).max() < 1e-14
    else:
        assert maxrel(got, ref) < 1e-12
    r.close()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("tangent", ["recompute", "full81", "sym45"])
def test_operator_fp64_matches_oracle(shape, tangent):
    r, F, K, mu, rng = _random_problem(shape, 3, "fp64", tangent)
    _, K4 = svk.constitutive(F, K, mu)
    dF = rng.standard_normal((3, 3) + shape)
    got = r.apply_operator(dF)
    ref = fourier.G(svk.tangent_apply(K4, dF))
    if np.abs(ref).max() == 0:
        assert np.abs(got).max() < 1e-13
    else:
        assert maxrel(got, ref) < 1e-12
    r.close()


@pytest.mark.parametrize("shape", [(9, 11, 13), (31, 31, 31), (63, 63, 63), (27, 3, 125),
                                   (81, 75, 7), (7, 5, 225), (15, 21, 125), (45, 63, 27),
                                   (16, 20, 24), (15, 16, 17), (125, 16, 32),
                                   (243, 7, 5), (5, 243, 3), (315, 5, 3), (3, 315, 5)])
@pytest.mark.parametrize("tangent", ["recompute", "full81", "sym45"])
def test_operator_mixed_matches_oracle(shape, tangent):
    r, F, K, mu, rng = _random_problem(shape, 4, "mixed", tangent)
    _, K4 = svk.constitutive(F, K, mu)
    dF = rng.standard_normal((3, 3) + shape)
    got = r.apply_operator(dF)
    ref = fourier.G(svk.tangent_apply(K4, dF))
    assert rel(got, ref) < 5e-6
    r.close()


@pytest.mark.parametrize("shape", [(3, 5, 7), (15, 15, 15), (33, 21, 27)])
def test_constitutive_matches_oracle(shape):
    r, F, K, mu, rng = _random_problem(shape, 5)
    P_ref, K4_ref = svk.constitutive(F, K, mu)
    assert maxrel(r.get_P(), P_ref) < 1e-13
    assert maxrel(r.get_K4(), K4_ref) < 1e-13
    assert np.array_equal(r.get_F(), F)
    r.close()


@pytest.mark.parametrize("amp", [3e-3, 0.15])
@pytest.mark.parametrize("shape", [(15, 15, 15), (33, 21, 27)])
def test_constitutive_mixed_matches_oracle(shape, amp):
    """P of a mixed handle with the recomputed tangent (float-float update
    written in H = F - I), Eq. elas:S-P, against the oracle's stress
    evaluated in extended precision (in float64 its F^T F - I cancels about
    log10(1/|E|) digits at small strains).  At strains of 3e-3 an update
    formed from F itself (2^-47 of |F^T F| ~ 1) would be off by about 2e-12
    of the largest stress; the H form stays near 1e-14."""
    r, F, K, mu, rng = _random_problem(shape, 6, "mixed", "recompute", amp=amp)
    ld = np.longdouble
    P_ref = svk.stress(F.astype(ld), K.astype(ld), mu.astype(ld))
    assert maxrel(r.get_P(), P_ref) < 1e-13
    assert np.array_equal(r.get_F(), F)
    r.close()


def test_constitutive_mixed_float64_residual_matches_oracle():
    """residual="fp64" keeps the float64 SVK kernel for mixed handles: its P
    follows the float64 oracle as the float64 path does."""
    shape = (15, 15, 15)
    rng = np.random.default_rng(6)
    phase = (rng.uniform(size=shape) < 0.35).astype(np.uint8)
    params = synth.two_phase_params(7.0)
    r = RVE(shape, phase=phase, phase_params=params, precision="mixed", tangent="recompute",
            residual="fp64")
    F = synth.random_F(shape, rng, 3e-3)
    r.set_F(F)
    P_ref, _ = svk.constitutive(F, params[phase, 0], params[phase, 1])
    assert maxrel(r.get_P(), P_ref) < 1e-13
    r.close()


@pytest.fixture(scope="module")
def cube31_oracle():
    cfg = synth.config_cube31()
    prob = solver.SVKProblem.from_phase(cfg["phase"], cfg["phase_params"])
    res = []
    for Fbar in cfg["schedule"][:3]:
        prob.increment(Fbar, tol_newton=cfg["tol_newton"], tol_cg=cfg["tol_cg"])
        res.append((prob.F.copy(), prob.P.copy()))
    return cfg, res


def test_cube31_fp64_schedule_matches_oracle(cube31_oracle):
    cfg, ref = cube31_oracle
    gold = json.load(open(os.path.join(GOLDEN, "svk31_cube_schedule.json")))
    r = RVE(cfg["shape"], phase=cfg["phase"], phase_params=cfg["phase_params"],
            precision="fp64")
    for k, Fbar in enumerate(cfg["schedule"]):
        r.set_macro_F(Fbar)
        st = r.solve_increment(cfg["tol_newton"], cfg["tol_cg"])
        g = gold["config_tolerances"]["increments"][k]
        assert st["newton_iters"] == g["newton_iters"]
        assert all(abs(a - b) <= 1 for a, b in zip(st["cg_iters"], g["cg_iters"]))
        assert maxrel(r.homogenized_P(), np.array(g["Pbar"])) < 1e-10
        if k < len(ref):
            assert rel(r.get_F(), ref[k][0]) < 1e-10
            assert rel(r.get_P(), ref[k][1]) < 1e-10
    # the prescribed macroscopic deformation is held (Eq. mean:zero)
    assert maxrel(r.get_F().mean(axis=(2, 3, 4)), cfg["schedule"][-1]) < 1e-14
    r.close()


@pytest.fixture(scope="module")
def cube31_tight_oracle():
    """The whole 31^3 schedule solved by the oracle to eta_NW = 1e-10,
    eta_CG = 1e-12, and the P field of the oracle's own solve at the config
    tolerances (scipy.fft backend on all host cores for speed; the backend
    is pinned against the naive DFT in the oracle tests)."""
    cfg = synth.config_cube31()
    prob = solver.SVKProblem.from_phase(cfg["phase"], cfg["phase_params"])
    loose = solver.SVKProblem.from_phase(cfg["phase"], cfg["phase_params"])
    old = fourier.get_backend()
    try:
        fourier.set_backend("scipy", workers=os.cpu_count() or 1)
    except RuntimeError:
        fourier.set_backend("numpy")
    res = []
    try:
        for Fbar in cfg["schedule"]:
            prob.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=1e-12)
            loose.increment(Fbar, tol_newton=cfg["tol_newton"], tol_cg=cfg["tol_cg"])
            res.append((prob.F.copy(), prob.P.copy(), prob.homogenized_P(), loose.P.copy()))
    finally:
        fourier.set_backend(old["name"], old["workers"])
    return cfg, res


def test_cube31_mixed_schedule_matches_tight_oracle(cube31_tight_oracle):
    """Mixed path at the config tolerances (eta_NW = 1e-5, eta_CG = 1e-8,
    floored at 1e-5 in float32) against the tight oracle, every increment:
    F element-wise (relative 2-norm 1e-7, largest entry 1e-7), P-bar 1e-8
    (also against the stored tight values), and P within 1e-7 or twice the
    oracle's own distance from the tight solution at the config tolerances
    (the Newton truncation of eta_NW = 1e-5, the same in float64)."""
    cfg, ref = cube31_tight_oracle
    gold = json.load(open(os.path.join(GOLDEN, "svk31_cube_schedule.json")))
    r = RVE(cfg["shape"], phase=cfg["phase"], phase_params=cfg["phase_params"],
            precision="mixed")
    for k, Fbar in enumerate(cfg["schedule"]):
        r.set_macro_F(Fbar)
        r.solve_increment(cfg["tol_newton"], cfg["tol_cg"])
        F_ref, P_ref, pb_ref, P_loose = ref[k]
        F, P = r.get_F(), r.get_P()
        assert rel(F, F_ref) < 1e-7, k
        assert maxrel(F, F_ref) < 1e-7, k
        assert rel(P, P_ref) < max(1e-7, 2 * rel(P_loose, P_ref)), k
        assert maxrel(r.homogenized_P(), pb_ref) < 1e-8, k
        g = gold["tight"]["increments"][k]
        assert maxrel(r.homogenized_P(), np.array(g["Pbar"])) < 1e-8, k
    r.close()


def test_cube31_mixed_tight_newton_matches_tight_oracle(cube31_tight_oracle):
    """The mixed path solved to eta_NW = 1e-10: F and P element-wise within
    1e-7 of the tight oracle (the float32 CG inside an iterative refinement
    by the float64 residual), P-bar 1e-8."""
    cfg, ref = cube31_tight_oracle
    r = RVE(cfg["shape"], phase=cfg["phase"], phase_params=cfg["phase_params"],
            precision="mixed", cg_atol=1e-13)
    for k, Fbar in enumerate(cfg["schedule"]):
        r.set_macro_F(Fbar)
        r.solve_increment(1e-10, cfg["tol_cg"])
        F_ref, P_ref, pb_ref, _ = ref[k]
        assert rel(r.get_F(), F_ref) < 1e-7, k
        assert rel(r.get_P(), P_ref) < 1e-7, k
        assert maxrel(r.get_P(), P_ref) < 1e-7, k
        assert maxrel(r.homogenized_P(), pb_ref) < 1e-8, k
    r.close()


@pytest.mark.parametrize("shape", [(15, 21, 125), (27, 33, 45), (16, 18, 20), (7, 5, 243),
                                   (5, 3, 315), (243, 5, 3), (3, 315, 5)])
def test_mixed_solve_matches_tight_oracle(shape):
    """Converged mixed solve on axis lengths served by the four-step kernels
    (the fused float CG iteration on every pass) against the tightly
    converged float64 oracle: P-bar 1e-8, fields 1e-7."""
    rng = np.random.default_rng(11)
    phase = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    params = synth.two_phase_params(10.0)
    Fbar = synth.simple_shear(0.03)
    prob = solver.SVKProblem.from_phase(phase, params)
    prob.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=1e-13)
    r = RVE(shape, phase=phase, phase_params=params, precision="mixed")
    r.set_macro_F(Fbar)
    r.solve_increment(1e-5, 1e-8)
    assert maxrel(r.homogenized_P(), prob.homogenized_P()) < 1e-8
    assert rel(r.get_F(), prob.F) < 1e-7
    assert rel(r.get_P(), prob.P) < 1e-7
    r.close()


@pytest.mark.parametrize("shape", [(31, 31, 31), (27, 33, 45)])
def test_floatfloat_residual_matches_fp64_residual(shape):
    """The mixed path's float64-accuracy transforms in float-float arithmetic
    (default) against hardware float64: same Newton path, P-bar within 1e-11,
    F within 1e-10."""
    rng = np.random.default_rng(12)
    phase = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    params = synth.two_phase_params(10.0)
    out = {}
    for res in ("floatfloat", "fp64"):
        r = RVE(shape, phase=phase, phase_params=params, precision="mixed", residual=res)
        r.set_macro_F(synth.simple_shear(0.03))
        st = r.solve_increment(1e-5, 1e-8)
        out[res] = (st["newton_iters"], r.homogenized_P(), r.get_F())
        r.close()
    assert out["floatfloat"][0] == out["fp64"][0]
    assert maxrel(out["floatfloat"][1], out["fp64"][1]) < 1e-11
    assert rel(out["floatfloat"][2], out["fp64"][2]) < 1e-10


def test_homogeneous_cell_gives_uniform_F():
    shape = (15, 9, 21)
    r = RVE(shape, phase=np.zeros(shape, np.uint8), phase_params=[[0.833, 0.386]])
    Fbar = np.eye(3) + 0.1 * np.random.default_rng(1).uniform(-1, 1, (3, 3))
    r.set_macro_F(Fbar)
    r.solve_increment(1e-5, 1e-8)
    F = r.get_F()
    assert np.abs(F - Fbar[:, :, None, None, None]).max() < 1e-14
    assert maxrel(r.homogenized_P(), svk.stress(Fbar, 0.833, 0.386)) < 1e-13
    r.close()


def test_single_voxel_cell():
    r = RVE((1, 1, 1), phase=np.ones((1, 1, 1), np.uint8), phase_params=[[1, 1], [2.0, 0.7]])
    Fbar = synth.simple_shear(0.2)
    r.set_macro_F(Fbar)
    st = r.solve_increment(1e-5, 1e-8)
    assert st["cg_iters"] == [0, 0]
    assert np.abs(r.get_F()[:, :, 0, 0, 0] - Fbar).max() < 1e-15
    r.close()


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-7)])
def test_laminate_closed_form(axis, prec, tol):
    from test_oracle_solver import _laminate_exact
    shape = [15, 15, 15]
    shape[axis] = 27
    shape = tuple(shape)
    ph = synth.laminate(shape, axis, fraction=12 / 27)
    params = synth.two_phase_params(20.0)
    Fbar = np.eye(3) + np.array([[0.05, 0.2, -0.03], [0.01, -0.04, 0.1], [0.02, 0.03, 0.06]])
    r = RVE(shape, phase=ph, phase_params=params, precision=prec, cg_atol=1e-12)
    r.set_macro_F(Fbar)
    r.solve_increment(1e-10 if prec == "fp64" else 1e-7, 1e-12)
    n = np.zeros(3)
    n[axis] = 1
    F1, F0 = _laminate_exact(Fbar, n, ph.mean(), tuple(params[1]), tuple(params[0]))
    exact = np.where(ph[None, None] == 1, F1[:, :, None, None, None], F0[:, :, None, None, None])
    assert np.abs(r.get_F() - exact).max() < tol
    r.close()


def test_invalid_arguments_are_rejected():
    with pytest.raises(RVEError) as e:
        RVE((0, 5, 5), phase=np.zeros((0, 5, 5), np.uint8), phase_params=[[1, 1]])
    assert e.value.code == -1
    with pytest.raises(RVEError):
        RVE((5, 5, 5), phase=np.full((5, 5, 5), 3, np.uint8), phase_params=[[1, 1], [2, 2]])


def test_negative_det_rolls_back():
    shape = (9, 9, 9)
    ph = synth.cube_inclusion(9, 3)
    r = RVE(shape, phase=ph, phase_params=synth.two_phase_params(5.0))
    r.set_macro_F(synth.simple_shear(0.05))
    r.solve_increment()
    F_ok = r.get_F()
    bad = np.diag([-1.0, 1.0, 1.0])  # an inversion: det F-bar < 0
    r.set_macro_F(bad)
    with pytest.raises(RVEError) as e:
        r.solve_increment()
    assert e.value.code == -8
    assert np.array_equal(r.get_F(), F_ok)
    r.close()


def test_per_voxel_moduli_match_phase_table():
    shape = (15, 15, 15)
    ph = synth.cube_inclusion(15, 5)
    params = synth.two_phase_params(10.0)
    vox = np.stack([params[ph, 0], params[ph, 1]])
    a = RVE(shape, phase=ph, phase_params=params)
    b = RVE(shape, voxel_params=vox)
    for r in (a, b):
        r.set_macro_F(synth.simple_shear(0.05))
        r.solve_increment()
    assert np.array_equal(a.get_F(), b.get_F())
    a.close()
    b.close()


def test_deterministic_repeat():
    cfg = synth.config_cube31()
    outs = []
    for _ in range(2):
        r = RVE(cfg["shape"], phase=cfg["phase"], phase_params=cfg["phase_params"],
                precision="mixed")
        r.set_macro_F(cfg["schedule"][0])
        r.solve_increment()
        outs.append(r.get_F())
        r.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("shape", [(15, 21, 125), (31, 31, 31)])
def test_projection_matches_cufft_cross_check(shape):
    """Cross-check of the library's transforms against cuFFT (through
    torch.fft, test-only): G:A = IFFT(G-hat : FFT(A)) with the reduced form
    of Eq. G_red, float64, on the device."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 3) + shape)
    r = RVE(shape, phase=np.zeros(shape, np.uint8), phase_params=[[1.0, 0.5]])
    got = r.project(A)
    r.close()
    At = torch.from_numpy(A).cuda()
    Ah = torch.fft.fftn(At, dim=(2, 3, 4))
    q = [torch.fft.fftfreq(n, d=1.0 / n, dtype=torch.float64, device="cuda") / n for n in shape]
    qx, qy, qz = torch.meshgrid(*q, indexing="ij")
    xi = torch.stack([qx, qy, qz])
    q2 = (xi * xi).sum(0)
    inv = torch.where(q2 > 0, 1.0 / torch.where(q2 > 0, q2, torch.ones_like(q2)), torch.zeros_like(q2))
    s = torch.einsum("ilxyz,lxyz->ixyz", Ah, xi.to(Ah.dtype))
    Gh = torch.einsum("ixyz,jxyz->ijxyz", s, xi.to(Ah.dtype)) * inv
    ref = torch.fft.ifftn(Gh, dim=(2, 3, 4)).real.cpu().numpy()
    assert maxrel(got, ref) < 1e-12


def test_autotuned_handle_matches_oracle():
    """A mixed handle with the autotuner on picks kernel variants (reported by
    rve_tuning), caches them per grid, and still reaches the oracle's
    converged state (P-bar 1e-8, fields 1e-7)."""
    shape = (27, 33, 45)
    rng = np.random.default_rng(13)
    phase = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    params = synth.two_phase_params(10.0)
    Fbar = synth.simple_shear(0.03)
    prob = solver.SVKProblem.from_phase(phase, params)
    prob.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=1e-13)
    for _ in range(2):  # second handle takes the cached choice
        r = RVE(shape, phase=phase, phase_params=params, precision="mixed", autotune=True)
        t = r.tuning()
        assert t["autotuned"] == 1 and t["z_blocks_per_sm"] in (1, 2, 3)
        r.set_macro_F(Fbar)
        r.solve_increment(1e-5, 1e-8)
        assert maxrel(r.homogenized_P(), prob.homogenized_P()) < 1e-8
        assert rel(r.get_F(), prob.F) < 1e-7
        r.close()


@pytest.mark.parametrize("shape", [(45, 63, 125), (243, 15, 21), (15, 315, 27)])
@pytest.mark.parametrize("halves", [(1, 0), (0, 1), (1, 1)])
def test_operator_tile_variants_match_oracle(shape, halves):
    """The autotuner's alternative tile heights of the four-step x and y
    passes (half the kz values per tile), set explicitly with
    rve_set_tuning: one float32 operator application against the oracle."""
    r, F, K, mu, rng = _random_problem(shape, 6, "mixed", "recompute")
    r.set_tuning(x_tile_half=halves[0], y_tile_half=halves[1])
    t = r.tuning()
    assert (t["x_tile_half"], t["y_tile_half"]) == halves and t["autotuned"] == 0
    _, K4 = svk.constitutive(F, K, mu)
    dF = rng.standard_normal((3, 3) + shape)
    got = r.apply_operator(dF)
    ref = fourier.G(svk.tangent_apply(K4, dF))
    assert rel(got, ref) < 5e-6
    r.close()


def test_mixed_solve_with_half_tiles_matches_tight_oracle():
    shape = (27, 33, 45)
    rng = np.random.default_rng(17)
    phase = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    params = synth.two_phase_params(10.0)
    Fbar = synth.simple_shear(0.03)
    prob = solver.SVKProblem.from_phase(phase, params)
    prob.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=1e-13)
    r = RVE(shape, phase=phase, phase_params=params, precision="mixed")
    r.set_tuning(x_tile_half=1, y_tile_half=1)
    r.set_macro_F(Fbar)
    r.solve_increment(1e-5, 1e-8)
    assert maxrel(r.homogenized_P(), prob.homogenized_P()) < 1e-8
    assert rel(r.get_F(), prob.F) < 1e-7
    r.close()


def test_set_tuning_rejects_bad_values():
    r = RVE((9, 9, 9), phase=np.zeros((9, 9, 9), np.uint8), phase_params=[[1.0, 0.5]],
            precision="mixed")
    with pytest.raises(RVEError):
        r.set_tuning(z_blocks_per_sm=4)
    with pytest.raises(RVEError):
        r.set_tuning(x_tile_half=2)
    r.close()
