"""Benchmark of the Newton-CG solver on the 125^3 two-phase sphere cell.

Workload (synthetic, seeded): Saint Venant-Kirchhoff, 125^3 voxels, random
non-overlapping spheres (radii 4-10, volume fraction 0.3, stiffness contrast
100, matrix K = 0.833, mu = 0.386), uniaxial F-bar = diag(1 + eps, 1, 1) with
eps ramped to 0.2 in 20 equal increments; eta_NW = 1e-5, eta_CG = 1e-8.

A step is one load increment: constitutive update, predictor solve, Newton
iterations with matrix-free CG to convergence, commit.  The headline value
is voxel * CG-iterations per second of the mixed-precision path (float32 CG
operator, float64 residual / update / reductions), timed with CUDA events on
the solver's stream with the cell resident in HBM; the plain float64 path is
timed on the same increments for the solve-time ratio, and the mixed path's
homogenised stress is compared with the float64 path's.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank solves its own replica of the
cell (the method has no exchange step between independent cells); the value
is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "voxel*CG-iterations/s, mixed FP32-CG/FP64-residual solver (vs plain FP64 GPU solver)"
UNIT = "voxel*CG-iter/s"
# algorithmic bytes per voxel of each kernel family of the float32 CG
# iteration (the five fused passes), on-the-fly SVK tangent (F in float32 +
# 1-byte phase), half spectrum of h = N//2+1 planes (nine complex values per
# (x, y, kz)).


def family_bytes_per_voxel(nz, fam):
    s = 4.0
    spec = 9 * 2 * s * (nz // 2 + 1) / nz
    return {
        # r, p, x in; p, x out; F; phase; spectrum out
        "zfwd": 9 * s * 5 + 9 * s + 1 + spec,
        "fft_y_fwd": 2 * spec,
        "fft_x_proj": 2 * spec,
        "fft_y_inv": 2 * spec,
        "zinv": spec + 9 * s * 2,               # spectrum in; r in, r out
    }[fam]


# dram__bytes_read.sum + dram__bytes_write.sum per launch of the current
# kernel version from one ncu capture of this workload; a kernel changed
# since its capture has no entry (traffic null)
NCU_TRAFFIC_BYTES = {"zfwd": 298.848256e6 + 157.713152e6}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.mkdtemp(prefix="rve_clocks_"), "clocks.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(rows), "reasons": sorted(reasons)}


def dist_setup(ngpus):
    if ngpus <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend)
    rank, world = dist.get_rank(), dist.get_world_size()
    if torch.cuda.is_available():
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
    return rank, world, dist


def reduce_max_sum(dist, t_max, s_sum):
    """(max over ranks of t_max, sum over ranks of s_sum)."""
    if dist is None:
        return t_max, s_sum
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    a = torch.tensor([t_max], dtype=torch.float64, device=dev)
    b = torch.tensor([s_sum], dtype=torch.float64, device=dev)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(a.item()), float(b.item())


def workload():
    cfg = synth.config_spheres(125, seed=1, nincr=20, eps=0.2)
    cfg["workload"] = "svk125_spheres_uniaxial"
    return cfg


def run_schedule(RVE, cfg, precision, steps, torch, e2e_buf=None, collect_pbar=False):
    """Solve `steps` increments of the ramp on a fresh cell.  Returns a dict
    with device time (CUDA events on the solver stream), CG iterations,
    P-bar per increment and the kernel launch count."""
    sched = cfg["schedule"]
    r = RVE(cfg["shape"], phase=cfg["phase"], phase_params=cfg["phase_params"],
            precision=precision)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cg = 0
    newton = 0
    pbars = []
    l0 = r.launch_count()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ev0.record(stream)
    for k in range(steps):
        if k and k % len(sched) == 0:
            r.set_F(np.broadcast_to(np.eye(3)[:, :, None, None, None],
                                    (3, 3) + cfg["shape"]).copy())
        r.set_macro_F(sched[k % len(sched)])
        st = r.solve_increment(cfg["tol_newton"], cfg["tol_cg"])
        cg += st["cg_iters_total"]
        newton += st["newton_iters"]
        if e2e_buf is not None:
            r.get_P(out=e2e_buf)
        if collect_pbar or e2e_buf is not None:
            pbars.append(r.homogenized_P())
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    ms = ev0.elapsed_time(ev1)
    out = dict(ms=ms, wall_s=wall, cg=cg, newton=newton, pbars=pbars,
               launches=r.launch_count() - l0, rve=r)
    return out


def kernel_profile(RVE, cfg, torch, families, steps=1):
    """Average device time per launch of each CG-iteration kernel family,
    from CUDA events recorded around every launch on the solver stream."""
    from paper_1603_08893_gb300 import rve as api
    res = {}
    for fi, fam in enumerate(families):
        r = RVE(cfg["shape"], phase=cfg["phase"], phase_params=cfg["phase_params"],
                precision="mixed")
        api.rve_kernel_timing(r.h, fi, True)
        for k in range(steps):
            r.set_macro_F(cfg["schedule"][k])
            r.solve_increment(cfg["tol_newton"], cfg["tol_cg"])
        ms, cnt = api.rve_kernel_time(r.h)
        if cnt:  # the float32 iteration has no separate vector-update pass
            res[fam] = dict(total_ms=ms, launches=cnt, avg_ms=ms / cnt)
        r.close()
    return res


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def cpu_model():
    """CPU model name of the host (x86 'model name', or lscpu's 'Model name'
    on Arm hosts whose /proc/cpuinfo has none)."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


class OracleSample:
    """The FP64 oracle, as it stands, on the host cores: the scipy.fft
    backend with one worker per core for its DFTs (its other steps are
    numpy as written), the tangent of the first increment's predictor and
    CG iterations of that predictor solve on the same cell."""

    def __init__(self, cfg):
        from oracle import fourier
        from oracle import solver as osolver
        from oracle import tensor as otensor
        self.cores = host_cores()
        self.cpu = cpu_model()
        self.fourier, self.osolver = fourier, osolver
        self.old = fourier.get_backend()
        fourier.set_backend("scipy", workers=self.cores)
        self.cfg = cfg
        self.n = int(np.prod(cfg["shape"]))
        prob = osolver.SVKProblem.from_phase(cfg["phase"], cfg["phase_params"])
        t0 = time.perf_counter()
        _, K4 = prob.constitutive(prob.F)
        self.t_const = time.perf_counter() - t0
        self.op = osolver.tangent_operator(K4)
        self.b = -self.op(otensor.uniform(cfg["schedule"][0] - np.eye(3), prob.shape))

    def iterate(self, k):
        """Seconds for k CG iterations (operator G:(K:p) + vector updates)."""
        t0 = time.perf_counter()
        try:
            self.osolver.cg(self.op, self.b, self.cfg["tol_cg"], maxiter=k)
        except self.osolver.SolverError:
            pass
        return time.perf_counter() - t0

    def close(self):
        self.fourier.set_backend(self.old["name"], self.old["workers"])

    def describe(self, iters, what):
        return (f"{what} CG iterations of the first increment's predictor solve on the "
                f"{self.cfg['shape'][0]}^3 cell, oracle with the scipy.fft backend on "
                f"{self.cores} workers (DFTs; its other steps single-threaded numpy), "
                f"{self.cpu}")


def cpu_baseline_sample(cfg, gpu_cg_iters=None, gpu_newton_iters=None, iters=10):
    """The oracle on a bounded sample of the workload (`iters` CG iterations
    plus the constitutive evaluation they need), with the full run
    extrapolated from the GPU run's CG and Newton counts (labelled as such:
    the oracle's own counts differ slightly)."""
    o = OracleSample(cfg)
    try:
        o.iterate(1)  # plans and page faults
        t_cg = o.iterate(iters)
    finally:
        o.close()
    out = dict(value=o.n * iters / t_cg, unit=UNIT, cores=o.cores, kind="oracle",
               sample=o.describe(iters, iters) +
               f"; one constitutive evaluation (tangent) {o.t_const:.1f} s",
               cpu_model=o.cpu, seconds=t_cg + o.t_const)
    if gpu_cg_iters:
        out["extrapolated_full_run_s"] = round(
            gpu_cg_iters * t_cg / iters + (gpu_newton_iters or 0) * o.t_const, 1)
        out["extrapolation"] = ("per-iteration CG time x the GPU run's CG iterations + one "
                                "constitutive evaluation per Newton iteration of the GPU run")
    return out


def reference_arm(args):
    """The oracle, as it stands, on the host cores: one step is one CG
    iteration (operator G:(K:p) and vector updates) of the first increment's
    predictor solve on the same 125^3 cell; the constitutive evaluation and
    the right-hand side are set up once, untimed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = workload()
    o = OracleSample(cfg)
    try:
        if args.warmup > 0:
            o.iterate(args.warmup)
        dt = o.iterate(args.steps)
    finally:
        o.close()
    v = o.n * args.steps / dt
    sample = (o.describe(args.steps, args.steps) +
              f", after {args.warmup} warm-up iterations; constitutive evaluation and "
              f"right-hand side untimed")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * dt / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": cfg["workload"], "grid": 125},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": o.cores, "kind": "oracle",
                            "sample": sample, "cpu_model": o.cpu},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# Secondary workloads (one JSON line each; `--workload NAME`).  The default
# workload above is the headline; these measure the other synthetic configs
# and the stored-vs-recomputed tangent choice on one GPU.
# ---------------------------------------------------------------------------
def _line(workload, metric, value, unit, **extra):
    d = {"workload": workload, "metric": metric, "value": value, "unit": unit,
         "n_gpus": 1, "data": "synthetic"}
    d.update(extra)  # may override n_gpus
    print(json.dumps(d), flush=True)


def _events(torch):
    return (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.current_stream())


def bench_cube31(args, torch, RVE):
    """31^3 corner cube, contrast 10, simple shear to 0.1 in 10 increments,
    plain float64 path (config 1)."""
    cfg = synth.config_cube31()
    n = int(np.prod(cfg["shape"]))
    w = RVE(cfg["shape"], phase=cfg["phase"], phase_params=cfg["phase_params"], precision="fp64")
    w.set_macro_F(cfg["schedule"][0])
    w.solve_increment(cfg["tol_newton"], cfg["tol_cg"])
    w.close()
    r = RVE(cfg["shape"], phase=cfg["phase"], phase_params=cfg["phase_params"], precision="fp64")
    e0, e1, s = _events(torch)
    cg = newton = 0
    torch.cuda.synchronize()
    e0.record(s)
    for Fb in cfg["schedule"]:
        r.set_macro_F(Fb)
        st = r.solve_increment(cfg["tol_newton"], cfg["tol_cg"])
        cg += st["cg_iters_total"]
        newton += st["newton_iters"]
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pbar = r.homogenized_P()
    r.close()
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "svk31_cube_schedule.json")))
    tight = np.array(gold["tight"]["increments"][-1]["Pbar"])
    # the oracle's whole schedule at the same tolerances on the host cores
    from oracle import fourier
    from oracle import solver as osolver
    old = fourier.get_backend()
    fourier.set_backend("scipy", workers=host_cores())
    try:
        prob = osolver.SVKProblem.from_phase(cfg["phase"], cfg["phase_params"])
        t0 = time.perf_counter()
        ocg = 0
        for Fb in cfg["schedule"]:
            ocg += sum(prob.increment(Fb, cfg["tol_newton"], cfg["tol_cg"]).cg_iters)
        t_or = time.perf_counter() - t0
    finally:
        fourier.set_backend(old["name"], old["workers"])
    _line("svk31_cube_shear_fp64", "voxel*CG-iterations/s, float64 GPU solver", n * cg / (ms / 1e3),
          UNIT, dtype="f64", increments=len(cfg["schedule"]), cg_iters=cg, newton_iters=newton,
          solve_ms=ms, pbar_xy=float(pbar[0, 1]),
          pbar_rel_err_vs_tight_oracle=float(np.abs(pbar - tight).max() / np.abs(tight).max()),
          cpu_oracle={"full_run_s": round(t_or, 2), "cg_iters": ocg, "cores": host_cores(),
                      "cpu_model": cpu_model(), "value": n * ocg / t_or,
                      "sample": "the whole 10-increment schedule, scipy.fft backend"})


def bench_j2_315(args, torch, RVE):
    """315^3 Voronoi, J2 plasticity, simple shear to 0.2 in 20 increments,
    mixed path with increment cutting (config 3); the first --j2-steps
    increments."""
    cfg = synth.config_voronoi_j2()
    n = int(np.prod(cfg["shape"]))
    r = RVE(cfg["shape"], model="j2", phase=cfg["phase"], phase_params=cfg["phase_params"],
            precision="mixed")
    e0, e1, s = _events(torch)
    cg = newton = subs = cuts = 0
    steps = min(args.j2_steps, len(cfg["schedule"]))
    torch.cuda.synchronize()
    e0.record(s)
    for Fb in cfg["schedule"][:steps]:
        st = r.solve_step(Fb, cfg["tol_newton"], cfg["tol_cg"], max_cuts=10)
        cg += st["cg_iters_total"]
        newton += st["newton_iters"]
        subs += st["substeps"]
        cuts += st["cuts"]
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ep = r.get_history()[6]
    value = n * cg / (ms / 1e3)
    # algorithmic bytes of one float32 CG iteration with the stored SYM45
    # tangent: the first pass reads 45 tangent reals instead of F and phase
    spec = 9 * 2 * 4.0 * (cfg["shape"][2] // 2 + 1) / cfg["shape"][2]
    b_iter = (9 * 4 * 5 + 45 * 4 + spec) + 3 * 2 * spec + (spec + 9 * 4 * 2)
    peak, peak_kind = load_peaks()
    _line("j2_315_voronoi_shear_mixed", METRIC, value, UNIT, dtype="f32/f64",
          increments=steps, substeps=subs, cuts=cuts, cg_iters=cg, newton_iters=newton,
          solve_ms=ms, pbar_xy=float(r.homogenized_P()[0, 1]), max_eps_p=float(ep.max()),
          plastic_fraction=float((ep > 0).mean()),
          cg_iteration_bytes_per_voxel=round(b_iter, 1),
          hbm_frac_whole_step=round(value * b_iter / 1e9 / peak, 4), peak_kind=peak_kind,
          note="hbm_frac_whole_step counts only CG-iteration bytes against the time of "
               "whole increments (return maps, residuals and cut attempts included)")
    r.close()


def bench_batch256(args, torch):
    """256 SVK cells of uneven size, one increment each, CUDA graph, autotuned
    kernels, mixed path with per-cell increment cutting (config 4).  Under
    torchrun the cells are sharded over the ranks (largest first to the least
    loaded rank, no data-path collective); value = all ranks' units / the
    slowest rank's time (strong scaling: the batch is fixed)."""
    from paper_1603_08893_gb300 import RVEBatch
    from paper_1603_08893_gb300.shard import partition_cells
    rank, world, dist = dist_setup(args.gpus)
    all_cells = synth.config_batch()
    mine = partition_cells([c["shape"] for c in all_cells], world)[rank]
    cells = [all_cells[i] for i in mine]
    shapes = [c["shape"] for c in cells]
    t0 = time.perf_counter()
    b = RVEBatch(shapes, [c["phase"] for c in cells], [c["phase_params"] for c in cells],
                 precision="mixed", autotune=True)
    setup_s = time.perf_counter() - t0
    F = np.stack([c["Fbar"] for c in cells])
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    stats = b.solve(F, 1e-5, 1e-8, check=False, max_cuts=4)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    units = sum(int(np.prod(sh)) * st["cg_iters_total"] for sh, st in zip(shapes, stats))
    failed = sum(1 for st in stats if st["status"] != 0)
    wall_max, units_all = reduce_max_sum(dist, wall, float(units))
    _, failed_all = reduce_max_sum(dist, 0.0, float(failed))
    if rank == 0:
        _line("svk_batch256_uneven_mixed", METRIC, units_all / wall_max, UNIT, dtype="f32/f64",
              n_gpus=world, scaling="strong", cells=len(all_cells),
              voxels=int(sum(int(np.prod(c["shape"])) for c in all_cells)),
              failed_cells=int(failed_all), solve_s=wall_max, setup_and_autotune_s=setup_s,
              cg_iters_rank0=int(sum(st["cg_iters_total"] for st in stats)),
              timing="host wall clock around the batch solve (its calls return when "
                     "idle), max over ranks")
    b.close()


def bench_adjoint243(args, torch, RVE):
    """243^3 lognormal shear modulus, simple shear 0.05, one increment, then
    the adjoint gradient of P-bar_xy (config 5), mixed path."""
    cfg = synth.config_lognormal()
    n = int(np.prod(cfg["shape"]))
    r = RVE(cfg["shape"], voxel_params=cfg["voxel_params"], precision="mixed")
    e0, e1, s = _events(torch)
    torch.cuda.synchronize()
    e0.record(s)
    r.set_macro_F(cfg["schedule"][0])
    st = r.solve_increment(cfg["tol_newton"], cfg["tol_cg"])
    e1.record(s)
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1)
    W = np.zeros((3, 3))
    W[0, 1] = 1.0
    e0.record(s)
    g, its = r.adjoint_grad_mu(W, tol_cg=1e-8)
    e1.record(s)
    torch.cuda.synchronize()
    ms_adj = e0.elapsed_time(e1)
    _line("svk243_lognormal_adjoint_mixed", "voxel*CG-iterations/s of the adjoint solve",
          n * its / (ms_adj / 1e3), UNIT, dtype="f32/f64", adjoint_cg_iters=its,
          adjoint_ms=ms_adj, forward_ms=ms_fwd, forward_cg_iters=st["cg_iters_total"],
          forward_value=n * st["cg_iters_total"] / (ms_fwd / 1e3),
          grad_abs_max=float(np.abs(g).max()))
    r.close()


def bench_tangent125(args, torch, RVE):
    """Stored K4 (81 float32 per voxel) against the recomputed SVK tangent in
    the first pass of the float32 CG iteration, 125^3 spheres: device time per
    launch of that kernel family and whole-increment throughput."""
    cfg = workload()
    from paper_1603_08893_gb300 import rve as api

    def run(model, tan, cfgx, Fb):
        kw = (dict(phase=cfgx["phase"], phase_params=cfgx["phase_params"]))
        r = RVE(cfgx["shape"], model=model, precision="mixed", tangent=tan, **kw)
        api.rve_kernel_timing(r.h, 0, True)
        e0, e1, s = _events(torch)
        torch.cuda.synchronize()
        e0.record(s)
        r.set_macro_F(Fb)
        st = r.solve_increment(cfgx["tol_newton"], cfgx["tol_cg"])
        e1.record(s)
        torch.cuda.synchronize()
        zms, cnt = api.rve_kernel_time(r.h)
        r.close()
        return {"first_pass_ms": zms / max(cnt, 1), "increment_ms": e0.elapsed_time(e1),
                "cg_iters": st["cg_iters_total"]}

    svk = {tan: run("svk", tan, cfg, cfg["schedule"][0]) for tan in ("recompute", "sym45", "full81")}
    j2cfg = synth.config_voronoi_j2(n=125)
    j2 = {tan: run("j2", tan, j2cfg, synth.simple_shear(0.002)) for tan in ("sym45", "full81")}
    best = min(svk, key=lambda k: svk[k]["first_pass_ms"])
    best_j2 = min(j2, key=lambda k: j2[k]["first_pass_ms"])
    _line("svk125_tangent_choice", "first-pass ms per CG iteration", svk[best]["first_pass_ms"],
          "ms", chosen=best, variants=svk, j2_125_chosen=best_j2, j2_125_variants=j2,
          algorithmic_bytes_per_voxel={"recompute": 253.3, "sym45": 253.3 - 37 + 180,
                                       "full81": 253.3 - 37 + 324})


def bench_project125(args, torch, RVE):
    """The float64-accuracy projection G:A of the mixed solver (the residual
    G:P and the projection of dF take the same passes) on the 125^3 and
    243^3 grids: float-float arithmetic on the float32 pipe (the default of
    mixed handles) against hardware float64 (residual="fp64"), device
    buffers, the two device copies of rve_project (A in, result out)
    included; the largest difference of the two results."""
    out = {}
    for nn in (125, 243):
        shape = (nn, nn, nn)
        rng = np.random.default_rng(7)
        A = rng.standard_normal((3, 3) + shape)
        At = torch.from_numpy(A).cuda()
        o = torch.empty_like(At)
        row = {}
        got = {}
        for res in ("floatfloat", "fp64"):
            r = RVE(shape, phase=np.zeros(shape, np.uint8), phase_params=[[1.0, 0.5]],
                    precision="mixed", residual=res)
            for _ in range(3):
                r.project(At, o)
            torch.cuda.synchronize()
            reps = 20 if nn == 125 else 5
            t0 = time.perf_counter()
            for _ in range(reps):
                r.project(At, o)
            torch.cuda.synchronize()
            row[res + "_ms"] = (time.perf_counter() - t0) / reps * 1e3
            got[res] = o.clone()
            r.close()
        d = (got["floatfloat"] - got["fp64"]).abs().max() / got["fp64"].abs().max()
        row["maxrel_floatfloat_vs_fp64"] = float(d)
        row["copy_bytes"] = 2 * A.nbytes
        del got
        out[str(nn)] = row
    _line("project125_floatfloat", "ms per G application (two 9-component device copies included)",
          out["125"]["floatfloat_ms"], "ms", dtype="float-float (f32 pairs) / f64", grids=out)


def bench_mixed125(args, torch, RVE):
    """Mixed macroscopic control on the 125^3 spheres, mixed precision:
    uniaxial stress along x (F11 = 1.01 prescribed, the lateral and shear
    P-bar components zero) against the uniaxial-strain increment to the same
    F11, both as one increment from F = I."""
    cfg = workload()
    n = int(np.prod(cfg["shape"]))
    kw = dict(phase=cfg["phase"], phase_params=cfg["phase_params"], precision="mixed")
    Fb = synth.uniaxial(0.01)
    res = {}
    for mode in ("strain", "stress"):
        r = RVE(cfg["shape"], **kw)
        e0, e1, s = _events(torch)
        torch.cuda.synchronize()
        e0.record(s)
        if mode == "strain":
            r.set_macro_F(Fb)
            st = r.solve_increment(cfg["tol_newton"], cfg["tol_cg"])
        else:
            st = r.solve_mixed(Fb, np.zeros(9), synth.uniaxial_stress_mask(), tol_stress=1e-6,
                               tol_newton=cfg["tol_newton"], tol_cg=cfg["tol_cg"])
        e1.record(s)
        torch.cuda.synchronize()
        res[mode] = (e0.elapsed_time(e1), st, r.homogenized_P(), r.macro_F())
        r.close()
    ms, st, Pb, Fm = res["stress"]
    ms_e, st_e, Pb_e, _ = res["strain"]
    _line("svk125_spheres_uniaxial_stress_mixed", METRIC, n * st["cg_iters_total"] / (ms / 1e3),
          UNIT, dtype="f32/f64", ms=ms, cg_iters=st["cg_iters_total"],
          macro_iters=st["macro_iters"], tangent_solves=st["tangent_solves"],
          newton_iters=st["newton_iters"], lateral_F=float(Fm[1, 1]), P11=float(Pb[0, 0]),
          strain_control_ms=ms_e, strain_control_cg_iters=st_e["cg_iters_total"],
          strain_control_P11=float(Pb_e[0, 0]), time_ratio=ms / ms_e)


def bench_precond125(args, torch, RVE):
    """Reference-medium preconditioned float32 CG against plain CG on the
    125^3 spheres (contrast 100): the first 4 increments of the uniaxial ramp,
    mixed precision, solve time and CG iterations of each, P-bar agreement."""
    cfg = workload()
    n = int(np.prod(cfg["shape"]))
    k = 4
    res = {}
    for pc in ("none", "reference"):
        r = RVE(cfg["shape"], phase=cfg["phase"], phase_params=cfg["phase_params"],
                precision="mixed", precond=pc)
        e0, e1, s = _events(torch)
        cg = 0
        torch.cuda.synchronize()
        e0.record(s)
        for Fb in cfg["schedule"][:k]:
            r.set_macro_F(Fb)
            cg += r.solve_increment(cfg["tol_newton"], cfg["tol_cg"])["cg_iters_total"]
        e1.record(s)
        torch.cuda.synchronize()
        res[pc] = (e0.elapsed_time(e1), cg, r.homogenized_P())
        r.close()
    ms, cg, Pb = res["reference"]
    ms0, cg0, Pb0 = res["none"]
    _line("svk125_spheres_uniaxial_precond_mixed", METRIC, n * cg / (ms / 1e3), UNIT,
          dtype="f32/f64", increments=k, solve_ms=ms, cg_iters=cg, plain_solve_ms=ms0,
          plain_cg_iters=cg0, plain_value=n * cg0 / (ms0 / 1e3), solve_time_ratio=ms0 / ms,
          pbar_rel_diff=float(np.abs(Pb - Pb0).max() / np.abs(Pb0).max()))


def bench_contrast63(args, torch, RVE):
    """Phase-contrast sweep of the paper's Sec. 5.5 experiment on a synthetic
    stand-in (the micrograph is not available): 63^3 periodic Voronoi cell
    (64 cells, half hard), J2 with E = 1, nu = 0.3, soft tau_y0 = 0.003 and
    H = 0.01, hard ones chi times larger, chi in {sqrt 2, 2, 4, 8}; pure shear
    F-bar = diag(l, 1/l, 1) to l = 1.2 in --contrast-increments increments
    (250 in the paper), mixed precision with load-step cutting, plain and
    reference-preconditioned CG.  Cumulative Newton and CG iterations and
    device time per chi, also at equivalent strains 0.05 / 0.1 / 0.2."""
    n = 63
    ph, _ = synth.voronoi(n, 64, np.random.default_rng(2))
    K, mu = 1.0 / 1.2, 1.0 / 2.6
    m = args.contrast_increments
    lams = [1.0 + 0.2 * (k + 1) / m for k in range(m)]
    marks = (0.05, 0.1, 0.2)
    out = {}
    for pc in ("none", "reference"):
        for chi in (np.sqrt(2.0), 2.0, 4.0, 8.0):
            params = np.array([[K, mu, 0.003, 0.01], [K, mu, 0.003 * chi, 0.01 * chi]])
            r = RVE((n, n, n), model="j2", phase=ph, phase_params=params, precision="mixed",
                    precond=pc)
            e0, e1, s = _events(torch)
            newton = cg = cuts = 0
            at = {}
            torch.cuda.synchronize()
            e0.record(s)
            for lam in lams:
                st = r.solve_step(np.diag([lam, 1.0 / lam, 1.0]), 1e-5, 1e-8, max_cuts=10)
                newton += st["newton_iters"]
                cg += st["cg_iters_total"]
                cuts += st["cuts"]
                eq = 2.0 / np.sqrt(3.0) * np.log(lam)
                for mk in marks:
                    if eq >= mk and mk not in at:
                        at[mk] = (newton, cg)
            e1.record(s)
            torch.cuda.synchronize()
            out[f"{pc}/chi={chi:.3g}"] = {
                "newton_iters": newton, "cg_iters": cg, "cuts": cuts,
                "solve_ms": e0.elapsed_time(e1),
                "at_eq_strain": {str(k): {"newton": v[0], "cg": v[1]} for k, v in at.items()},
                "pbar_xx": float(r.homogenized_P()[0, 0]),
                "max_eps_p": float(r.get_history()[6].max())}
            r.close()
    tot_cg = sum(v["cg_iters"] for v in out.values())
    tot_ms = sum(v["solve_ms"] for v in out.values())
    _line("j2_63_voronoi_pure_shear_contrast_sweep", METRIC, n ** 3 * tot_cg / (tot_ms / 1e3),
          UNIT, dtype="f32/f64", increments=m, sweep=out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--mixed-only", action="store_true",
                    help="time the mixed path only (no float64 comparison, no e2e); "
                         "used for profiler captures")
    ap.add_argument("--j2-steps", type=int, default=2,
                    help="increments of the 315^3 J2 ramp timed by --workload j2_315")
    ap.add_argument("--contrast-increments", type=int, default=250,
                    help="increments of the pure-shear ramp of --workload contrast63")
    ap.add_argument("--workload", default="svk125",
                    choices=["svk125", "cube31", "j2_315", "batch256", "adjoint243", "tangent125",
                             "mixed125", "precond125", "contrast63", "project125"],
                    help="svk125 (default) is the headline; the others print one line each")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload != "svk125":
        import torch
        from paper_1603_08893_gb300 import RVE
        fn = {"cube31": lambda: bench_cube31(args, torch, RVE),
              "j2_315": lambda: bench_j2_315(args, torch, RVE),
              "batch256": lambda: bench_batch256(args, torch),
              "adjoint243": lambda: bench_adjoint243(args, torch, RVE),
              "tangent125": lambda: bench_tangent125(args, torch, RVE),
              "mixed125": lambda: bench_mixed125(args, torch, RVE),
              "precond125": lambda: bench_precond125(args, torch, RVE),
              "contrast63": lambda: bench_contrast63(args, torch, RVE),
              "project125": lambda: bench_project125(args, torch, RVE)}[args.workload]
        fn()
        return None

    import torch
    rank, world, dist = dist_setup(args.gpus)
    from paper_1603_08893_gb300 import KERNEL_FAMILIES, RVE

    cfg = workload()
    n = int(np.prod(cfg["shape"]))
    # warm-up: W increments of the ramp on a separate cell (both precisions)
    for prec in (("mixed",) if args.mixed_only else ("mixed", "fp64")):
        w = run_schedule(RVE, cfg, prec, max(1, args.warmup if prec == "mixed" else 1), torch)
        w["rve"].close()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    mixed = run_schedule(RVE, cfg, "mixed", args.steps, torch)
    ck = clocks.stop()
    mixed["rve"].close()
    t_max, units = reduce_max_sum(dist, mixed["ms"], float(n) * mixed["cg"])
    value = units / (t_max / 1e3)

    if args.mixed_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT,
                              "steps": args.steps, "cg_iters": mixed["cg"],
                              "ms_per_step": t_max / args.steps, "mixed_only": True}))
        return None
    # float64 GPU path on the first increments, for the solve-time ratio and
    # the accuracy of the mixed path
    k64 = min(args.fp64_steps, args.steps)
    fp64 = run_schedule(RVE, cfg, "fp64", k64, torch, collect_pbar=True)
    fp64["rve"].close()
    mixed_k = run_schedule(RVE, cfg, "mixed", k64, torch, collect_pbar=True)
    mixed_k["rve"].close()
    perr = max(float(np.abs(a - b).max() / np.abs(b).max())
               for a, b in zip(mixed_k["pbars"], fp64["pbars"]))

    # end to end through the public API: per step the macroscopic F-bar goes
    # host -> device and the stress field P comes back into pinned host memory
    pinned = torch.empty(9 * n, dtype=torch.float64, pin_memory=True)
    e2e = run_schedule(RVE, cfg, "mixed", args.steps, torch, e2e_buf=pinned.numpy())
    e2e["rve"].close()
    t_e2e, u_e2e = reduce_max_sum(dist, e2e["wall_s"], float(n) * e2e["cg"])

    result = None
    if rank == 0:
        peak, peak_kind = load_peaks()
        roof = None
        prof = None
        if not args.no_profile:
            prof = kernel_profile(RVE, cfg, torch, KERNEL_FAMILIES)
            fam = max(prof, key=lambda f: prof[f]["total_ms"])
            bpl = family_bytes_per_voxel(cfg["shape"][2], fam) * n
            ach = bpl / (prof[fam]["avg_ms"] / 1e3) / 1e9
            roof = {"bound": "hbm", "kernel": fam, "achieved": round(ach, 1),
                    "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                    "traffic": NCU_TRAFFIC_BYTES.get(fam), "peak_kind": peak_kind,
                    "algorithmic_bytes_per_launch": bpl,
                    "avg_launch_ms": prof[fam]["avg_ms"]}
            # every family against the same peak, and the whole five-pass
            # iteration (algorithmic bytes of one iteration / its kernel time)
            per = {}
            tot_b = tot_ms = 0.0
            for f, v in prof.items():
                b_f = family_bytes_per_voxel(cfg["shape"][2], f) * n
                per[f] = round(b_f / (v["avg_ms"] / 1e3) / 1e9 / peak, 4)
                tot_b += b_f
                tot_ms += v["avg_ms"]
            roof["per_family_frac"] = per
            roof["iteration"] = {"bytes": tot_b, "ms": round(tot_ms, 5),
                                 "achieved": round(tot_b / (tot_ms / 1e3) / 1e9, 1),
                                 "frac": round(tot_b / (tot_ms / 1e3) / 1e9 / peak, 4)}
        cpu = (None if args.no_cpu_baseline else
               cpu_baseline_sample(cfg, mixed["cg"], mixed["newton"]))
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic",
            "config": {"workload": cfg["workload"], "grid": 125, "model": "svk",
                       "sphere_fraction": round(cfg["fraction"], 4), "contrast": 100,
                       "increments": args.steps, "tol_newton": cfg["tol_newton"],
                       "tol_cg": cfg["tol_cg"], "mixed_cg_tol_floor": 1e-5,
                       "l2": "working set ~1 GB > 129 MB L2, no flush needed",
                       "parallelism": f"replicas{world}"},
            "cg_iters": mixed["cg"], "newton_iters": mixed["newton"],
            "solve_ms_mixed": mixed["ms"],
            "fp64": {"steps": k64, "value": float(n) * fp64["cg"] / (fp64["ms"] / 1e3),
                     "cg_iters": fp64["cg"], "solve_ms": fp64["ms"],
                     "mixed_solve_ms_same_steps": mixed_k["ms"],
                     "mixed_cg_iters_same_steps": mixed_k["cg"],
                     "solve_time_ratio_fp64_over_mixed": fp64["ms"] / mixed_k["ms"],
                     "pbar_rel_err_mixed_vs_fp64": perr},
            "roofline": roof,
            "kernel_profile_ms": ({k: round(v["avg_ms"], 5) for k, v in prof.items()}
                                  if prof else None),
            "cpu_baseline": ({k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample",
                                                  "cpu_model", "extrapolated_full_run_s",
                                                  "extrapolation") if k in cpu}
                             if cpu else None),
            "e2e": {"value": u_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 72,
                    "d2h_bytes_per_step": 9 * n * 8 + 72},
            "clocks": ck,
            "gpu_launches": mixed["launches"],
        }
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return result


if __name__ == "__main__":
    main()
