"""Writes oracle results used as stored expected values by the GPU tests.

Calls only ``oracle/`` (and the seeded inputs of ``synth``).  Run from the
repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import solver  # noqa: E402


def cube31(tight):
    cfg = synth.config_cube31()
    prob = solver.SVKProblem.from_phase(cfg["phase"], cfg["phase_params"])
    out = []
    for Fbar in cfg["schedule"]:
        if tight:
            st = prob.increment(Fbar, tol_newton=1e-10, tol_cg=1e-12, cg_atol=1e-12)
        else:
            st = prob.increment(Fbar, tol_newton=cfg["tol_newton"], tol_cg=cfg["tol_cg"])
        out.append(dict(Fbar=Fbar.tolist(), Pbar=prob.homogenized_P().tolist(),
                        newton_iters=st.newton_iters, cg_iters=st.cg_iters,
                        Fnorm=float(np.linalg.norm(prob.F)),
                        Pnorm=float(np.linalg.norm(prob.P))))
    return out


if __name__ == "__main__":
    t = time.time()
    data = {
        "what": "SVK 31^3, 9^3 corner cube (x>=22, y<9, z>=22), contrast 10, "
                "simple shear gamma = 0.01 k, k = 1..10",
        "generator": "tests/golden/make_golden.py (oracle only)",
        "config_tolerances": {"tol_newton": 1e-5, "tol_cg": 1e-8,
                              "increments": cube31(False)},
        "tight": {"tol_newton": 1e-10, "tol_cg": 1e-12, "cg_atol": 1e-12,
                  "increments": cube31(True)},
    }
    with open(os.path.join(HERE, "svk31_cube_schedule.json"), "w") as f:
        json.dump(data, f, indent=1)
    print("written in", time.time() - t, "s")
