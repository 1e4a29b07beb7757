"""The bounds-checking build (LBM_DEBUG_BOUNDS): every population access of
the sweep kernels is checked against the population arrays, and an access
outside them is recorded and reported as LBM_E_BOUNDS by the next
synchronising call instead of faulting.  This test builds that library and
runs every sweep kind on it (dense periodic, FP16 two-cell, fluid-cell list
with inlet/outlet cells, separate boundary kernels, CUDA-graph replay): the
results must match the oracle and no call may report LBM_E_BOUNDS.  (No test
provokes an out-of-array access on the GPU.)"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np
from paper_2001_11806_gb300 import _lib, inputs
from paper_2001_11806_gb300.sim import Sim
from oracle import collision as oco, lattice as olat, lbm as olbm
assert _lib.LIB_PATH.endswith("liblbm_debug.so"), _lib.LIB_PATH
TOL = {"f64": 1e-12, "f32": 1e-5, "f16s": 5e-3}

def flags(shape):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[:, 0, :] = olbm.NOSLIP
    fl[:, -1, :] = olbm.NOSLIP
    fl[:, 1:-1, 0] = olbm.INLET
    fl[:, 1:-1, -1] = olbm.OUTLET
    r = inputs.uniform(3, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.08) & (fl == 0)] = olbm.NOSLIP
    return fl

cases = []
for pattern in ["pull", "aa", "eso"]:
    for storage in ["f32", "f16s"]:
        cases.append(("D3Q19", "trt", [1.6, 1.1], storage, pattern, (34, 6, 5), None, "in_sweep", 5))
        cases.append(("D3Q19", "mrt", [1.7, 1.1, 1.3, 1.3], storage, pattern, (40, 7, 5), "channel", "in_sweep", 5))
    cases.append(("D3Q27", "cumulant", [1.9, 1.0, 1.0], "f32", pattern, (36, 5, 4), "channel", "in_sweep", 4))
    cases.append(("D2Q9", "srt", [1.4], "f64", pattern, (30, 9, 1), None, "in_sweep", 70))
cases.append(("D3Q19", "trt", [1.6, 1.1], "f32", "pull", (40, 7, 5), "channel", "separate", 5))
cases.append(("D3Q19", "kbc", [1.9, 1.9], "f32", "aa", (36, 7, 5), "channel", "in_sweep", 5))
for st, coll, om, storage, pattern, shape, geo, bmode, steps in cases:
    lat = olat.get(st)
    fl = flags(shape) if geo else None
    per = (False, False, True) if geo else (True, True, True)
    sim = Sim(st, coll, storage, pattern, shape, periodic=per, omega=om, u_wall=(0.04, 0.0, 0.0), flags=fl,
              boundary=bmode)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=7)
    sim.set_state(P.reshape(lat.q, -1))
    sim.step(steps)
    sim.sync()
    ref = olbm.Sim(oco.Method(lat, coll, om), shape, periodic=per, flags=fl, u_wall=(0.04, 0.0, 0.0))
    ref.P = P.copy()
    ref.step(steps)
    fluid = ref.fluid.reshape(-1)
    fg = sim.populations().cpu().numpy()[:, fluid]
    fr = ref.populations().reshape(lat.q, -1)[:, fluid]
    err = np.linalg.norm(fg - fr) / np.linalg.norm(fr - lat.w[:, None])
    # rounding grows with the number of steps (the 70-step case replays graphs)
    assert err < TOL[storage] * max(1.0, steps / 10), (st, coll, storage, pattern, geo, bmode, err)
    sim.close()
print("ok", len(cases))
'''


def test_bounds_checking_build_runs_clean():
    b = subprocess.run([sys.executable, "-c",
                        "from paper_2001_11806_gb300 import build; build.build(debug_bounds=True)"],
                       cwd=ROOT, capture_output=True, text=True, timeout=3600)
    assert b.returncode == 0, b.stderr[-3000:]
    env = dict(os.environ, LBM_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-3000:])
    assert r.stdout.strip().startswith("ok")
