"""lbm_reduce_noalloc: the conservation sums for callers that cannot allocate
device memory (their GPU memory belongs to another allocator, or they cannot
pay cudaMalloc's device-wide synchronisation inside a time-step loop).

The entry point is called through the C ABI on the raw population array of a
running simulation and must agree with lbm_reduce of the same state, on two
calls in a row (the second call reuses the library's fixed scratch array that
the first one left behind).  The buffers below are allocated by the test; the
entry point itself allocates nothing.  This file is collected last so that a
run stopping at its first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import lattice as olat
from paper_2001_11806_gb300 import _lib, inputs
from paper_2001_11806_gb300.sim import Sim

pytestmark = pytest.mark.gpu


def _flags(shape):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[:, 0, :] = 1
    fl[:, -1, :] = 1
    fl[:, 1:-1, 0] = 2
    fl[:, 1:-1, -1] = 4
    r = inputs.uniform(3, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.08) & (fl == 0)] = 1
    return fl


@pytest.mark.parametrize("stencil,collision,storage,pattern,steps", [
    ("D3Q19", "trt", "f32", "aa", 3),
    ("D3Q19", "mrt", "f64", "pull", 2),
    ("D2Q9", "srt", "f16s", "aa", 4),
    ("D3Q27", "cumulant", "f32s", "pull", 3),
])
def test_noalloc_matches_lbm_reduce_twice(stencil, collision, storage, pattern, steps):
    shape = (150, 5, 1) if stencil == "D2Q9" else (150, 5, 4)
    om = {"srt": [1.37], "trt": [1.8, 8 / 31], "mrt": [1.7, 1.1, 0.9, 1.3], "cumulant": [1.95, 1.0, 1.0]}[collision]
    fl = _flags(shape)
    force = [2e-4, -1e-4, 0.0] if collision != "cumulant" else [0.0, 0.0, 0.0]
    sim = Sim(stencil, collision, storage, pattern, shape, periodic=(False, False, True), omega=om,
              u_wall=(0.05, 0.0, 0.0), force=force, flags=fl)
    lat = olat.get(stencil)
    sim.set_state(inputs.random_pdfs(lat.w, shape[::-1], seed=4).reshape(lat.q, -1))
    sim.step(steps)
    ref = sim.reduce()
    raw, t = sim.get_pdfs()
    out = torch.full((5,), float("nan"), dtype=torch.float64, device=sim.device)
    stream = torch.cuda.current_stream(sim.device).cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        status = _lib.lib().lbm_reduce_noalloc(ctypes.byref(sim.params), raw.data_ptr(), sim.flags.data_ptr(),
                                               t, out.data_ptr(), stream)
        assert status == 0
        got = out.cpu().numpy()
        assert abs(got[0] / ref[0] - 1) < 1e-13
        for a in range(1, 5):
            assert abs(got[a] - ref[a]) <= 1e-12 * max(abs(ref[a]), 1.0), (a, got[a], ref[a])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    p = _lib.Params()
    _lib.lib().lbm_default_params(ctypes.byref(p))
    p.nx, p.ny, p.nz = 4096, 4096, 5  # 83.9 M cells > 67,108,864
    out = torch.zeros(5, dtype=torch.float64, device="cuda:0")
    status = _lib.lib().lbm_reduce_noalloc(ctypes.byref(p), out.data_ptr(), None, 0, out.data_ptr(), None)
    assert status == 1  # LBM_E_INVAL
