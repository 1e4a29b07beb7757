"""lbm_reduce_noalloc: the conservation sums for callers that cannot allocate
device memory (their GPU memory belongs to another allocator, or they cannot
pay cudaMalloc's device-wide synchronisation inside a time-step loop).

The entry point is called through the C ABI on the raw population array of a
running simulation and must agree with lbm_reduce of the same state and with
the oracle's sums, on two calls in a row (the second call reuses the
library's fixed scratch array that the first one left behind).  Cases cover
flags and the periodic flag-free path, the pull, AA and esoteric-twist
layouts at both parities, and a domain of several scratch rows whose last
chunk is partial, followed by a smaller one that must not see the rows the
larger call left behind.  The call does not synchronise and so cannot report
a non-finite sum: a NaN is left in its output (checked below).  The buffers
below are allocated by the test; the entry point itself allocates nothing.
This file is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import _lib, inputs
from paper_2001_11806_gb300.sim import Sim

pytestmark = pytest.mark.gpu

OMEGAS = {"srt": [1.37], "trt": [1.8, 8 / 31], "mrt": [1.7, 1.1, 0.9, 1.3], "cumulant": [1.95, 1.0, 1.0]}
# oracle tolerance of each storage, relative to the sum of the magnitudes of
# the summed terms (the field tolerances of the parity tests)
TOL = {"f64": 1e-12, "f32": 1e-5, "f32s": 1e-5, "f16s": 5e-3}


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


def _case(stencil, collision, storage, pattern, shape, steps, with_flags=True):
    om = OMEGAS[collision]
    force = [2e-4, -1e-4, 0.0] if collision != "cumulant" else [0.0, 0.0, 0.0]
    fl = _flags(shape) if with_flags else None
    per = (False, False, True) if with_flags else (True, True, True)
    sim = Sim(stencil, collision, storage, pattern, shape, periodic=per, omega=om, u_wall=(0.05, 0.0, 0.0),
              force=force, flags=fl)
    lat = olat.get(stencil)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=4)
    sim.set_state(P.reshape(lat.q, -1))
    sim.step(steps)
    ref = olbm.Sim(oco.Method(lat, collision, OMEGAS[collision], force=None if collision == "cumulant" else force[:lat.d]),
                   shape, periodic=per, flags=fl, u_wall=(0.05, 0.0, 0.0))
    ref.P = P.copy()
    ref.step(steps)
    rho, u = ref.macroscopic()
    fluid = ref.fluid
    scale = [np.abs(rho[fluid]).sum()] + [np.abs(rho * u[a])[fluid].sum() for a in range(lat.d)]
    scale += [0.0] * (3 - lat.d) + [abs(ref.reduce()[4])]
    return sim, ref.reduce(), np.array(scale)


def _noalloc(sim, raw, t, out):
    stream = torch.cuda.current_stream(sim.device).cuda_stream
    flags = sim.flags.data_ptr() if sim.flags is not None else None
    return _lib.lib().lbm_reduce_noalloc(ctypes.byref(sim.params), raw.data_ptr(), flags, t, out.data_ptr(), stream)


def _check(sim, oracle_sums, scale, storage, calls=2):
    ref = sim.reduce()
    raw, t = sim.get_pdfs()
    out = torch.full((5,), float("nan"), dtype=torch.float64, device=sim.device)
    for _ in range(calls):
        out.fill_(float("nan"))
        assert _noalloc(sim, raw, t, out) == 0
        got = out.cpu().numpy()
        assert abs(got[0] / ref[0] - 1) < 1e-13
        for a in range(1, 5):
            assert abs(got[a] - ref[a]) <= 1e-12 * max(abs(ref[a]), 1.0), (a, got[a], ref[a])
        err = np.abs(got - oracle_sums)
        assert np.all(err <= TOL[storage] * np.maximum(scale, 1e-300)), (got, oracle_sums, scale)


@pytest.mark.parametrize("stencil,collision,storage,pattern,steps,with_flags", [
    ("D3Q19", "trt", "f32", "aa", 3, True),
    ("D3Q19", "mrt", "f64", "pull", 2, True),
    ("D2Q9", "srt", "f16s", "aa", 4, True),
    ("D3Q27", "cumulant", "f32s", "pull", 3, True),
    ("D3Q19", "trt", "f64", "eso", 3, True),
    ("D3Q19", "trt", "f64", "eso", 4, True),
    ("D3Q27", "trt", "f32", "eso", 5, True),
    ("D3Q19", "trt", "f64", "aa", 3, False),
    ("D3Q19", "srt", "f32", "eso", 3, False),
    ("D2Q9", "trt", "f64", "pull", 2, False),
])
def test_noalloc_matches_lbm_reduce_and_oracle_twice(stencil, collision, storage, pattern, steps, with_flags):
    shape = (150, 5, 1) if stencil == "D2Q9" else (150, 5, 4)
    sim, oracle_sums, scale = _case(stencil, collision, storage, pattern, shape, steps, with_flags)
    _check(sim, oracle_sums, scale, storage)


def test_noalloc_several_rows_then_a_smaller_domain():
    """64 x 64 x 9 = 36,864 cells fill three scratch rows of 16,384 cells, the
    last one partial; the smaller domain that follows (one row) must agree
    with its own lbm_reduce, whatever the larger call left in the array."""
    big, ref_b, sc_b = _case("D3Q19", "trt", "f64", "aa", (64, 64, 9), 3)
    _check(big, ref_b, sc_b, "f64")
    small, ref_s, sc_s = _case("D3Q19", "trt", "f64", "eso", (40, 6, 5), 3)
    _check(small, ref_s, sc_s, "f64")
    _check(big, ref_b, sc_b, "f64", calls=1)


def test_noalloc_leaves_a_nonfinite_sum_in_its_output():
    lat = olat.d3q19()
    shape = (12, 6, 5)
    sim = Sim("D3Q19", "trt", "f32", "aa", shape, omega=[1.6, 1.1])
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=41).reshape(19, -1)
    P[3, 17] = np.nan
    sim.set_state(P)
    sim.step(2)
    raw, t = sim.get_pdfs()
    out = torch.zeros(5, dtype=torch.float64, device=sim.device)
    assert _noalloc(sim, raw, t, out) == 0
    assert not np.all(np.isfinite(out.cpu().numpy()))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    p = _lib.Params()
    _lib.lib().lbm_default_params(ctypes.byref(p))
    p.nx, p.ny, p.nz = 4096, 4096, 5  # 83.9 M cells > 67,108,864
    out = torch.zeros(5, dtype=torch.float64, device="cuda:0")
    status = _lib.lib().lbm_reduce_noalloc(ctypes.byref(p), out.data_ptr(), None, 0, out.data_ptr(), None)
    assert status == 1  # LBM_E_INVAL
