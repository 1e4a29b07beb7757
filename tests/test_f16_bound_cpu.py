"""The element-wise tolerance of the FP16-shifted GPU tests, checked on the CPU.

FP16-shifted storage rounds every stored h = f - w to binary16 once per step
(round to nearest even, unit roundoff U16 = 2^-11).  The GPU tests hold each
population to |f_gpu - f_ref| <= 3 U16 max|h_ref|.  Here that bound is checked
against a rounding model: the oracle's FP64 step followed by the RNE rounding
of its state to binary16 (numpy's float64 -> float16 conversion), on the
walls-inlet-outlet-obstacle box of the GPU channel tests, for five steps.  The
model has to stay well inside the bound (1.5 U16 max|h|, leaving the rest for
the GPU's FP32 arithmetic and for the single-array patterns, which round
boundary values when they write them).  A wrong wall velocity, planted in the
oracle, has to exceed the bound by far, so that the bound still detects the
boundary errors it is there for."""
import numpy as np
import pytest

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs

U16 = 2.0 ** -11


def _flags(shape, seed=3):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[:, 0, :] = olbm.NOSLIP
    fl[:, -1, :] = olbm.NOSLIP
    fl[:, 1:-1, 0] = olbm.INLET
    fl[:, 1:-1, -1] = olbm.OUTLET
    r = inputs.uniform(seed, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.08) & (fl == 0)] = olbm.NOSLIP
    return fl


def _round16(P, w):
    return (P - w).astype(np.float16).astype(np.float64) + w


def test_binary16_rounding_is_round_to_nearest_even():
    """The rounding model is the library conversion: exact on representable
    values, ties to even, 11 significant bits."""
    one_ulp = 2.0 ** -10
    x = np.array([1.0, 1.0 + one_ulp, 1.0 + one_ulp / 2, 1.0 + 1.5 * one_ulp, 3e-3])
    r = x.astype(np.float16).astype(np.float64)
    assert r[0] == 1.0 and r[1] == 1.0 + one_ulp
    assert r[2] == 1.0 and r[3] == 1.0 + 2 * one_ulp
    assert abs(r[4] - 3e-3) <= U16 * 3e-3


@pytest.mark.parametrize("stencil,collision,omegas", [("D2Q9", "srt", [1.37]), ("D3Q19", "mrt", [1.7, 1.1, 0.9, 1.3]),
                                                      ("D3Q19", "kbc", [1.9, 1.3])])
def test_rounding_model_within_elementwise_bound(stencil, collision, omegas):
    lat = olat.get(stencil)
    shape = (150, 7, 1) if stencil == "D2Q9" else (150, 5, 4)
    fl = _flags(shape)
    m = oco.Method(lat, collision, omegas)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=5)
    w = lat.w.reshape((-1,) + (1,) * 3)
    kw = dict(periodic=(False, False, True), flags=fl, u_wall=(0.05, 0.01, 0.0))
    exact, model = olbm.Sim(m, shape, **kw), olbm.Sim(m, shape, **kw)
    wrong = olbm.Sim(m, shape, periodic=(False, False, True), flags=fl, u_wall=(-0.05, 0.01, 0.0))
    exact.P = P.copy()
    wrong.P = P.copy()
    model.P = _round16(P, w)
    fluid = fl.reshape(-1) == 0
    for _ in range(5):
        exact.step(1)
        wrong.step(1)
        model.P = _round16(model.step_state(model.P), w)
        fr = exact.populations().reshape(lat.q, -1)[:, fluid]
        bound = 3 * U16 * np.abs(fr - lat.w[:, None]).max()
        d_model = np.abs(model.populations().reshape(lat.q, -1)[:, fluid] - fr).max()
        d_wrong = np.abs(wrong.populations().reshape(lat.q, -1)[:, fluid] - fr).max()
        assert d_model <= 0.5 * bound, (d_model, bound)
        assert d_wrong >= 20 * bound, (d_wrong, bound)
