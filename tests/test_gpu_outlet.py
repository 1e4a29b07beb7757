"""Outlet density on the GPU: parity with the FP64 oracle at rho_out != 1,
and the steady state of a channel that is periodic across the flow.

From rest, a channel with a velocity bounce-back inlet (rho_0 = 1) and a
pressure outlet, periodic in y and z, settles to rho = rho_out and momentum
j = rho_0 u_in everywhere (mass conservation makes j_x uniform, nothing
holds a pressure gradient); the oracle reaches it too, so the GPU kernels
are checked against the flow as well as against the oracle.  Tolerances as
in the other parity tests: 1e-12 for FP64 storage, 1e-5 for FP32."""
import numpy as np
import pytest

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs
from paper_2001_11806_gb300.sim import Sim

pytestmark = pytest.mark.gpu

U_IN, RHO_OUT = 0.03, 1.03
OMEGAS = {"srt": [1.37], "trt": [1.8, 8 / 31], "mrt": [1.7, 1.1, 0.9, 1.3, 1.2, 1.05]}
TOL = {"f64": 1e-12, "f32": 1e-5}


def _shape(stencil):
    return (150, 7, 1) if stencil == "D2Q9" else (150, 5, 4)


def _flags(shape, seed=4):
    # walls on y, inlet at x = 0, outlet at x = nx - 1, a few obstacles
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[:, 0, :] = olbm.NOSLIP
    fl[:, -1, :] = olbm.NOSLIP
    fl[:, 1:-1, 0] = olbm.INLET
    fl[:, 1:-1, -1] = olbm.OUTLET
    r = inputs.uniform(seed, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.06) & (fl == 0)] = olbm.NOSLIP
    return fl


def _rates(stencil, collision):
    om = OMEGAS[collision]
    if collision == "mrt":
        om = om[:6] if stencil == "D3Q27" else om[:4]
    return om


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("collision", ["srt", "trt", "mrt"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
@pytest.mark.parametrize("incompressible", [False, True])
def test_outlet_density_parity(stencil, collision, storage, pattern, incompressible):
    lat = olat.get(stencil)
    shape = _shape(stencil)
    fl = _flags(shape)
    per = (False, False, True)
    om = _rates(stencil, collision)
    sim = Sim(stencil, collision, storage, pattern, shape, periodic=per, omega=OMEGAS[collision],
              incompressible=incompressible, u_wall=(U_IN, 0.0, 0.0), rho_outlet=RHO_OUT, flags=fl)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=6)
    sim.set_state(P.reshape(lat.q, -1))
    sim.step(4)
    f_gpu = sim.populations().cpu().numpy()
    ref = olbm.Sim(oco.Method(lat, collision, om, incompressible=incompressible), shape, periodic=per,
                   flags=fl, u_wall=(U_IN, 0.0, 0.0), rho_out=RHO_OUT)
    ref.P = P.copy()
    ref.step(4)
    f_ref = ref.populations().reshape(lat.q, -1)
    m = ref.fluid.reshape(-1)
    err = np.linalg.norm(f_gpu[:, m] - f_ref[:, m]) / np.linalg.norm(f_ref[:, m] - lat.w[:, None])
    assert err < TOL[storage], err


@pytest.mark.parametrize("stencil,shape,steps,tol", [("D2Q9", (16, 2, 1), 6000, 1e-8),
                                                     ("D3Q19", (12, 2, 2), 4000, 1e-12)])
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
@pytest.mark.parametrize("incompressible", [False, True])
def test_channel_from_rest_reaches_outlet_pressure(stencil, shape, steps, tol, pattern, incompressible):
    lat = olat.get(stencil)
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[..., 0] = olbm.INLET
    fl[..., -1] = olbm.OUTLET
    sim = Sim(stencil, "srt", "f64", pattern, shape, periodic=(False, True, True), omega=[1.0],
              incompressible=incompressible, u_wall=(U_IN, 0.0, 0.0), rho_outlet=RHO_OUT, flags=fl)
    rho0 = np.ones(shape[::-1])
    u0 = np.zeros((lat.d,) + shape[::-1])
    sim.init_equilibrium(rho0, u0)
    sim.step(steps)
    rho, u = (t.cpu().numpy() for t in sim.macroscopic(True))
    m = (fl == 0).reshape(-1)
    rho = rho.reshape(-1)[m]
    u = u.reshape(lat.d, -1)[:, m]
    jx = u[0] * (1.0 if incompressible else rho)
    assert np.abs(rho - RHO_OUT).max() < tol
    assert np.abs(jx - U_IN).max() < tol
    for a in range(1, lat.d):
        assert np.abs(u[a]).max() < tol
