"""Pins of the inlet/outlet pair against the flow it must produce.

The outlet (B_q = f^eq_q(rho_out, u_P(x))) is a reading: the paper names
pressure boundaries but prints none.  What any correct pair of a velocity
bounce-back inlet (UBB listing of Sec. III-C, rho_0 = 1) and a pressure
outlet must do in a channel that is periodic across the flow:

- the uniform state rho = rho_out, momentum j = rho_0 u_in is a fixed point.
  In it every collision is the identity (f = f^eq), the UBB link gives
  f^eq_qbar + 6 w_q rho_0 c_q.u_in, which is f^eq_q exactly because
  f^eq_q - f^eq_qbar = 6 w_q c_q.j for both equilibria (the quadratic terms
  are even in c), and the outlet returns f^eq(rho_out, j / rho) of that state;
- from rest it is also the steady state: with no walls, mass conservation
  makes j_x uniform, the inlet fixes it to rho_0 u_in, there is no friction
  to hold a pressure gradient, and the outlet fixes the pressure.

A wrong sign of u at the outlet, an outlet that ignores rho_out, a UBB term
scaled by the local density or an outlet velocity that is not divided by
rho each leave a different state (the density errors are 3e-2, the tests
ask for 1e-8).
"""
import numpy as np
import pytest

from oracle import collision as co
from oracle import lattice
from oracle import lbm

U_IN, RHO_OUT = 0.03, 1.03


def _channel(lat, n):
    shp = n if lat.d == 3 else (n[0], n[1], 1)
    flags = np.zeros(shp[::-1], np.uint8)
    flags[..., 0] = lbm.INLET
    flags[..., -1] = lbm.OUTLET
    return shp, flags


def _method(lat, op, incompressible):
    omegas = {"srt": [1.3], "trt": [1.3, 0.9], "mrt": [1.3, 1.1, 0.9, 1.2]}[op]
    return co.Method(lat, op, omegas, incompressible=incompressible)


def _uniform(lat, shp, incompressible):
    # j = rho_0 u_in with rho_0 = 1: u = u_in (incompressible, u = j / rho_0)
    # or u_in / rho_out (compressible, u = j / rho)
    ux = U_IN if incompressible else U_IN / RHO_OUT
    u = np.zeros((lat.d,) + shp[::-1])
    u[0] = ux
    return np.full(shp[::-1], RHO_OUT), u


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("op", ["srt", "trt", "mrt"])
@pytest.mark.parametrize("incompressible", [False, True])
def test_outlet_density_state_is_fixed_point(name, op, incompressible):
    lat = lattice.get(name)
    shp, flags = _channel(lat, (7, 3, 3))
    s = lbm.Sim(_method(lat, op, incompressible), shp, periodic=(False, True, True), flags=flags,
                u_wall=(U_IN, 0.0, 0.0), rho_out=RHO_OUT)
    rho0, u0 = _uniform(lat, shp, incompressible)
    s.init_equilibrium(rho0, u0)
    P0 = s.P.copy()
    s.step(4)
    fl = s.fluid
    assert np.abs(s.P[:, fl] - P0[:, fl]).max() < 1e-15


@pytest.mark.parametrize("name,n,steps,tol", [("D2Q9", (16, 2, 1), 6000, 1e-8), ("D3Q19", (12, 2, 2), 4000, 1e-12)])
@pytest.mark.parametrize("incompressible", [False, True])
def test_channel_from_rest_reaches_outlet_pressure(name, n, steps, tol, incompressible):
    lat = lattice.get(name)
    shp, flags = _channel(lat, n)
    m = co.Method(lat, "srt", [1.0], incompressible=incompressible)
    s = lbm.Sim(m, shp, periodic=(False, True, True), flags=flags, u_wall=(U_IN, 0.0, 0.0), rho_out=RHO_OUT)
    s.init_equilibrium(np.ones(shp[::-1]), np.zeros((lat.d,) + shp[::-1]))
    s.step(steps)
    rho, u = s.macroscopic()
    fl = s.fluid
    jx = u[0] * (1.0 if incompressible else rho)
    assert np.abs(rho[fl] - RHO_OUT).max() < tol
    assert np.abs(jx[fl] - U_IN).max() < tol
    for a in range(1, lat.d):
        assert np.abs(u[a][fl]).max() < tol
