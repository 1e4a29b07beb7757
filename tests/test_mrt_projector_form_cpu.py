"""MRT whose moments of order >= 3 share one rate equals its projector form
(the form the sweep uses when the rates allow it), checked on the CPU
against the oracle's moment-matrix MRT (Eq. mrt) with and without a Guo
force:

  h* = h + G - omega_h y - (omega_s - omega_h) Ys - (omega_b - omega_h) Yb,
  y = h - h^eq + G/2,  Ys_q = 4.5 w_q c_q.dev(Pi_y).c_q,
  Yb_q = (4.5/D) w_q (|c_q|^2 - D/3) tr(Pi_y),  Pi_y = sum_q c_q c_q y_q.

A wrong sign, a missing G/2 or a projector of the wrong span fails this."""
import numpy as np
import pytest

from oracle import collision as co
from oracle import lattice


def _projector_form(lat, f, om_s, om_b, om_h, force):
    d = lat.d
    c = lat.c.astype(np.float64)
    rho, u = co.velocity(lat, f, force)
    feq = co.equilibrium(lat, rho, u)
    G = co.guo_source(lat, u, force) if force is not None else np.zeros_like(f)
    y = f - feq + 0.5 * G
    pi = np.einsum("qa,qb,q...->ab...", c, c, y)
    tr = np.trace(pi)
    dev = pi - tr / d * np.eye(d)[:, :, None]
    w = lat.w[:, None]
    quad = np.einsum("qa,qb,ab...->q...", c, c, dev)
    c2 = (c * c).sum(1)[:, None]
    Ys = 4.5 * w * quad
    Yb = (4.5 / d) * w * (c2 - d / 3.0) * tr
    return f + G - om_h * y - (om_s - om_h) * Ys - (om_b - om_h) * Yb


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("with_force", [False, True])
def test_projector_form_equals_moment_matrix_mrt(name, with_force):
    lat = lattice.get(name)
    rng = np.random.default_rng(5)
    n = 30
    rho = 1 + 0.02 * rng.uniform(-1, 1, n)
    u = 0.05 * rng.uniform(-1, 1, (lat.d, n))
    f = co.equilibrium(lat, rho, u) * (1 + 0.1 * rng.uniform(-1, 1, (lat.q, n)))
    om_s, om_b, om_h = 1.7, 1.1, 1.3
    nrates = 6 if name == "D3Q27" else 4
    omegas = [om_s, om_b] + [om_h] * (nrates - 2)
    force = np.array([2e-4, -1e-4, 5e-5][: lat.d]) if with_force else None
    ref = co.collide(co.Method(lat, "mrt", omegas, force=force), f)
    got = _projector_form(lat, f, om_s, om_b, om_h, force)
    assert np.abs(got - ref).max() < 1e-15
    # a distinct higher-order rate is not captured by the projector form
    omegas2 = [om_s, om_b, om_h, 0.9] + [om_h] * (nrates - 4)
    ref2 = co.collide(co.Method(lat, "mrt", omegas2, force=force), f)
    assert np.abs(got - ref2).max() > 1e-6
