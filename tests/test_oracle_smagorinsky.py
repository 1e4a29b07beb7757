"""Pins for the Smagorinsky model of the oracle (Sec. III-C, turbulence
models): the solved rate satisfies both printed equations, C_S = 0 gives the
plain operator, conservation, equilibrium fixed point, and the model adds
dissipation to a decaying vortex."""
import numpy as np
import pytest

from oracle import collision as co
from oracle import lattice, lbm
from paper_2001_11806_gb300 import inputs


def _rand_f(lat, n=64, seed=0, amp=0.3):
    rng = np.random.default_rng(seed)
    return lat.w[:, None] * (1.0 + amp * rng.uniform(-1, 1, (lat.q, n)))


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q27"])
def test_rate_satisfies_both_equations(name):
    lat = lattice.get(name)
    f = _rand_f(lat)
    rho, u = co.velocity(lat, f)
    feq = co.equilibrium(lat, rho, u)
    om0, cs = 1.7, 0.17
    om = co.smagorinsky_omega(lat, f, feq, rho, om0, cs)
    # Eq. smag_shear: S_ij = -(3 omega / (2 rho)) Pi^neq_ij, |S| = sqrt(2 S_ij S_ij)
    c = lat.c.astype(float)
    S2 = 0.0
    for a in range(lat.d):
        for b in range(lat.d):
            Pi = ((c[:, a] * c[:, b])[:, None] * (f - feq)).sum(0)
            S = -3.0 * om / (2.0 * rho) * Pi
            S2 = S2 + S * S
    absS = np.sqrt(2.0 * S2)
    nu0 = (1.0 / om0 - 0.5) / 3.0
    # Eq. smag_omega
    assert np.abs(om - 2.0 / (6.0 * cs * cs * absS + 6.0 * nu0 + 1.0)).max() < 1e-14
    assert np.all(om < om0) and np.all(om > 0)


@pytest.mark.parametrize("op,omegas", [("srt", [1.6]), ("trt", [1.6, 0.9])])
def test_zero_constant_and_invariants(op, omegas):
    lat = lattice.d3q19()
    f = _rand_f(lat, seed=2)
    plain = co.collide(co.Method(lat, op, omegas), f)
    assert np.array_equal(co.collide(co.Method(lat, op, omegas, cs=0.0), f), plain)
    m = co.Method(lat, op, omegas, cs=0.2, magic=3 / 16 if op == "trt" else None)
    fs = co.collide(m, f)
    assert np.abs(fs.sum(0) - f.sum(0)).max() < 1e-15
    assert np.abs(co.momentum(lat, fs) - co.momentum(lat, f)).max() < 1e-15
    rho, u = co.velocity(lat, f)
    feq = co.equilibrium(lat, rho, u)
    assert np.abs(co.collide(m, feq) - feq).max() < 1e-15


def test_model_adds_dissipation():
    lat = lattice.d2q9()
    n = 32
    rho, u = inputs.tgv2d(n, 0.05)
    e = {}
    for cs in (0.0, 0.3):
        s = lbm.Sim(co.Method(lat, "srt", [1.95], cs=cs), (n, n, 1))
        s.init_equilibrium(rho, u)
        s.step(200)
        e[cs] = s.reduce()[4]
    assert e[0.3] < 0.99 * e[0.0]
