"""Pins for oracle.cumulant.

The strongest pin re-derives every cumulant straight from
Eq. cumulant_generating_function, K(xi) = ln sum_q f_q exp(c_q.xi), without
the ring: Taylor coefficients of the analytic K are extracted with Cauchy's
integral formula, discretised by the trapezoid rule on small circles in each
complex xi_a plane (spectrally accurate), using numpy's complex log."""
import itertools
from math import factorial

import numpy as np
import pytest

from oracle import collision as co
from oracle import cumulant as cu
from oracle import lattice

LAT = lattice.d3q27()
CS2 = 1.0 / 3.0


def _rand_f(n=6, seed=0, amp=0.3):
    rng = np.random.default_rng(seed)
    return LAT.w[:, None] * (1.0 + amp * rng.uniform(-1, 1, (27, n))) * (1 + 0.1 * rng.uniform(-1, 1, n))


def _cauchy_cumulants(f_cell, r=0.15, n=24):
    th = 2 * np.pi * np.arange(n) / n
    z = r * np.exp(1j * th)
    X, Y, Z = np.meshgrid(z, z, z, indexing="ij")
    c = LAT.c.astype(float)
    S = sum(f_cell[q] * np.exp(c[q, 0] * X + c[q, 1] * Y + c[q, 2] * Z) for q in range(27))
    K = np.log(S)
    out = {}
    for a, b, cc in itertools.product(range(3), repeat=3):
        coef = (K * X ** (-a) * Y ** (-b) * Z ** (-cc)).mean()
        out[(a, b, cc)] = (coef * factorial(a) * factorial(b) * factorial(cc)).real
    return out


def test_cumulants_match_cauchy_integral_of_definition():
    f = _rand_f(n=3, seed=4)
    rho, kap = cu.cumulants(LAT, f)
    for cell in range(3):
        ref = _cauchy_cumulants(f[:, cell])
        for e, i in cu.IDX.items():
            val = kap[i, cell] + (np.log(rho[cell]) if e == (0, 0, 0) else 0.0)
            assert abs(val - ref[e]) < 1e-11, (e, val, ref[e])


def test_round_trip_identity():
    f = _rand_f(n=50)
    rho, kap = cu.cumulants(LAT, f)
    assert np.abs(cu.populations_from_cumulants(LAT, rho, kap) - f).max() < 1e-15


def _product_eq(rho, u):
    def p(c, v):
        return np.where(c == 0, 1 - CS2 - v * v, (CS2 + v * v + c * v) / 2)
    return np.stack([rho * p(c[0], u[0]) * p(c[1], u[1]) * p(c[2], u[2]) for c in LAT.c_list])


def test_all_rates_one_gives_product_equilibrium():
    f = _rand_f(n=40, seed=2)
    fs = co.collide(co.Method(LAT, "cumulant", [1.0, 1.0, 1.0]), f)
    rho, u = co.velocity(LAT, f)
    assert np.abs(fs - _product_eq(rho, u)).max() < 1e-15


def test_conservation_and_fixed_point():
    f = _rand_f(n=40, seed=3)
    m = co.Method(LAT, "cumulant", [1.95, 1.0, 1.0])
    fs = co.collide(m, f)
    assert np.abs(fs.sum(0) - f.sum(0)).max() < 1e-15
    assert np.abs(co.momentum(LAT, fs) - co.momentum(LAT, f)).max() < 1e-16
    rho, u = co.velocity(LAT, f)
    eq = _product_eq(rho, u)
    for rates in ([1.95, 1.0, 1.0], [1.3, 0.7, 1.4]):
        assert np.abs(co.collide(co.Method(LAT, "cumulant", rates), eq) - eq).max() < 1e-15


def test_second_order_is_covariance_and_mixed_vanish_for_products():
    f = _rand_f(n=10, seed=6)
    rho, kap = cu.cumulants(LAT, f)
    c = LAT.c.astype(float)
    u = (c.T @ f) / rho
    for a, b in itertools.product(range(3), range(3)):
        e = [0, 0, 0]
        e[a] += 1
        e[b] += 1
        cov = ((c[:, a, None] - u[a]) * (c[:, b, None] - u[b]) * f).sum(0) / rho
        assert np.abs(kap[cu.IDX[tuple(e)]] - cov).max() < 1e-15
    # independent axes: K separates, every mixed cumulant is zero
    rng = np.random.default_rng(9)
    px, py, pz = (rng.uniform(0.1, 1.0, (3, 4)) for _ in range(3))
    fp = np.stack([px[c[0] + 1] * py[c[1] + 1] * pz[c[2] + 1] for c in LAT.c_list])
    _, kp = cu.cumulants(LAT, fp)
    for e, i in cu.IDX.items():
        if sum(x > 0 for x in e) >= 2:
            assert np.abs(kp[i]).max() < 1e-15, e


@pytest.mark.parametrize("bad", ["D2Q9", "D3Q19"])
def test_other_stencils_rejected(bad):
    lat = lattice.get(bad)
    with pytest.raises(ValueError):
        co.collide(co.Method(lat, "cumulant", [1.5, 1.0, 1.0]), lat.w[:, None] * np.ones((lat.q, 2)))
