"""Pins for oracle.collision: equilibrium moments, conservation, fixed
point, operator equivalences (SRT == TRT(we=wo) == MRT(all equal);
TRT == MRT with even/odd rates), Guo momentum input."""
import numpy as np
import pytest

from oracle import collision as co
from oracle import lattice

NAMES = ["D2Q9", "D3Q19", "D3Q27"]
CS2 = 1.0 / 3.0


def _rand_f(lat, n=64, seed=0, amp=0.3):
    rng = np.random.default_rng(seed)
    return lat.w[:, None] * (1.0 + amp * rng.uniform(-1, 1, (lat.q, n)))


def _rand_ru(lat, n=64, seed=1):
    rng = np.random.default_rng(seed)
    return 1.0 + 0.05 * rng.uniform(-1, 1, n), 0.08 * rng.uniform(-1, 1, (lat.d, n))


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("incomp", [False, True])
def test_equilibrium_moments(name, incomp):
    lat = lattice.get(name)
    rho, u = _rand_ru(lat)
    feq = co.equilibrium(lat, rho, u, incomp)
    rho0 = 1.0 if incomp else rho
    c = lat.c.astype(float)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-15)
    for a in range(lat.d):
        assert np.allclose((c[:, a, None] * feq).sum(0), rho0 * u[a], rtol=0, atol=1e-16)
        for b in range(lat.d):
            pi = (c[:, a, None] * c[:, b, None] * feq).sum(0)
            ref = rho * CS2 * (a == b) + rho0 * u[a] * u[b]
            assert np.allclose(pi, ref, rtol=0, atol=1e-15)


def _methods(lat, force=None):
    out = [co.Method(lat, "srt", [1.3], force=force),
           co.Method(lat, "trt", [1.7, co.trt_odd_rate(1.7, 3 / 16)], force=force),
           co.Method(lat, "mrt", [1.6, 1.1, 0.9, 1.3, 1.2, 1.05], force=force)]
    if lat.name == "D3Q27" and force is None:
        out.append(co.Method(lat, "cumulant", [1.6, 1.1, 0.8]))
    return out


@pytest.mark.parametrize("name", NAMES)
def test_conservation_and_fixed_point(name):
    lat = lattice.get(name)
    f = _rand_f(lat)
    rho, u = _rand_ru(lat)
    for m in _methods(lat):
        fs = co.collide(m, f)
        assert np.abs(fs.sum(0) - f.sum(0)).max() < 1e-14
        assert np.abs(co.momentum(lat, fs) - co.momentum(lat, f)).max() < 1e-15
        if m.op == "cumulant":
            continue  # its fixed point is the product-form Maxwellian (test_oracle_cumulant)
        feq = co.equilibrium(lat, rho, u)
        assert np.abs(co.collide(m, feq) - feq).max() < 2e-15, m.op


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("force", [None, (2e-3, -1e-3, 5e-4)])
def test_operator_equivalence(name, force):
    lat = lattice.get(name)
    F = None if force is None else force[: lat.d]
    f = _rand_f(lat)
    om = 1.37
    srt = co.collide(co.Method(lat, "srt", [om], force=F), f)
    trt = co.collide(co.Method(lat, "trt", [om, om], force=F), f)
    mrt = co.collide(co.Method(lat, "mrt", [om] * 6, force=F), f)
    assert np.abs(srt - trt).max() < 1e-15
    assert np.abs(srt - mrt).max() < 1e-14


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("force", [None, (2e-3, -1e-3, 5e-4)])
def test_trt_equals_mrt_with_parity_rates(name, force):
    """Even moments (orders 0, 2, 4, 6) with omega_e, odd (1, 3, 5) with omega_o."""
    lat = lattice.get(name)
    F = None if force is None else force[: lat.d]
    f = _rand_f(lat, seed=5)
    we, wo = 1.8, co.trt_odd_rate(1.8, 3 / 16)
    assert abs(wo - 8 / 31) < 1e-15
    trt = co.collide(co.Method(lat, "trt", [we, wo], force=F), f)
    mrt = co.collide(co.Method(lat, "mrt", [we, we, wo, we, wo, we], force=F), f)
    assert np.abs(trt - mrt).max() < 1e-14


@pytest.mark.parametrize("name", NAMES)
def test_guo_momentum_input(name):
    lat = lattice.get(name)
    F = np.array([3e-3, -2e-3, 1e-3][: lat.d])
    f = _rand_f(lat, seed=3)
    for m in _methods(lat, force=F):
        fs = co.collide(m, f)
        assert np.abs(fs.sum(0) - f.sum(0)).max() < 1e-14
        dj = co.momentum(lat, fs) - co.momentum(lat, f)
        assert np.abs(dj - F[:, None]).max() < 1e-15, m.op
