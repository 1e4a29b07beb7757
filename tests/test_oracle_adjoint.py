"""Pins for oracle.adjoint: per-step dot-product identity against the
forward map's own directional derivative, per-cell collision Jacobian against
central finite differences, and the whole-run gradient (initial velocity and
body force) against central finite differences of the forward oracle."""
import numpy as np
import pytest

from oracle import adjoint as ad
from oracle import collision as co
from oracle import lattice, lbm
from paper_2001_11806_gb300 import inputs

CASES = [("D2Q9", "srt", [1.3]), ("D3Q19", "trt", [1.8, 8 / 31]),
         ("D3Q19", "mrt", [1.6, 1.1, 0.9, 1.3]), ("D3Q27", "cumulant", [1.5, 1.1, 0.8])]


def _sim(name, op, om, force=True):
    lat = lattice.get(name)
    F = None if (op == "cumulant" or not force) else [1e-3, -2e-3, 5e-4][: lat.d]
    shp = (5, 4, 3) if lat.d == 3 else (6, 5, 1)
    flags = np.zeros(shp[::-1], np.uint8)
    flags[:, 0, :] = lbm.NOSLIP
    flags[:, -1, 1:3] = lbm.INLET
    return lbm.Sim(co.Method(lat, op, om, force=F), shp, periodic=(True, False, True), flags=flags,
                   u_wall=(0.02, 0.01, 0.0))


@pytest.mark.parametrize("name,op,om", CASES)
def test_dot_product_identity(name, op, om):
    s = _sim(name, op, om)
    rng = np.random.default_rng(0)
    P = inputs.random_pdfs(s.lat.w, s.shape3, seed=8)
    v = rng.standard_normal(P.shape)
    w = rng.standard_normal(P.shape)
    Jv = s.step_state(P.astype(np.complex128) + 1j * 1e-30 * v).imag / 1e-30
    JTw, _ = ad.adjoint_step(s, P, w)
    lhs, rhs = (Jv * w).sum(), (v * JTw).sum()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("name,op,om", CASES)
def test_collision_jacobian_vs_central_differences(name, op, om):
    s = _sim(name, op, om)
    f = inputs.random_pdfs(s.lat.w, (4,), seed=9)
    lam = np.random.default_rng(1).standard_normal(f.shape)
    mu = ad.collide_vjp(s.m, f, lam)
    h = 1e-6
    for j in range(s.lat.q):
        e = np.zeros_like(f)
        e[j] = h
        col = (co.collide(s.m, f + e) - co.collide(s.m, f - e)) / (2 * h)
        assert np.abs((col * lam).sum(0) - mu[j]).max() < 1e-8


@pytest.mark.parametrize("name,op,om", CASES)
def test_gradient_vs_finite_differences(name, op, om):
    s = _sim(name, op, om)
    rho0, u0 = inputs.random_fields(s.shape3, s.lat.d, seed=3)
    box = (1, 4, 1, 3, 0, 2)
    T = 3
    L, gu, gF = ad.gradient(s, rho0, u0, T, box)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(u0.shape)
    e = 1e-6
    fd = (ad.forward_loss(s, rho0, u0 + e * v, T, box) - ad.forward_loss(s, rho0, u0 - e * v, T, box)) / (2 * e)
    assert abs((gu * v).sum() - fd) <= 1e-7 * abs(fd)
    if s.m.force is not None:
        F0 = np.asarray(s.m.force)
        dv = rng.standard_normal(F0.shape)

        def loss_at(F):
            s2 = lbm.Sim(s.m.with_force(F), (s.nx, s.ny, s.nz), s.periodic, s.flags, (0.02, 0.01, 0.0))
            return ad.forward_loss(s2, rho0, u0, T, box)
        fdF = (loss_at(F0 + e * dv) - loss_at(F0 - e * dv)) / (2 * e)
        assert abs((gF * dv).sum() - fdF) <= 1e-7 * abs(fdF)
