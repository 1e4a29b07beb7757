"""Pins of the oracle's outputs on states whose moments are known in closed
form: the conservation sums (mass, momentum rho_0 u, kinetic energy
(1/2) sum rho |u|^2 over fluid cells), the velocity of Eq. density with the
Guo half force, and the kinetic-energy box loss of the adjoint.

A uniform equilibrium f^eq(rho, u) is unchanged by streaming and collision,
so its populations and moments are those of the state itself; with walls the
sums run over the fluid cells only."""
import numpy as np
import pytest

from oracle import adjoint as ad
from oracle import collision as co
from oracle import lattice
from oracle import lbm

NAMES = ["D2Q9", "D3Q19", "D3Q27"]


def _uniform_sim(name, incompressible, force=None, walls=False, rho=1.04, u=(0.03, -0.02, 0.01)):
    lat = lattice.get(name)
    shp = (6, 5, 4) if lat.d == 3 else (6, 5, 1)
    flags = None
    if walls:
        flags = np.zeros(shp[::-1], np.uint8)
        flags[:, 0, :] = lbm.NOSLIP
        flags[:, -1, :] = lbm.NOSLIP
    m = co.Method(lat, "srt", [1.2], incompressible=incompressible, force=force)
    s = lbm.Sim(m, shp, periodic=(True, not walls, True), flags=flags)
    uu = np.array(u[: lat.d])
    s.init_equilibrium(np.full(shp[::-1], rho), np.broadcast_to(uu.reshape((-1,) + (1,) * 3), (lat.d,) + shp[::-1]))
    return s, lat, rho, uu


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("incompressible", [False, True])
@pytest.mark.parametrize("walls", [False, True])
def test_reduce_closed_form(name, incompressible, walls):
    # with walls the fluid is at rest, which bounce-back leaves unchanged
    u_init = (0.0, 0.0, 0.0) if walls else (0.03, -0.02, 0.01)
    s, lat, rho, u = _uniform_sim(name, incompressible, walls=walls, u=u_init)
    n = int(s.fluid.sum())
    got = s.reduce()
    rho0 = 1.0 if incompressible else rho
    want = [n * rho] + [n * rho0 * ua for ua in u] + [0.0] * (3 - lat.d) + [0.5 * n * rho * float(u @ u)]
    assert np.allclose(got, want, rtol=1e-14, atol=1e-15), (got, want)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("incompressible", [False, True])
def test_macroscopic_adds_half_force(name, incompressible):
    lat = lattice.get(name)
    F = np.array([2e-3, -1e-3, 5e-4][: lat.d])
    s, lat, rho, u = _uniform_sim(name, incompressible, force=F)
    # the populations right after initialisation are f^eq(rho, u) itself
    r, v = s.macroscopic()
    rho0 = 1.0 if incompressible else rho
    assert np.abs(r - rho).max() < 1e-15
    for a in range(lat.d):
        assert np.abs(v[a] - (u[a] + F[a] / (2 * rho0))).max() < 1e-15


@pytest.mark.parametrize("name", NAMES)
def test_ke_box_loss_closed_form(name):
    s, lat, rho, u = _uniform_sim(name, False)
    nz = s.shape3[0]
    box = (1, 4, 1, 3, 0, nz)
    n_box = 3 * 2 * nz
    L = ad.ke_box_loss(s, s.P, box)
    assert abs(L - 0.5 * n_box * rho * float(u @ u)) <= 1e-14 * L


@pytest.mark.parametrize("name", NAMES)
def test_ke_box_loss_counts_only_the_box(name):
    # fluid at rest in and around the box, moving two or more cells away from
    # it: one pull cannot carry momentum into the box, so the loss is exactly 0
    lat = lattice.get(name)
    shp = (12, 8, 3) if lat.d == 3 else (12, 8, 1)
    s = lbm.Sim(co.Method(lat, "srt", [1.2]), shp)
    u0 = np.zeros((lat.d,) + shp[::-1])
    u0[0][..., 6:11] = 0.04
    s.init_equilibrium(np.ones(shp[::-1]), u0)
    assert ad.ke_box_loss(s, s.P, (1, 4, 1, 3, 0, shp[2])) == 0.0
    assert ad.ke_box_loss(s, s.P, (7, 10, 1, 3, 0, shp[2])) > 0.0
