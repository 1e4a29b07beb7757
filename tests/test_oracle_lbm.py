"""Pins for oracle.lbm: pull streaming direction convention, bounce-back,
UBB momentum input (closed form), inlet/outlet preserving a uniform flow,
out-of-domain = wall, mass conservation in a closed box, link mask against a
brute-force loop."""
import itertools

import numpy as np
import pytest

from oracle import collision as co
from oracle import lattice, lbm
from paper_2001_11806_gb300 import inputs

NAMES = ["D2Q9", "D3Q19", "D3Q27"]


def _shape(lat, n=(5, 4, 3)):
    return n if lat.d == 3 else (n[0], n[1], 1)


@pytest.mark.parametrize("name", NAMES)
def test_pull_streaming_matches_roll(name):
    lat = lattice.get(name)
    shp = _shape(lat)
    s = lbm.Sim(co.Method(lat, "srt", [0.0]), shp)  # omega = 0: collision is the identity
    P = inputs.random_pdfs(lat.w, shp[::-1], seed=3)
    s.P = P.copy()
    s.step(1)
    for q in range(lat.q):
        c = list(lat.c[q]) + [0] * (3 - lat.d)
        ref = np.roll(P[q], shift=(c[2], c[1], c[0]), axis=(0, 1, 2))  # value moves along +c
        assert np.array_equal(s.P[q], ref), q


@pytest.mark.parametrize("name", NAMES)
def test_bounce_back_reverses_links(name):
    lat = lattice.get(name)
    shp = _shape(lat, (4, 5, 3))
    flags = np.zeros(shp[::-1], np.uint8)
    flags[:, 0, :] = lbm.NOSLIP
    s = lbm.Sim(co.Method(lat, "srt", [0.0]), shp, flags=flags)
    P = inputs.random_pdfs(lat.w, shp[::-1], seed=4)
    s.P = P.copy()
    s.step(1)
    for q in range(lat.q):
        if lat.c[q][1] == 1:  # source below is the wall row y = 0 for cells at y = 1
            assert np.array_equal(s.P[q][:, 1, :], P[lat.opp[q]][:, 1, :]), q


def test_ubb_momentum_closed_form():
    lat = lattice.d2q9()
    U = 0.05
    flags = np.zeros((1, 6, 4), np.uint8)
    flags[:, 5, :] = lbm.INLET  # moving lid at the top row
    s = lbm.Sim(co.Method(lat, "srt", [0.0]), (4, 6, 1), flags=flags, u_wall=(U, 0, 0))
    s.init_equilibrium(np.ones((1, 6, 4)), np.zeros((2, 1, 6, 4)))
    f = s.populations()
    jx = (lat.c[:, 0, None, None, None] * f).sum(0)
    # incoming links (c_y = -1): 2 w_q (c_q.u_w)/cs2 -> +U/6 and -U/6 on x-momentum +1 and -1
    assert np.allclose(jx[0, 4, :], U / 3, rtol=0, atol=1e-16)
    assert np.allclose(jx[0, 1:4, :], 0.0, atol=1e-17)


@pytest.mark.parametrize("name", NAMES)
def test_inlet_outlet_keep_uniform_flow(name):
    lat = lattice.get(name)
    U = np.array([0.04, 0.0, 0.0])[: lat.d]
    shp = _shape(lat, (8, 4, 3))
    flags = np.zeros(shp[::-1], np.uint8)
    flags[..., 0] = lbm.INLET
    flags[..., -1] = lbm.OUTLET
    s = lbm.Sim(co.Method(lat, "srt", [1.3]), shp, periodic=(False, True, True), flags=flags,
                u_wall=(0.04, 0, 0))
    s.init_equilibrium(np.ones(shp[::-1]), np.broadcast_to(U.reshape((-1, 1, 1, 1)), (lat.d,) + shp[::-1]))
    s.step(5)
    rho, u = s.macroscopic()
    fl = s.fluid
    assert np.abs(rho[fl] - 1).max() < 1e-15
    assert np.abs(u[0][fl] - 0.04).max() < 1e-15


@pytest.mark.parametrize("name", NAMES)
def test_out_of_domain_is_noslip(name):
    lat = lattice.get(name)
    shp = _shape(lat, (5, 4, 3))
    m = co.Method(lat, "trt", [1.2, 0.9])
    rho, u = inputs.random_fields(shp[::-1], lat.d, seed=2)
    a = lbm.Sim(m, shp, periodic=(False, False, lat.d == 2))
    a.init_equilibrium(rho, u)
    a.step(3)
    pad = (shp[0] + 2, shp[1] + 2, shp[2] + 2 if lat.d == 3 else 1)
    flags = np.full(pad[::-1], lbm.NOSLIP, np.uint8)
    inner = (slice(1, -1) if lat.d == 3 else slice(None), slice(1, -1), slice(1, -1))
    flags[inner] = 0
    rp = np.ones(pad[::-1])
    up = np.zeros((lat.d,) + pad[::-1])
    rp[inner] = rho
    for k in range(lat.d):
        up[k][inner] = u[k]
    b = lbm.Sim(m, pad, periodic=(True, True, True), flags=flags)
    b.init_equilibrium(rp, up)
    b.step(3)
    assert np.abs(b.populations()[(slice(None),) + inner] - a.populations()).max() < 1e-16


@pytest.mark.parametrize("name", NAMES)
def test_closed_box_mass_conservation(name):
    lat = lattice.get(name)
    shp = _shape(lat, (6, 5, 4))
    flags = inputs.channel_flags(*shp, margin=1, rmin=1, rmax=1, porosity=0.9) if lat.d == 3 else None
    if flags is not None:
        flags[flags != 0] = lbm.NOSLIP
    s = lbm.Sim(co.Method(lat, "mrt", [1.7, 1.2, 1.1, 1.3, 1.0, 1.0]), shp,
                periodic=(False, False, False), flags=flags)
    rho, u = inputs.random_fields(shp[::-1], lat.d, seed=5)
    s.init_equilibrium(rho, u)
    m0 = s.reduce()[0]
    s.step(40)
    assert abs(s.reduce()[0] / m0 - 1) < 1e-13


def test_link_mask_brute_force():
    lat = lattice.d3q19()
    shp = (6, 5, 4)
    flags = np.zeros(shp[::-1], np.uint8)
    flags[1, 2, 3] = lbm.NOSLIP
    flags[:, 0, :] = lbm.INLET
    flags[2, 3, 0] = lbm.OUTLET
    s = lbm.Sim(co.Method(lat, "srt", [1.0]), shp, periodic=(True, False, True), flags=flags)
    mask = s.link_mask()
    for z, y, x in itertools.product(range(4), range(5), range(6)):
        ref = 0
        if flags[z, y, x] != 0:
            ref = 1 << 31
        else:
            for q, c in enumerate(lat.c_list):
                sx, sy, sz = (x - c[0]) % 6, y - c[1], (z - c[2]) % 4
                if not (0 <= sy < 5) or flags[sz, sy, sx] != 0:
                    ref |= 1 << q
                    if 0 <= sy < 5 and flags[sz, sy, sx] in (lbm.INLET, lbm.OUTLET):
                        ref |= 1 << 30
        assert mask[z, y, x] == ref, (z, y, x)


def test_link_kind_of_every_flag_value():
    # the documented rule for a uint8 flag: 0 is fluid; the GHOST bit (8)
    # without bits 0-2 is a ghost source, which streams like fluid; otherwise
    # NOSLIP if bit 0 is set or no known bit is set, else INLET if bit 1,
    # else OUTLET
    for v in range(256):
        if v == 0 or (v & 8 and not v & 7):
            want = lbm.FLUID
        elif v & 1 or not v & 6:
            want = lbm.NOSLIP
        elif v & 2:
            want = lbm.INLET
        else:
            want = lbm.OUTLET
        assert lbm.link_kind(np.uint8(v)) == want, v


@pytest.mark.parametrize("name", NAMES)
def test_ubb_at_rest_is_bounce_back(name):
    # the UBB listing with wall velocity 0 adds nothing: an inlet at rest
    # must give exactly the populations of a no-slip wall
    lat = lattice.get(name)
    shp = _shape(lat, (6, 5, 3))
    P = inputs.random_pdfs(lat.w, shp[::-1], seed=12)
    out = []
    for kind in (lbm.INLET, lbm.NOSLIP):
        flags = np.zeros(shp[::-1], np.uint8)
        flags[:, 0, :] = kind
        flags[:, -1, :] = lbm.NOSLIP
        s = lbm.Sim(co.Method(lat, "trt", [1.3, 0.9]), shp, periodic=(True, False, True), flags=flags,
                    u_wall=(0.0, 0.0, 0.0))
        s.P = P.copy()
        s.step(3)
        out.append(s.populations())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("periodic_x", [True, False])
def test_ghost_blocks_reproduce_the_undivided_domain(name, periodic_x):
    """A block partition in x (Sec. IV-D, the framework's block-structured
    domain): each block carries one ghost layer per x face, flagged GHOST
    where the neighbouring block's cell is fluid, and after every step the
    ghost cells take the post-collision populations of the cells they stand
    for.  Then every block's interior equals the undivided domain exactly;
    a plausible mistake (ghosts treated as walls, a ghost not refreshed, a
    block boundary shifted by one) breaks it."""
    lat = lattice.get(name)
    shp = _shape(lat, (12, 5, 4))
    nx = shp[0]
    flags = np.zeros(shp[::-1], np.uint8)
    r = inputs.uniform(17, flags.size).reshape(flags.shape)
    flags[r < 0.12] = lbm.NOSLIP
    if not periodic_x:
        flags[..., 0] = lbm.INLET
        flags[..., -1] = lbm.OUTLET
    per = (periodic_x, True, True)
    m = co.Method(lat, "trt", [1.6, 0.9])
    whole = lbm.Sim(m, shp, periodic=per, flags=flags, u_wall=(0.03, 0.0, 0.0))
    P = inputs.random_pdfs(lat.w, shp[::-1], seed=18)
    whole.P = P.copy()
    cuts = [0, 5, nx]
    blocks = []
    for b in range(2):
        x0, x1 = cuts[b], cuts[b + 1]
        xs = [(x - 1) for x in range(x0, x1 + 2)]  # global x of local 0 .. nb + 1
        fl = np.zeros(shp[::-1][:-1] + (len(xs),), np.uint8)
        for i, gx in enumerate(xs):
            inside = 0 <= gx < nx
            g = gx % nx
            if 1 <= i <= x1 - x0:
                fl[..., i] = flags[..., g]
            elif not inside and not periodic_x:
                fl[..., i] = lbm.NOSLIP
            else:
                fl[..., i] = np.where(flags[..., g] == 0, lbm.GHOST, flags[..., g])
        s = lbm.Sim(m, (len(xs), shp[1], shp[2]), periodic=(False, True, True), flags=fl, u_wall=(0.03, 0.0, 0.0))
        s.P = P[..., [x % nx for x in xs]].copy()
        blocks.append((s, xs, fl))

    def refresh():
        for s, xs, fl in blocks:
            for i in (0, len(xs) - 1):
                gx = xs[i]
                owner = [o for o in blocks if o[1][1] <= gx % nx <= o[1][-2]]
                if (0 <= gx < nx or periodic_x) and owner:
                    o, oxs, _ = owner[0]
                    s.P[..., i] = o.P[..., oxs.index(gx % nx)]
    refresh()
    for _ in range(4):
        whole.step(1)
        for s, _, _ in blocks:
            s.step(1)
        refresh()
    for s, xs, fl in blocks:
        inner = slice(1, len(xs) - 1)
        assert np.array_equal(s.populations()[..., inner], whole.populations()[..., xs[1]:xs[-2] + 1])
    # the ghost bit in the mask
    s, xs, fl = blocks[0]
    mk = s.link_mask()
    assert np.all(((mk >> 29) & 1).astype(bool) == lbm.is_ghost(fl))
