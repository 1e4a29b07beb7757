"""GPU parity against the FP64 oracle, through the C ABI.

Tolerances (relative L2 over fluid cells): populations are compared as
||f_gpu - f_ref|| / ||f_ref - w||, densities as rho - 1, velocities per
component.  FP64 storage: 1e-12.  FP32 and FP32-shifted storage: 1e-5.
FP16-shifted storage keeps h = f - w in binary16 (11-bit significand, unit
roundoff 2^-11 = 4.9e-4 of |h| per stored value), so it is held to 5e-3 over
at most five steps, and element-wise to 3 * 2^-11 max|h_ref| (derivation at
U16 below).  Boxes are 150 cells long in x (two 128-thread tiles and a
ragged tail of 22) so every kernel runs full and partial tiles."""
import numpy as np
import pytest
import torch

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs
from paper_2001_11806_gb300.sim import Sim

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32s": 1e-5, "f16s": 5e-3}
# Element-wise bound for FP16-shifted storage: every step rounds each stored
# h = f - w once to binary16 (error <= U16 |h|, U16 = 2^-11); streaming moves
# those errors unchanged and a collision with rates in (0, 2) does not
# amplify them (a contraction in the w-weighted norm), so a value's error
# stays at the rounding of the largest values that feed it.  Bound:
# |f_gpu - f_ref| <= 3 U16 max|h_ref| for every population of every fluid
# cell.  A rounding model of the oracle stays below 1.2 U16 max|h| over five
# steps (tests/test_f16_bound_cpu.py); a wrong UBB or outlet value is off by
# 6 w_q |c.u| (8e-3 for a D3Q19 edge at u = 0.05), about 80 times the bound.
U16 = 2.0 ** -11


def assert_f16_elementwise(fg, fr, w):
    """fg, fr: [q][cells] GPU and oracle populations of the fluid cells."""
    h = np.abs(fr - np.asarray(w)[:, None])
    bound = 3.0 * U16 * h.max()
    d = np.abs(fg - fr)
    assert d.max() <= bound, (d.max(), bound, np.unravel_index(d.argmax(), d.shape))
OMEGAS = {"srt": [1.37], "trt": [1.8, 8 / 31], "mrt": [1.7, 1.1, 0.9, 1.3, 1.2, 1.05], "cumulant": [1.95, 1.0, 1.0],
          "kbc": [1.9, 1.3]}


def _shape(stencil, big=True):
    if stencil == "D2Q9":
        return (150, 7, 1) if big else (9, 7, 1)
    return (150, 5, 4) if big else (7, 6, 5)


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


def _oracle_method(stencil, collision, force=None, incompressible=False):
    lat = olat.get(stencil)
    om = OMEGAS[collision]
    if collision == "mrt":
        om = om[:6] if stencil == "D3Q27" else om[:4]
    return oco.Method(lat, collision, om, incompressible=incompressible, force=force)


def run_pair(stencil, collision, storage, pattern, shape, steps, periodic=(True, True, True), flags=None,
             force=None, u_wall=(0.0, 0.0, 0.0), incompressible=False, seed=5):
    lat = olat.get(stencil)
    d = lat.d
    F3 = list(force) + [0.0] * (3 - len(force)) if force is not None else [0.0, 0.0, 0.0]
    sim = Sim(stencil, collision, storage, pattern, shape, periodic=periodic, omega=OMEGAS[collision],
              incompressible=incompressible, u_wall=u_wall, force=F3, flags=flags)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=seed)
    sim.set_state(P.reshape(lat.q, -1))
    sim.step(steps)
    f_gpu = sim.populations().cpu().numpy()
    rho_g, u_g = (t.cpu().numpy() for t in sim.macroscopic(True))
    red_g = sim.reduce()
    ref = olbm.Sim(_oracle_method(stencil, collision, None if force is None else force[:d], incompressible),
                   shape, periodic=periodic, flags=flags, u_wall=u_wall)
    ref.P = P.copy()
    ref.step(steps)
    f_ref = ref.populations().reshape(lat.q, -1)
    rho_r, u_r = ref.macroscopic()
    fl = ref.fluid.reshape(-1)
    return dict(sim=sim, ref=ref, fluid=fl, lat=lat,
                f=(f_gpu[:, fl], f_ref[:, fl]), rho=(rho_g[fl], rho_r.reshape(-1)[fl]),
                u=(u_g[:, fl], u_r.reshape(d, -1)[:, fl]), red=(red_g, ref.reduce()))


def _errs(r):
    (fg, fr), (rg, rr), (ug, ur) = r["f"], r["rho"], r["u"]
    w = r["lat"].w[:, None]
    ef = np.linalg.norm(fg - fr) / np.linalg.norm(fr - w)
    er = np.linalg.norm(rg - rr) / np.linalg.norm(rr - 1.0)
    eu = max(np.linalg.norm(ug[a] - ur[a]) / np.linalg.norm(ur[a]) for a in range(ur.shape[0]))
    return ef, er, eu


COMBOS = [(s, c) for s in ["D2Q9", "D3Q19", "D3Q27"] for c in ["srt", "trt", "mrt", "kbc"]] + [("D3Q27", "cumulant")]


@pytest.mark.parametrize("stencil,collision", COMBOS)
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
@pytest.mark.parametrize("steps", [1, 4])
def test_periodic_parity(stencil, collision, storage, pattern, steps):
    r = run_pair(stencil, collision, storage, pattern, _shape(stencil), steps)
    ef, er, eu = _errs(r)
    tol = TOL[storage]
    assert ef < tol and er < tol and eu < tol, (ef, er, eu)


@pytest.mark.parametrize("stencil,collision", COMBOS)
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "f32s"])
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
@pytest.mark.parametrize("steps", [3, 4])
def test_channel_parity(stencil, collision, storage, pattern, steps):
    shape = _shape(stencil)
    fl = _flags(shape)
    per = (False, False, True)
    r = run_pair(stencil, collision, storage, pattern, shape, steps, periodic=per, flags=fl,
                 u_wall=(0.05, 0.01, 0.0))
    ef, er, eu = _errs(r)
    tol = TOL[storage]
    assert ef < tol and er < tol and eu < tol, (ef, er, eu)
    if storage == "f16s":
        assert_f16_elementwise(*r["f"], r["lat"].w)
    mask = r["sim"].link_mask().cpu().numpy().view(np.uint32)
    assert np.array_equal(mask, r["ref"].link_mask().reshape(-1))


@pytest.mark.parametrize("stencil,collision", [c for c in COMBOS if c[1] not in ("cumulant", "kbc")])
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
@pytest.mark.parametrize("incompressible", [False, True])
def test_force_parity(stencil, collision, pattern, incompressible):
    shape = _shape(stencil)
    fl = _flags(shape)
    r = run_pair(stencil, collision, "f64", pattern, shape, 3, periodic=(False, False, True), flags=fl,
                 force=[2e-4, -1e-4, 5e-5], u_wall=(0.03, 0.0, 0.0), incompressible=incompressible)
    ef, er, eu = _errs(r)
    assert ef < 1e-12 and er < 1e-12 and eu < 1e-12, (ef, er, eu)


@pytest.mark.parametrize("stencil,collision", COMBOS)
def test_reduction_parity(stencil, collision):
    shape = _shape(stencil)
    r = run_pair(stencil, collision, "f64", "aa", shape, 3, periodic=(False, False, True), flags=_flags(shape),
                 u_wall=(0.05, 0.0, 0.0))
    g, o = r["red"]
    assert abs(g[0] / o[0] - 1) < 1e-13
    for a in range(1, 5):
        assert abs(g[a] - o[a]) <= 1e-12 * max(abs(o[a]), 1.0), (a, g[a], o[a])


@pytest.mark.parametrize("stencil,collision", COMBOS)
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_aa_matches_two_grid_bitwise(stencil, collision, storage):
    """Same arithmetic in all three patterns (pull, AA, esoteric twist):
    identical bits after an even number of steps for FP64 and FP32 storage.
    No-slip walls only: UBB and outlet values are rounded to the storage type
    when written (AA, esoteric twist) but not when read (pull).  The patterns
    are separate kernel instantiations, so the compiler may round an FP32
    intermediate differently; with FP16 storage that can flip the last
    binary16 bit of a value, so FP16 is held to two binary16 ulps of
    h = f - w."""
    shape = _shape(stencil)
    fl = _flags(shape)
    fl[fl != 0] = olbm.NOSLIP
    lat = olat.get(stencil)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=9).reshape(lat.q, -1)
    out = []
    for pattern in ["pull", "aa", "eso"]:
        sim = Sim(stencil, collision, storage, pattern, shape, periodic=(False, False, True),
                  omega=OMEGAS[collision], u_wall=(0.05, 0.0, 0.0), flags=fl)
        sim.set_state(P)
        sim.step(6)
        out.append(sim.populations().cpu().numpy())
    fluid = fl.reshape(-1) == 0
    a = out[0][:, fluid]
    for other in out[1:]:
        b = other[:, fluid]
        if storage != "f16s":
            assert np.array_equal(a, b)
        else:
            h = np.abs(a - lat.w[:, None])
            diff = np.abs(a - b)
            frac = np.mean(diff > 0)
            print(f"f16s vs pull: {frac:.2e} of values differ, max {diff.max():.2e}")
            assert np.all(diff <= 2.0 ** -10 * h + 1e-7)


def test_degenerate_domains():
    lat = olat.d3q19()
    # one periodic cell: every neighbour is the cell itself
    for pattern in ["pull", "aa", "eso"]:
        r = run_pair("D3Q19", "trt", "f64", pattern, (1, 1, 1), 3)
        assert np.abs(r["f"][0] - r["f"][1]).max() < 1e-14
    # a box that is entirely solid: nothing moves, reductions are zero
    fl = np.full((3, 4, 5), olbm.NOSLIP, np.uint8)
    sim = Sim("D3Q19", "srt", "f32", "aa", (5, 4, 3), omega=[1.2], flags=fl)
    sim.set_state(inputs.random_pdfs(lat.w, (3, 4, 5)).reshape(19, -1))
    sim.step(2)
    assert np.all(sim.reduce() == 0.0)
    assert np.all(np.isnan(sim.populations().cpu().numpy()))
    # zero steps is a no-op and an isolated fluid cell only bounces back
    fl = np.full((3, 3, 3), olbm.NOSLIP, np.uint8)
    fl[1, 1, 1] = 0
    for pattern in ["pull", "aa", "eso"]:
        r = run_pair("D3Q19", "mrt", "f64", pattern, (3, 3, 3), 0, flags=fl)
        assert np.abs(r["f"][0] - r["f"][1]).max() < 1e-15
        r = run_pair("D3Q19", "mrt", "f64", pattern, (3, 3, 3), 5, flags=fl)
        assert np.abs(r["f"][0] - r["f"][1]).max() < 1e-14


@pytest.mark.parametrize("pattern", ["aa", "eso"])
def test_checkpoint_restore_roundtrip(pattern):
    shape = _shape("D3Q19", big=False)
    lat = olat.d3q19()
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=2).reshape(19, -1)
    sim = Sim("D3Q19", "trt", "f32", pattern, shape, omega=OMEGAS["trt"])
    sim.set_state(P)
    sim.step(3)
    raw, t = sim.get_pdfs()
    sim.step(4)
    after = sim.populations().cpu().numpy()
    sim.set_pdfs(raw, t)
    assert sim.t == 3
    sim.step(4)
    assert np.array_equal(sim.populations().cpu().numpy(), after)


def test_tgv2d_config1_full_parity_and_decay():
    """D2Q9 SRT FP64, 64^2, TGV u0 = 0.01, omega = 1.6, 200 steps: full-field
    parity with the oracle and the viscous decay rate of exp(-2 nu k^2 t)."""
    n, om = 64, 1.6
    rho0, u0 = inputs.tgv2d(n, 0.01)
    sim = Sim("D2Q9", "srt", "f64", "pull", (n, n, 1), omega=[om])
    sim.init_equilibrium(rho0.reshape(-1), u0.reshape(2, -1))
    ref = olbm.Sim(oco.Method(olat.d2q9(), "srt", [om]), (n, n, 1))
    ref.init_equilibrium(rho0, u0)
    ts, amps = [], []
    w = olat.d2q9().w[:, None]
    for t in range(0, 201, 10):
        if t >= 20:
            _, u = sim.macroscopic(True)
            ts.append(t)
            amps.append(float(torch.linalg.norm(u)))
        if t in (100, 200):
            ref.step(100)
            f_g = sim.populations().cpu().numpy()
            f_r = ref.populations().reshape(9, -1)
            err = np.linalg.norm(f_g - f_r) / np.linalg.norm(f_r - w)
            # FP64 rounding (FMA contraction, summation order) differs from
            # numpy by ~1e-14 of ||f - w|| per step for this low-amplitude
            # vortex (||f - w|| is ~3 % of ||f||) and adds up linearly, so the
            # bound is 3e-14 per step: 3e-12 at t = 100, 6e-12 at t = 200
            assert err < 3e-14 * t, (t, err)
        if t < 200:
            sim.step(10)
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    expect = 2 * (1 / om - 0.5) / 3 * (2 * np.pi / n) ** 2
    assert abs(rate / expect - 1) < 1e-2


def test_poiseuille_exact_on_gpu():
    """TRT with Lambda = 3/16, halfway bounce-back and Guo force gives the
    exact parabola (FP64 storage)."""
    H, F, oe = 8, 1e-5, 1.0
    fl = np.zeros((1, H + 2, 4), np.uint8)
    fl[:, 0, :] = olbm.NOSLIP
    fl[:, H + 1, :] = olbm.NOSLIP
    for pattern in ["pull", "aa"]:
        sim = Sim("D2Q9", "trt", "f64", pattern, (4, H + 2, 1), periodic=(True, False, True), omega=[oe],
                  trt_magic=3 / 16, force=[F, 0, 0], flags=fl)
        sim.init_equilibrium(np.ones(4 * (H + 2)), np.zeros((2, 4 * (H + 2))))
        sim.step(3000)
        u = sim.macroscopic(True)[1].cpu().numpy()[0].reshape(H + 2, 4)
        nu = (1 / oe - 0.5) / 3
        y = np.arange(1, H + 1)
        exact = F / (2 * nu) * (y - 0.5) * (H + 0.5 - y)
        assert np.abs(u[1:H + 1, :] - exact[:, None]).max() / exact.max() < 1e-10


@pytest.mark.parametrize("stencil,collision", [("D2Q9", "trt"), ("D3Q19", "trt"), ("D3Q19", "mrt"),
                                               ("D3Q27", "srt"), ("D3Q27", "cumulant"), ("D3Q19", "kbc")])
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
@pytest.mark.parametrize("nx", [534, 151])
def test_f16_two_cell_kernel_parity(stencil, collision, pattern, nx):
    """Periodic FP16-shifted runs with even nx use the two-cells-per-thread
    kernel (534 = 267 cell pairs: two full 128-thread tiles and a ragged
    tail); odd nx falls back to one cell per thread."""
    shape = (nx, 3, 1) if stencil == "D2Q9" else (nx, 3, 2)
    for steps in (3, 4):
        r = run_pair(stencil, collision, "f16s", pattern, shape, steps)
        ef, er, eu = _errs(r)
        assert ef < 5e-3 and er < 5e-3 and eu < 5e-3, (steps, ef, er, eu)
        assert_f16_elementwise(*r["f"], r["lat"].w)


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("collision,magic", [("srt", None), ("trt", None), ("trt", 3 / 16)])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
def test_smagorinsky_parity(stencil, collision, magic, storage, pattern):
    """Per-cell Smagorinsky rate (C_S = 0.17) on random populations with walls,
    an inlet, an outlet and a body force."""
    lat = olat.get(stencil)
    shape = _shape(stencil)
    fl = _flags(shape)
    om = [1.7] if collision == "srt" else [1.7, 0.9]
    force = [2e-4, -1e-4, 5e-5]
    sim = Sim(stencil, collision, storage, pattern, shape, periodic=(False, False, True), omega=om,
              trt_magic=magic, u_wall=(0.05, 0.0, 0.0), force=force, flags=fl, smagorinsky_cs=0.17)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=12)
    sim.set_state(P.reshape(lat.q, -1))
    sim.step(3)
    m = oco.Method(lat, collision, om, force=force[: lat.d], cs=0.17, magic=magic)
    ref = olbm.Sim(m, shape, periodic=(False, False, True), flags=fl, u_wall=(0.05, 0.0, 0.0))
    ref.P = P.copy()
    ref.step(3)
    fluid = fl.reshape(-1) == 0
    fg = sim.populations().cpu().numpy()[:, fluid]
    fr = ref.populations().reshape(lat.q, -1)[:, fluid]
    err = np.linalg.norm(fg - fr) / np.linalg.norm(fr - lat.w[:, None])
    assert err < TOL[storage], err
    if storage == "f16s":
        assert_f16_elementwise(fg, fr, lat.w)


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("pattern", ["aa", "eso"])
def test_kbc_incompressible_and_two_rate_form(stencil, storage, pattern):
    """KBC with the incompressible equilibrium, and with omega_b = omega_s
    (the paper's two-rate form), walls and a moving inlet."""
    lat = olat.get(stencil)
    shape = _shape(stencil)
    fl = _flags(shape)
    for om, inc in (([1.95, 1.95], False), ([1.6, 0.7], True)):
        sim = Sim(stencil, "kbc", storage, pattern, shape, periodic=(False, False, True), omega=om,
                  incompressible=inc, u_wall=(0.05, 0.0, 0.0), flags=fl)
        P = inputs.random_pdfs(lat.w, shape[::-1], amp=0.05, seed=31)
        sim.set_state(P.reshape(lat.q, -1))
        sim.step(5)
        ref = olbm.Sim(oco.Method(lat, "kbc", om, incompressible=inc), shape, periodic=(False, False, True), flags=fl,
                       u_wall=(0.05, 0.0, 0.0))
        ref.P = P.copy()
        ref.step(5)
        fluid = fl.reshape(-1) == 0
        fg = sim.populations().cpu().numpy()[:, fluid]
        fr = ref.populations().reshape(lat.q, -1)[:, fluid]
        err = np.linalg.norm(fg - fr) / np.linalg.norm(fr - lat.w[:, None])
        assert err < TOL[storage], (om, inc, err)


def test_kbc_unsupported_combinations():
    from paper_2001_11806_gb300 import LbmError
    with pytest.raises(LbmError):
        Sim("D3Q19", "kbc", "f32", "pull", (8, 8, 8), omega=[1.9, 1.0], force=(1e-4, 0.0, 0.0))
    with pytest.raises(LbmError):
        Sim("D3Q19", "kbc", "f32", "pull", (8, 8, 8), omega=[1.9, 1.0], smagorinsky_cs=0.1)


def test_esotwist_refuses_fluid_last_layer():
    """The esoteric twist wraps its locations on every axis, so along a
    non-periodic axis the last layer must be non-fluid (LBM_E_UNSUPPORTED
    otherwise); the first layer may be fluid."""
    from paper_2001_11806_gb300 import LbmError
    shape = (8, 6, 5)
    fl = np.zeros(shape[::-1], np.uint8)
    fl[:, -1, :] = olbm.NOSLIP
    Sim("D3Q19", "trt", "f32", "eso", shape, periodic=(True, False, True), omega=[1.5, 1.2], flags=fl).close()
    for per in [(True, False, True), (True, True, False)]:
        bad = np.zeros(shape[::-1], np.uint8)
        if not per[1]:
            bad[:, 0, :] = olbm.NOSLIP
        with pytest.raises(LbmError) as e:
            Sim("D3Q19", "trt", "f32", "eso", shape, periodic=per, omega=[1.5, 1.2], flags=bad)
        assert e.value.status == 2
    with pytest.raises(LbmError) as e:
        Sim("D3Q19", "trt", "f32", "eso", shape, periodic=(False, True, True), omega=[1.5, 1.2])
    assert e.value.status == 2


@pytest.mark.parametrize("stencil,collision", [("D2Q9", "srt"), ("D3Q19", "trt"), ("D3Q27", "cumulant")])
def test_esotwist_channel_with_open_first_layer(stencil, collision):
    """Fluid first layer against a wall-only last layer: the first layer's
    boundary links read the wrapped locations of the solid last layer."""
    lat = olat.get(stencil)
    shape = _shape(stencil)
    fl = np.zeros(shape[::-1], np.uint8)
    fl[:, -1, :] = olbm.NOSLIP
    fl[..., -1] = olbm.OUTLET
    r = run_pair(stencil, collision, "f64", "eso", shape, 5, periodic=(False, False, True), flags=fl,
                 u_wall=(0.05, 0.0, 0.0))
    ef, er, eu = _errs(r)
    assert ef < 1e-12 and er < 1e-12 and eu < 1e-12, (ef, er, eu)


@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
def test_replayed_steps_match_single_steps(pattern):
    """Small domains replay 32-step CUDA graphs inside lbm_step(n); the bits
    must equal n single steps, from either pull buffer or AA parity, and a
    force change must reach the replayed steps."""
    from paper_2001_11806_gb300 import _lib
    import ctypes
    lat = olat.d3q19()
    shape = (12, 10, 8)
    fl = _flags(shape)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=14).reshape(19, -1)
    out = []
    for chunks in ([1] * 75, [3, 70, 2], [75]):
        sim = Sim("D3Q19", "trt", "f32", pattern, shape, periodic=(False, False, True), omega=[1.6, 1.1],
                  u_wall=(0.04, 0.0, 0.0), flags=fl, force=(1e-5, 0.0, 0.0))
        sim.set_state(P)
        for i, k in enumerate(chunks):
            sim.step(k)
        F = (ctypes.c_double * 3)(2e-5, -1e-5, 0.0)
        _lib.check(_lib.lib().lbm_set_force(sim.ctx, F), sim.ctx, "set_force")
        for k in chunks:
            sim.step(k)
        assert sim.t == 150
        out.append(sim.populations().cpu().numpy())
        sim.close()
    fluid = fl.reshape(-1) == 0
    assert np.array_equal(out[0][:, fluid], out[1][:, fluid])
    assert np.array_equal(out[0][:, fluid], out[2][:, fluid])


@pytest.mark.parametrize("storage", ["f64", "f32", "f32s"])
@pytest.mark.parametrize("pattern", ["pull", "aa"])
def test_cumulant_with_higher_order_rate_not_one(storage, pattern):
    """The cumulant sweep skips the pre-collision orders >= 3 when
    omega_higher = 1; this covers the general branch (omega_higher = 1.4,
    bulk rate 1.2) on walls, an inlet and an outlet."""
    lat = olat.d3q27()
    shape = _shape("D3Q27")
    fl = _flags(shape)
    om = [1.8, 1.2, 1.4]
    sim = Sim("D3Q27", "cumulant", storage, pattern, shape, periodic=(False, False, True), omega=om,
              u_wall=(0.05, 0.0, 0.0), flags=fl)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=23)
    sim.set_state(P.reshape(lat.q, -1))
    sim.step(4)
    ref = olbm.Sim(oco.Method(lat, "cumulant", om), shape, periodic=(False, False, True), flags=fl,
                   u_wall=(0.05, 0.0, 0.0))
    ref.P = P.copy()
    ref.step(4)
    fluid = fl.reshape(-1) == 0
    fg = sim.populations().cpu().numpy()[:, fluid]
    fr = ref.populations().reshape(lat.q, -1)[:, fluid]
    err = np.linalg.norm(fg - fr) / np.linalg.norm(fr - lat.w[:, None])
    assert err < TOL[storage], err


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
@pytest.mark.parametrize("force", [False, True])
def test_mrt_with_one_higher_order_rate(stencil, storage, pattern, force):
    """MRT whose moments of order >= 3 share one rate runs the projector form
    of the operator; against the oracle's moment-matrix MRT on walls, an
    inlet, an outlet and (optionally) a body force."""
    lat = olat.get(stencil)
    shape = _shape(stencil)
    fl = _flags(shape)
    om = [1.7, 1.1, 1.3, 1.3, 1.3, 1.3] if stencil == "D3Q27" else [1.7, 1.1, 1.3, 1.3]
    F = [2e-4, -1e-4, 5e-5] if force else [0.0, 0.0, 0.0]
    sim = Sim(stencil, "mrt", storage, pattern, shape, periodic=(False, False, True), omega=om,
              u_wall=(0.05, 0.0, 0.0), flags=fl, force=F)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=27)
    sim.set_state(P.reshape(lat.q, -1))
    sim.step(4)
    ref = olbm.Sim(oco.Method(lat, "mrt", om, force=F[: lat.d] if force else None), shape,
                   periodic=(False, False, True), flags=fl, u_wall=(0.05, 0.0, 0.0))
    ref.P = P.copy()
    ref.step(4)
    fluid = fl.reshape(-1) == 0
    fg = sim.populations().cpu().numpy()[:, fluid]
    fr = ref.populations().reshape(lat.q, -1)[:, fluid]
    err = np.linalg.norm(fg - fr) / np.linalg.norm(fr - lat.w[:, None])
    assert err < TOL[storage], err
    if storage == "f16s":
        assert_f16_elementwise(fg, fr, lat.w)
    # periodic box: the dense sweep kernels
    shape2 = (34, 6, 1) if lat.d == 2 else (34, 6, 5)
    sim = Sim(stencil, "mrt", storage, pattern, shape2, omega=om, force=F)
    P = inputs.random_pdfs(lat.w, shape2[::-1], seed=28)
    sim.set_state(P.reshape(lat.q, -1))
    sim.step(3)
    ref = olbm.Sim(oco.Method(lat, "mrt", om, force=F[: lat.d] if force else None), shape2)
    ref.P = P.copy()
    ref.step(3)
    fg = sim.populations().cpu().numpy()
    fr = ref.populations().reshape(lat.q, -1)
    err = np.linalg.norm(fg - fr) / np.linalg.norm(fr - lat.w[:, None])
    assert err < TOL[storage], err
    if storage == "f16s":
        assert_f16_elementwise(fg, fr, lat.w)


SEPARATE_COMBOS = [("D2Q9", "srt"), ("D2Q9", "mrt"), ("D3Q19", "trt"), ("D3Q19", "mrt"), ("D3Q19", "kbc"),
                   ("D3Q27", "cumulant"), ("D3Q27", "mrt")]


@pytest.mark.parametrize("stencil,collision", SEPARATE_COMBOS)
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "f32s"])
def test_separate_boundary_kernel_parity(stencil, collision, storage):
    """Two-grid pull with a separate boundary kernel before each sweep (the
    sweep then streams every link as fluid): walls, a moving inlet, an
    outlet and obstacles, against the oracle and against the in-sweep
    boundaries."""
    lat = olat.get(stencil)
    shape = _shape(stencil)
    fl = _flags(shape)
    per = (False, False, True)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=33)
    out = {}
    for mode in ["separate", "in_sweep"]:
        sim = Sim(stencil, collision, storage, "pull", shape, periodic=per, omega=OMEGAS[collision],
                  u_wall=(0.05, 0.01, 0.0), flags=fl, boundary=mode)
        sim.set_state(P.reshape(lat.q, -1))
        sim.step(5)
        out[mode] = sim.populations().cpu().numpy()
        sim.close()
    ref = olbm.Sim(_oracle_method(stencil, collision), shape, periodic=per, flags=fl, u_wall=(0.05, 0.01, 0.0))
    ref.P = P.copy()
    ref.step(5)
    fluid = fl.reshape(-1) == 0
    fr = ref.populations().reshape(lat.q, -1)[:, fluid]
    for mode, f in out.items():
        err = np.linalg.norm(f[:, fluid] - fr) / np.linalg.norm(fr - lat.w[:, None])
        assert err < TOL[storage], (mode, err)
        if storage == "f16s":
            assert_f16_elementwise(f[:, fluid], fr, lat.w)
    d = np.linalg.norm(out["separate"][:, fluid] - out["in_sweep"][:, fluid]) / np.linalg.norm(fr - lat.w[:, None])
    assert d < {"f64": 1e-14, "f32": 1e-6, "f32s": 1e-6, "f16s": 2e-3}[storage], d


def test_separate_boundary_kernel_needs_closed_faces():
    """Boundary-link sources must lie inside the box; AA and the adjoint
    refuse the mode."""
    from paper_2001_11806_gb300 import LbmError, _lib
    shape = (8, 6, 5)
    fl = np.zeros(shape[::-1], np.uint8)
    fl[:, 0, :] = olbm.NOSLIP
    fl[:, -1, :] = olbm.NOSLIP
    Sim("D3Q19", "trt", "f32", "pull", shape, periodic=(True, False, True), omega=[1.5, 1.2], flags=fl,
        boundary="separate").close()
    for per in [(True, True, False), (False, False, True)]:
        with pytest.raises(LbmError) as e:
            Sim("D3Q19", "trt", "f32", "pull", shape, periodic=per, omega=[1.5, 1.2], flags=fl, boundary="separate")
        assert e.value.status == 2
    with pytest.raises(LbmError) as e:
        Sim("D3Q19", "trt", "f32", "aa", shape, periodic=(True, False, True), omega=[1.5, 1.2], flags=fl,
            boundary="separate")
    assert e.value.status == 2
    sim = Sim("D3Q19", "trt", "f64", "pull", shape, periodic=(True, False, True), omega=[1.5, 1.2], flags=fl,
              boundary="separate")
    buf = torch.zeros((19, sim.N), dtype=torch.float64, device=sim.device)
    out = torch.zeros_like(buf)
    assert _lib.lib().lbm_adjoint_step(sim.ctx, sim.pdf.data_ptr(), buf.data_ptr(), out.data_ptr(), None) == 2


def test_nonfinite_state_is_reported_and_context_stays_usable():
    """A NaN in the populations reaches the FP64 reduction, which returns
    LBM_E_NONFINITE; the context keeps working after a new state is set."""
    from paper_2001_11806_gb300 import LbmError
    lat = olat.d3q19()
    shape = (12, 6, 5)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=41).reshape(19, -1)
    sim = Sim("D3Q19", "trt", "f32", "aa", shape, omega=[1.6, 1.1])
    bad = P.copy()
    bad[3, 17] = np.nan
    sim.set_state(bad)
    sim.step(2)
    with pytest.raises(LbmError) as e:
        sim.reduce()
    assert e.value.status == 6
    assert b"non-finite" in _lib_last_error(sim)
    sim.set_state(P)
    sim.step(2)
    assert np.all(np.isfinite(sim.reduce()))


def test_injected_allocation_failure_with_flags():
    """A context with a flag field allocates the host offsets of its
    fluid-cell list; an injected failure there returns LBM_E_NOMEM."""
    from paper_2001_11806_gb300 import LbmError, _lib
    fl = _flags(_shape("D3Q19", big=False))
    _lib.lib().lbm_debug_fail_host_allocs(2)  # the context, then the list offsets
    try:
        with pytest.raises(LbmError) as e:
            Sim("D3Q19", "trt", "f32", "pull", _shape("D3Q19", big=False), periodic=(False, False, True),
                omega=[1.6, 1.1], flags=fl)
        assert e.value.status == 4
        with pytest.raises(LbmError) as e:
            Sim("D3Q19", "trt", "f32", "pull", _shape("D3Q19", big=False), periodic=(False, False, True),
                omega=[1.6, 1.1], flags=fl)
        assert e.value.status == 4
    finally:
        _lib.lib().lbm_debug_fail_host_allocs(0)
    Sim("D3Q19", "trt", "f32", "pull", _shape("D3Q19", big=False), periodic=(False, False, True),
        omega=[1.6, 1.1], flags=fl).close()


def _lib_last_error(sim):
    from paper_2001_11806_gb300 import _lib
    return _lib.lib().lbm_last_error(sim.ctx)


@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
@pytest.mark.parametrize("shape", [(150, 5, 4), (149, 5, 3)])
def test_f16_list_sweep_even_and_odd_cell_counts(pattern, shape):
    """The FP16 list sweep (capped main launch) on even and odd cell counts,
    so that the population streams start on 4-byte and on 2-byte
    boundaries; against the oracle, element-wise."""
    fl = _flags(shape)
    r = run_pair("D3Q19", "trt", "f16s", pattern, shape, 4, periodic=(False, False, True), flags=fl,
                 u_wall=(0.05, 0.01, 0.0))
    ef, er, eu = _errs(r)
    assert ef < 5e-3 and er < 5e-3 and eu < 5e-3, (ef, er, eu)
    assert_f16_elementwise(*r["f"], r["lat"].w)
