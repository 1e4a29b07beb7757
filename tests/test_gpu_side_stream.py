"""The list sweep's second launch on its side stream.

Masked domains are swept over a fluid-cell list in two launches: the main
launch, and a second one for the cells on a face of a periodic axis (and,
for the two-grid pull, the cells with inlet or outlet links).  The second
launch runs on a stream of its own, forked from the sweep's stream before
the main launch and joined back after it, so the two overlap within a step.
A fully periodic porous 40 x 12 x 10 box has over a third of its fluid
cells on its six faces, so both launches carry many cells.  Checked here:
parity with the FP64 oracle for the pull, AA and esoteric-twist patterns,
the pull's inlet and outlet cells on periodic y and z, and lbm_step(n)
replayed as 32-step CUDA graphs (whose capture holds the fork and the join)
against n single steps, bit for bit."""
import numpy as np
import pytest

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs
from paper_2001_11806_gb300.sim import Sim

SHAPE = (40, 12, 10)
OMEGA = [1.8, 8 / 31]
TOL = {"f64": 1e-12, "f32": 1e-5}


def porous_flags(shape, seed=29, fraction=0.12):
    nx, ny, nz = shape
    r = inputs.uniform(seed, nx * ny * nz).reshape(nz, ny, nx)
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[r < fraction] = olbm.NOSLIP
    return fl


def channel_flags(shape, seed=31):
    fl = porous_flags(shape, seed, 0.08)
    fl[..., 0] = olbm.INLET
    fl[..., -1] = olbm.OUTLET
    return fl


def run(storage, pattern, shape, flags, periodic, steps, u_wall=(0.0, 0.0, 0.0)):
    lat = olat.d3q19()
    sim = Sim("D3Q19", "trt", storage, pattern, shape, periodic=periodic, omega=OMEGA, flags=flags,
              u_wall=u_wall, rho_outlet=1.01)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=17)
    sim.set_state(P.reshape(lat.q, -1))
    sim.step(steps)
    f_gpu = sim.populations().cpu().numpy()
    sim.close()
    ref = olbm.Sim(oco.Method(lat, "trt", OMEGA), shape, periodic=periodic, flags=flags, u_wall=u_wall,
                   rho_out=1.01)
    ref.P = P.copy()
    ref.step(steps)
    f_ref = ref.populations().reshape(lat.q, -1)
    fl = ref.fluid.reshape(-1)
    w = lat.w[:, None]
    return np.linalg.norm(f_gpu[:, fl] - f_ref[:, fl]) / np.linalg.norm(f_ref[:, fl] - w)


def test_porous_box_puts_cells_in_both_launches():
    """The premise: fluid cells on the faces of the periodic box (second
    launch) and inside it (main launch)."""
    fl = porous_flags(SHAPE)
    fluid = fl == 0
    face = np.zeros_like(fluid)
    face[0], face[-1] = True, True
    face[:, 0], face[:, -1] = True, True
    face[..., 0], face[..., -1] = True, True
    assert (fluid & face).sum() > 1000 and (fluid & ~face).sum() > 1000


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
def test_periodic_porous_box_matches_the_oracle(storage, pattern):
    err = run(storage, pattern, SHAPE, porous_flags(SHAPE), (True, True, True), 7)
    assert err < TOL[storage], err


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_pull_inlet_outlet_cells_with_periodic_faces(storage):
    """Two-grid pull: the inlet/outlet cells and the y/z face cells share the
    second launch."""
    shape = (40, 10, 8)
    err = run(storage, "pull", shape, channel_flags(shape), (False, True, True), 7, u_wall=(0.04, 0.0, 0.0))
    assert err < TOL[storage], err


@pytest.mark.gpu
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
def test_graph_replay_equals_single_steps(pattern):
    lat = olat.d3q19()
    fl = porous_flags(SHAPE)
    P = inputs.random_pdfs(lat.w, SHAPE[::-1], seed=19).reshape(lat.q, -1)
    out = []
    for chunks in ([1] * 70, [70]):
        sim = Sim("D3Q19", "trt", "f32", pattern, SHAPE, periodic=(True, True, True), omega=OMEGA, flags=fl)
        sim.set_state(P)
        for k in chunks:
            sim.step(k)
        assert sim.t == 70
        out.append(sim.populations().cpu().numpy())
        sim.close()
    fluid = fl.reshape(-1) == 0
    assert np.array_equal(out[0][:, fluid], out[1][:, fluid])
