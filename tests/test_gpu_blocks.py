"""x-slab block partition on one GPU (Sec. IV-D "Framework Integration": the
domain split into blocks that exchange the populations crossing their faces
through pack and unpack kernels, which depend on the pattern and the step
parity).  Two and three blocks with ghost layers, exchanging through
lbm_halo_pack / lbm_halo_unpack after the initialisation and after every step,
must give bit for bit the populations of the undivided domain, for the pull
and AA patterns, odd and even step counts, obstacles across the block faces
and a periodic or an inlet/outlet x axis; and the partition agrees with the
oracle within the storage tolerance."""
import numpy as np
import pytest

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs
from paper_2001_11806_gb300.blocks import SlabBlocks
from paper_2001_11806_gb300.sim import Sim

pytestmark = pytest.mark.gpu

OMEGAS = {"srt": [1.37], "trt": [1.8, 8 / 31], "mrt": [1.7, 1.1, 0.9, 1.3, 1.2, 1.05], "cumulant": [1.95, 1.0, 1.0]}


def _flags(shape, periodic_x, seed=13):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    r = inputs.uniform(seed, fl.size).reshape(fl.shape)
    fl[r < 0.1] = olbm.NOSLIP
    if not periodic_x:
        fl[..., 0] = olbm.INLET
        fl[..., -1] = olbm.OUTLET
    return fl


@pytest.mark.parametrize("stencil,collision", [("D2Q9", "srt"), ("D3Q19", "trt"), ("D3Q19", "mrt"),
                                               ("D3Q27", "cumulant")])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("pattern", ["pull", "aa"])
@pytest.mark.parametrize("periodic_x", [True, False])
def test_blocks_equal_the_undivided_domain(stencil, collision, storage, pattern, periodic_x):
    lat = olat.get(stencil)
    shape = (40, 7, 1) if lat.d == 2 else (40, 6, 5)
    fl = _flags(shape, periodic_x)
    per = (periodic_x, True, True)
    kw = dict(omega=OMEGAS[collision], u_wall=(0.04, 0.0, 0.0), rho_outlet=1.01)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=21).reshape(lat.q, -1)
    whole = Sim(stencil, collision, storage, pattern, shape, periodic=per, flags=fl, **kw)
    whole.set_state(P)
    fluid = fl.reshape(-1) == 0
    for cuts in ([0, 17, 40], [0, 9, 10, 40]):
        blk = SlabBlocks(stencil, collision, storage, pattern, shape, cuts, periodic=per, flags=fl, **kw)
        blk.set_state(P)
        ref = Sim(stencil, collision, storage, pattern, shape, periodic=per, flags=fl, **kw)
        ref.set_state(P)
        for n in (5, 1):  # odd, then even step counts
            blk.step(n)
            ref.step(n)
            got = blk.populations().cpu().numpy()
            want = ref.populations().cpu().numpy()
            assert np.array_equal(got[:, fluid], want[:, fluid]), (cuts, n)
        blk.close()
        ref.close()
    whole.close()


@pytest.mark.parametrize("pattern", ["pull", "aa"])
def test_blocks_from_equilibrium_against_the_oracle(pattern):
    """Initialisation by lbm_init_equilibrium (the AA push writes across the
    block faces), then the oracle's undivided run."""
    lat = olat.d3q19()
    shape = (36, 6, 5)
    fl = _flags(shape, False)
    per = (False, True, True)
    rho, u = inputs.random_fields(shape[::-1], 3, seed=22)
    blk = SlabBlocks("D3Q19", "trt", "f64", pattern, shape, [0, 12, 25, 36], periodic=per, flags=fl,
                     omega=OMEGAS["trt"], u_wall=(0.04, 0.0, 0.0))
    blk.init_equilibrium(rho.reshape(-1), u.reshape(3, -1))
    blk.step(7)
    ref = olbm.Sim(oco.Method(lat, "trt", OMEGAS["trt"]), shape, periodic=per, flags=fl, u_wall=(0.04, 0.0, 0.0))
    ref.init_equilibrium(rho, u)
    ref.step(7)
    fluid = fl.reshape(-1) == 0
    fr = ref.populations().reshape(19, -1)[:, fluid]
    fg = blk.populations().cpu().numpy()[:, fluid]
    assert np.linalg.norm(fg - fr) / np.linalg.norm(fr - lat.w[:, None]) < 1e-12
    blk.close()


def test_halo_refuses_what_it_does_not_serve():
    from paper_2001_11806_gb300 import LbmError, _lib
    import torch
    sim = Sim("D3Q19", "trt", "f32", "eso", (8, 6, 5), periodic=(False, True, True), omega=[1.6, 1.1],
              flags=np.where(np.arange(8)[None, None, :] % 7 == 0, olbm.NOSLIP, 0).astype(np.uint8)
              * np.ones((5, 6, 8), np.uint8))
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device=sim.device)
    assert _lib.lib().lbm_halo_pack(sim.ctx, 1, buf.data_ptr()) == 2  # LBM_E_UNSUPPORTED
    per = Sim("D3Q19", "trt", "f32", "aa", (8, 6, 5), omega=[1.6, 1.1])
    assert _lib.lib().lbm_halo_pack(per.ctx, 1, buf.data_ptr()) == 1  # periodic x: LBM_E_INVAL
    assert _lib.lib().lbm_halo_unpack(per.ctx, 2, buf.data_ptr()) == 1  # unknown face
    with pytest.raises(LbmError):
        SlabBlocks("D3Q19", "trt", "f32", "eso", (8, 6, 5), [0, 4, 8])
