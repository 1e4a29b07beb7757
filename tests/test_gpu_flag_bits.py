"""Flag values with several bits set, or with bits the library does not name,
on the GPU: the link mask stays bit-exact with the oracle and the populations
match it (a link takes NOSLIP if its source flag has bit 0 or no known bit,
else INLET if bit 1, else OUTLET; the GHOST bit 8 counts only without the
other three).  The same channel with the flags reduced
to their single types gives bitwise the same GPU result."""
import numpy as np
import pytest

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs
from paper_2001_11806_gb300.sim import Sim

pytestmark = pytest.mark.gpu

OMEGAS = {"srt": [1.37], "trt": [1.8, 8 / 31], "mrt": [1.7, 1.1, 0.9, 1.3, 1.2, 1.05]}
TOL = {"f64": 1e-12, "f32": 1e-5}


def _flags(shape, seed=9):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[:, 0, :] = olbm.NOSLIP
    fl[:, -1, :] = olbm.NOSLIP
    fl[:, 1:-1, 0] = olbm.INLET
    fl[:, 1:-1, -1] = olbm.OUTLET
    r = inputs.uniform(seed, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.08) & (fl == 0)] = olbm.NOSLIP
    return fl


def _mixed(fl, seed=10):
    """Same link types, other bit patterns: NOSLIP -> 1|2, 1|4, 16 or 255;
    INLET -> 2|4 or 2|8; OUTLET -> 4|16."""
    r = inputs.uniform(seed, fl.size).reshape(fl.shape)
    out = fl.copy()
    ns = fl == olbm.NOSLIP
    out[ns & (r < 0.25)] = 3
    out[ns & (r >= 0.25) & (r < 0.5)] = 5
    out[ns & (r >= 0.5) & (r < 0.75)] = 16
    out[ns & (r >= 0.75)] = 255
    out[(fl == olbm.INLET) & (r < 0.5)] = 6
    out[(fl == olbm.INLET) & (r >= 0.5) & (r < 0.75)] = 10
    out[(fl == olbm.OUTLET) & (r < 0.5)] = 20
    return out


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("collision", ["srt", "trt", "mrt"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("pattern", ["pull", "aa", "eso"])
def test_mixed_flag_bits(stencil, collision, storage, pattern):
    lat = olat.get(stencil)
    shape = (150, 7, 1) if stencil == "D2Q9" else (150, 5, 4)
    base = _flags(shape)
    mixed = _mixed(base)
    assert (mixed != base).any()
    per = (False, False, True)
    om = OMEGAS[collision]
    if collision == "mrt":
        om_ref = om[:6] if stencil == "D3Q27" else om[:4]
    else:
        om_ref = om
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=11)
    out = {}
    for name, fl in (("base", base), ("mixed", mixed)):
        sim = Sim(stencil, collision, storage, pattern, shape, periodic=per, omega=om, u_wall=(0.04, 0.01, 0.0),
                  rho_outlet=1.01, flags=fl)
        sim.set_state(P.reshape(lat.q, -1))
        sim.step(4)
        out[name] = (sim.populations().cpu().numpy(), sim.link_mask().cpu().numpy().view(np.uint32))
    ref = olbm.Sim(oco.Method(lat, collision, om_ref), shape, periodic=per, flags=mixed, u_wall=(0.04, 0.01, 0.0),
                   rho_out=1.01)
    assert np.array_equal(out["mixed"][1], ref.link_mask().reshape(-1))
    assert np.array_equal(out["mixed"][1], out["base"][1])
    assert np.array_equal(out["mixed"][0], out["base"][0], equal_nan=True)  # non-fluid cells read NaN
    ref.P = P.copy()
    ref.step(4)
    f_ref = ref.populations().reshape(lat.q, -1)
    m = ref.fluid.reshape(-1)
    err = np.linalg.norm(out["mixed"][0][:, m] - f_ref[:, m]) / np.linalg.norm(f_ref[:, m] - lat.w[:, None])
    assert err < TOL[storage], err
