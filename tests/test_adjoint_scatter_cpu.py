"""The premise of the GPU adjoint's reverse streaming, checked on the CPU:
without outlet links, pull streaming with bounce-back and UBB links maps the
post-collision slots of the fluid cells one-to-one onto the populations the
fluid cells collide next (each slot (q, y) of a fluid cell feeds f_q(y + c_q)
if that cell is fluid, else f_qbar(y) through the bounce-back link).  Its
transpose therefore gives every adjoint slot exactly one contribution, so
the adjoint kernel writes it with a plain store (no atomics, no zeroing)."""
import numpy as np
import pytest

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs


def _flags(shape, seed):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[:, 0, :] = olbm.NOSLIP
    fl[:, -1, 1:-1] = olbm.INLET
    r = inputs.uniform(seed, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.15) & (fl == 0)] = olbm.NOSLIP
    return fl


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("periodic", [(True, False, True), (False, False, False)])
def test_fluid_streaming_is_a_bijection_of_fluid_slots(stencil, periodic):
    lat = olat.get(stencil)
    shape = (8, 7, 1) if lat.d == 2 else (7, 6, 5)
    if lat.d == 2:
        periodic = (periodic[0], periodic[1], True)
    s = olbm.Sim(oco.Method(lat, "srt", [1.2]), shape, periodic=periodic, flags=_flags(shape, 3),
                 u_wall=(0.03, 0.0, 0.0))
    assert not (s.kind == olbm.OUTLET).any()
    fluid = s.fluid.reshape(-1)
    cells = np.flatnonzero(fluid)
    src = s.src.reshape(lat.q, -1)[:, cells].reshape(-1)  # flat indices q * N + cell
    assert len(np.unique(src)) == src.size, "two populations pull the same slot"
    q_src, cell_src = np.divmod(src, s.N)
    assert fluid[cell_src].all(), "a fluid population pulls a slot of a non-fluid cell"
    assert src.size == lat.q * len(cells)
