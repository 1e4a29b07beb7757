"""The premise of the main fluid-cell-list launch, checked on the CPU.

Masked domains are swept over the list of their fluid cells.  The main
launch takes the cells that are not on a face of a periodic axis and
addresses every neighbour as the cell's own index plus a fixed per-direction
offset, -(c_x + nx c_y + nx ny c_z), without any wrap; boundary links of
every type read the cell's own index (slot qbar), and inlet and outlet links
then have their value replaced.  That is right only if, for every such cell,
each fluid link (x, q) pulls from exactly x minus that offset (no wrap,
inside the box) and every link whose source would leave the box is a
boundary link.  The oracle's link table (independent pull with wraps and
boundary tests) must agree with the offset rule on all of them (the
periodic-face cells go to the second launch, which addresses by
coordinates)."""
import numpy as np
import pytest

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs


def _flags(shape, periodic, seed):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    if not periodic[1]:
        fl[:, 0, :] = olbm.NOSLIP
        fl[:, -1, :] = olbm.NOSLIP
    if not periodic[0]:
        fl[:, 1:-1, 0] = olbm.INLET
        fl[:, 1:-1, -1] = olbm.OUTLET
    r = inputs.uniform(seed, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.1) & (fl == 0)] = olbm.NOSLIP
    return fl


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("periodic", [(True, True, True), (False, False, True), (True, False, False),
                                      (False, False, False)])
def test_plain_cells_pull_through_fixed_offsets(stencil, periodic):
    lat = olat.get(stencil)
    shape = (10, 7, 1) if lat.d == 2 else (8, 7, 6)
    if lat.d == 2:
        periodic = (periodic[0], periodic[1], True)
    s = olbm.Sim(oco.Method(lat, "srt", [1.2]), shape, periodic=periodic, flags=_flags(shape, periodic, 2),
                 u_wall=(0.04, 0.0, 0.0))
    nx, ny, nz = shape
    N = s.N
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X, Y, Z = X.reshape(-1), Y.reshape(-1), Z.reshape(-1)
    fluid = s.fluid.reshape(-1)
    kind = s.kind.reshape(lat.q, -1)
    special = ((kind == olbm.INLET) | (kind == olbm.OUTLET)).any(axis=0)
    face = np.zeros(N, bool)
    for a, (v, n) in enumerate(((X, nx), (Y, ny), (Z, nz))):
        if periodic[a] and not (a == 2 and lat.d == 2):
            face |= (v == 0) | (v == n - 1)
    plain = fluid & ~face
    assert plain.any()
    if not periodic[0]:
        assert (plain & special).any()
    src = s.src.reshape(lat.q, -1)
    c3 = np.zeros((lat.q, 3), np.int64)
    c3[:, : lat.d] = lat.c
    cells = np.flatnonzero(plain)
    for q in range(lat.q):
        off = c3[q, 0] + nx * c3[q, 1] + nx * ny * c3[q, 2]
        fl_link = kind[q, cells] == olbm.FLUID
        # fluid links: slot q of cell - offset, which is inside the box and fluid
        assert np.array_equal(src[q, cells[fl_link]], q * N + cells[fl_link] - off), q
        x0, y0, z0 = X[cells] - c3[q, 0], Y[cells] - c3[q, 1], Z[cells] - c3[q, 2]
        inside = (x0 >= 0) & (x0 < nx) & (y0 >= 0) & (y0 < ny) & (z0 >= 0) & (z0 < nz)
        assert inside[fl_link].all(), q
        # every source outside the box is a boundary link, read from the cell itself
        assert (~fl_link[~inside]).all(), q
        assert np.array_equal(src[q, cells[~fl_link]], lat.opp[q] * N + cells[~fl_link]), q


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
def test_dense_inner_rows_pull_through_offsets_with_an_x_correction(stencil):
    """The periodic sweep's fast path: in a row whose y and z neighbours do
    not wrap, the source of link (x, q) is the cell index minus the fixed
    offset, corrected by +-nx where x - c_x wraps."""
    lat = olat.get(stencil)
    shape = (9, 6, 1) if lat.d == 2 else (9, 6, 5)
    s = olbm.Sim(oco.Method(lat, "srt", [1.2]), shape)
    nx, ny, nz = shape
    N = s.N
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X, Y, Z = X.reshape(-1), Y.reshape(-1), Z.reshape(-1)
    inner = (Y > 0) & (Y < ny - 1)
    if lat.d == 3:
        inner &= (Z > 0) & (Z < nz - 1)
    cells = np.flatnonzero(inner)
    src = s.src.reshape(lat.q, -1)
    c3 = np.zeros((lat.q, 3), np.int64)
    c3[:, : lat.d] = lat.c
    for q in range(lat.q):
        off = c3[q, 0] + nx * c3[q, 1] + nx * ny * c3[q, 2]
        xs = X[cells] - c3[q, 0]
        corr = np.where(xs < 0, nx, np.where(xs >= nx, -nx, 0))
        assert np.array_equal(src[q, cells], q * N + cells - off + corr), q
