"""Host model of the separate boundary kernels of the two-grid pull (Sec.
IV-B offers boundary handling in kernels run before the sweep), checked on
the CPU.

Before each pull sweep, for every boundary link (x, q) of a fluid cell x the
boundary kernel writes B_q(P(x)) into slot q of the link's source cell
x - c_q, which is non-fluid and inside the box; the sweep then pulls every
link as a fluid one, f_q(x) = P_q(x - c_q).  The model checks that (1) every
slot the boundary kernel writes belongs to exactly one link and to a
non-fluid cell (no race, no fluid population overwritten), and (2) the
populations the sweep pulls equal the oracle's pull streaming with boundary
links, step after step.  A fluid first or last layer of a non-periodic axis
has link sources outside the box, which have no slot: that case is refused
by the library and shown here."""
import numpy as np
import pytest

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs


def _flags(shape, periodic, seed=8):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    if not periodic[1]:
        fl[:, 0, :] = olbm.NOSLIP
        fl[:, -1, :] = olbm.NOSLIP
    if not periodic[0]:
        fl[:, 1:-1, 0] = olbm.INLET
        fl[:, 1:-1, -1] = olbm.OUTLET
    if not periodic[2] and nz > 1:
        fl[0] = olbm.NOSLIP
        fl[-1] = olbm.NOSLIP
    r = inputs.uniform(seed, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.1) & (fl == 0)] = olbm.NOSLIP
    return fl


def _sources(ref):
    """[q][cell] location of x - c_q (wrapped on periodic axes) or -1 outside."""
    lat = ref.lat
    nz, ny, nx = ref.shape3
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c3 = np.zeros((lat.q, 3), np.int64)
    c3[:, : lat.d] = lat.c
    out = np.empty((lat.q, ref.N), np.int64)
    for q in range(lat.q):
        x, y, z = X - c3[q, 0], Y - c3[q, 1], Z - c3[q, 2]
        ok = np.ones(x.shape, bool)
        for a, (v, n) in enumerate(((x, nx), (y, ny), (z, nz))):
            if not ref.periodic[a]:
                ok &= (v >= 0) & (v < n)
        out[q] = np.where(ok, (x % nx) + nx * ((y % ny) + ny * (z % nz)), -1).reshape(-1)
    return out


def _boundary_values(ref, P):
    """B_q(P(x)) for every link: bounce-back (+ UBB term) or outlet value."""
    lat = ref.lat
    Pf = P.reshape(lat.q, -1)
    kind = ref.kind.reshape(lat.q, -1)
    out_v = ref.outlet_values(P).reshape(lat.q, -1)
    ubb = ref.ubb_const.reshape(lat.q, -1)
    B = np.empty_like(Pf)
    for q in range(lat.q):
        B[q] = np.where(kind[q] == olbm.OUTLET, out_v[q], Pf[lat.opp[q]] + ubb[q])
    return B


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("periodic", [(True, True, True), (False, False, True), (False, False, False)])
def test_separate_boundary_kernel_then_plain_pull(stencil, periodic):
    lat = olat.get(stencil)
    shape = (9, 7, 1) if lat.d == 2 else (7, 6, 5)
    if lat.d == 2:
        periodic = (periodic[0], periodic[1], True)
    fl = _flags(shape, periodic)
    ref = olbm.Sim(oco.Method(lat, "trt", [1.7, 1.1]), shape, periodic=periodic, flags=fl,
                   u_wall=(0.05, 0.01, 0.0), rho_out=1.02)
    ref.P = inputs.random_pdfs(lat.w, shape[::-1], seed=5)
    src = _sources(ref)
    fluid = ref.fluid.reshape(-1)
    cells = np.flatnonzero(fluid)
    kind = ref.kind.reshape(lat.q, -1)
    for t in range(4):
        A = ref.P.reshape(lat.q, -1).copy()
        B = _boundary_values(ref, ref.P)
        written = {}
        for q in range(lat.q):
            for x in cells:
                if kind[q, x] == olbm.FLUID:
                    continue
                s = src[q, x]
                assert s >= 0, "a boundary link with its source outside the box"
                assert not fluid[s], "the boundary kernel would overwrite a fluid population"
                assert written.setdefault((q, s), x) == x, "two links write one slot"
                A[q, s] = B[q, x]
        f = np.stack([A[q, src[q, cells]] for q in range(lat.q)])
        f_ref = ref.populations().reshape(lat.q, -1)[:, cells]
        assert np.array_equal(f, f_ref), t
        ref.step(1)


def test_fluid_face_of_a_non_periodic_axis_has_no_slot():
    lat = olat.get("D3Q19")
    shape = (6, 5, 4)
    fl = np.zeros(shape[::-1], np.uint8)
    fl[:, 0, :] = olbm.NOSLIP
    fl[:, -1, :] = olbm.NOSLIP  # y closed; z open and non-periodic
    ref = olbm.Sim(oco.Method(lat, "srt", [1.2]), shape, periodic=(True, False, False), flags=fl)
    src = _sources(ref)
    kind = ref.kind.reshape(lat.q, -1)
    fluid = ref.fluid.reshape(-1)
    outside = [(q, x) for q in range(lat.q) for x in np.flatnonzero(fluid)
               if kind[q, x] != olbm.FLUID and src[q, x] < 0]
    assert outside, "the open z faces must have links with no source slot"
