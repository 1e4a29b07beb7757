"""Host model of the esoteric-twist addressing of the sweep kernels (Sec.
IV-B, single array run as even and odd kernels), checked on the CPU.

Cell x reads f_q(x) from location x + max(-c_q, 0) (slot q after an even
number of steps, qbar after an odd number) and writes P_q(x) to location
x + max(c_q, 0) (slot qbar in even steps, q in odd steps); for a boundary
link (x, qbar) it writes B_qbar(P(x)) to the other slot of that location.
Locations wrap on every axis, also on non-periodic ones, which is why the
last layer of a non-periodic axis must be non-fluid.  The model checks that
(1) within a step every (slot, location) pair is touched by at most one cell
(the update is in place and race-free, including the wrapped pairs of
non-periodic faces and the slots of solid cells), (2) the populations it
reads equal the oracle's pull streaming with boundary links, step after
step, and (3) a fluid last layer does produce a race."""
import numpy as np
import pytest

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs


def _flags(shape, periodic, seed=3):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    if not periodic[1]:
        fl[:, 0, :] = olbm.NOSLIP
        fl[:, -1, :] = olbm.NOSLIP
    if not periodic[0]:
        fl[:, 1:-1, 0] = olbm.INLET
        fl[:, 1:-1, -1] = olbm.OUTLET
    if not periodic[2] and len(fl) > 1:
        fl[0] = olbm.NOSLIP
        fl[-1] = olbm.NOSLIP
    r = inputs.uniform(seed, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.1) & (fl == 0)] = olbm.NOSLIP
    return fl


class EsoModel:
    def __init__(self, ref):
        self.ref = ref
        lat = ref.lat
        self.lat = lat
        nz, ny, nx = ref.shape3
        Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        self.cells = np.flatnonzero(ref.fluid.reshape(-1))
        xs, ys, zs = X.reshape(-1)[self.cells], Y.reshape(-1)[self.cells], Z.reshape(-1)[self.cells]
        c3 = np.zeros((lat.q, 3), np.int64)
        c3[:, : lat.d] = lat.c

        def loc(m):
            return ((xs + m[0]) % nx) + nx * (((ys + m[1]) % ny) + ny * ((zs + m[2]) % nz))

        self.rd = np.stack([loc(np.maximum(-c3[q], 0)) for q in range(lat.q)])
        self.wr = np.stack([loc(np.maximum(c3[q], 0)) for q in range(lat.q)])
        kind = ref.kind.reshape(lat.q, -1)[:, self.cells]
        self.bnd = kind != olbm.FLUID  # [p][cell]: link (x, p) is a boundary link
        self.A = np.full((lat.q, ref.N), np.nan)
        self.touched = None

    def _touch(self, slots, locs):
        owner = np.broadcast_to(np.arange(len(self.cells)), slots.shape)
        key = slots.reshape(-1) * self.ref.N + locs.reshape(-1)
        for k, o in zip(key, owner.reshape(-1)):
            prev = self.touched.setdefault(int(k), int(o))
            assert prev == o, "a (slot, location) pair is touched by two cells in one step"

    def _outgoing(self, P):
        """Value each fluid cell writes for direction q: P_q(x), or B_qbar(P(x))
        if (x, qbar) is a boundary link."""
        ref, lat = self.ref, self.lat
        Pc = P.reshape(lat.q, -1)[:, self.cells]
        out_v = ref.outlet_values(P).reshape(lat.q, -1)[:, self.cells]
        ubb = ref.ubb_const.reshape(lat.q, -1)[:, self.cells]
        kind = ref.kind.reshape(lat.q, -1)[:, self.cells]
        vals = Pc.copy()
        for q in range(lat.q):
            p = lat.opp[q]
            vals[q] = np.where(kind[p] == olbm.OUTLET, out_v[p], Pc[q] + ubb[p])
        return vals

    def write(self, P, even):
        """The write phase of a step (even=False: also the initialisation)."""
        lat = self.lat
        vals = self._outgoing(P)
        slots = np.empty_like(self.wr)
        for q in range(lat.q):
            p = lat.opp[q]
            b = self.bnd[p]
            slots[q] = np.where(even != b, p, q)
        self._touch(slots, self.wr)
        self.A[slots, self.wr] = vals

    def read(self, even):
        lat = self.lat
        slots = np.array([q if even else lat.opp[q] for q in range(lat.q)])[:, None] * np.ones_like(self.rd)
        self._touch(slots, self.rd)
        return self.A[slots, self.rd]


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("periodic", [(True, True, True), (False, False, True), (False, False, False)])
def test_esoteric_twist_is_in_place_and_streams_like_pull(stencil, periodic):
    lat = olat.get(stencil)
    shape = (9, 7, 1) if lat.d == 2 else (7, 6, 5)
    fl = _flags(shape, periodic)
    m = oco.Method(lat, "trt", [1.7, 1.1])
    ref = olbm.Sim(m, shape, periodic=periodic, flags=fl, u_wall=(0.05, 0.01, 0.0), rho_out=1.02)
    ref.P = inputs.random_pdfs(lat.w, shape[::-1], seed=4)
    model = EsoModel(ref)
    model.touched = {}
    model.write(ref.P, even=False)  # initialisation = the writes of an odd step
    for t in range(5):
        even = t % 2 == 0
        model.touched = {}
        f = model.read(even)
        f_ref = ref.populations().reshape(lat.q, -1)[:, model.cells]
        assert np.array_equal(f, f_ref), t
        ref.step(1)
        model.write(ref.P, even)


def test_fluid_last_layer_races():
    """Why lbm_create refuses the esoteric twist when the last layer of a
    non-periodic axis is fluid: the first layer's boundary links share the
    wrapped locations with it."""
    lat = olat.get("D3Q19")
    shape = (6, 5, 4)
    fl = np.zeros(shape[::-1], np.uint8)
    fl[:, 0, :] = olbm.NOSLIP
    fl[:, -1, :] = olbm.NOSLIP  # y walls on both sides, but z open and non-periodic
    ref = olbm.Sim(oco.Method(lat, "srt", [1.2]), shape, periodic=(True, False, False), flags=fl)
    ref.P = inputs.random_pdfs(lat.w, shape[::-1], seed=5)
    model = EsoModel(ref)
    model.touched = {}
    model.write(ref.P, even=False)
    model.touched = {}
    model.read(True)
    with pytest.raises(AssertionError, match="two cells"):
        model.write(ref.P, even=True)
