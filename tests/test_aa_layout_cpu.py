"""Host model of the AA-pattern addressing of the sweep kernels (Sec. IV-B,
one array, even and odd steps), boundary links included, checked on the CPU.

Array state between steps: after an odd step (and after initialisation)
slot q at x holds f_q(x), the population arriving at x.  Even step: cell x
reads slot q at x and writes its outgoing value for direction q to slot qbar
at x.  Odd step: cell x reads slot qbar at x - c_q (the neighbour's outgoing
value) or, for a boundary link (x, q), slot q at x; it writes its outgoing
value for direction q to slot q at x + c_q or, when (x, qbar) is a boundary
link, to slot qbar at x.  The outgoing value for direction q is P_q(x), or
B_qbar(P(x)) when (x, qbar) is a boundary link (no-slip: P_q(x) itself; UBB:
plus the wall term; outlet: the equilibrium value), so the consumer reads
boundary links like any other.  No access leaves the box on a non-periodic
axis.

The model checks that (1) within a step every (slot, location) pair is
touched by at most one cell (the update is in place and race-free), (2) no
slot of a non-fluid cell is touched, and (3) the populations it reads equal
the oracle's pull streaming with boundary links, step after step."""
import numpy as np
import pytest

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs


def _flags(shape, periodic, seed=6):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    if not periodic[1]:
        fl[:, 0, :] = olbm.NOSLIP
        fl[:, -1, :] = olbm.NOSLIP
    if not periodic[0]:
        fl[:, 1:-1, 0] = olbm.INLET
        fl[:, 1:-1, -1] = olbm.OUTLET
    r = inputs.uniform(seed, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.12) & (fl == 0)] = olbm.NOSLIP
    return fl


class AAModel:
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
        per = ref.periodic

        def shifted(s):
            # location x + s; -1 where it leaves the box on a non-periodic axis
            x, y, z = xs + s[0], ys + s[1], zs + s[2]
            ok = np.ones_like(x, bool)
            for a, (v, n) in enumerate(((x, nx), (y, ny), (z, nz))):
                if not per[a]:
                    ok &= (v >= 0) & (v < n)
            loc = (x % nx) + nx * ((y % ny) + ny * (z % nz))
            return np.where(ok, loc, -1)

        self.up = np.stack([shifted(-c3[q]) for q in range(lat.q)])   # x - c_q
        self.down = np.stack([shifted(c3[q]) for q in range(lat.q)])  # x + c_q
        kind = ref.kind.reshape(lat.q, -1)[:, self.cells]
        self.bnd = kind != olbm.FLUID  # [q][cell]: link (x, q) is a boundary link
        self.own = np.broadcast_to(self.cells, self.bnd.shape)
        self.A = np.full((lat.q, ref.N), np.nan)
        self.touched = None

    def _touch(self, slots, locs):
        assert (locs >= 0).all(), "an access left the box"
        assert ref_fluid_at(self.ref, locs).all(), "a slot of a non-fluid cell was touched"
        owner = np.broadcast_to(np.arange(len(self.cells)), slots.shape)
        key = slots.reshape(-1) * self.ref.N + locs.reshape(-1)
        for k, o in zip(key, owner.reshape(-1)):
            prev = self.touched.setdefault(int(k), int(o))
            assert prev == o, "a (slot, location) pair is touched by two cells in one step"

    def _outgoing(self, P):
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

    def read(self, even):
        lat = self.lat
        if even:
            slots = np.arange(lat.q)[:, None] * np.ones_like(self.own)
            locs = self.own
        else:
            opp = np.array(lat.opp)[:, None] * np.ones_like(self.own)
            slots = np.where(self.bnd, np.arange(lat.q)[:, None], opp)
            locs = np.where(self.bnd, self.own, self.up)
        self._touch(slots, locs)
        return self.A[slots, locs]

    def write(self, P, even):
        """The write phase of a step (even=False: also the initialisation)."""
        lat = self.lat
        vals = self._outgoing(P)
        opp = np.array(lat.opp)
        if even:
            slots = opp[:, None] * np.ones_like(self.own)
            locs = self.own
        else:
            b = self.bnd[opp]  # [q][cell]: (x, qbar) is a boundary link
            slots = np.where(b, opp[:, None], np.arange(lat.q)[:, None])
            locs = np.where(b, self.own, self.down)
        self._touch(slots, locs)
        self.A[slots, locs] = vals


def ref_fluid_at(ref, locs):
    return ref.fluid.reshape(-1)[np.where(locs >= 0, locs, 0)]


@pytest.mark.parametrize("stencil", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("periodic", [(True, True, True), (False, False, True), (False, False, False)])
def test_aa_is_in_place_and_streams_like_pull(stencil, periodic):
    lat = olat.get(stencil)
    shape = (9, 7, 1) if lat.d == 2 else (7, 6, 5)
    if lat.d == 2:
        periodic = (periodic[0], periodic[1], True)
    fl = _flags(shape, periodic)
    m = oco.Method(lat, "trt", [1.7, 1.1])
    ref = olbm.Sim(m, shape, periodic=periodic, flags=fl, u_wall=(0.05, 0.01, 0.0), rho_out=1.02)
    ref.P = inputs.random_pdfs(lat.w, shape[::-1], seed=4)
    model = AAModel(ref)
    model.touched = {}
    model.write(ref.P, even=False)  # initialisation = the writes of an odd step
    for t in range(6):
        even = t % 2 == 0
        model.touched = {}
        f = model.read(even)
        f_ref = ref.populations().reshape(lat.q, -1)[:, model.cells]
        assert np.array_equal(f, f_ref), t
        ref.step(1)
        model.write(ref.P, even)
