"""Two-grid stream-pull-collide time stepping (oracle; test only).

State convention.  The array P holds post-collision populations of the last
completed step (the two-array pull scheme of Sec. IV-B "Streaming and
Collision"); initialisation sets P = f^eq(rho_0, u_0).  One time step:

  f_q(x) = P_q(x - c_q)             if the source cell x - c_q is fluid,
  f_q(x) = B_q(P(x))                otherwise (boundary link),
  P'(x)  = collide(f(x))            for fluid x; non-fluid cells keep P.

Periodic axes wrap; a source outside a non-periodic axis counts as a no-slip
wall.  Boundaries are per link (Sec. III-C "Boundary Conditions"), decided by
the flag of the source cell with precedence NOSLIP > INLET > OUTLET (a flag
with none of these bits counts as NOSLIP, unless it has the GHOST bit):

- NOSLIP (halfway bounce-back): B_q = P_qbar(x).
- INLET (velocity bounce-back, UBB listing with c the fluid-to-wall
  direction c_qbar and rho_0 = 1): B_q = P_qbar(x) - 2 w_q (c_qbar.u_w)/cs2.
- OUTLET (not in the paper; reading): B_q = f^eq_q(rho_out, u_P(x)) with
  u_P = (sum_q c_q P_q - F/2) / rho_0(P) the velocity of the cell's own last
  collision.  Pinned by what a velocity inlet and a pressure outlet must
  produce in a channel periodic across the flow (tests/test_oracle_outlet.py):
  the uniform state rho = rho_out, j = rho_0 u_in is a fixed point, and the
  steady state reached from rest.  Which velocity it takes in a transient is
  the reading, which only oracle-vs-GPU agreement checks.

- GHOST (the GHOST bit without NOSLIP, INLET or OUTLET): a ghost cell of a
  block partition (Sec. IV-D "Framework Integration": the domain is split
  into blocks that exchange the populations crossing their faces).  It is
  not updated, like any non-fluid cell, but a link whose source is a ghost
  cell streams like a fluid link: the ghost holds the populations of the
  neighbouring block's cell, set from outside.

Output.  ``populations`` returns f(x) (the pre-collision populations the next
step would collide); ``macroscopic`` returns their moments (Eq. density, with
the Guo half-force); ``reduce`` returns sum rho, sum rho_0 u and
(1/2) sum rho |u|^2 over fluid cells; ``link_mask`` sets bit q for every
boundary link (x, q) of a fluid cell, bit 30 for a fluid cell with an INLET
or OUTLET link, bit 31 for non-fluid cells and bit 29 (beside bit 31) for
ghost cells.

Pins: tests/test_oracle_lbm.py (pull streaming against an independent
np.roll shift, global mass conservation with walls, bounce-back reversing a
free-streaming packet, UBB momentum input, mask bits against a brute-force
loop), tests/test_oracle_outlet.py (inlet/outlet fixed point and steady
state) and tests/test_oracle_flows.py (TGV decay, Poiseuille parabola).
"""
import numpy as np

from . import collision as co
from .lattice import CS2

FLUID, NOSLIP, INLET, OUTLET, GHOST = 0, 1, 2, 4, 8
SELF = -1
CS2F = float(CS2)


def is_ghost(flag):
    flag = np.asarray(flag)
    return ((flag & (NOSLIP | INLET | OUTLET)) == 0) & ((flag & GHOST) != 0)


def link_kind(flag):
    """Type of a link by its source flag: FLUID for a fluid or ghost source,
    else NOSLIP > INLET > OUTLET (NOSLIP when none of the three bits is set)."""
    flag = np.asarray(flag)
    kind = np.full(flag.shape, NOSLIP, dtype=np.int8)
    kind[((flag & NOSLIP) == 0) & ((flag & INLET) != 0)] = INLET
    kind[((flag & (NOSLIP | INLET)) == 0) & ((flag & OUTLET) != 0)] = OUTLET
    kind[(flag == 0) | is_ghost(flag)] = FLUID
    return kind


class Sim:
    """Oracle simulation on an nx x ny x nz box (nz = 1 for D2Q9)."""

    def __init__(self, method, shape, periodic=(True, True, True), flags=None,
                 u_wall=(0.0, 0.0, 0.0), rho_out=1.0):
        self.m = method
        self.lat = method.lat
        self.nx, self.ny, self.nz = shape
        self.periodic = tuple(bool(p) for p in periodic)
        self.shape3 = (self.nz, self.ny, self.nx)
        self.N = self.nx * self.ny * self.nz
        if flags is None:
            flags = np.zeros(self.shape3, dtype=np.uint8)
        self.flags = np.asarray(flags, dtype=np.uint8).reshape(self.shape3)
        self.fluid = self.flags == 0
        self.u_wall = np.asarray(u_wall, dtype=np.float64)[: self.lat.d]
        self.rho_out = float(rho_out)
        self._build_links()
        self.P = np.zeros((self.lat.q,) + self.shape3)
        self.t = 0

    # ------------------------------------------------------------- geometry
    def _build_links(self):
        lat = self.lat
        Z, Y, X = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx), indexing="ij")
        own = (Z * self.ny + Y) * self.nx + X
        self.src = np.empty((lat.q,) + self.shape3, dtype=np.int64)
        self.kind = np.empty((lat.q,) + self.shape3, dtype=np.int8)
        c3 = np.zeros((lat.q, 3), dtype=np.int64)
        c3[:, : lat.d] = lat.c
        for q in range(lat.q):
            s = [X - c3[q, 0], Y - c3[q, 1], Z - c3[q, 2]]
            n = [self.nx, self.ny, self.nz]
            inside = np.ones(self.shape3, dtype=bool)
            for a in range(3):
                if self.periodic[a]:
                    s[a] = s[a] % n[a]
                else:
                    inside &= (s[a] >= 0) & (s[a] < n[a])
                    s[a] = np.clip(s[a], 0, n[a] - 1)
            src_cell = (s[2] * self.ny + s[1]) * self.nx + s[0]
            src_flag = np.where(inside, self.flags.reshape(-1)[src_cell], NOSLIP)
            kind = link_kind(src_flag)
            kind[~self.fluid] = SELF
            self.kind[q] = kind
            # flat index into P.reshape(-1) that feeds f_q(x)
            pulled = q * self.N + src_cell
            bounced = lat.opp[q] * self.N + own
            itself = q * self.N + own
            self.src[q] = np.where(kind == FLUID, pulled, np.where(kind == SELF, itself, bounced))
        # UBB constant per link: -2 w_q (c_qbar . u_w) / cs2
        cqb = lat.c[lat.opp].astype(np.float64)
        ubb = -2.0 * lat.w * (cqb @ self.u_wall) / CS2F
        self.ubb_const = np.where(self.kind == INLET, ubb.reshape((-1, 1, 1, 1)), 0.0)

    def link_mask(self):
        mask = np.zeros(self.shape3, dtype=np.uint64)
        special = np.zeros(self.shape3, dtype=bool)
        for q in range(self.lat.q):
            b = (self.kind[q] != FLUID) & self.fluid
            mask |= b.astype(np.uint64) << np.uint64(q)
            special |= self.fluid & ((self.kind[q] == INLET) | (self.kind[q] == OUTLET))
        mask |= special.astype(np.uint64) << np.uint64(30)
        mask |= (~self.fluid).astype(np.uint64) << np.uint64(31)
        mask |= is_ghost(self.flags).astype(np.uint64) << np.uint64(29)
        return mask.astype(np.uint32)

    # -------------------------------------------------------------- stepping
    def init_equilibrium(self, rho0, u0):
        rho0 = np.asarray(rho0, dtype=np.float64).reshape(self.shape3)
        u0 = np.asarray(u0, dtype=np.float64).reshape((self.lat.d,) + self.shape3)
        self.P = co.equilibrium(self.lat, rho0, u0, self.m.incompressible)
        self.t = 0

    def outlet_values(self, P):
        """f^eq(rho_out, u_P(x)) for every cell (used on OUTLET links)."""
        lat, m = self.lat, self.m
        rho = co.density(P)
        j = co.momentum(lat, P)
        if m.force is not None:
            j = j - 0.5 * co._force_array(lat, m.force, P)
        u = j / (1.0 if m.incompressible else rho)
        rho_o = np.full_like(rho, self.rho_out)
        return co.equilibrium(lat, rho_o, u, m.incompressible)

    def stream(self, P):
        """Pull streaming with boundary links: returns f from P."""
        f = P.reshape(-1)[self.src] + self.ubb_const
        if (self.kind == OUTLET).any():
            f = np.where(self.kind == OUTLET, self.outlet_values(P), f)
        return f

    def step_state(self, P, method=None):
        method = self.m if method is None else method
        f = self.stream(P)
        Pn = method_collide(method, f)
        return np.where(self.fluid[None], Pn, P)

    def step(self, n=1):
        for _ in range(n):
            self.P = self.step_state(self.P)
            self.t += 1

    # ---------------------------------------------------------------- output
    def populations(self):
        return self.stream(self.P)

    def macroscopic(self):
        f = self.populations()
        rho, u = co.velocity(self.lat, f, self.m.force, self.m.incompressible)
        return rho, u

    def reduce(self):
        rho, u = self.macroscopic()
        fl = self.fluid
        rho0 = np.ones_like(rho) if self.m.incompressible else rho
        mass = rho[fl].sum()
        mom = [(rho0 * u[a])[fl].sum() for a in range(self.lat.d)]
        mom += [0.0] * (3 - self.lat.d)
        ke = 0.5 * (rho * (u * u).sum(axis=0))[fl].sum()
        return np.array([mass] + mom + [ke])


def method_collide(method, f):
    return co.collide(method, f)
