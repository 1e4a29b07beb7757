"""Discrete adjoint of the time step (oracle; test only).

The paper has no adjoint; this is the reverse-mode derivative of the oracle's
own time step P_t = C(S(P_{t-1})) (S = pull streaming with boundary links,
C = per-cell collision), written from the chain rule:

  lambda_{t-1} = S^T [ C'(f_t)^T lambda_t ],   f_t = S(P_{t-1}),
  dL/dF       += (dC/dF)(f_t)^T lambda_t,
  dL/du_0      = (d f^eq(rho_0, u_0)/du_0)^T lambda_{-1}.

Per-cell Jacobians come from complex-step differentiation
(d/dx g(x) = Im g(x + i h)/h, exact to rounding for analytic g; h = 1e-30),
which shares nothing with the CUDA path's hand-derived transposes.  S is
linear plus UBB constants, so S^T is the scatter-add of the link table
Sim.src; OUTLET links (non-linear) are not supported here.  Non-fluid cells
are the identity map.

Loss: L = (1/2) sum_{x in box, fluid} rho |u|^2 of f_T = S(P_{T-1})
(kinetic energy in a box), with u from Eq. density including F/2.

Pins (tests/test_oracle_adjoint.py): dot-product identity
<J v, w> = <v, J^T w> per step against the forward map, per-cell Jacobian
against central finite differences, whole-run gradients against central
finite differences of the forward oracle.
"""
import numpy as np

from . import collision as co
from .lbm import OUTLET

H = 1e-30


def collide_vjp(method, f, lam):
    """mu = (dC/df)^T lam, cell by cell."""
    mu = np.zeros_like(f)
    fc = f.astype(np.complex128)
    for j in range(f.shape[0]):
        fp = fc.copy()
        fp[j] = fp[j] + 1j * H
        col = co.collide(method, fp).imag / H
        mu[j] = (col * lam).sum(axis=0)
    return mu


def collide_force_vjp(method, f, lam, cellmask):
    """sum over masked cells of (dC/dF_a)^T lam for each force component a."""
    d = method.lat.d
    g = np.zeros(d)
    F0 = np.zeros(d) if method.force is None else np.asarray(method.force, dtype=np.float64)
    for a in range(d):
        Fc = F0.astype(np.complex128)
        Fc[a] += 1j * H
        dC = co.collide(method.with_force(Fc), f.astype(np.complex128)).imag / H
        g[a] = ((dC * lam).sum(axis=0))[cellmask].sum()
    return g


def stream_transpose(sim, mu):
    if (sim.kind == OUTLET).any():
        raise ValueError("outlet links are not differentiated")
    out = np.zeros(mu.size)
    np.add.at(out, sim.src.reshape(-1), mu.reshape(-1))
    return out.reshape(mu.shape)


def adjoint_step(sim, P_prev, lam):
    """Return (lambda_{t-1}, dL/dF contribution) for one step."""
    f = sim.stream(P_prev)
    fl = sim.fluid
    mu = np.where(fl[None], collide_vjp(sim.m, f, lam), lam)
    gF = collide_force_vjp(sim.m, f, lam, fl) if sim.m.force is not None else np.zeros(sim.lat.d)
    return stream_transpose(sim, mu), gF


def box_mask(sim, box):
    x0, x1, y0, y1, z0, z1 = box
    m = np.zeros(sim.shape3, dtype=bool)
    m[z0:z1, y0:y1, x0:x1] = True
    return m & sim.fluid


def _ke_density(method, f):
    rho, u = co.velocity(method.lat, f, method.force, method.incompressible)
    return 0.5 * rho * (u * u).sum(axis=0)


def ke_box_loss(sim, P, box):
    f = sim.stream(P)
    return float(_ke_density(sim.m, f)[box_mask(sim, box)].sum())


def ke_box_seed(sim, P, box):
    """Return (L, dL/dP_{T-1}, direct dL/dF)."""
    f = sim.stream(P)
    bm = box_mask(sim, box)
    dLdf = np.zeros_like(f)
    fc = f.astype(np.complex128)
    for j in range(f.shape[0]):
        fp = fc.copy()
        fp[j] = fp[j] + 1j * H
        dLdf[j] = np.where(bm, _ke_density(sim.m, fp).imag / H, 0.0)
    gF = np.zeros(sim.lat.d)
    if sim.m.force is not None:
        for a in range(sim.lat.d):
            Fc = np.asarray(sim.m.force, dtype=np.complex128).copy()
            Fc[a] += 1j * H
            gF[a] = (_ke_density(sim.m.with_force(Fc), fc).imag / H)[bm].sum()
    L = float(_ke_density(sim.m, f)[bm].sum())
    return L, stream_transpose(sim, dLdf), gF


def eq_vjp(sim, rho0, u0, lam):
    """(d f^eq(rho_0, u_0)/d u_0)^T lam per cell, shape (d, ...cells)."""
    lat = sim.lat
    rho0 = np.asarray(rho0, dtype=np.float64).reshape(sim.shape3)
    u0 = np.asarray(u0, dtype=np.float64).reshape((lat.d,) + sim.shape3)
    g = np.zeros_like(u0)
    for a in range(lat.d):
        uc = u0.astype(np.complex128)
        uc[a] = uc[a] + 1j * H
        dfeq = co.equilibrium(lat, rho0, uc, sim.m.incompressible).imag / H
        g[a] = (dfeq * lam).sum(axis=0)
    return g


def gradient(sim, rho0, u0, T, box):
    """Forward T steps from f^eq(rho_0, u_0), then the reverse sweep.

    Returns (L, dL/du_0, dL/dF) with dL/dF zero-length-d when unforced."""
    sim.init_equilibrium(rho0, u0)
    states = [sim.P.copy()]
    for _ in range(T):
        sim.step(1)
        states.append(sim.P.copy())
    L, lam, gF = ke_box_seed(sim, states[T], box)
    gF = gF.copy()
    for t in range(T, 0, -1):
        lam, g = adjoint_step(sim, states[t - 1], lam)
        gF += g
    g_u0 = eq_vjp(sim, rho0, u0, lam)
    return L, g_u0, gF


def forward_loss(sim, rho0, u0, T, box):
    sim.init_equilibrium(rho0, u0)
    sim.step(T)
    return ke_box_loss(sim, sim.P, box)
