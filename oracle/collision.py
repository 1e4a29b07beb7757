"""Equilibrium, macroscopic moments and collision operators (oracle; test only).

Arrays hold one population per row: f has shape (q, ...cells); velocities
u have shape (d, ...cells).  Everything works for float64 and for complex128
(the adjoint uses complex-step differentiation), so no abs/conj is used.

- Eq. density: rho = sum_q f_q, u = sum_q c_q f_q / rho_0, with rho_0 = rho
  (compressible) or rho_0 = 1 (incompressible, Sec. III-A).  With a body
  force F (Guo scheme, cited in Sec. I) the velocity is (sum c f + F/2)/rho_0.
- Eq. discrete_eq, second order only (the third-order term of the printed
  equation is garbled; second order suffices for Navier-Stokes, Sec. III-A):
  f^eq_q = w_q [rho + rho_0 (c.u/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2))].
- SRT, Eq. bgk: f* = f + omega (f^eq - f).
- TRT (Sec. III-C, TRT example and table): even moments relax with omega_e,
  odd ones with omega_o; in population form with f^+- = (f_q +- f_qbar)/2:
  f*_q = f_q - omega_e (f+_q - feq+_q) - omega_o (f-_q - feq-_q).
- MRT, Eq. mrt: f* = M^-1 [S m^eq + (I - S) M f] with m^eq = M f^eq, the
  basis and rates of moments.weighted_orthogonal_basis / relaxation_rates.
- Smagorinsky (Sec. III-C, turbulence models): per-cell omega from Pi^neq,
  see smagorinsky_omega.
- Entropic KBC (Sec. III-C): collide_kbc, op 'kbc' with omegas [omega_s]
  or [omega_s, omega_bulk]; omega_h per cell from the entropy condition.
- Guo forcing: raw source G_q = w_q [(c_q - u)/cs2 + (c_q.u) c_q/cs2^2].F;
  SRT adds (1 - omega/2) G, TRT adds (1 - omega_e/2) G+ + (1 - omega_o/2) G-,
  MRT adds M^-1 (I - S/2) M G.

Pins (tests/test_oracle_collision.py): moments of f^eq (rho, rho u,
rho cs2 I + rho u u) exactly; mass/momentum conservation of every operator;
f^eq is a fixed point; SRT == TRT(omega_e = omega_o) == MRT(all rates equal);
Guo momentum change equal to F; TGV viscous decay and the Poiseuille profile
(tests/test_oracle_flows.py).
"""
import numpy as np

from . import moments as mo
from .lattice import CS2

CS2F = float(CS2)


def _cdot(lat, vec):
    """c_q . vec for every q; vec has shape (d, ...)."""
    return np.tensordot(lat.c.astype(np.float64), vec, axes=([1], [0]))


def density(f):
    return f.sum(axis=0)


def momentum(lat, f):
    return np.tensordot(lat.c.T.astype(np.float64), f, axes=([1], [0]))


def _force_array(lat, force, like):
    if force is None:
        return None
    F = np.asarray(force)
    return F.reshape((lat.d,) + (1,) * (like.ndim - 1)) * np.ones_like(like[: lat.d])


def velocity(lat, f, force=None, incompressible=False):
    rho = density(f)
    j = momentum(lat, f)
    if force is not None:
        j = j + 0.5 * _force_array(lat, force, f)
    rho0 = 1.0 if incompressible else rho
    return rho, j / rho0


def equilibrium(lat, rho, u, incompressible=False):
    rho0 = 1.0 if incompressible else rho
    cu = _cdot(lat, u)
    usq = (u * u).sum(axis=0)
    w = lat.w.reshape((lat.q,) + (1,) * (cu.ndim - 1))
    return w * (rho + rho0 * (cu / CS2F + cu * cu / (2 * CS2F * CS2F) - usq / (2 * CS2F)))


def guo_source(lat, u, force):
    F = _force_array(lat, force, u)
    cF = _cdot(lat, F)
    cu = _cdot(lat, u)
    uF = (u * F).sum(axis=0)
    w = lat.w.reshape((lat.q,) + (1,) * (cu.ndim - 1))
    return w * ((cF - uF) / CS2F + cu * cF / (CS2F * CS2F))


def trt_odd_rate(omega_e, magic):
    """omega_o from the magic parameter Lambda = (1/omega_e - 1/2)(1/omega_o - 1/2)."""
    return 1.0 / (magic / (1.0 / omega_e - 0.5) + 0.5)


def smagorinsky_omega(lat, f, feq, rho, omega0, cs):
    """Per-cell relaxation rate of the Smagorinsky model (Sec. III-C,
    "Turbulence models"): nu = nu_0 + (C_S Delta)^2 |S| with Delta = 1,
    |S| = sqrt(2 S_ij S_ij), S_ij = -(3 omega / (2 rho)) Pi^neq_ij,
    Pi^neq_ij = sum_q c_qi c_qj (f_q - f^eq_q), omega = 2 / (6 C_S^2 |S| + 6 nu_0 + 1).
    With P = sqrt(2 Pi^neq : Pi^neq) the pair is solved for tau = 1/omega:
    2 tau^2 - 2 tau_0 tau - 9 C_S^2 P / rho = 0 (positive root)."""
    c = lat.c.astype(np.float64)
    fneq = f - feq
    pp = 0.0
    for a in range(lat.d):
        for b in range(lat.d):
            pab = np.tensordot(c[:, a] * c[:, b], fneq, axes=([0], [0]))
            pp = pp + pab * pab
    P = np.sqrt(2.0 * pp)
    tau0 = 1.0 / omega0
    tau = 0.5 * (tau0 + np.sqrt(tau0 * tau0 + 18.0 * cs * cs * P / rho))
    return 1.0 / tau


class Method:
    """A collision operator with its parameters.

    op: 'srt' (omegas=[omega]), 'trt' ([omega_e, omega_o]), 'mrt'
    ([omega_shear, omega_bulk, omega_3, omega_4(, omega_5, omega_6)]) or
    'cumulant' ([omega_shear, omega_bulk, omega_higher]) or 'kbc'
    ([omega_shear(, omega_bulk)], omega_h chosen per cell).
    cs > 0 adds the Smagorinsky model to SRT/TRT: the (even) rate becomes the
    per-cell smagorinsky_omega; with magic set, the TRT odd rate follows it
    through Lambda = magic, otherwise omega_o stays as given.
    """

    def __init__(self, lat, op, omegas, incompressible=False, force=None, cs=0.0, magic=None):
        self.lat = lat
        self.op = op
        self.omegas = list(omegas)
        self.incompressible = incompressible
        self.force = None if force is None else np.asarray(force)
        self.cs = float(cs)
        self.magic = magic
        if op in ("mrt", "kbc"):
            basis = mo.weighted_orthogonal_basis(lat)
            Mx = mo.moment_matrix(basis, lat)
            self.basis = basis
            self.M = np.array([[float(v) for v in r] for r in Mx])
            self.Minv = np.array([[float(v) for v in r] for r in mo.exact_inverse(Mx)])
            self.s = np.array(mo.relaxation_rates(basis, self.omegas + [1.0] * 6))

    def with_force(self, force):
        m = Method.__new__(Method)
        m.__dict__.update(self.__dict__)
        m.force = None if force is None else np.asarray(force)
        return m


def _pm(lat, f):
    fb = f[lat.opp]
    return 0.5 * (f + fb), 0.5 * (f - fb)


def collide(method, f):
    """Post-collision populations for pre-collision populations f."""
    lat = method.lat
    if method.op == "cumulant":
        from .cumulant import collide_cumulant
        if method.force is not None:
            raise ValueError("cumulant collision with a body force is not defined here")
        return collide_cumulant(lat, f, method.omegas)
    rho, u = velocity(lat, f, method.force, method.incompressible)
    feq = equilibrium(lat, rho, u, method.incompressible)
    G = guo_source(lat, u, method.force) if method.force is not None else None
    if method.cs > 0.0 and method.op in ("srt", "trt"):
        om = smagorinsky_omega(lat, f, feq, density(f), method.omegas[0], method.cs)
        if method.op == "srt":
            oo = om
        elif method.magic is not None:
            oo = 1.0 / (method.magic / (1.0 / om - 0.5) + 0.5)
        else:
            oo = method.omegas[1]
        fp, fm = _pm(lat, f)
        ep, em = _pm(lat, feq)
        out = f - om * (fp - ep) - oo * (fm - em)
        if G is not None:
            gp, gm = _pm(lat, G)
            out = out + (1 - om / 2) * gp + (1 - oo / 2) * gm
        return out
    if method.op == "kbc":
        return collide_kbc(method, f, feq)
    if method.op == "srt":
        om = method.omegas[0]
        out = f + om * (feq - f)
        if G is not None:
            out = out + (1 - om / 2) * G
        return out
    if method.op == "trt":
        oe, oo = method.omegas[0], method.omegas[1]
        fp, fm = _pm(lat, f)
        ep, em = _pm(lat, feq)
        out = f - oe * (fp - ep) - oo * (fm - em)
        if G is not None:
            gp, gm = _pm(lat, G)
            out = out + (1 - oe / 2) * gp + (1 - oo / 2) * gm
        return out
    if method.op == "mrt":
        M, Minv = method.M, method.Minv
        S = method.s.reshape((-1,) + (1,) * (f.ndim - 1))
        m = np.tensordot(M, f, axes=([1], [0]))
        meq = np.tensordot(M, feq, axes=([1], [0]))
        mstar = S * meq + (1 - S) * m
        if G is not None:
            mstar = mstar + (1 - S / 2) * np.tensordot(M, G, axes=([1], [0]))
        return np.tensordot(Minv, mstar, axes=([1], [0]))
    raise ValueError(method.op)


def kbc_parts(method, f, feq):
    """(Delta s, Delta b, Delta h): the non-equilibrium part f - f^eq projected
    onto the moment groups of the w-orthogonal MRT basis (Eq. mrt): shear
    (the traceless second-order moments), bulk (the trace) and h (every
    moment of order >= 3), so that f = f^eq + Delta s + Delta b + Delta h."""
    M, Minv = method.M, method.Minv
    kinds = [m.kind for m in method.basis]
    m = np.tensordot(M, f - feq, axes=([1], [0]))
    out = []
    for group in (("shear",), ("bulk",), ("higher",)):
        sel = np.array([1.0 if k in group else 0.0 for k in kinds]).reshape((-1,) + (1,) * (f.ndim - 1))
        out.append(np.tensordot(Minv, sel * m, axes=([1], [0])))
    return tuple(out)


def kbc_omega_h(method, f, feq):
    """omega_h from the paper's linearised optimality condition
    sum_q Delta h_q f'_q / f^eq_q = 0 (Sec. III-C, entropic KBC), with
    f' = f - omega_s Delta s - omega_b Delta b - omega_h Delta h:
    omega_h = 1 + [(1 - omega_s) <Ds, Dh>_E + (1 - omega_b) <Db, Dh>_E] / <Dh, Dh>_E,
    <a, b>_E = sum_q a_q b_q / f^eq_q.  For omega_b = omega_s this is
    Eq. entropic_direct_omega_eq with Delta s + Delta b in the role of the
    paper's Delta s.  Where <Dh, Dh>_E <= 1e-30 (no higher-order
    deviation to tune) omega_h = 1."""
    om_s, om_b = method.omegas[0], method.omegas[1] if len(method.omegas) > 1 else method.omegas[0]
    ds, db, dh = kbc_parts(method, f, feq)
    num = (1.0 - om_s) * (ds * dh / feq).sum(axis=0) + (1.0 - om_b) * (db * dh / feq).sum(axis=0)
    den = (dh * dh / feq).sum(axis=0)
    safe = den > 1e-30
    return np.where(safe, 1.0 + num / np.where(safe, den, 1.0), 1.0), (ds, db, dh)


def collide_kbc(method, f, feq):
    """Entropic KBC (Sec. III-C, Eq. entropic_linear_update extended by a
    fixed bulk rate): f' = f - omega_s Delta s - omega_b Delta b - omega_h Delta h,
    omega_h per cell from kbc_omega_h.  omegas = [omega_s] or [omega_s, omega_b];
    a body force is not defined for this operator."""
    if method.force is not None:
        raise ValueError("KBC collision with a body force is not defined here")
    om_s, om_b = method.omegas[0], method.omegas[1] if len(method.omegas) > 1 else method.omegas[0]
    om_h, (ds, db, dh) = kbc_omega_h(method, f, feq)
    return f - om_s * ds - om_b * db - om_h * dh
