"""Moment polynomials and the automatic MRT moment basis (oracle; test only).

Follows Sec. III-A "Moment Space" step by step, in exact rational arithmetic:

1. Moments are polynomials P(c_q) in the lattice velocity components; the
   moment value is Pi_P(f) = sum_q P(c_q) f_q (Eq. disrete_moment_def) and
   M_kq = P_k(c_q).
2. Because c_qi is in {-1, 0, 1}, c^3 aliases c and even powers >= 4 alias
   c^2, so candidate monomials are x^e0 y^e1 z^e2 with e_i in {0, 1, 2}
   (27 in 3-D, 9 in 2-D).  Monomials whose row of M is zero are discarded
   (8 of 27 for D3Q19).
3. The candidates are sorted by order, then lexicographically.
4. The second-order diagonal monomials are split into one bulk moment
   (x^2 + y^2 [+ z^2]) and traceless shear differences before
   orthogonalisation (the MRT example of Sec. III-C).
5. Gram-Schmidt with the standard or the w_q-weighted scalar product
   <a, b> = sum_q w_q a(c_q) b(c_q).
6. Relaxation rates as in the MRT example: order < 2 -> 0, shear -> omega_0,
   bulk -> omega_1, order k >= 3 -> omega_{k-1}.

Equilibrium moments from the continuous Maxwellian (Eqs. cont_maxwellian,
cont_moment_integral): each axis is a normal law with mean u_a and variance
c_s^2, so E[xi^0] = 1, E[xi] = u, E[xi^2] = c_s^2 + u^2; the result is
optionally truncated in u.  Polynomials in (rho, u) are dicts keyed by the
exponent tuple (p_rho, p_u0, p_u1[, p_u2]).

Pins: tests/test_oracle_moments.py (the D2Q9 TRT and weighted-MRT tables of
Sec. III-C reproduced exactly; 8 zero rows for D3Q19; aliasing c^3 = c;
Maxwellian moments equal M f^eq for D2Q9/D3Q27; invertibility; weighted
orthogonality).
"""
import itertools
from fractions import Fraction as Fr
from math import gcd

from .lattice import CS2

# ---------------------------------------------------------------- polynomials


def mono(exps):
    return {tuple(exps): Fr(1)}


def padd(a, b, sb=Fr(1)):
    out = dict(a)
    for k, v in b.items():
        out[k] = out.get(k, Fr(0)) + sb * v
        if out[k] == 0:
            del out[k]
    return out


def pscale(a, s):
    return {k: v * s for k, v in a.items() if v * s != 0}


def peval(poly, c):
    """Value of a velocity polynomial at one lattice velocity c."""
    tot = Fr(0)
    for exps, coef in poly.items():
        term = coef
        for ci, e in zip(c, exps):
            term *= Fr(ci) ** e
        tot += term
    return tot


def porder(poly):
    return max(sum(e) for e in poly)


def prow(poly, lat):
    return [peval(poly, c) for c in lat.c_list]


def normalise(poly):
    """Scale to a primitive integer polynomial whose leading monomial (highest
    order, then lexicographically first) has a positive coefficient."""
    den = 1
    for v in poly.values():
        den = den * v.denominator // gcd(den, v.denominator)
    ints = {k: int(v * den) for k, v in poly.items()}
    g = 0
    for v in ints.values():
        g = gcd(g, abs(v))
    lead = sorted(ints, key=lambda e: (-sum(e), [-x for x in e]))[0]
    sgn = 1 if ints[lead] > 0 else -1
    return {k: Fr(sgn * v, g) for k, v in ints.items()}


# ------------------------------------------------------------ basis building


class Moment:
    """A moment polynomial with its bookkeeping class.

    kind is one of 'conserved' (order < 2), 'shear', 'bulk', 'higher'.
    """

    def __init__(self, poly, kind):
        self.poly = poly
        self.kind = kind

    @property
    def order(self):
        return porder(self.poly)

    def is_even(self):
        return all(sum(e) % 2 == 0 for e in self.poly)


def _sort_key(exps):
    return (sum(exps), [-e for e in exps])


def independent_raw_moments(lat):
    """Step 2-3: monomials with e_i <= 2 giving a non-zero row, sorted by order
    then lexicographically (x before y before z, higher power first)."""
    out = []
    for exps in itertools.product(range(3), repeat=lat.d):
        row = prow(mono(exps), lat)
        if any(v != 0 for v in row):
            out.append(exps)
    out.sort(key=_sort_key)
    return [Moment(mono(e), "conserved" if sum(e) < 2 else "higher") for e in out]


def zero_row_monomials(lat):
    out = []
    for exps in itertools.product(range(3), repeat=lat.d):
        if all(v == 0 for v in prow(mono(exps), lat)):
            out.append(exps)
    return out


def split_shear_bulk(moments, d):
    """Step 4: replace x^2, y^2 (, z^2) by shear differences x^2 - y^2
    (, x^2 - z^2) and the bulk sum, keep the mixed second-order monomials as
    shear moments.  The order-2 block becomes: diagonal differences, mixed
    monomials, bulk."""
    diag = [tuple(2 if i == a else 0 for i in range(d)) for a in range(d)]
    lower = [m for m in moments if m.order < 2]
    second = [m for m in moments if m.order == 2]
    higher = [m for m in moments if m.order > 2]
    present = [k for m in second for k in m.poly]
    assert all(e in present for e in diag), "stencil lacks a diagonal second moment"
    mixed = [m for m in second if list(m.poly)[0] not in diag]
    shear_diag = [Moment(padd(mono(diag[0]), mono(diag[a]), Fr(-1)), "shear")
                  for a in range(1, d)]
    bulk = {}
    for e in diag:
        bulk = padd(bulk, mono(e))
    block = shear_diag + [Moment(m.poly, "shear") for m in mixed] + [Moment(bulk, "bulk")]
    return lower + block + higher


def inner(a, b, lat, weighted):
    ra, rb = prow(a, lat), prow(b, lat)
    if weighted:
        return sum(w * x * y for w, x, y in zip(lat.w_exact, ra, rb))
    return sum(x * y for x, y in zip(ra, rb))


def gram_schmidt(moments, lat, weighted=True):
    """Step 5: classical Gram-Schmidt in list order, each result normalised
    to a primitive integer polynomial (scaling does not change the MRT
    operator)."""
    done = []
    for m in moments:
        p = dict(m.poly)
        for prev in done:
            num = inner(m.poly, prev.poly, lat, weighted)
            if num != 0:
                p = padd(p, prev.poly, -num / inner(prev.poly, prev.poly, lat, weighted))
        done.append(Moment(normalise(p), m.kind))
    return done


def weighted_orthogonal_basis(lat):
    """The weighted-orthogonal MRT basis of the Sec. III-C MRT example."""
    return gram_schmidt(split_shear_bulk(independent_raw_moments(lat), lat.d), lat, True)


def relaxation_rates(moments, omegas):
    """Step 6.  omegas = [omega_shear, omega_bulk, omega_3, omega_4, ...]."""
    out = []
    for m in moments:
        if m.order < 2:
            out.append(0.0)
        elif m.kind == "shear":
            out.append(omegas[0])
        elif m.kind == "bulk":
            out.append(omegas[1])
        else:
            out.append(omegas[m.order - 1])
    return out


# ------------------------------------------------------------- exact matrices


def moment_matrix(moments, lat):
    return [prow(m.poly, lat) for m in moments]


def exact_inverse(mat):
    """Gauss-Jordan elimination over the rationals; raises if singular."""
    n = len(mat)
    a = [list(row) + [Fr(int(i == j)) for j in range(n)] for i, row in enumerate(mat)]
    for col in range(n):
        piv = next((r for r in range(col, n) if a[r][col] != 0), None)
        if piv is None:
            raise ValueError("moment matrix is singular")
        a[col], a[piv] = a[piv], a[col]
        pv = a[col][col]
        a[col] = [v / pv for v in a[col]]
        for r in range(n):
            if r != col and a[r][col] != 0:
                fac = a[r][col]
                a[r] = [x - fac * y for x, y in zip(a[r], a[col])]
    return [row[n:] for row in a]


# ------------------------------------------- equilibrium moments (symbolic u)


def _rp_mul(a, b):
    out = {}
    for ka, va in a.items():
        for kb, vb in b.items():
            k = tuple(x + y for x, y in zip(ka, kb))
            out[k] = out.get(k, Fr(0)) + va * vb
    return {k: v for k, v in out.items() if v != 0}


def _u_power(d, axis, p):
    k = [0] * (d + 1)
    k[1 + axis] = p
    return tuple(k)


def maxwellian_moment(poly, d, max_u_order=None):
    """rho * E[P(xi)] for xi ~ N(u, c_s^2 I) (Eq. cont_moment_integral), as a
    polynomial in (rho, u); optionally truncated at total u-degree."""
    total = {}
    for exps, coef in poly.items():
        term = {tuple([1] + [0] * d): coef}
        for axis, e in enumerate(exps):
            if e == 0:
                axis_m = {tuple([0] * (d + 1)): Fr(1)}
            elif e == 1:
                axis_m = {_u_power(d, axis, 1): Fr(1)}
            elif e == 2:
                axis_m = {tuple([0] * (d + 1)): CS2, _u_power(d, axis, 2): Fr(1)}
            else:
                raise ValueError("exponent > 2 never occurs after aliasing")
            term = _rp_mul(term, axis_m)
        total = padd(total, term)
    if max_u_order is not None:
        total = {k: v for k, v in total.items() if sum(k[1:]) <= max_u_order}
    return total


def discrete_equilibrium_poly(lat, q, incompressible=False):
    """Second-order Eq. discrete_eq for direction q as a polynomial in
    (rho, u): w_q [rho + rho0 (c.u/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2))]."""
    d = lat.d
    c = lat.c_list[q]
    w = lat.w_exact[q]
    r0 = (0 if incompressible else 1,)
    out = {tuple([1] + [0] * d): w}
    for a in range(d):
        if c[a] != 0:
            out = padd(out, {r0 + _u_power(d, a, 1)[1:]: w * c[a] / CS2})
    for a in range(d):
        for b in range(d):
            coef = Fr(c[a] * c[b]) / (2 * CS2 * CS2)
            if a == b:
                coef -= Fr(1) / (2 * CS2)
            if coef != 0:
                k = [0] * d
                k[a] += 1
                k[b] += 1
                out = padd(out, {r0 + tuple(k): w * coef})
    return out


def discrete_equilibrium_moment(poly, lat, incompressible=False):
    """sum_q P(c_q) f^eq_q as a polynomial in (rho, u)."""
    total = {}
    for q in range(lat.q):
        pv = peval(poly, lat.c_list[q])
        if pv != 0:
            total = padd(total, pscale(discrete_equilibrium_poly(lat, q, incompressible), pv))
    return total


def to_incompressible(rpoly):
    """Sec. III-C: set rho = 1 in every term containing a velocity."""
    out = {}
    for k, v in rpoly.items():
        nk = k if sum(k[1:]) == 0 else (0,) + k[1:]
        out[nk] = out.get(nk, Fr(0)) + v
    return {k: v for k, v in out.items() if v != 0}
