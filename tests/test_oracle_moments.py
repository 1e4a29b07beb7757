"""Pins for oracle.moments: the two D2Q9 tables printed in Sec. III-C
(tests/golden), the D3Q19 zero-row count, aliasing, Maxwellian vs discrete
equilibrium moments, weighted orthogonality."""
import os
import random
from fractions import Fraction as Fr

import pytest

from oracle import lattice
from oracle import moments as mo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([s.strip() for s in line.split(";")])
    return rows


def _points(n, k, seed):
    r = random.Random(seed)
    return [[Fr(r.randint(-50, 50), r.randint(1, 13)) for _ in range(k)] for _ in range(n)]


def _eval_text(expr, env):
    return eval(expr, {"__builtins__": {}}, dict(env))  # committed fixture text only


def _eval_vpoly(poly, x, y):
    return mo.peval(poly, (x, y))


def _eval_rpoly(rp, rho, u):
    tot = Fr(0)
    for k, v in rp.items():
        t = v * rho ** k[0]
        for a, e in enumerate(k[1:]):
            t *= u[a] ** e
        tot += t
    return tot


def _same_vpoly(poly, text):
    return all(_eval_vpoly(poly, x, y) == _eval_text(text, {"x": x, "y": y})
               for x, y in _points(12, 2, 1))


def _same_rpoly(rp, text):
    return all(_eval_rpoly(rp, r, (a, b)) == _eval_text(text, {"rho": r, "u0": a, "u1": b})
               for r, a, b in _points(12, 3, 2))


def test_d2q9_trt_table():
    lat = lattice.d2q9()
    rows = _read_table("d2q9_trt_table.txt")
    moms = mo.independent_raw_moments(lat)
    assert len(moms) == len(rows) == 9
    for mtext, eqtext, rate in rows:
        match = [m for m in moms if _same_vpoly(m.poly, mtext)]
        assert len(match) == 1, mtext
        m = match[0]
        # equilibrium from the continuous Maxwellian, truncated to second order
        assert _same_rpoly(mo.maxwellian_moment(m.poly, 2, max_u_order=2), eqtext), mtext
        # ... and equal to the moment of the discrete equilibrium (Sec. III-A)
        assert _same_rpoly(mo.discrete_equilibrium_moment(m.poly, lat), eqtext), mtext
        assert ("we" if m.is_even() else "wo") == rate, mtext


def test_d2q9_weighted_mrt_table():
    lat = lattice.d2q9()
    rows = _read_table("d2q9_mrt_table.txt")
    basis = mo.weighted_orthogonal_basis(lat)
    assert len(basis) == len(rows)
    names = {"0": 0.0, "w0": 0.11, "w1": 0.22, "w2": 0.33, "w3": 0.44}
    rates = mo.relaxation_rates(basis, [0.11, 0.22, 0.33, 0.44])
    for (mtext, eqtext, rate), m, s in zip(rows, basis, rates):
        assert _same_vpoly(m.poly, mtext), (m.poly, mtext)
        eq = mo.to_incompressible(mo.discrete_equilibrium_moment(m.poly, lat))
        assert _same_rpoly(eq, eqtext), mtext
        assert s == names[rate]


def test_d3q19_zero_rows_and_aliasing():
    lat = lattice.d3q19()
    zero = mo.zero_row_monomials(lat)
    assert len(zero) == 8
    assert (1, 1, 1) in zero and (2, 1, 1) in zero
    assert len(mo.independent_raw_moments(lat)) == 19
    for lat in [lattice.d2q9(), lattice.d3q19(), lattice.d3q27()]:
        for a in range(lat.d):
            e1 = tuple(1 if i == a else 0 for i in range(lat.d))
            e3 = tuple(3 if i == a else 0 for i in range(lat.d))
            e4 = tuple(4 if i == a else 0 for i in range(lat.d))
            e2 = tuple(2 if i == a else 0 for i in range(lat.d))
            assert mo.prow(mo.mono(e3), lat) == mo.prow(mo.mono(e1), lat)
            assert mo.prow(mo.mono(e4), lat) == mo.prow(mo.mono(e2), lat)


@pytest.mark.parametrize("name,equal", [("D2Q9", True), ("D3Q27", True), ("D3Q19", False)])
def test_maxwellian_vs_discrete_equilibrium(name, equal):
    lat = lattice.get(name)
    same = all(
        mo.maxwellian_moment(m.poly, lat.d, max_u_order=2) == mo.discrete_equilibrium_moment(m.poly, lat)
        for m in mo.independent_raw_moments(lat))
    assert same == equal


@pytest.mark.parametrize("name,q", [("D2Q9", 9), ("D3Q19", 19), ("D3Q27", 27)])
def test_basis_orthogonal_and_invertible(name, q):
    lat = lattice.get(name)
    basis = mo.weighted_orthogonal_basis(lat)
    assert len(basis) == q
    M = mo.moment_matrix(basis, lat)
    for i in range(q):
        for j in range(i):
            assert sum(w * a * b for w, a, b in zip(lat.w_exact, M[i], M[j])) == 0
    Mi = mo.exact_inverse(M)
    for i in range(q):
        for j in range(q):
            assert sum(M[i][k] * Mi[k][j] for k in range(q)) == (1 if i == j else 0)
    kinds = [m.kind for m in basis]
    assert kinds.count("bulk") == 1
    assert kinds.count("shear") == (2 if lat.d == 2 else 5)
    assert kinds.count("conserved") == 1 + lat.d
