"""Pins for oracle.lattice: isotropy of the weights (exact rationals), the
opposite-pair rule of the direction order, tensor-product weights."""
import itertools
from fractions import Fraction as Fr

import pytest

from oracle import lattice

CS2 = Fr(1, 3)
NAMES = ["D2Q9", "D3Q19", "D3Q27"]


@pytest.mark.parametrize("name", NAMES)
def test_isotropy_to_fourth_order(name):
    lat = lattice.get(name)
    d, w, cs = lat.d, lat.w_exact, lat.c_list
    assert sum(w) == 1
    rng = range(d)
    for a in rng:
        assert sum(wq * c[a] for wq, c in zip(w, cs)) == 0
    for a, b in itertools.product(rng, rng):
        assert sum(wq * c[a] * c[b] for wq, c in zip(w, cs)) == (CS2 if a == b else 0)
    for a, b, g in itertools.product(rng, rng, rng):
        assert sum(wq * c[a] * c[b] * c[g] for wq, c in zip(w, cs)) == 0
    for a, b, g, e in itertools.product(rng, rng, rng, rng):
        lhs = sum(wq * c[a] * c[b] * c[g] * c[e] for wq, c in zip(w, cs))
        rhs = CS2 * CS2 * (int(a == b and g == e) + int(a == g and b == e) + int(a == e and b == g))
        assert lhs == rhs, (a, b, g, e)


@pytest.mark.parametrize("name,q", [("D2Q9", 9), ("D3Q19", 19), ("D3Q27", 27)])
def test_pairs_and_order(name, q):
    lat = lattice.get(name)
    assert lat.q == q and len(set(lat.c_list)) == q
    assert lat.c_list[0] == (0,) * lat.d
    for i in range(1, q):
        j = i + 1 if i % 2 == 1 else i - 1
        assert lat.opp[i] == j
        assert tuple(-x for x in lat.c_list[i]) == lat.c_list[j]
    # faces, then edges, then corners
    nz = [sum(abs(x) for x in c) for c in lat.c_list]
    assert nz == sorted(nz)


def test_weight_values():
    d19 = lattice.d3q19()
    assert d19.w_exact[0] == Fr(1, 3) and set(d19.w_exact[1:7]) == {Fr(1, 18)}
    assert set(d19.w_exact[7:]) == {Fr(1, 36)}
    d27 = lattice.d3q27()
    assert sorted(set(d27.w_exact)) == [Fr(1, 216), Fr(1, 54), Fr(2, 27), Fr(8, 27)]
    d9 = lattice.d2q9()
    assert sorted(set(d9.w_exact)) == [Fr(1, 36), Fr(1, 9), Fr(4, 9)]
