"""DdQq lattice velocity sets and weights (oracle; test infrastructure only).

Sec. III-A: a DdQq stencil is a list of q integer lattice velocities with
components in {-1, 0, 1}; populations f_q travel along c_q.  The speed of
sound is c_s^2 = 1/3 for first-neighbourhood stencils (Sec. III-A,
"Equilibrium State").  D2Q9 and D3Q27 are Cartesian products of the 1-D
three-velocity set; the D3Q19 weights are the standard ones obtained by
Hermite projection (same subsection).

Direction order (shared interface with the C ABI, written out independently
here): index 0 is the rest velocity; then opposite pairs (2k-1, 2k) in the
order faces (+x,-x,+y,-y,+z,-z), edges per axis pair (xy, xz, yz; signs
(+,+),(-,-),(+,-),(-,+)), corners ((+,+,+),(-,-,-)), ((+,+,-),(-,-,+)),
((+,-,+),(-,+,-)), ((-,+,+),(+,-,-)).

Pins: tests/test_oracle_lattice.py (isotropy to fourth order in exact
rationals, opposite pairs, tensor-product weights).
"""
from fractions import Fraction as Fr

import numpy as np

CS2 = Fr(1, 3)

_FACES3 = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
_EDGES3 = [(1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
           (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
           (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
_CORNERS3 = [(1, 1, 1), (-1, -1, -1), (1, 1, -1), (-1, -1, 1),
             (1, -1, 1), (-1, 1, -1), (-1, 1, 1), (1, -1, -1)]
_FACES2 = [(1, 0), (-1, 0), (0, 1), (0, -1)]
_EDGES2 = [(1, 1), (-1, -1), (1, -1), (-1, 1)]

_W1D = {0: Fr(2, 3), 1: Fr(1, 6), -1: Fr(1, 6)}


class Lattice:
    """Velocity set: ``c`` (q, d) int array, ``w`` exact weights, ``opp``."""

    def __init__(self, name, vels, weights):
        self.name = name
        self.c_list = [tuple(v) for v in vels]
        self.q = len(vels)
        self.d = len(vels[0])
        self.c = np.array(vels, dtype=np.int64)
        self.w_exact = list(weights)
        self.w = np.array([float(x) for x in weights])
        self.opp = np.array([self.c_list.index(tuple(-x for x in v)) for v in self.c_list])

    def __repr__(self):
        return f"Lattice({self.name})"


def _product_weights(vels):
    out = []
    for v in vels:
        w = Fr(1)
        for comp in v:
            w *= _W1D[comp]
        out.append(w)
    return out


def d2q9():
    vels = [(0, 0)] + _FACES2 + _EDGES2
    return Lattice("D2Q9", vels, _product_weights(vels))


def d3q19():
    vels = [(0, 0, 0)] + _FACES3 + _EDGES3
    w = [Fr(1, 3)] + [Fr(1, 18)] * 6 + [Fr(1, 36)] * 12
    return Lattice("D3Q19", vels, w)


def d3q27():
    vels = [(0, 0, 0)] + _FACES3 + _EDGES3 + _CORNERS3
    return Lattice("D3Q27", vels, _product_weights(vels))


def get(name):
    return {"D2Q9": d2q9, "D3Q19": d3q19, "D3Q27": d3q27}[name]()
