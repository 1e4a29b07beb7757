"""Cumulant collision from its definition (oracle; test only).

Sec. III-B, Eq. cumulant_generating_function: K(xi) = ln sum_q f_q exp(c_q.xi);
cumulants are the derivatives of K at xi = 0.  For D3Q27 the populations are
determined by the 27 raw moments with per-axis exponent <= 2, so all
arithmetic is done in the quotient ring R[xi]/(xi_x^3, xi_y^3, xi_z^3):
an element is the 27 coefficients of xi_x^a xi_y^b xi_z^c, a, b, c <= 2.
Coefficients of monomials with exponents <= 2 are exact in this ring
(exponents only add under multiplication).

Steps, in the paper's order (populations -> moments -> cumulants, relax,
back): Z = (1/rho) sum_q f_q prod_a exp(c_qa xi_a) (each factor exact since
c is in {-1,0,1}); K = ln Z = sum_{n=1..6} (-1)^{n+1} (Z-1)^n / n (the series
ends because (Z-1) has no constant term and total degree <= 6);
kappa_abc = a! b! c! [xi^abc] K.  Relaxation (reading of the unspecified
cumulant set): kappa_110, kappa_101, kappa_011, kappa_200 - kappa_020 and
kappa_200 - kappa_002 relax with omega_shear toward 0; the trace
kappa_200 + kappa_020 + kappa_002 relaxes with omega_bulk toward 3 c_s^2;
every cumulant of order >= 3 relaxes with omega_higher toward 0; rho and u
are conserved.  Back: Z' = exp(K') (finite series), raw moments
m_abc = rho a! b! c! [xi^abc] Z', and populations from the per-axis inverse
Vandermonde matrix on {-1, 0, 1} (tensor product).

Pins (tests/test_oracle_cumulant.py): round trip f -> kappa -> f; all rates 1
gives the product-form Maxwellian equilibrium rho prod_a p(c_a, u_a) with
p(+-1, u) = (cs2 + u^2 +- u)/2, p(0, u) = 1 - cs2 - u^2; conservation;
equilibrium fixed point; second-order cumulants equal the covariance of c
under f/rho computed directly; low-Re 3-D TGV decay.
"""
import itertools
from math import factorial

import numpy as np

from .lattice import CS2

CS2F = float(CS2)

EXPS = list(itertools.product(range(3), repeat=3))
IDX = {e: i for i, e in enumerate(EXPS)}
FACT = np.array([factorial(a) * factorial(b) * factorial(c) for a, b, c in EXPS], dtype=np.float64)
MUL = [(i, j, IDX[(a + x, b + y, c + z)])
       for i, (a, b, c) in enumerate(EXPS) for j, (x, y, z) in enumerate(EXPS)
       if a + x <= 2 and b + y <= 2 and c + z <= 2]


def ring_mul(A, B):
    out = np.zeros_like(A * B[:1])
    for i, j, k in MUL:
        out[k] = out[k] + A[i] * B[j]
    return out


def ring_log1p(X):
    """ln(1 + X) for X without constant term."""
    out = np.zeros_like(X)
    p = X.copy()
    for n in range(1, 7):
        out = out + ((-1) ** (n + 1) / n) * p
        p = ring_mul(p, X)
    return out


def ring_exp(K):
    """exp(K) for K without constant term."""
    out = np.zeros_like(K)
    out[IDX[(0, 0, 0)]] = 1.0
    p = K.copy()
    for n in range(1, 7):
        out = out + p / factorial(n)
        p = ring_mul(p, K)
    return out


def _exp_coeffs(c):
    """Coefficients of prod_a exp(c_a xi_a) truncated at exponent 2."""
    out = np.zeros(27)
    for i, e in enumerate(EXPS):
        v = 1.0
        for ca, ea in zip(c, e):
            v *= ca ** ea / factorial(ea)
        out[i] = v
    return out


def _vandermonde_inverse():
    V = np.array([[1.0, 1.0, 1.0], [-1.0, 0.0, 1.0], [1.0, 0.0, 1.0]])  # rows c^0,c^1,c^2; cols c=-1,0,1
    Vi = np.linalg.inv(V)
    return np.kron(np.kron(Vi, Vi), Vi)  # maps m[abc] (a-major) to f[ijk] (i-major)


_VINV = _vandermonde_inverse()


def cumulants(lat, f):
    """Return (rho, kappa[27, ...]) with kappa_000 = 0 (normalised K)."""
    E = np.stack([_exp_coeffs(c) for c in lat.c_list], axis=1)  # (27, q)
    rho = f.sum(axis=0)
    Z = np.tensordot(E, f, axes=([1], [0])) / rho
    X = Z.copy()
    X[IDX[(0, 0, 0)]] = X[IDX[(0, 0, 0)]] - 1.0
    K = ring_log1p(X)
    fact = FACT.reshape((27,) + (1,) * (f.ndim - 1))
    return rho, K * fact


def populations_from_cumulants(lat, rho, kappa):
    fact = FACT.reshape((27,) + (1,) * (kappa.ndim - 1))
    Zp = ring_exp(kappa / fact)
    m = rho * Zp * fact
    fijk = np.tensordot(_VINV, m, axes=([1], [0]))
    out = np.empty((lat.q,) + kappa.shape[1:], dtype=fijk.dtype)
    for q, c in enumerate(lat.c_list):
        out[q] = fijk[9 * (c[0] + 1) + 3 * (c[1] + 1) + (c[2] + 1)]
    return out


def relax(kappa, omegas):
    om, omb, omh = omegas[0], omegas[1], omegas[2]
    k = kappa.copy()
    i200, i020, i002 = IDX[(2, 0, 0)], IDX[(0, 2, 0)], IDX[(0, 0, 2)]
    for e in [(1, 1, 0), (1, 0, 1), (0, 1, 1)]:
        k[IDX[e]] = (1 - om) * kappa[IDX[e]]
    d1 = (1 - om) * (kappa[i200] - kappa[i020])
    d2 = (1 - om) * (kappa[i200] - kappa[i002])
    tr = kappa[i200] + kappa[i020] + kappa[i002]
    tr = tr + omb * (3 * CS2F - tr)
    k[i200] = (tr + d1 + d2) / 3
    k[i020] = (tr - 2 * d1 + d2) / 3
    k[i002] = (tr + d1 - 2 * d2) / 3
    for e in EXPS:
        if sum(e) >= 3:
            k[IDX[e]] = (1 - omh) * kappa[IDX[e]]
    return k


def collide_cumulant(lat, f, omegas):
    if lat.name != "D3Q27":
        raise ValueError("the cumulant operator is built for D3Q27 only")
    rho, kappa = cumulants(lat, f)
    return populations_from_cumulants(lat, rho, relax(kappa, omegas))
