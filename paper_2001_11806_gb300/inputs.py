"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds no lattice Boltzmann arithmetic: it only draws numbers and
builds initial fields and geometry.  Random numbers come from SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): state_i = seed + (i + 1) * 0x9E3779B97F4A7C15, then the mix
z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
z ^= z >> 31.  A double in [0, 1) is (z >> 11) * 2^-53.

Workloads (shapes follow the paper's periodic and channel benchmarks):
- ``tgv2d``: 2-D Taylor-Green vortex, nodes at integer coordinates,
  k = 2 pi / N, u_x = -u0 cos(kx) sin(ky), u_y = u0 sin(kx) cos(ky), rho = 1.
- ``tgv3d``: u = u0 sin(kx) cos(ky) cos(kz), v = -u0 cos(kx) sin(ky) cos(kz),
  w = 0, rho = 1, plus additive U(-a, a) noise per component per cell.
- ``channel_flags``: box with no-slip layers at y, z = 0 and n-1, an inlet
  layer at x = 0 and an outlet layer at x = nx-1 (interior y, z), and random
  spheres (integer centres uniform in x in [32, nx-32), y, z in [1, n-1),
  integer radius uniform in [rmin, rmax]) until the interior solid fraction
  reaches 1 - porosity.
- ``random_pdfs``: positive populations base_q * (1 + amp * U(-1, 1)).
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

FLUID, NOSLIP, INLET, OUTLET = 0, 1, 2, 4


def splitmix64(seed, n, offset=0):
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def uniform(seed, n, offset=0):
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def tgv2d(n, u0):
    k = 2 * np.pi / n
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")  # [y][x]
    ux = -u0 * np.cos(k * X) * np.sin(k * Y)
    uy = u0 * np.sin(k * X) * np.cos(k * Y)
    rho = np.ones((1, n, n))
    return rho, np.stack([ux, uy])[:, None]


def tgv3d(n, u0, noise=0.0, seed=42):
    k = 2 * np.pi / n
    x = np.arange(n, dtype=np.float64)
    sx, cx = np.sin(k * x), np.cos(k * x)
    u = np.empty((3, n, n, n))  # [comp][z][y][x]
    u[0] = u0 * (cx[:, None, None] * cx[None, :, None]) * sx[None, None, :]
    u[1] = -u0 * (cx[:, None, None] * sx[None, :, None]) * cx[None, None, :]
    u[2] = 0.0
    if noise:
        N = n ** 3
        for comp in range(3):
            u[comp] += (2.0 * uniform(seed, N, comp * N) - 1.0).reshape(n, n, n) * noise
    return np.ones((n, n, n)), u


def channel_flags(nx, ny, nz, seed=1234, porosity=0.8, rmin=4, rmax=10, margin=32):
    flags = np.zeros((nz, ny, nx), dtype=np.uint8)
    interior = np.zeros_like(flags, dtype=bool)
    interior[1:nz - 1, 1:ny - 1, 1:nx - 1] = True
    n_int = int(interior.sum())
    solid = np.zeros_like(interior)
    target = 1.0 - porosity
    k = 0
    zz, yy, xx = np.arange(nz), np.arange(ny), np.arange(nx)
    while solid[interior].sum() < target * n_int:
        r4 = uniform(seed, 4, 4 * k)
        k += 1
        cx = margin + int(r4[0] * (nx - 2 * margin))
        cy = 1 + int(r4[1] * (ny - 2))
        cz = 1 + int(r4[2] * (nz - 2))
        r = rmin + int(r4[3] * (rmax - rmin + 1))
        x0, x1 = max(cx - r, 0), min(cx + r + 1, nx)
        y0, y1 = max(cy - r, 0), min(cy + r + 1, ny)
        z0, z1 = max(cz - r, 0), min(cz + r + 1, nz)
        d2 = ((zz[z0:z1, None, None] - cz) ** 2 + (yy[None, y0:y1, None] - cy) ** 2
              + (xx[None, None, x0:x1] - cx) ** 2)
        solid[z0:z1, y0:y1, x0:x1] |= d2 <= r * r
    solid &= interior
    flags[solid] = NOSLIP
    flags[:, :, 0] = INLET
    flags[:, :, nx - 1] = OUTLET
    flags[:, 0, :] = NOSLIP
    flags[:, ny - 1, :] = NOSLIP
    flags[0, :, :] = NOSLIP
    flags[nz - 1, :, :] = NOSLIP
    return flags


def random_pdfs(base, shape3, amp=0.2, seed=7):
    q = len(base)
    N = int(np.prod(shape3))
    r = 2.0 * uniform(seed, q * N) - 1.0
    return (np.asarray(base, dtype=np.float64)[:, None] * (1.0 + amp * r.reshape(q, N))).reshape((q,) + tuple(shape3))


def random_fields(shape3, d, amp_rho=0.01, amp_u=0.03, seed=11):
    N = int(np.prod(shape3))
    rho = 1.0 + amp_rho * (2.0 * uniform(seed, N) - 1.0)
    u = amp_u * (2.0 * uniform(seed + 1, d * N) - 1.0)
    return rho.reshape(shape3), u.reshape((d,) + tuple(shape3))
