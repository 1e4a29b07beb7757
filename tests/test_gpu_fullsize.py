"""Parity at the full workload sizes, on sampled cells.

The GPU runs the whole domain in the configuration the benchmark times; the
oracle recomputes each sampled cell on its own: after s steps a cell's
populations depend only on initial values within s + 1 cells (s pulls plus
the final streaming of the output), so the oracle steps a (2s + 3)^3 box cut
from the same seeded initial fields around the cell.  The box edges are wrong
(wrapped), but that error travels one cell per step and never reaches the
centre.  Tolerances as in test_gpu_parity.py: FP32 1e-5, FP16-shifted 5e-3,
relative L2 of f - f_ref over the sampled cells against ||f_ref - w||, and
for FP16-shifted storage also element-wise, 3 * 2^-11 max|f_ref - w|."""
import numpy as np
import pytest
import torch

from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import inputs
from paper_2001_11806_gb300.sim import Sim

pytestmark = pytest.mark.gpu


def _sample_cells(shape, n, seed, fluid=None):
    nx, ny, nz = shape
    r = inputs.uniform(seed, 3 * 4 * n)
    cells = []
    for i in range(4 * n):
        c = (int(r[3 * i] * nx), int(r[3 * i + 1] * ny), int(r[3 * i + 2] * nz))
        if fluid is None or fluid[c[2], c[1], c[0]]:
            cells.append(c)
        if len(cells) == n:
            break
    return cells


def _cut(arr, c, h, shape, periodic):
    """arr [..., z, y, x] -> the (2h+1)^3 block around cell c; outside a
    non-periodic axis the block is filled with edge values (the caller marks
    those cells solid)."""
    idx = []
    for a, (ca, na) in enumerate(zip(c[::-1], shape[::-1])):
        rng = np.arange(ca - h, ca + h + 1)
        per = periodic[2 - a]
        idx.append(rng % na if per else np.clip(rng, 0, na - 1))
    return arr[..., idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]]


def _outside(c, h, shape, periodic):
    out = np.zeros((2 * h + 1,) * 3, bool)
    for a in range(3):
        if periodic[a]:
            continue
        rng = np.arange(c[a] - h, c[a] + h + 1)
        bad = (rng < 0) | (rng >= shape[a])
        sl = [slice(None)] * 3
        sl[2 - a] = bad
        out[tuple(sl)] = True
    return out


def _check(sim, method, shape, rho0, u0, steps, cells, periodic=(True, True, True), flags=None, u_wall=(0, 0, 0),
           tol=1e-5, f16_elementwise=False):
    lat = method.lat
    f = sim.populations()
    idx = torch.tensor([x + shape[0] * (y + shape[1] * z) for x, y, z in cells], device=f.device)
    got = f[:, idx].cpu().numpy()
    h = steps + 1
    worst = 0.0
    num = den = 0.0
    dmax = hmax = 0.0
    for k, c in enumerate(cells):
        r = _cut(rho0, c, h, shape, periodic)
        u = _cut(u0, c, h, shape, periodic)
        fl = None
        if flags is not None:
            fl = _cut(flags, c, h, shape, periodic).copy()
            fl[_outside(c, h, shape, periodic)] = olbm.NOSLIP
        box = (2 * h + 1,) * 3
        ref = olbm.Sim(method, box, periodic=(True, True, True), flags=fl, u_wall=u_wall)
        ref.init_equilibrium(r, u)
        ref.step(steps)
        fr = ref.populations()[:, h, h, h]
        worst = max(worst, np.linalg.norm(got[:, k] - fr) / np.linalg.norm(fr - lat.w))
        num += np.sum((got[:, k] - fr) ** 2)
        den += np.sum((fr - lat.w) ** 2)
        dmax = max(dmax, np.abs(got[:, k] - fr).max())
        hmax = max(hmax, np.abs(fr - lat.w).max())
    err = np.sqrt(num / den)
    # the norm is over the sampled set (as the field norms of the small-box
    # tests); single cells near a vortex node have ||f - w|| ~ 1e-4 w, below
    # what unshifted FP32 storage resolves, so their own ratio is only printed
    print(f"sampled parity: relative L2 {err:.2e}, worst single cell {worst:.2e}")
    assert err < tol, err
    if f16_elementwise:
        # binary16 storage, element-wise: 3 U16 max|h_ref| (U16 = 2^-11; the
        # derivation is in test_gpu_parity.py)
        print(f"FP16 element-wise: max |f - f_ref| {dmax:.2e}, bound {3 * 2.0 ** -11 * hmax:.2e}")
        assert dmax <= 3 * 2.0 ** -11 * hmax, (dmax, hmax)
    return err


def test_config2_d3q19_trt_f32_aa_256():
    """The benchmark workload: D3Q19 TRT FP32, 256^3 periodic TGV, AA."""
    n, steps = 256, 4
    rho0, u0 = inputs.tgv3d(n, 0.02, 1e-4, 42)
    sim = Sim("D3Q19", "trt", "f32", "aa", (n, n, n), omega=[1.8], trt_magic=3 / 16)
    sim.init_equilibrium(rho0.reshape(-1), u0.reshape(3, -1))
    sim.step(steps)
    lat = olat.d3q19()
    m = oco.Method(lat, "trt", [1.8, oco.trt_odd_rate(1.8, 3 / 16)])
    cells = _sample_cells((n, n, n), 24, 11) + [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 7)]
    _check(sim, m, (n, n, n), rho0, u0, steps, cells)
    # the two-grid pull sweep and the esoteric twist on the same workload
    for pattern in ["pull", "eso"]:
        sim2 = Sim("D3Q19", "trt", "f32", pattern, (n, n, n), omega=[1.8], trt_magic=3 / 16)
        sim2.init_equilibrium(rho0.reshape(-1), u0.reshape(3, -1))
        sim2.step(steps)
        _check(sim2, m, (n, n, n), rho0, u0, steps, cells[:8])
        del sim2
        torch.cuda.empty_cache()


@pytest.mark.parametrize("stencil", ["D3Q19", "D3Q27"])
def test_kbc_256_benchmark_variant(stencil):
    """The KBC variants of the benchmark: 256^3 TGV, omega_s = omega_b = 1.95, AA."""
    n, steps = 256, 3
    rho0, u0 = inputs.tgv3d(n, 0.02, 1e-4, 42)
    sim = Sim(stencil, "kbc", "f32", "aa", (n, n, n), omega=[1.95, 1.95])
    sim.init_equilibrium(rho0.reshape(-1), u0.reshape(3, -1))
    sim.step(steps)
    m = oco.Method(olat.get(stencil), "kbc", [1.95, 1.95])
    cells = _sample_cells((n, n, n), 6, 17) + [(0, 0, 0), (n - 1, n - 1, n - 1)]
    _check(sim, m, (n, n, n), rho0, u0, steps, cells)


def test_config3_d3q19_mrt_channel_512x128x128():
    """D3Q19 MRT channel: walls, UBB inlet 0.05, outlet, random spheres
    (porosity 0.8); FP32 (pull and AA) and FP16-shifted (AA) storage, the
    patterns of the benchmark's channel variants."""
    shape = (512, 128, 128)
    steps = 3
    flags = inputs.channel_flags(*shape)
    fluid = flags == 0
    rho0, u0 = inputs.random_fields(shape[::-1], 3, amp_rho=0.01, amp_u=0.03, seed=21)
    lat = olat.d3q19()
    m = oco.Method(lat, "mrt", [1.7, 1.0, 1.0, 1.0])
    per = (False, False, False)
    cells = _sample_cells(shape, 24, 5, fluid)
    # cells next to the inlet, the outlet and a wall
    cells += [(1, 64, 64), (510, 64, 64), (200, 1, 1)]
    for storage, pattern, tol in [("f32", "pull", 1e-5), ("f32", "aa", 1e-5), ("f16s", "aa", 5e-3)]:
        sim = Sim("D3Q19", "mrt", storage, pattern, shape, periodic=per, omega=[1.7, 1.0, 1.0, 1.0],
                  u_wall=(0.05, 0.0, 0.0), flags=flags)
        sim.init_equilibrium(rho0.reshape(-1), u0.reshape(3, -1))
        sim.step(steps)
        _check(sim, m, shape, rho0, u0, steps, cells, periodic=per, flags=flags, u_wall=(0.05, 0, 0), tol=tol,
               f16_elementwise=storage == "f16s")
        del sim
        torch.cuda.empty_cache()


def test_config4_d3q27_cumulant_384():
    """D3Q27 cumulant, omega 1.95, higher orders rate 1, 384^3 TGV u0 = 0.05."""
    n, steps = 384, 3
    rho0, u0 = inputs.tgv3d(n, 0.05, 0.0, 42)
    sim = Sim("D3Q27", "cumulant", "f32", "aa", (n, n, n), omega=[1.95, 1.0, 1.0])
    sim.init_equilibrium(rho0.reshape(-1), u0.reshape(3, -1))
    sim.step(steps)
    m = oco.Method(olat.d3q27(), "cumulant", [1.95, 1.0, 1.0])
    cells = _sample_cells((n, n, n), 12, 3) + [(0, 0, 0), (n - 1, 5, n - 1)]
    _check(sim, m, (n, n, n), rho0, u0, steps, cells)
