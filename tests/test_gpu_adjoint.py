"""GPU adjoint against the oracle's complex-step adjoint and against finite
differences.

Per-kernel parity (FP64 storage, 1e-12 relative): one adjoint step
(transposed streaming of the transposed collision Jacobian, with no-slip and
UBB links and a Guo force), the kinetic-energy seed, the equilibrium VJP.
Whole-run parity: L, dL/du_0 and dL/dF of the checkpointed reverse sweep
against the oracle's full reverse sweep (FP64: 1e-10; FP32 storage and
adjoint: 1e-4; FP16-shifted storage: 5e-3).  FP16-shifted single steps: the
oracle linearised around the same binary16 state, 1e-5.  Finite differences: directional derivatives of the FP64
forward on random directions (relative 1e-6 for the FP64 adjoint)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import adjoint as oad
from oracle import collision as oco
from oracle import lattice as olat
from oracle import lbm as olbm
from paper_2001_11806_gb300 import _lib, inputs
from paper_2001_11806_gb300.adjoint import LBMRollout, Rollout
from paper_2001_11806_gb300.sim import Sim

pytestmark = pytest.mark.gpu

OMEGAS = {"srt": [1.37], "trt": [1.8, 8 / 31], "mrt": [1.7, 1.1, 0.9, 1.3, 1.2, 1.05]}
COMBOS = [(s, c) for s in ["D2Q9", "D3Q19", "D3Q27"] for c in ["srt", "trt", "mrt"]]
FORCE = [2e-4, -1e-4, 5e-5]


def _shape(stencil):
    return (37, 6, 1) if stencil == "D2Q9" else (37, 5, 4)


def _flags(shape):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[:, 0, :] = olbm.NOSLIP
    fl[:, -1, 3:20] = olbm.INLET
    fl[:, -1, 20:] = olbm.NOSLIP
    fl[:, -1, :3] = olbm.NOSLIP
    r = inputs.uniform(5, nx * ny * nz).reshape(nz, ny, nx)
    fl[(r < 0.06) & (fl == 0)] = olbm.NOSLIP
    return fl


def _oracle(stencil, collision, shape, fl, force=FORCE):
    lat = olat.get(stencil)
    om = OMEGAS[collision][:6 if stencil == "D3Q27" else 4]
    m = oco.Method(lat, collision, om, force=force[: lat.d])
    return olbm.Sim(m, shape, periodic=(True, False, True), flags=fl, u_wall=(0.03, 0.0, 0.0))


def _gpu(stencil, collision, storage, shape, fl, force=FORCE):
    return Sim(stencil, collision, storage, "pull", shape, periodic=(True, False, True), omega=OMEGAS[collision],
               u_wall=(0.03, 0.0, 0.0), force=force, flags=fl)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("stencil,collision", COMBOS)
def test_adjoint_step_parity(stencil, collision):
    shape = _shape(stencil)
    fl = _flags(shape)
    lat = olat.get(stencil)
    sim = _gpu(stencil, collision, "f64", shape, fl)
    ref = _oracle(stencil, collision, shape, fl)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=6)
    lam = np.random.default_rng(2).standard_normal((lat.q,) + shape[::-1])
    lam[:, fl != 0] = 0.0
    sim.set_state(P.reshape(lat.q, -1))
    raw, _ = sim.get_pdfs()
    lam_in = torch.tensor(lam.reshape(lat.q, -1), device=sim.device)
    lam_out = torch.full_like(lam_in, float("nan"))
    dF = torch.zeros(3, dtype=torch.float64, device=sim.device)
    st = _lib.lib().lbm_adjoint_step(sim.ctx, raw.data_ptr(), lam_in.data_ptr(), lam_out.data_ptr(), dF.data_ptr())
    assert st == 0
    ref_lam, ref_gF = oad.adjoint_step(ref, P, lam)
    fluid = fl.reshape(-1) == 0
    got = lam_out.cpu().numpy()
    assert np.all(got[:, ~fluid] == 0.0)
    assert _rel(got[:, fluid], ref_lam.reshape(lat.q, -1)[:, fluid]) < 1e-12
    assert _rel(dF.cpu().numpy()[: lat.d], ref_gF) < 1e-12


@pytest.mark.parametrize("stencil,collision", [("D2Q9", "srt"), ("D3Q19", "trt"), ("D3Q19", "mrt"), ("D3Q27", "trt")])
def test_f16s_adjoint_step_parity(stencil, collision):
    """FP16-shifted storage: the adjoint step reads P_prev from binary16
    storage and computes in FP32 with FP32 lambda.  The oracle linearises
    around the same stored state (the binary16 values converted exactly to
    FP64), so only the FP32 arithmetic differs: 1e-5 relative, the FP32
    tolerance."""
    shape = _shape(stencil)
    fl = _flags(shape)
    lat = olat.get(stencil)
    sim = _gpu(stencil, collision, "f16s", shape, fl)
    ref = _oracle(stencil, collision, shape, fl)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=16)
    lam = np.random.default_rng(3).standard_normal((lat.q,) + shape[::-1])
    lam[:, fl != 0] = 0.0
    sim.set_state(P.reshape(lat.q, -1))
    raw, _ = sim.get_pdfs()
    h16 = raw.view(torch.float16).reshape(lat.q, sim.N).double().cpu().numpy()
    P16 = (h16 + lat.w[:, None]).reshape(P.shape)
    lam_in = torch.tensor(lam.reshape(lat.q, -1), dtype=torch.float32, device=sim.device)
    lam_out = torch.full_like(lam_in, float("nan"))
    dF = torch.zeros(3, dtype=torch.float64, device=sim.device)
    st = _lib.lib().lbm_adjoint_step(sim.ctx, raw.data_ptr(), lam_in.data_ptr(), lam_out.data_ptr(), dF.data_ptr())
    assert st == 0
    ref_lam, ref_gF = oad.adjoint_step(ref, P16, lam.astype(np.float32).astype(np.float64))
    fluid = fl.reshape(-1) == 0
    got = lam_out.cpu().numpy()
    assert np.all(got[:, ~fluid] == 0.0)
    assert _rel(got[:, fluid], ref_lam.reshape(lat.q, -1)[:, fluid]) < 1e-5
    assert _rel(dF.cpu().numpy()[: lat.d], ref_gF) < 1e-5


@pytest.mark.parametrize("stencil,collision", COMBOS)
def test_seed_and_eq_vjp_parity(stencil, collision):
    shape = _shape(stencil)
    fl = _flags(shape)
    lat = olat.get(stencil)
    sim = _gpu(stencil, collision, "f64", shape, fl)
    ref = _oracle(stencil, collision, shape, fl)
    P = inputs.random_pdfs(lat.w, shape[::-1], seed=7)
    sim.set_state(P.reshape(lat.q, -1))
    raw, _ = sim.get_pdfs()
    box = (3, 30, 1, 4, 0, shape[2])
    L = torch.zeros(1, dtype=torch.float64, device=sim.device)
    lam = torch.full((lat.q, sim.N), float("nan"), dtype=torch.float64, device=sim.device)
    dF = torch.zeros(3, dtype=torch.float64, device=sim.device)
    st = _lib.lib().lbm_ke_loss_seed(sim.ctx, raw.data_ptr(), (ctypes.c_int32 * 6)(*box), L.data_ptr(),
                                     lam.data_ptr(), dF.data_ptr())
    assert st == 0
    rL, rlam, rgF = oad.ke_box_seed(ref, P, box)
    assert abs(L.item() / rL - 1) < 1e-12
    fluid = fl.reshape(-1) == 0
    assert _rel(lam.cpu().numpy()[:, fluid], rlam.reshape(lat.q, -1)[:, fluid]) < 1e-12
    assert _rel(dF.cpu().numpy()[: lat.d], rgF) < 1e-12
    # equilibrium VJP
    rho0, u0 = inputs.random_fields(shape[::-1], lat.d, seed=8)
    g = torch.empty((lat.d, sim.N), dtype=torch.float64, device=sim.device)
    r_t = torch.tensor(rho0.reshape(-1), device=sim.device)
    u_t = torch.tensor(u0.reshape(lat.d, -1), device=sim.device)
    st = _lib.lib().lbm_eq_vjp(sim.ctx, r_t.data_ptr(), u_t.data_ptr(), lam.data_ptr(), g.data_ptr())
    assert st == 0
    lam_np = lam.cpu().numpy().reshape((lat.q,) + shape[::-1])
    rg = oad.eq_vjp(ref, rho0, u0, np.where(np.isnan(lam_np), 0.0, lam_np))
    assert _rel(g.cpu().numpy()[:, fluid], rg.reshape(lat.d, -1)[:, fluid]) < 1e-12


@pytest.mark.parametrize("stencil,collision", [("D2Q9", "srt"), ("D3Q19", "trt"), ("D3Q19", "mrt"), ("D3Q27", "trt")])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-4), ("f16s", 5e-3)])
def test_whole_run_gradient_parity(stencil, collision, storage, tol):
    """FP16-shifted storage differentiates its own binary16 trajectory, which
    leaves the FP64 one by about the storage rounding per step; it is held to
    the FP16 field tolerance, 5e-3."""
    shape = _shape(stencil)
    fl = _flags(shape)
    lat = olat.get(stencil)
    T = 11  # k = 4: three segments, the last one short
    box = (5, 25, 1, 4, 0, shape[2])
    ro = Rollout(stencil, collision, storage, shape, OMEGAS[collision], T, box, periodic=(True, False, True),
                 flags=fl, u_wall=(0.03, 0.0, 0.0))
    rho0, u0 = inputs.random_fields(shape[::-1], lat.d, amp_u=0.04, seed=9)
    L, g_u0, g_F = ro.gradient(rho0, u0, FORCE)
    ref = _oracle(stencil, collision, shape, fl)
    rL, rg, rgF = oad.gradient(ref, rho0, u0, T, box)
    fluid = fl.reshape(-1) == 0
    assert abs(L.item() / rL - 1) < tol
    assert _rel(g_u0.cpu().numpy()[:, fluid], rg.reshape(lat.d, -1)[:, fluid]) < tol
    assert _rel(g_F.cpu().numpy()[: lat.d], rgF) < tol


def test_autograd_function_and_unsupported_cases():
    shape = (16, 12, 10)
    ro = Rollout("D3Q19", "trt", "f64", shape, [1.8], 9, (4, 12, 3, 9, 2, 8), trt_magic=3 / 16)
    rho0, u0 = inputs.tgv3d(16, 0.02, 1e-4, 42)
    rho0, u0 = rho0[:10, :12, :16], u0[:, :10, :12, :16]
    u_t = torch.tensor(u0.reshape(3, -1), device="cuda:0", requires_grad=True)
    F_t = torch.tensor([1e-5, 0.0, 0.0], dtype=torch.float64, requires_grad=True)
    L = LBMRollout.apply(u_t, F_t, ro, rho0.reshape(-1))
    (2.0 * L).backward()
    Lr, g_u0, g_F = ro.gradient(rho0.reshape(-1), u0.reshape(3, -1), [1e-5, 0.0, 0.0])
    assert abs(L.item() - Lr.item()) <= 1e-14 * abs(Lr.item())
    assert torch.allclose(u_t.grad, 2.0 * g_u0, rtol=0, atol=1e-300)
    # the force gradient is summed in a fixed order (per-block rows, then one
    # final sum), so the two calls agree bit for bit
    assert np.array_equal(F_t.grad.numpy(), 2.0 * g_F.cpu().numpy())
    # the adjoint refuses what it does not differentiate
    fl = np.zeros((4, 5, 6), np.uint8)
    fl[:, :, -1] = olbm.OUTLET
    for kw, status in [(dict(collision="trt", pattern="aa"), 8), (dict(collision="trt", flags=fl), 2),
                       (dict(collision="kbc"), 2)]:
        sim = Sim("D3Q19", kw["collision"], "f64", kw.get("pattern", "pull"), (6, 5, 4), omega=[1.2, 1.1],
                  flags=kw.get("flags"), periodic=(False, True, True))
        buf = torch.zeros((19, sim.N), dtype=torch.float64, device=sim.device)
        out = torch.zeros_like(buf)
        st = _lib.lib().lbm_adjoint_step(sim.ctx, sim.pdf.data_ptr(), buf.data_ptr(), out.data_ptr(), None)
        assert st == status


def test_finite_differences_config5_size():
    """D3Q19 TRT, 128^3 periodic, T = 1000, L = kinetic energy in the central
    32^3 box, TGV u0 = 0.02 + noise, uniform force F = (1e-6, 0, 0): adjoint
    directional derivatives against central finite differences of the FP64
    forward, on 20 random directions of (u0, F), 10 of u0 alone and 10 of F
    alone.  Each error is divided by the RMS of the finite differences over
    its set of directions (a random projection of the gradient can come out
    arbitrarily small, which would make a plain ratio meaningless).
    FP64 adjoint: 1e-6 on every set.  The FP32 adjoint (FP32 arithmetic,
    FP32 or shifted-FP32 storage) differentiates the FP32 forward, which stays
    within ~1e-5 of the FP64 trajectory over 1000 steps now that the Guo
    force's constant odd increment is no longer rounded on the populations'
    coarse grid (before, the forced momentum lost 1e-4 of F and the force
    gradient was off by 1.8e-4).  Bar for FP32 and shifted-FP32 storage:
    directional derivatives within 1e-4 of the finite differences of the FP64
    forward on every set (u0, F, joint), and the gradient within 1e-4 of the
    FP64 gradient in norm, for u0 and for F."""
    n, T = 128, 1000
    box = (48, 80, 48, 80, 48, 80)
    rho0, u0 = inputs.tgv3d(n, 0.02, 1e-4, 42)
    rho0 = rho0.reshape(-1)
    u0 = u0.reshape(3, -1)
    F0 = np.array([1e-6, 0.0, 0.0])
    grads = {}
    for storage in ["f64", "f32s", "f32"]:
        ro = Rollout("D3Q19", "trt", storage, (n, n, n), [1.8], T, box, trt_magic=3 / 16)
        _, g, gF = ro.gradient(rho0, u0, F0)
        grads[storage] = (g.cpu().numpy(), gF.cpu().numpy())
        if storage == "f64":
            ro64 = ro
        else:
            del ro
            torch.cuda.empty_cache()
    rng = np.random.default_rng(2024)
    err = {}
    for kind, ndir in [("joint", 20), ("u0", 10), ("F", 10)]:
        fds, ds = [], {k: [] for k in grads}
        for i in range(ndir):
            v = rng.standard_normal(u0.shape) if kind != "F" else np.zeros(u0.shape)
            if kind == "joint":
                vF = rng.standard_normal(3) * 1e-2 * np.linalg.norm(v) / np.sqrt(v.size)
            elif kind == "F":
                vF = rng.standard_normal(3)
            else:
                vF = np.zeros(3)
            eps = 1e-4 * (np.linalg.norm(u0) / np.linalg.norm(v) if kind != "F"
                          else np.linalg.norm(F0) / np.linalg.norm(vF))
            Lp = ro64.loss(rho0, u0 + eps * v, F0 + eps * vF).item()
            Lm = ro64.loss(rho0, u0 - eps * v, F0 - eps * vF).item()
            fds.append((Lp - Lm) / (2 * eps))
            for k, (g, gF) in grads.items():
                ds[k].append((g * v).sum() + gF @ vF)
        fds = np.array(fds)
        rms = np.sqrt(np.mean(fds ** 2))
        for k in grads:
            err[(k, kind)] = np.max(np.abs(np.array(ds[k]) - fds)) / rms
    print("FD check, max |adjoint - FD| / RMS(FD): " + ", ".join(f"{k}/{kind} {v:.2e}" for (k, kind), v in err.items()))
    for kind in ["joint", "u0", "F"]:
        assert err[("f64", kind)] < 1e-6
    g64, gF64 = grads["f64"]
    for k in ["f32s", "f32"]:
        g, gF = grads[k]
        eu = np.linalg.norm(g - g64) / np.linalg.norm(g64)
        eF = np.linalg.norm(gF - gF64) / np.linalg.norm(gF64)
        print(f"{k} gradient vs FP64 gradient: u0 {eu:.2e}, F {eF:.2e}")
        assert eu < 1e-4 and eF < 1e-4
        for kind in ["joint", "u0", "F"]:
            assert err[(k, kind)] < 1e-4, (k, kind, err[(k, kind)])
