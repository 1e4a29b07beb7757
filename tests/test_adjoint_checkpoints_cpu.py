"""Host logic of the sqrt(T) checkpointing in ``paper_2001_11806_gb300.adjoint``,
checked on the CPU against a stand-in for the library.

The stand-in replaces the C calls ``Rollout`` makes with a small non-linear
map on numpy arrays that live in the same memory as the torch tensors the
rollout allocates (addressed through their data pointers, as the library
does):

  P_{t+1} = M P_t + alpha P_t^2 + G F,   P_0 = E u_0,   L = (1/2) |W P_T|^2,

so the reverse sweep is right only if every adjoint step receives the state
it linearises about.  The gradients (L, dL/du_0, dL/dF) from
``Rollout.gradient`` must equal a plain reverse sweep over all stored states
and agree with central differences, for step counts that are and are not
multiples of the segment length, and the rollout must hold ceil(T/k) + k
state buffers (k = ceil(sqrt T))."""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_2001_11806_gb300 import adjoint

Q, NC, D = 3, 4, 2  # "populations" per cell, cells, velocity components
S = Q * NC
ALPHA = 0.05


def _view(ptr, n):
    return np.ctypeslib.as_array((ctypes.c_double * n).from_address(int(ptr)))


class Model:
    def __init__(self, seed=0):
        rng = np.random.default_rng(seed)
        self.M = 0.3 * rng.standard_normal((S, S)) / math.sqrt(S)
        self.G = rng.standard_normal((S, 3))
        self.E = rng.standard_normal((S, D * NC))
        self.W = rng.standard_normal((5, S))
        self.F = np.zeros(3)

    def step(self, P):
        return self.M @ P + ALPHA * P * P + self.G @ self.F

    def vjp(self, P, lam):
        return self.M.T @ lam + 2 * ALPHA * P * lam


class FakeLib:
    """The C calls of Rollout, on the model."""

    def __init__(self, model):
        self.m = model
        self.calls = {"step_pull": 0, "adjoint_step": 0}

    def lbm_set_force(self, ctx, F3):
        self.m.F = np.array([F3[0], F3[1], F3[2]])
        return 0

    def lbm_get_pdfs(self, ctx, dst):
        _view(dst, S)[:] = ctx.state
        return 0

    def lbm_step_pull(self, ctx, src, dst):
        self.calls["step_pull"] += 1
        _view(dst, S)[:] = self.m.step(_view(src, S).copy())
        return 0

    def lbm_ke_loss_seed(self, ctx, P, box, L, lam_out, dLdF):
        WP = self.m.W @ _view(P, S)
        _view(L, 1)[0] += 0.5 * WP @ WP
        if lam_out:
            _view(lam_out, S)[:] = self.m.W.T @ WP
        return 0

    def lbm_adjoint_step(self, ctx, P_prev, lam_in, lam_out, dLdF):
        self.calls["adjoint_step"] += 1
        lam = _view(lam_in, S).copy()
        _view(lam_out, S)[:] = self.m.vjp(_view(P_prev, S).copy(), lam)
        _view(dLdF, 3)[:] += self.m.G.T @ lam
        return 0

    def lbm_adjoint_segment(self, ctx, states, n, lam0, lam1, cur, dLdF):
        """The documented schedule: recompute states[1 .. n-1], then n adjoint
        steps backwards, alternating lam0/lam1 from *cur."""
        for i in range(1, n):
            self.lbm_step_pull(ctx, states[i - 1], states[i])
        lam = [lam0, lam1]
        k = cur._obj.value
        for t in range(n, 0, -1):
            self.lbm_adjoint_step(ctx, states[t - 1], lam[k], lam[1 - k], dLdF)
            k = 1 - k
        cur._obj.value = k
        return 0

    def lbm_eq_vjp(self, ctx, rho0, u0, lam, g_u0):
        _view(g_u0, D * NC)[:] = self.m.E.T @ _view(lam, S)
        return 0


class FakeSim:
    def __init__(self, model):
        self.m = model
        self.ctx = self  # the fake calls read the state through ctx
        self.q, self.N, self.d = Q, NC, D
        self.pdf_bytes = S * 8
        self.device = torch.device("cpu")
        self.state = np.zeros(S)

    def init_equilibrium(self, rho0, u0):
        self.state = self.m.E @ np.asarray(u0, dtype=np.float64).reshape(-1)

    def step(self, n):
        for _ in range(int(n)):
            self.state = self.m.step(self.state)

    def get_pdfs(self):
        return torch.from_numpy(self.state.copy()), 0


def _rollout(model, T, monkeypatch):
    fake = FakeLib(model)
    monkeypatch.setattr(adjoint, "lib", lambda: fake)
    r = object.__new__(adjoint.Rollout)
    r.sim = FakeSim(model)
    r.T = T
    r.k = max(1, math.ceil(math.sqrt(T)))
    r.box = (ctypes.c_int32 * 6)(0, 1, 0, 1, 0, 1)
    r.lam_dtype = torch.float64
    r.device = torch.device("cpu")
    r._ckpt, r._seg = [], []
    return r, fake


def _direct(model, u0, F, T):
    model.F = np.asarray(F, dtype=np.float64)
    states = [model.E @ u0.reshape(-1)]
    for _ in range(T):
        states.append(model.step(states[-1]))
    WP = model.W @ states[-1]
    L = 0.5 * WP @ WP
    lam = model.W.T @ WP
    gF = np.zeros(3)
    for t in range(T, 0, -1):
        gF += model.G.T @ lam
        lam = model.vjp(states[t - 1], lam)
    return L, model.E.T @ lam, gF


@pytest.mark.parametrize("T", [1, 2, 3, 4, 5, 9, 10, 17, 50])
def test_checkpointed_reverse_sweep_equals_plain_reverse(T, monkeypatch):
    model = Model()
    rng = np.random.default_rng(T)
    u0 = 0.1 * rng.standard_normal((D, NC))
    F = [0.01, -0.02, 0.005]
    r, fake = _rollout(model, T, monkeypatch)
    L, g_u0, g_F = r.gradient(np.ones(NC), u0, F)
    L_ref, gu_ref, gF_ref = _direct(model, u0, F, T)
    assert abs(float(L) - L_ref) <= 1e-13 * abs(L_ref)
    assert np.allclose(g_u0.numpy().reshape(-1), gu_ref, rtol=1e-12, atol=1e-14)
    assert np.allclose(g_F.numpy(), gF_ref, rtol=1e-12, atol=1e-14)
    k = r.k
    assert len(r._ckpt) == math.ceil(T / k) and len(r._seg) == k
    assert fake.calls["adjoint_step"] == T
    # each segment recomputes all but its checkpointed first state
    assert fake.calls["step_pull"] == T - math.ceil(T / k)


def test_gradient_against_central_differences(monkeypatch):
    model = Model(seed=3)
    T = 12
    rng = np.random.default_rng(1)
    u0 = 0.1 * rng.standard_normal((D, NC))
    F = np.array([0.01, -0.02, 0.005])
    r, _ = _rollout(model, T, monkeypatch)
    _, g_u0, g_F = r.gradient(np.ones(NC), u0, F.tolist())
    h = 1e-6
    for _ in range(5):
        du = rng.standard_normal(u0.shape)
        Lp = _direct(model, u0 + h * du, F, T)[0]
        Lm = _direct(model, u0 - h * du, F, T)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - float((g_u0.numpy() * du).sum())) <= 1e-6 * max(1.0, abs(fd))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (_direct(model, u0, F + e, T)[0] - _direct(model, u0, F - e, T)[0]) / (2 * h)
        assert abs(fd - float(g_F.numpy()[a])) <= 1e-6 * max(1.0, abs(fd))


def test_autograd_function_routes_the_gradients(monkeypatch):
    model = Model(seed=5)
    T = 7
    rng = np.random.default_rng(2)
    u0_np = 0.1 * rng.standard_normal((D, NC))
    F_np = np.array([0.01, -0.02, 0.005])
    r, _ = _rollout(model, T, monkeypatch)
    u0 = torch.tensor(u0_np, dtype=torch.float64, requires_grad=True)
    F = torch.tensor(F_np, dtype=torch.float64, requires_grad=True)
    L = adjoint.LBMRollout.apply(u0, F, r, np.ones(NC))
    (3.0 * L).backward()
    L_ref, gu_ref, gF_ref = _direct(model, u0_np, F_np, T)
    assert abs(float(L.detach()) - L_ref) <= 1e-13 * abs(L_ref)
    assert np.allclose(u0.grad.numpy().reshape(-1), 3.0 * gu_ref, rtol=1e-12, atol=1e-14)
    assert np.allclose(F.grad.numpy(), 3.0 * gF_ref, rtol=1e-12, atol=1e-14)
