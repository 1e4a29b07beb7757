"""Gradients of a flow objective through the adjoint kernels.

``Rollout`` runs T pull steps from f^eq(rho_0, u_0) with a uniform Guo body
force F and returns the kinetic energy in a box at the end,
L = (1/2) sum_{x in box} rho |u|^2.  ``Rollout.gradient`` returns
(L, dL/du_0, dL/dF) by the discrete adjoint: the seed kernel gives
lambda_T = dL/dP_T, then for t = T .. 1 lambda_{t-1} = adjoint_step(P_{t-1},
lambda_t) and finally dL/du_0 = (d f^eq / d u_0)^T lambda_0.

Checkpointing (sqrt(T) scheme): the forward keeps the raw state every
k = ceil(sqrt(T)) steps; the reverse sweep recomputes one segment of at most k
states at a time from its checkpoint (one pull step per state, written
straight into the segment buffers) and runs the adjoint backwards through it,
one lbm_adjoint_segment call per segment, so the host issues one call per k
steps.
Device memory: (ceil(T/k) + k) population arrays plus two adjoint arrays; for
D3Q19 FP32 at 128^3 and T = 1000 that is 64 x 159 MB = 10.2 GB.

``LBMRollout`` wraps this as a torch.autograd.Function of (u_0, F).
"""
import ctypes
import math

import numpy as np
import torch

from ._lib import LbmError, check, lib
from .sim import Sim


class Rollout:
    def __init__(self, stencil, collision, storage, shape, omega, T, box, periodic=(True, True, True), flags=None,
                 trt_magic=None, incompressible=False, u_wall=(0.0, 0.0, 0.0), device="cuda:0"):
        self.sim = Sim(stencil, collision, storage, "pull", shape, periodic=periodic, omega=omega,
                       trt_magic=trt_magic, incompressible=incompressible, u_wall=u_wall, flags=flags,
                       device=device)
        self.T = int(T)
        self.k = max(1, math.ceil(math.sqrt(self.T)))
        self.box = (ctypes.c_int32 * 6)(*[int(b) for b in box])
        self.lam_dtype = torch.float64 if storage == "f64" else torch.float32
        self.device = self.sim.device
        self._ckpt = []
        self._seg = []

    # ----------------------------------------------------------- primitives
    def _set_force(self, F):
        F3 = (ctypes.c_double * 3)(*[float(v) for v in list(F) + [0.0] * (3 - len(F))])
        check(lib().lbm_set_force(self.sim.ctx, F3), self.sim.ctx, "set_force")

    def _raw(self):
        return torch.empty(self.sim.pdf_bytes, dtype=torch.uint8, device=self.device)

    def _loss(self, P, lam_out=None, dLdF=None):
        L = torch.zeros(1, dtype=torch.float64, device=self.device)
        check(lib().lbm_ke_loss_seed(self.sim.ctx, P.data_ptr(), self.box, L.data_ptr(),
                                     lam_out.data_ptr() if lam_out is not None else None,
                                     dLdF.data_ptr() if dLdF is not None else None), self.sim.ctx, "ke_loss_seed")
        return L

    # -------------------------------------------------------------- forward
    def loss(self, rho0, u0, F, keep=False):
        """L for initial fields (rho0, u0) and force F; keep=True stores the
        checkpoints for a following ``backward``."""
        self._set_force(F)
        self.sim.init_equilibrium(rho0, u0)
        self._rho0 = torch.as_tensor(rho0, dtype=torch.float64).to(self.device).reshape(-1).contiguous()
        self._u0 = torch.as_tensor(u0, dtype=torch.float64).to(self.device).reshape(self.sim.d, -1).contiguous()
        if keep:
            while len(self._ckpt) < math.ceil(self.T / self.k):
                self._ckpt.append(self._raw())
        done = 0
        while done < self.T:
            if keep:
                check(lib().lbm_get_pdfs(self.sim.ctx, self._ckpt[done // self.k].data_ptr()), self.sim.ctx,
                      "get_pdfs")
            n = min(self.k, self.T - done)
            self.sim.step(n)
            done += n
        self._final = self.sim.get_pdfs()[0]
        return self._loss(self._final)

    # -------------------------------------------------------------- reverse
    def backward(self):
        """(dL/du_0 [d][N] FP64, dL/dF [3] FP64) for the last ``loss(keep=True)``."""
        L = lib()
        ctx = self.sim.ctx
        q, N = self.sim.q, self.sim.N
        lam = [torch.empty((q, N), dtype=self.lam_dtype, device=self.device) for _ in range(2)]
        dLdF = torch.zeros(3, dtype=torch.float64, device=self.device)
        self._loss(self._final, lam_out=lam[0], dLdF=dLdF)
        while len(self._seg) < self.k:
            self._seg.append(self._raw())
        cur = ctypes.c_int32(0)
        nseg = math.ceil(self.T / self.k)
        for s in range(nseg - 1, -1, -1):
            base = s * self.k
            n = min(base + self.k, self.T) - base
            # the library recomputes the segment into the buffers and runs its
            # n adjoint steps backwards (lbm_adjoint_segment)
            states = (ctypes.c_void_p * n)(self._ckpt[s].data_ptr(), *[self._seg[i].data_ptr() for i in range(1, n)])
            check(L.lbm_adjoint_segment(ctx, states, n, lam[0].data_ptr(), lam[1].data_ptr(), ctypes.byref(cur),
                                        dLdF.data_ptr()), ctx, "adjoint_segment")
        cur = cur.value
        g_u0 = torch.empty((self.sim.d, N), dtype=torch.float64, device=self.device)
        check(L.lbm_eq_vjp(ctx, self._rho0.data_ptr(), self._u0.data_ptr(), lam[cur].data_ptr(), g_u0.data_ptr()),
              ctx, "eq_vjp")
        return g_u0, dLdF

    def gradient(self, rho0, u0, F):
        Lval = self.loss(rho0, u0, F, keep=True)
        g_u0, g_F = self.backward()
        return Lval, g_u0, g_F


class LBMRollout(torch.autograd.Function):
    """L = LBMRollout.apply(u0, F, rollout, rho0) with gradients for u0 ([d][N]
    FP64 on the rollout's device) and F ([3] FP64)."""

    @staticmethod
    def forward(ctx, u0, F, rollout, rho0):
        L = rollout.loss(rho0, u0.detach(), F.detach().cpu().numpy().tolist(), keep=True)
        ctx.rollout = rollout
        ctx.F_device = F.device
        return L.reshape(())

    @staticmethod
    def backward(ctx, gL):
        g_u0, g_F = ctx.rollout.backward()
        g_u0 = g_u0 * gL
        g_F = (g_F * gL).to(ctx.F_device)
        return g_u0, g_F, None, None


__all__ = ["Rollout", "LBMRollout", "LbmError"]
