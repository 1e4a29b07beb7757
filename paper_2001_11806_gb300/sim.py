"""Python handle over one lbm_ctx: torch owns the device buffers, the C ABI
does all the work.

    sim = Sim("D3Q19", "trt", "f32", "aa", (256, 256, 256), omega=[1.8],
              trt_magic=3/16)
    sim.init_equilibrium(rho, u)        # torch/numpy FP64, [N] and [d][N]
    sim.step(1000)
    rho, u = sim.macroscopic()

stencil "D2Q9" | "D3Q19" | "D3Q27"; collision "srt" | "trt" | "mrt" |
"cumulant" | "kbc"; storage "f64" | "f32" | "f32s" | "f16s" (s = shifted,
h = f - w); pattern "pull" | "aa" | "eso" (esoteric twist); boundary
"in_sweep" | "separate" (separate boundary kernel, pull only); omega as in
lbm_params.omega of include/lbm.h.
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import LbmError, Params, check, lib


def _dev_f64(a, device):
    t = torch.as_tensor(a, dtype=torch.float64)
    return t.to(device).contiguous()


class Sim:
    def __init__(self, stencil="D3Q19", collision="trt", storage="f32", pattern="pull", shape=(1, 1, 1),
                 periodic=(True, True, True), omega=(1.0,), trt_magic=None, incompressible=False,
                 u_wall=(0.0, 0.0, 0.0), rho_outlet=1.0, force=(0.0, 0.0, 0.0), flags=None,
                 device="cuda:0", stream=None, smagorinsky_cs=0.0, boundary="in_sweep"):
        L = lib()
        self.device = torch.device(device)
        p = Params()
        L.lbm_default_params(ctypes.byref(p))
        p.stencil = _lib.STENCILS[stencil]
        p.collision = _lib.COLLISIONS[collision]
        p.storage = _lib.STORAGES[storage]
        p.pattern = _lib.PATTERNS[pattern]
        p.nx, p.ny, p.nz = (int(v) for v in shape)
        for i in range(3):
            p.periodic[i] = 1 if periodic[i] else 0
        om = list(omega) + [1.0] * (6 - len(omega))
        for i in range(6):
            p.omega[i] = float(om[i])
        if trt_magic is not None:
            p.trt_magic = 1
            p.magic = float(trt_magic)
        p.incompressible = 1 if incompressible else 0
        for i in range(3):
            p.u_wall[i] = float(u_wall[i])
            p.force[i] = float(force[i])
        p.rho_outlet = float(rho_outlet)
        p.smagorinsky_cs = float(smagorinsky_cs)
        p.boundary_mode = {"in_sweep": 0, "separate": 1}[boundary]
        self.params = p
        self.stencil, self.collision, self.storage, self.pattern = stencil, collision, storage, pattern
        self.shape = tuple(int(v) for v in shape)
        self.N = p.nx * p.ny * p.nz
        self.q, self.d, self.c, self.w = _lib.stencil_info(stencil)
        pdf_b, aux_b = ctypes.c_size_t(), ctypes.c_size_t()
        check(L.lbm_query_sizes(ctypes.byref(p), ctypes.byref(pdf_b), ctypes.byref(aux_b)), what="query_sizes")
        self.pdf_bytes = pdf_b.value
        self.pdf = torch.empty(self.pdf_bytes, dtype=torch.uint8, device=self.device)
        self.pdf2 = torch.empty(self.pdf_bytes, dtype=torch.uint8, device=self.device) if pattern == "pull" else None
        self.aux = torch.zeros(aux_b.value, dtype=torch.uint8, device=self.device)
        self.flags = None
        if flags is not None:
            self.flags = torch.as_tensor(np.ascontiguousarray(flags), dtype=torch.uint8).reshape(-1).to(self.device)
            if self.flags.numel() != self.N:
                raise LbmError("flags must have N entries")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = ctypes.c_void_p()
        check(L.lbm_create(ctypes.byref(ctx), ctypes.byref(p), self.pdf.data_ptr(), self.pdf_bytes,
                           self.pdf2.data_ptr() if self.pdf2 is not None else None,
                           self.pdf_bytes if self.pdf2 is not None else 0,
                           self.aux.data_ptr(), self.aux.numel(),
                           self.flags.data_ptr() if self.flags is not None else None,
                           self.stream.cuda_stream), what="create")
        self.ctx = ctx

    # ------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "ctx", None):
            lib().lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status, what):
        check(status, self.ctx, what)

    # ------------------------------------------------------------ operations
    def init_equilibrium(self, rho, u):
        rho_t = _dev_f64(rho, self.device).reshape(-1)
        u_t = _dev_f64(u, self.device).reshape(self.d, -1)
        if rho_t.numel() != self.N or u_t.shape[1] != self.N:
            raise LbmError("rho must have N entries and u d*N entries")
        self._keep = (rho_t, u_t)
        self._check(lib().lbm_init_equilibrium(self.ctx, rho_t.data_ptr(), u_t.data_ptr()), "init_equilibrium")

    def set_state(self, P):
        P_t = _dev_f64(P, self.device).reshape(self.q, -1)
        if P_t.shape[1] != self.N:
            raise LbmError("P must have q*N entries")
        self._keep = (P_t,)
        self._check(lib().lbm_set_state(self.ctx, P_t.data_ptr()), "set_state")

    def step(self, n=1):
        self._check(lib().lbm_step(self.ctx, int(n)), "step")

    @property
    def t(self):
        v = ctypes.c_int64()
        self._check(lib().lbm_get_time(self.ctx, ctypes.byref(v)), "get_time")
        return v.value

    def populations(self):
        out = torch.empty((self.q, self.N), dtype=torch.float64, device=self.device)
        self._check(lib().lbm_populations(self.ctx, out.data_ptr()), "populations")
        return out

    def macroscopic(self, f64=True):
        dt = torch.float64 if f64 else torch.float32
        rho = torch.empty(self.N, dtype=dt, device=self.device)
        u = torch.empty((self.d, self.N), dtype=dt, device=self.device)
        self._check(lib().lbm_macroscopic(self.ctx, rho.data_ptr(), u.data_ptr(), 1 if f64 else 0), "macroscopic")
        return rho, u

    def reduce(self):
        out = (ctypes.c_double * 5)()
        self._check(lib().lbm_reduce(self.ctx, out), "reduce")
        return np.array(list(out))

    def link_mask(self):
        out = torch.empty(self.N, dtype=torch.int32, device=self.device)
        self._check(lib().lbm_link_mask(self.ctx, out.data_ptr()), "link_mask")
        return out

    def get_pdfs(self):
        out = torch.empty(self.pdf_bytes, dtype=torch.uint8, device=self.device)
        self._check(lib().lbm_get_pdfs(self.ctx, out.data_ptr()), "get_pdfs")
        return out, self.t

    def set_pdfs(self, raw, t):
        """Restore a state saved by get_pdfs; raw must be a contiguous tensor
        of exactly pdf_bytes on the device (the C call copies pdf_bytes from
        it and cannot check its size)."""
        if not isinstance(raw, torch.Tensor) or not raw.is_contiguous() or \
                raw.numel() * raw.element_size() != self.pdf_bytes or raw.device.type != self.device.type:
            raise LbmError(f"set_pdfs needs a contiguous {self.device.type} tensor of {self.pdf_bytes} bytes")
        self._check(lib().lbm_set_pdfs(self.ctx, raw.data_ptr(), int(t)), "set_pdfs")

    def sync(self):
        self._check(lib().lbm_sync(self.ctx), "sync")
