"""ctypes declarations for liblbm.so (C ABI in include/lbm.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  ``lib()`` loads the in-tree library and raises ``LbmError`` if it
has not been built (there is no fallback path).
"""
import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_size_t, c_uint8, c_uint32, c_void_p

# LBM_DEBUG_BOUNDS=1 selects the bounds-checking build (build(debug_bounds=True))
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "liblbm_debug.so" if os.environ.get("LBM_DEBUG_BOUNDS") == "1" else "liblbm.so")

STENCILS = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2}
COLLISIONS = {"srt": 0, "trt": 1, "mrt": 2, "cumulant": 3, "kbc": 4}
STORAGES = {"f64": 0, "f32": 1, "f16s": 2, "f32s": 3}
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16s": 2, "f32s": 4}
PATTERNS = {"pull": 0, "aa": 1, "eso": 2}
STATUS = ["LBM_OK", "LBM_E_INVAL", "LBM_E_UNSUPPORTED", "LBM_E_CUDA", "LBM_E_NOMEM", "LBM_E_BUFSIZE",
          "LBM_E_NONFINITE", "LBM_E_BOUNDS", "LBM_E_STATE"]
FLUID, NOSLIP, INLET, OUTLET = 0, 1, 2, 4
MASK_SOLID = 0x80000000


class LbmError(RuntimeError):
    def __init__(self, msg, status=None):
        super().__init__(msg)
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("stencil", c_int32), ("collision", c_int32), ("storage", c_int32), ("pattern", c_int32),
                ("nx", c_int32), ("ny", c_int32), ("nz", c_int32), ("periodic", c_int32 * 3),
                ("omega", c_double * 6), ("trt_magic", c_int32), ("incompressible", c_int32),
                ("magic", c_double), ("u_wall", c_double * 3), ("rho_outlet", c_double),
                ("force", c_double * 3), ("smagorinsky_cs", c_double), ("boundary_mode", c_int32)]


_LIB = None

_SIGS = {
    "lbm_default_params": (None, [POINTER(Params)]),
    "lbm_stencil_info": (c_int32, [c_int32, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32), POINTER(c_double)]),
    "lbm_query_sizes": (c_int32, [POINTER(Params), POINTER(c_size_t), POINTER(c_size_t)]),
    "lbm_create": (c_int32, [POINTER(c_void_p), POINTER(Params), c_void_p, c_size_t, c_void_p, c_size_t,
                             c_void_p, c_size_t, c_void_p, c_void_p]),
    "lbm_set_stream": (c_int32, [c_void_p, c_void_p]),
    "lbm_init_equilibrium": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "lbm_set_state": (c_int32, [c_void_p, c_void_p]),
    "lbm_step": (c_int32, [c_void_p, c_int32]),
    "lbm_get_time": (c_int32, [c_void_p, POINTER(c_int64)]),
    "lbm_populations": (c_int32, [c_void_p, c_void_p]),
    "lbm_macroscopic": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "lbm_reduce": (c_int32, [c_void_p, POINTER(c_double)]),
    "lbm_get_pdfs": (c_int32, [c_void_p, c_void_p]),
    "lbm_set_pdfs": (c_int32, [c_void_p, c_void_p, c_int64]),
    "lbm_link_mask": (c_int32, [c_void_p, c_void_p]),
    "lbm_set_force": (c_int32, [c_void_p, POINTER(c_double)]),
    "lbm_step_pull": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "lbm_adjoint_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_adjoint_segment": (c_int32, [c_void_p, POINTER(c_void_p), c_int32, c_void_p, c_void_p, POINTER(c_int32),
                                      c_void_p]),
    "lbm_ke_loss_seed": (c_int32, [c_void_p, c_void_p, POINTER(c_int32), c_void_p, c_void_p, c_void_p]),
    "lbm_eq_vjp": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_reduce_noalloc": (c_int32, [POINTER(Params), c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "lbm_halo_bytes": (c_int32, [POINTER(Params), POINTER(c_size_t)]),
    "lbm_halo_pack": (c_int32, [c_void_p, c_int32, c_void_p]),
    "lbm_halo_unpack": (c_int32, [c_void_p, c_int32, c_void_p]),
    "lbm_sync": (c_int32, [c_void_p]),
    "lbm_status_str": (c_char_p, [c_int32]),
    "lbm_debug_fail_host_allocs": (None, [c_int32]),
    "lbm_last_error": (c_char_p, [c_void_p]),
    "lbm_destroy": (None, [c_void_p]),
}

EXPORTED = tuple(_SIGS)


def lib():
    """Load liblbm.so once; raise LbmError if it is missing."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise LbmError(f"{LIB_PATH} is not built; run paper_2001_11806_gb300.build.build()")
        dll = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(dll, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = dll
    return _LIB


def check(status, ctx=None, what=""):
    if status != 0:
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        detail = ""
        if ctx is not None:
            detail = (lib().lbm_last_error(ctx) or b"").decode()
        raise LbmError(f"{what}: {name} {detail}".strip(), status)


def stencil_info(name):
    q, d = c_int32(), c_int32()
    c = (c_int32 * 81)()
    w = (c_double * 27)()
    check(lib().lbm_stencil_info(STENCILS[name], ctypes.byref(q), ctypes.byref(d), c, w), what="stencil_info")
    Q = q.value
    return Q, d.value, [tuple(c[3 * k: 3 * k + 3]) for k in range(Q)], [w[k] for k in range(Q)]


__all__ = ["lib", "check", "LbmError", "Params", "EXPORTED", "STENCILS", "COLLISIONS", "STORAGES",
           "STORAGE_BYTES", "PATTERNS", "stencil_info", "c_uint8", "c_uint32"]
