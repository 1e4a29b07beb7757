"""Host-only checks of the C ABI (no GPU needed): the library loads, exports
every function include/lbm.h declares, validates arguments, and its stencil
table matches the documented direction order (compared with the oracle's
independently written table)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import lattice as olat
from paper_2001_11806_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _lib.lib()


def _header_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_function(L):
    declared = _header_functions()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(declared) == sorted(_lib.EXPORTED)


def _params(**kw):
    p = _lib.Params()
    _lib.lib().lbm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "omega":
            for i, x in enumerate(v):
                p.omega[i] = x
        elif k in ("periodic", "force"):
            for i, x in enumerate(v):
                getattr(p, k)[i] = x
        else:
            setattr(p, k, v)
    return p


def _query(p):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    s = _lib.lib().lbm_query_sizes(ctypes.byref(p), ctypes.byref(a), ctypes.byref(b))
    return s, a.value, b.value


def test_query_sizes(L):
    s, pdf, aux = _query(_params(nx=256, ny=256, nz=256))
    assert s == 0 and pdf == 19 * 256 ** 3 * 4
    assert aux >= 4 * 256 ** 3
    s, pdf, _ = _query(_params(stencil=2, storage=2, nx=8, ny=8, nz=8))
    assert s == 0 and pdf == 27 * 512 * 2
    s, pdf, _ = _query(_params(stencil=0, storage=0, nx=64, ny=64, nz=1))
    assert s == 0 and pdf == 9 * 64 * 64 * 8


@pytest.mark.parametrize("kw,status", [
    (dict(nx=0), 1), (dict(stencil=7), 1), (dict(collision=9), 1), (dict(storage=5), 1), (dict(pattern=3), 1),
    (dict(stencil=0, nz=2), 1), (dict(omega=[2.5]), 1), (dict(omega=[0.0]), 1), (dict(ny=70000), 1),
    (dict(collision=3, stencil=1, omega=[1.5, 1, 1]), 2), (dict(collision=3, stencil=0, nz=1, omega=[1.5, 1, 1]), 2),
    (dict(rho_outlet=-1.0), 1), (dict(collision=1, trt_magic=1, magic=-1.0), 1),
    (dict(collision=4, omega=[1.9, 0.0]), 1), (dict(collision=4, omega=[1.9, 1.0], force=(1e-4, 0.0, 0.0)), 2),
    (dict(collision=4, omega=[1.9, 1.0], smagorinsky_cs=0.1), 2), (dict(collision=2, smagorinsky_cs=0.1), 2),
    (dict(collision=5), 1), (dict(boundary_mode=2), 1), (dict(boundary_mode=1, pattern=1), 2),
    (dict(boundary_mode=1, pattern=2), 2),
])
def test_invalid_parameters(L, kw, status):
    s, _, _ = _query(_params(**kw))
    assert s == status


def test_create_rejects_bad_buffers_without_touching_the_gpu(L):
    p = _params(nx=4, ny=4, nz=4)
    ctx = ctypes.c_void_p()
    s, pdf, aux = _query(p)
    fake = 0x1000
    # pdf2 missing for the pull pattern
    assert L.lbm_create(ctypes.byref(ctx), ctypes.byref(p), fake, pdf, None, 0, fake, aux, None, None) == 1
    # buffers too small
    assert L.lbm_create(ctypes.byref(ctx), ctypes.byref(p), fake, pdf - 1, fake, pdf, fake, aux, None, None) == 5
    assert L.lbm_create(ctypes.byref(ctx), ctypes.byref(p), fake, pdf, fake, pdf, fake, aux - 1, None, None) == 5
    assert L.lbm_create(None, ctypes.byref(p), fake, pdf, fake, pdf, fake, aux, None, None) == 1
    assert L.lbm_status_str(5) == b"LBM_E_BUFSIZE"
    assert L.lbm_last_error(None) == b""


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q27"])
def test_stencil_table_matches_documented_order(L, name):
    q, d, c, w = _lib.stencil_info(name)
    ref = olat.get(name)
    assert q == ref.q and d == ref.d
    assert [tuple(v[:d]) for v in c] == ref.c_list
    assert np.allclose(w, ref.w, rtol=0, atol=1e-17)


def test_injected_host_allocation_failure(L):
    """lbm_create reports a failed host allocation as LBM_E_NOMEM and leaves
    nothing behind; the next create succeeds.  A periodic box without flags
    makes no CUDA call at create time, so fake device pointers suffice."""
    p = _params(nx=4, ny=4, nz=4)
    ctx = ctypes.c_void_p()
    s, pdf, aux = _query(p)
    fake = 0x1000
    L.lbm_debug_fail_host_allocs(1)
    assert L.lbm_create(ctypes.byref(ctx), ctypes.byref(p), fake, pdf, fake, pdf, fake, aux, None, None) == 4
    assert not ctx.value
    assert L.lbm_create(ctypes.byref(ctx), ctypes.byref(p), fake, pdf, fake, pdf, fake, aux, None, None) == 0
    assert ctx.value
    assert L.lbm_last_error(ctx) == b""
    L.lbm_destroy(ctx)
    L.lbm_debug_fail_host_allocs(0)
