"""Host logic of the Python binding, on the CPU.

(1) The ctypes mirror of lbm_params has the C layout: a small C program
compiled with the host compiler from include/lbm.h prints sizeof and every
field's offset, which must equal ctypes' (a mismatch would pass shifted
parameters to every call).  (2) ``Sim`` marshals its arguments into that
struct and the buffer sizes of lbm_query_sizes: lbm_create is intercepted
(the rest is the real library), the captured call is checked field by
field, and the intercepted call's error status is raised as LbmError.
(3) set_pdfs refuses a buffer that is not exactly pdf_bytes before the C
call, which copies pdf_bytes from whatever pointer it gets."""
import ctypes
import os
import shutil
import subprocess
import types

import pytest
import torch

from paper_2001_11806_gb300 import _lib
from paper_2001_11806_gb300 import sim as sim_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FIELDS = [f for f, _ in _lib.Params._fields_]

C_PROG = r"""
#include <stddef.h>
#include <stdio.h>
#include "lbm.h"
#define F(name) printf("%s %zu\n", #name, offsetof(lbm_params, name));
int main(void) {
  printf("sizeof %zu\n", sizeof(lbm_params));
  %FIELDS%
  return 0;
}
"""


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _lib.lib()


def test_params_layout_matches_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "layout.c"
    src.write_text(C_PROG.replace("%FIELDS%", " ".join(f"F({f})" for f in FIELDS)))
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    assert int(out["sizeof"]) == ctypes.sizeof(_lib.Params)
    for f in FIELDS:
        assert int(out[f]) == getattr(_lib.Params, f).offset, f


class _Stream:
    cuda_stream = 0x1234


class _Intercept:
    """The real library, with lbm_create recorded and refused."""

    def __init__(self, real):
        self.real = real
        self.call = None

    def __getattr__(self, name):
        return getattr(self.real, name)

    def lbm_create(self, out, p, pdf, pdf_bytes, pdf2, pdf2_bytes, aux, aux_bytes, flags, stream):
        prm = ctypes.cast(p, ctypes.POINTER(_lib.Params)).contents
        self.call = dict(params={f: (list(getattr(prm, f)) if hasattr(getattr(prm, f), "__len__")
                                     else getattr(prm, f)) for f in FIELDS},
                         pdf=pdf, pdf_bytes=pdf_bytes, pdf2=pdf2, pdf2_bytes=pdf2_bytes, aux=aux,
                         aux_bytes=aux_bytes, flags=flags, stream=stream)
        return 2  # LBM_E_UNSUPPORTED: Sim must raise


def _make(monkeypatch, L, **kw):
    fake = _Intercept(L)
    monkeypatch.setattr(sim_mod, "lib", lambda: fake)
    with pytest.raises(_lib.LbmError):
        sim_mod.Sim(device="cpu", stream=_Stream(), **kw)
    return fake.call


def test_sim_marshals_every_parameter(monkeypatch, L):
    shape = (5, 4, 3)
    flags = torch.zeros(shape[::-1], dtype=torch.uint8)
    flags[:, 0, :] = 1
    c = _make(monkeypatch, L, stencil="D3Q27", collision="mrt", storage="f16s", pattern="eso", shape=shape,
              periodic=(True, False, True), omega=[1.7, 1.1, 0.9, 1.3, 1.2, 1.05], incompressible=True,
              u_wall=(0.05, 0.01, 0.0), rho_outlet=1.02, force=(1e-5, -2e-5, 3e-5), flags=flags.numpy())
    p = c["params"]
    assert (p["stencil"], p["collision"], p["storage"], p["pattern"]) == (
        _lib.STENCILS["D3Q27"], _lib.COLLISIONS["mrt"], _lib.STORAGES["f16s"], _lib.PATTERNS["eso"])
    assert (p["nx"], p["ny"], p["nz"]) == shape
    assert p["periodic"] == [1, 0, 1]
    assert p["omega"] == [1.7, 1.1, 0.9, 1.3, 1.2, 1.05]
    assert p["trt_magic"] == 0 and p["incompressible"] == 1
    assert p["u_wall"] == [0.05, 0.01, 0.0] and p["rho_outlet"] == 1.02
    assert p["force"] == [1e-5, -2e-5, 3e-5]
    assert p["smagorinsky_cs"] == 0.0 and p["boundary_mode"] == 0
    N = 5 * 4 * 3
    assert c["pdf_bytes"] == 27 * N * 2
    assert not c["pdf2"] and c["pdf2_bytes"] == 0  # single-array pattern
    assert c["pdf"] and c["aux"] and c["flags"]
    assert c["stream"] == _Stream.cuda_stream


def test_sim_marshals_trt_magic_pull_and_separate_boundary(monkeypatch, L):
    c = _make(monkeypatch, L, stencil="D3Q19", collision="trt", storage="f32", pattern="pull", shape=(6, 5, 4),
              omega=[1.8], trt_magic=3 / 16, smagorinsky_cs=0.17, boundary="separate")
    p = c["params"]
    assert p["omega"] == [1.8, 1.0, 1.0, 1.0, 1.0, 1.0]  # unused rates padded with 1
    assert p["trt_magic"] == 1 and p["magic"] == 3 / 16
    assert p["smagorinsky_cs"] == 0.17 and p["boundary_mode"] == 1
    assert c["pdf2"] and c["pdf2_bytes"] == c["pdf_bytes"] == 19 * 6 * 5 * 4 * 4
    assert not c["flags"]


def test_sim_rejects_flags_of_the_wrong_size(monkeypatch, L):
    fake = _Intercept(L)
    monkeypatch.setattr(sim_mod, "lib", lambda: fake)
    with pytest.raises(_lib.LbmError, match="flags must have N entries"):
        sim_mod.Sim("D3Q19", "srt", "f32", "aa", (4, 4, 4), flags=torch.zeros(10, dtype=torch.uint8).numpy(),
                    device="cpu", stream=_Stream())
    assert fake.call is None


def test_set_pdfs_checks_the_buffer_before_the_copy(monkeypatch):
    # the C call copies pdf_bytes from the pointer it gets; the binding must
    # refuse anything else before the call
    calls = []
    fake = types.SimpleNamespace(lbm_set_pdfs=lambda *a: calls.append(a) or 0)
    monkeypatch.setattr(sim_mod, "lib", lambda: fake)
    s = object.__new__(sim_mod.Sim)
    s.ctx, s.pdf_bytes, s.device = None, 64, torch.device("cpu")
    for bad in (torch.zeros(63, dtype=torch.uint8), torch.zeros(8, dtype=torch.float32),
                torch.zeros(128, dtype=torch.uint8)[::2], b"x" * 64):
        with pytest.raises(_lib.LbmError, match="set_pdfs needs"):
            s.set_pdfs(bad, 3)
    assert not calls
    s.set_pdfs(torch.zeros(16, dtype=torch.float32), 3)  # 64 bytes, contiguous
    assert len(calls) == 1 and calls[0][2] == 3
