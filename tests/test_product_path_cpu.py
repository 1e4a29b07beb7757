"""The product path stands on its own: it never imports the oracle, and it
fails loudly (no CPU fallback) when liblbm.so is missing.  Runs in fresh
interpreters so that nothing another test imported leaks in."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PRODUCT_MODULES = ["paper_2001_11806_gb300", "paper_2001_11806_gb300._lib", "paper_2001_11806_gb300.sim",
                   "paper_2001_11806_gb300.adjoint", "paper_2001_11806_gb300.inputs", "paper_2001_11806_gb300.build"]


def _run(code):
    env = dict(os.environ)
    env.pop("LBM_DEBUG_BOUNDS", None)
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=300)


def test_product_modules_do_not_import_the_oracle():
    code = ("import importlib, sys\n"
            f"for m in {PRODUCT_MODULES!r}:\n"
            "    importlib.import_module(m)\n"
            "bad = sorted(k for k in sys.modules if k == 'oracle' or k.startswith('oracle.'))\n"
            "print('ORACLE_MODULES', bad)\n")
    r = _run(code)
    assert r.returncode == 0, r.stderr
    assert "ORACLE_MODULES []" in r.stdout, r.stdout


def test_missing_library_raises_instead_of_falling_back():
    code = ("from paper_2001_11806_gb300 import _lib\n"
            "_lib.LIB_PATH = _lib.LIB_PATH + '.absent'\n"
            "_lib._LIB = None\n"
            "from paper_2001_11806_gb300.sim import Sim\n"
            "try:\n"
            "    Sim('D3Q19', 'trt', 'f32', 'aa', (8, 8, 8), omega=[1.8], trt_magic=3 / 16, device='cpu')\n"
            "except _lib.LbmError as e:\n"
            "    print('RAISED', 'is not built' in str(e))\n"
            "else:\n"
            "    print('NO ERROR')\n")
    r = _run(code)
    assert r.returncode == 0, r.stderr
    assert "RAISED True" in r.stdout, (r.stdout, r.stderr)
