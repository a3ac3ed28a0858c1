"""The C example (paper_1903_04946_gb300/examples/rabi.c) uses the library
from plain C through include/dso.h: it compiles and links against the
in-tree library on any machine, and on a GPU it reproduces the exact Rabi
populations of a constant coupling, sin^2(c t), to 1e-12."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1903_04946_gb300")


def _build(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "rabi")
    cmd = [cc, "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(PKG, "examples", "rabi.c"), "-L", PKG, "-ldso_gb300", f"-Wl,-rpath,{PKG}", "-lm",
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_example_compiles_and_links(tmp_path):
    _build(tmp_path)


@pytest.mark.gpu
def test_c_example_reproduces_rabi_oscillation(tmp_path):
    from gpu_util import require_gpu
    require_gpu()
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "max |P2 - sin^2(ct)|" in r.stdout
