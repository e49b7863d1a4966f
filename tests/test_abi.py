"""CPU checks of the C-ABI boundary: the library builds, exports every symbol
the header declares, and its loader refuses to fall back to anything else."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "glasso.h")


def _declared():
    text = open(HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(glasso_[A-Za-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1607_00315_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("glasso_create", "glasso_destroy", "glasso_solve", "glasso_solve_batch",
                     "glasso_submit", "glasso_poll", "glasso_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(glasso_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_lists_match_header(lib_path):
    from paper_1607_00315_gb300 import glasso

    assert sorted(glasso.EXPORTED) == _declared()


def test_library_loads_and_reports_without_gpu(lib_path):
    import ctypes

    import torch

    from paper_1607_00315_gb300 import glasso

    L = glasso.load()
    assert L.glasso_strerror(glasso.EINVAL) == b"invalid argument"
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        cfg = glasso.Config(0, 0, glasso.FP64)
        s = L.glasso_create(ctypes.byref(cfg), ctypes.byref(h))
        assert s == glasso.ECUDA and not h.value
        # bad arguments are rejected before any device work
        assert L.glasso_create(None, ctypes.byref(h)) == glasso.EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1607_00315_gb300 import glasso

    monkeypatch.setattr(glasso, "_lib", None)
    monkeypatch.setattr(glasso, "LIB_PATH", str(tmp_path / "libglasso.so"))
    with pytest.raises(RuntimeError, match="not built"):
        glasso.load()
