"""The C-ABI library loads and exports every entry point include/bounce.h
declares (no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bounce.h")
LIB = os.path.join(ROOT, "paper_2002_07109_gb300", "libbounce.so")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bounce_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2002_07109_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("bounce_create", "bounce_set_topology", "bounce_set_lj", "bounce_set_state", "bounce_run",
                 "bounce_get_state", "bounce_get_energies", "bounce_last_error", "bounce_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header(lib):
    from paper_2002_07109_gb300 import bounce
    assert sorted(bounce.exported_symbols()) == _declared()


def test_host_only_entry_points(lib):
    """Calls that touch no device: config defaults and argument checks."""
    from paper_2002_07109_gb300 import bounce
    cfg = bounce.bounce_config()
    bounce.bounce_config_default(ctypes.byref(cfg))
    assert cfg.dt_fs == 1.0 and cfg.r_off == 5.0 and cfg.max_neighbors == 2048
    assert bounce.bounce_create(None, ctypes.byref(cfg)) == -1
    bad = bounce.bounce_config()
    bounce.bounce_config_default(ctypes.byref(bad))
    bad.dt_fs = -1.0
    h = ctypes.c_void_p()
    assert bounce.bounce_create(ctypes.byref(h), ctypes.byref(bad)) == -1
    assert bounce.bounce_last_error(None) == b"null context"
    assert bounce.bounce_run(None, 1, 1, None) == -1


def test_symbols_are_c_linkage(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (bounce_[a-z_]+)\b", out))
    assert set(_declared()) <= exported
