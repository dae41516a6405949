"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no compute calls: these run without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2009_10173_gb300 import binding, build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(oam_[A-Za-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return ctypes.CDLL(build_lib.OUT)


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("oam_build_model", "oam_forward", "oam_adjoint", "oam_lsqr", "oam_l1_fista"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert set(binding.EXPORTED) == declared_functions()


def test_status_strings_and_version(lib):
    binding._lib = None
    assert binding.status_string(binding.OAM_OK) == "ok"
    assert "window" in binding.status_string(binding.OAM_ERR_WINDOW)
    assert binding.oam_version() >= 100


def test_build_rejects_invalid_arguments_before_touching_the_gpu(lib):
    """Null or inconsistent parameters are refused by the host checks, which
    run before any CUDA call, so this works without a device."""
    from paper_2009_10173_gb300 import configs
    L = binding.lib()
    s, g, e = binding.structs_from_config(configs.TINY_32)
    h = ctypes.c_void_p()
    assert L.oam_build_model(None, ctypes.byref(g), ctypes.byref(e), 0, None, ctypes.byref(h)) == 1
    bad = binding.OamGrid.from_buffer_copy(g)
    bad.win = 10
    assert L.oam_build_model(ctypes.byref(s), ctypes.byref(bad), ctypes.byref(e), 0, None, ctypes.byref(h)) == 1
    bad = binding.OamSensor.from_buffer_copy(s)
    bad.n_patches = 2001
    assert L.oam_build_model(ctypes.byref(bad), ctypes.byref(g), ctypes.byref(e), 0, None, ctypes.byref(h)) == 1
    bad = binding.OamSensor.from_buffer_copy(s)
    bad.aperture_m = 9e-3
    assert L.oam_build_model(ctypes.byref(bad), ctypes.byref(g), ctypes.byref(e), 0, None, ctypes.byref(h)) == 1
    assert L.oam_build_model(ctypes.byref(s), ctypes.byref(g), ctypes.byref(e), 7, None, ctypes.byref(h)) == 1
    assert L.oam_forward(None, None, None, None) == 1
    assert L.oam_model_free(None) == 0
