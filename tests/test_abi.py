"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; argument validation happens before any device call."""
import ctypes
import glob
import os
import re

import pytest

from paper_1806_10251_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lbm_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_step", "lbm_run_to_steady", "lbm_fields", "lbm_destroy",
                     "lbm_set_option", "lbm_last_error", "lbm_save", "lbm_load"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = lbm.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(lbm.SIGNATURES)


def test_invalid_arguments_rejected_without_device():
    L = lbm.lib()
    h = ctypes.c_void_p()
    assert L.lbm_create(2, 16, 0.1, 0.5, 0.1, None, ctypes.byref(h)) == lbm.ERR_INVALID
    assert b"nx" in L.lbm_last_error()
    assert L.lbm_create(16, 16, -1.0, 0.5, 0.1, None, ctypes.byref(h)) == lbm.ERR_INVALID
    assert L.lbm_create(16, 16, 0.1, 1.5, 0.1, None, ctypes.byref(h)) == lbm.ERR_INVALID
    assert L.lbm_create(16, 16, 0.1, 0.0, 0.1, None, ctypes.byref(h)) == lbm.ERR_INVALID
    assert L.lbm_step(None, 1) == lbm.ERR_INVALID
    L.lbm_destroy(None)  # NULL-safe
    b, _ = lbm.make_boundaries([(0, 0, 0), (1, 0, 0), (1, 0, 0), (1, 0, 0)])
    assert L.lbm_create(16, 16, 0.1, 0.5, 0.1, ctypes.byref(b), ctypes.byref(h)) == lbm.ERR_INVALID
    assert b"periodic" in L.lbm_last_error()


def test_no_cpu_fallback_without_gpu():
    """On a machine without a usable GPU the library reports LBM_ERR_CUDA."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(lbm.LbmError) as e:
        lbm.Solver(16, 16, 0.1, 0.5, 0.1)
    assert e.value.status == lbm.ERR_CUDA
