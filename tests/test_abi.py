"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; argument validation happens before any device call."""
import ctypes
import glob
import os
import re
import subprocess

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
    n = ctypes.c_long(-1)
    assert L.lbm_residual_history(None, None, None, 0, ctypes.byref(n)) == lbm.ERR_INVALID and n.value == -1
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


def declared_prototypes():
    """name -> parameter count of every function prototype in include/*.h."""
    protos = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(lbm_\w+)\s*\(([^;{}]*?)\)\s*;", text):
            params = m.group(2).strip()
            protos[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return protos


def test_binding_arity_matches_prototypes():
    protos = declared_prototypes()
    assert set(protos) == set(declared_functions())
    for name, n in protos.items():
        assert len(lbm.SIGNATURES[name][1]) == n, (name, n, lbm.SIGNATURES[name][1])


STRUCTS = {"lbm_side": lbm.Side, "lbm_boundaries": lbm.Boundaries, "lbm_request": lbm.Request,
           "lbm_result": lbm.Result, "lbm_population_desc": lbm.PopulationDesc, "lbm_allocator": lbm.Allocator}


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets
    (gcc on the header itself)."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines))
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, py in STRUCTS.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
