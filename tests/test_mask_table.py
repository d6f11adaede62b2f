"""The host-side row table of a solid mask (csrc/mask_table.cu), which decides
whether a step kernel's work item may skip the per-cell solid logic: built
with the host compiler alone and compared with a brute-force table from its
definition (flag[r][b] = a solid cell in rows r-1 .. r+1 and columns
32b-34 .. 32b+65, periodic sides wrapping, wall sides clipping), and the device
layout (the 0/1 mask on its pitch, then the table).  A flag missing where a
solid lies in reach would let an item stream from a solid cell, so every
mask shape that stresses the ranges is covered: seams of 32-column blocks, the
last ragged block, the wrap in x and y, domains narrower than the range."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1806_10251_gb300", "csrc", "mask_table.cu")

SHIM = r"""
#include <stdint.h>
#include <string.h>
#include <vector>
namespace lbm {
std::vector<uint8_t> make_solid_rows(const uint8_t *mask, int nx, int ny, bool perx, bool pery);
std::vector<uint8_t> mask_with_row_table(const uint8_t *mask, int nx, int ny, int pitch, bool perx, bool pery);
}
extern "C" long table(const uint8_t *m, int nx, int ny, int px, int py, uint8_t *out) {
    const std::vector<uint8_t> v = lbm::make_solid_rows(m, nx, ny, px != 0, py != 0);
    memcpy(out, v.data(), v.size());
    return (long)v.size();
}
extern "C" long layout(const uint8_t *m, int nx, int ny, int pitch, int px, int py, uint8_t *out) {
    const std::vector<uint8_t> v = lbm::mask_with_row_table(m, nx, ny, pitch, px != 0, py != 0);
    memcpy(out, v.data(), v.size());
    return (long)v.size();
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("mask_table")
    shim = d / "shim.cpp"
    shim.write_text(SHIM)
    so = d / "libmask_table.so"
    subprocess.run([gxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-x", "c++", SRC, "-x", "c++", str(shim),
                    "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    for f in (L.table, L.layout):
        f.restype = ctypes.c_long
    return L


def brute(mask, perx, pery):
    ny, nx = mask.shape
    nb = (nx + 31) // 32
    out = np.zeros((ny, nb), np.uint8)
    for r in range(ny):
        for b in range(nb):
            hit = False
            for y in (r - 1, r, r + 1):
                if pery:
                    y %= ny
                elif not 0 <= y < ny:
                    continue
                for x in range(32 * b - 34, 32 * b + 66):
                    if perx:
                        x %= nx
                    elif not 0 <= x < nx:
                        continue
                    if mask[y, x]:
                        hit = True
                        break
                if hit:
                    break
            out[r, b] = hit
    return out


def masks():
    rng = np.random.default_rng(3)
    for nx, ny in ((301, 45), (64, 7), (97, 5), (40, 6), (130, 3)):
        m = np.zeros((ny, nx), np.uint8)
        for x in {0, 31, 32, 63, 64, 95, 96, nx - 1} & set(range(nx)):
            m[rng.integers(0, ny), x] = 1
        yield m
        yield (rng.random((ny, nx)) < 0.004).astype(np.uint8)
    yield np.zeros((9, 200), np.uint8)
    one = np.zeros((9, 200), np.uint8)
    one[0, 199] = 1
    yield one


@pytest.mark.parametrize("perx,pery", [(False, False), (True, False), (False, True), (True, True)])
def test_row_table_matches_its_definition(lib, perx, pery):
    for m in masks():
        ny, nx = m.shape
        nb = (nx + 31) // 32
        out = np.zeros(ny * nb, np.uint8)
        n = lib.table(m.ctypes.data_as(ctypes.c_void_p), nx, ny, int(perx), int(pery),
                      out.ctypes.data_as(ctypes.c_void_p))
        assert n == ny * nb
        assert np.array_equal(out.reshape(ny, nb), brute(m, perx, pery)), (m.shape, perx, pery)


def test_device_layout_is_mask_then_table(lib):
    m = (np.random.default_rng(5).random((33, 150)) < 0.02).astype(np.uint8) * 7  # any nonzero is solid
    ny, nx = m.shape
    pitch = 192
    nb = (nx + 31) // 32
    out = np.zeros(pitch * ny + ny * nb, np.uint8)
    n = lib.layout(m.ctypes.data_as(ctypes.c_void_p), nx, ny, pitch, 0, 1, out.ctypes.data_as(ctypes.c_void_p))
    assert n == out.size
    plane = out[:pitch * ny].reshape(ny, pitch)
    assert np.array_equal(plane[:, :nx], (m != 0).astype(np.uint8))
    assert not plane[:, nx:].any()
    assert np.array_equal(out[pitch * ny:].reshape(ny, nb), brute(m != 0, False, True))
