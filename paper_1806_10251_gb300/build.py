"""Compile the CUDA library in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_1806_10251_gb300/_build/liblbm_gb300.so``.  ``variants.cu`` is compiled
once per (storage type, group of kernel variants) with the defines of
``VARIANT_MATRIX``, so that the large step and batch kernels compile on all
cores at once.  Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm_gb300.so")
# debug build: every computed kernel index checked (LBM_DEBUG_BOUNDS=1)
DEBUG_BUILD = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_BUILD, "liblbm_gb300_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", INCLUDE]


# variants.cu: storage types 0..3 (LBM_STORAGE_*) x groups 0..3 of variants, and
# group 4 (the persistent batch kernel) for the packed storages 0..2
VARIANT_MATRIX = [(st, part) for st in range(4) for part in range(4)] + [(st, 4) for st in range(3)]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in sources() + _headers() + [__file__])


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Build the library (debug=True: the bounds-checking variant, into its own
    folder) and return its path."""
    out_dir, lib_path = (DEBUG_BUILD, DEBUG_LIB) if debug else (BUILD, LIB)
    if debug:
        extra_flags = (*extra_flags, "-DLBM_DEBUG_BOUNDS=1")
    if not force and up_to_date(lib_path):
        return lib_path
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    jobs = []  # (source, object, defines)
    for src in sources():
        stem = os.path.basename(src)[:-3]
        if stem == "variants":
            for st, part in VARIANT_MATRIX:
                jobs.append((src, os.path.join(out_dir, f"variants_s{st}_p{part}.o"),
                             [f"-DLBM_VARIANT_STORAGE={st}", f"-DLBM_VARIANT_PART={part}"]))
        else:
            jobs.append((src, os.path.join(out_dir, stem + ".o"), []))
    # the largest units first, so that the small ones fill in around them
    jobs.sort(key=lambda j: os.path.basename(j[0]) != "variants.cu")
    objs = [j[1] for j in jobs]

    def compile_one(job):
        src, obj, defines = job
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defines, *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}")
        return r.stderr

    with ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 1, len(jobs)))) as ex:
        list(ex.map(compile_one, jobs))
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    v = "-v" in sys.argv
    flags = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(flags), extra_flags=flags))
