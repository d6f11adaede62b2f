"""ctypes binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every step of the method runs in the CUDA library; nothing here computes.  If
the library cannot be built or loaded, :func:`lib` raises -- there is no CPU
fallback.  Function names match the C entry points.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_DIVERGED, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_IO = 0, -1, -2, -3, -4, -5, -6, -7
SIDE_PERIODIC, SIDE_WALL, SIDE_MOVING_WALL, SIDE_INLET, SIDE_OUTLET = 0, 1, 2, 3, 4
STORAGE_F32, STORAGE_F16, STORAGE_BF16, STORAGE_F64 = 0, 1, 2, 3
GI_UNCORRECTED, GI_CUBIC_ONLY, GI_FULL = 0, 1, 2
FD_CENTRAL, FD_ISOTROPIC = 0, 1  # values of the "fd" option (density-gradient stencil)

_STATUS = {0: "LBM_OK", -1: "LBM_ERR_INVALID", -2: "LBM_ERR_OOM", -3: "LBM_ERR_CUDA", -4: "LBM_ERR_DIVERGED",
           -5: "LBM_ERR_NOT_CONVERGED", -6: "LBM_ERR_TIMEOUT", -7: "LBM_ERR_IO"}


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class Side(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ux", ctypes.c_double), ("uy", ctypes.c_double)]


class Boundaries(ctypes.Structure):
    _fields_ = [("west", Side), ("east", Side), ("south", Side), ("north", Side),
                ("solid", ctypes.c_void_p)]


class Request(ctypes.Structure):
    """lbm_request: one steady solve submitted to a batch."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nu", ctypes.c_double), ("gamma", ctypes.c_double),
                ("U", ctypes.c_double), ("bnd", Boundaries), ("use_bnd", ctypes.c_int), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("tol", ctypes.c_double), ("max_steps", ctypes.c_long),
                ("check_every", ctypes.c_long)]


class Result(ctypes.Structure):
    """lbm_result: state of a submitted request."""
    _fields_ = [("state", ctypes.c_int), ("steps", ctypes.c_long), ("residual", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


REQ_QUEUED, REQ_RUNNING, REQ_CONVERGED, REQ_NOT_CONVERGED, REQ_DIVERGED, REQ_FAILED, REQ_CANCELLED = range(7)


class PopulationDesc(ctypes.Structure):
    """lbm_population_desc: a caller-owned device population array."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pitch", ctypes.c_int), ("storage", ctypes.c_int),
                ("gamma", ctypes.c_double), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("solid_dev", ctypes.c_void_p)]


NOALLOC_MAX_CELLS = 65536 * 256

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("release", _FREE_FN), ("user", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()

# C signatures: name -> (restype, argtypes)
_P = ctypes.c_void_p
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_L = ctypes.c_long
SIGNATURES = {
    "lbm_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _D, _D, _D, ctypes.POINTER(Boundaries),
                                  ctypes.POINTER(_P)]),
    "lbm_set_option": (ctypes.c_int, [_P, ctypes.c_char_p, _D]),
    "lbm_get_option": (ctypes.c_int, [_P, ctypes.c_char_p, _DP]),
    "lbm_set_stream": (ctypes.c_int, [_P, _P]),
    "lbm_set_force_field": (ctypes.c_int, [_P, _P, _P]),
    "lbm_init_fields": (ctypes.c_int, [_P, _P, _P, _P]),
    "lbm_step": (ctypes.c_int, [_P, _L]),
    "lbm_run_to_steady": (ctypes.c_int, [_P, _D, _L, _L, _D, ctypes.POINTER(_L), _DP]),
    "lbm_residual": (ctypes.c_int, [_P, _DP, _DP]),
    "lbm_residual_history": (ctypes.c_int, [_P, _P, _P, _L, ctypes.POINTER(_L)]),
    "lbm_fields": (ctypes.c_int, [_P, _P, _P, _P]),
    "lbm_get_populations": (ctypes.c_int, [_P, _P]),
    "lbm_set_populations": (ctypes.c_int, [_P, _P]),
    "lbm_steps_done": (ctypes.c_int, [_P, ctypes.POINTER(_L)]),
    "lbm_guard_count": (ctypes.c_int, [_P, ctypes.POINTER(_L)]),
    "lbm_drag": (ctypes.c_int, [_P, _P]),
    "lbm_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "lbm_load": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "lbm_destroy": (None, [_P]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_bounded_wait_selftest": (ctypes.c_int, [_P, _DP]),
    "lbm_set_allocator": (ctypes.c_int, [ctypes.POINTER(Allocator)]),
    "lbm_kernel_launches": (ctypes.c_int, [_P, ctypes.POINTER(_L)]),
    "lbm_residual_sums_noalloc": (ctypes.c_int, [ctypes.POINTER(PopulationDesc), _P, _P, _P, _P, _P]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)]),
    "lbm_batch_set_option": (ctypes.c_int, [_P, ctypes.c_char_p, _D]),
    "lbm_batch_submit": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.POINTER(_L)]),
    "lbm_batch_poll": (ctypes.c_int, [_P, _L, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Result)]),
    "lbm_batch_fields": (ctypes.c_int, [_P, _L, _P, _P, _P]),
    "lbm_batch_release": (ctypes.c_int, [_P, _L]),
    "lbm_batch_cancel": (ctypes.c_int, [_P, _L]),
    "lbm_batch_run": (ctypes.c_int, [_P, _D]),
    "lbm_batch_start": (ctypes.c_int, [_P]),
    "lbm_batch_stop": (ctypes.c_int, [_P]),
    "lbm_batch_stats": (ctypes.c_int, [_P, _DP]),
    "lbm_batch_destroy": (None, [_P]),
}


def debug_bounds() -> bool:
    """LBM_DEBUG_BOUNDS=1 in the environment selects the bounds-checking build."""
    return os.environ.get("LBM_DEBUG_BOUNDS", "0") not in ("", "0")


def library_path() -> str:
    return _build.DEBUG_LIB if debug_bounds() else _build.LIB


def lib() -> ctypes.CDLL:
    """Build (if stale) and load the CUDA library; raises if that fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(debug=debug_bounds())
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().lbm_last_error().decode()


def check(status: int) -> None:
    if status != OK:
        raise LbmError(status, last_error())


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def make_boundaries(sides: Sequence, solid: Optional[np.ndarray] = None):
    """sides: four (kind, ux, uy) tuples for west, east, south, north."""
    b = Boundaries()
    for name, (kind, uw, vw) in zip(("west", "east", "south", "north"), sides):
        setattr(b, name, Side(int(kind), float(uw), float(vw)))
    keep = None
    if solid is not None:
        keep = np.ascontiguousarray(solid, dtype=np.uint8)
        b.solid = keep.ctypes.data_as(ctypes.c_void_p)
    return b, keep


# ---- PyTorch as the device-memory provider -----------------------------------
_torch_blocks = {}
_torch_alloc_ref = None


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _torch_alloc_ref
    if not enable:
        check(lib().lbm_set_allocator(None))
        _torch_alloc_ref = None
        return
    import torch

    def _alloc(nbytes, _user):
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        except Exception:  # allocation failure is reported to the library as NULL
            return None
        ptr = t.data_ptr()
        _torch_blocks[ptr] = t
        return ptr

    def _free(ptr, _user):
        _torch_blocks.pop(int(ptr) if ptr else 0, None)

    a = Allocator(_ALLOC_FN(_alloc), _FREE_FN(_free), None)
    _torch_alloc_ref = a  # keep the callbacks alive
    check(lib().lbm_set_allocator(ctypes.byref(a)))


class Solver:
    """One domain (an ``lbm_ctx``).  Methods map one-to-one onto the C ABI."""

    def __init__(self, nx: int, ny: int, nu: float, gamma: float, U: float = 0.0,
                 sides: Optional[Sequence] = None, solid: Optional[np.ndarray] = None):
        L = lib()
        self.nx, self.ny = int(nx), int(ny)
        self._h = ctypes.c_void_p()
        if sides is None and solid is None:
            check(L.lbm_create(self.nx, self.ny, float(nu), float(gamma), float(U), None, ctypes.byref(self._h)))
        else:
            if sides is None:
                sides = ((SIDE_WALL, 0, 0), (SIDE_WALL, 0, 0), (SIDE_WALL, 0, 0), (SIDE_MOVING_WALL, U, 0))
            b, keep = make_boundaries(sides, solid)
            check(L.lbm_create(self.nx, self.ny, float(nu), float(gamma), float(U), ctypes.byref(b),
                               ctypes.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().lbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- options
    def set_option(self, key: str, value: float):
        check(lib().lbm_set_option(self._h, key.encode(), float(value)))

    def get_option(self, key: str) -> float:
        v = ctypes.c_double()
        check(lib().lbm_get_option(self._h, key.encode(), ctypes.byref(v)))
        return v.value

    def set_stream(self, stream_handle: Optional[int]):
        check(lib().lbm_set_stream(self._h, ctypes.c_void_p(stream_handle) if stream_handle else None))

    def set_force_field(self, fx: Optional[np.ndarray], fy: Optional[np.ndarray]):
        if fx is None:
            check(lib().lbm_set_force_field(self._h, None, None))
            return
        fx = np.ascontiguousarray(fx, dtype=np.float64).reshape(self.ny, self.nx)
        fy = np.ascontiguousarray(fy, dtype=np.float64).reshape(self.ny, self.nx)
        check(lib().lbm_set_force_field(self._h, _ptr(fx), _ptr(fy)))

    def init_fields(self, rho=None, ux=None, uy=None):
        arrs = [None if a is None else np.ascontiguousarray(np.broadcast_to(a, (self.ny, self.nx)), dtype=np.float64)
                for a in (rho, ux, uy)]
        check(lib().lbm_init_fields(self._h, *[_ptr(a) for a in arrs]))

    # -- stepping
    def step(self, n: int = 1):
        check(lib().lbm_step(self._h, int(n)))

    def run_to_steady(self, tol: float, check_every: int, max_steps: int, wall_seconds: float = 0.0,
                      raise_on_error: bool = True):
        steps = ctypes.c_long()
        r = ctypes.c_double()
        s = lib().lbm_run_to_steady(self._h, float(tol), int(check_every), int(max_steps), float(wall_seconds),
                                    ctypes.byref(steps), ctypes.byref(r))
        if s != OK and raise_on_error:
            raise LbmError(s, last_error())
        return s, steps.value, r.value

    def residual_history(self):
        """(steps, residuals) of the last run_to_steady, one entry per check."""
        n = ctypes.c_long()
        check(lib().lbm_residual_history(self._h, None, None, 0, ctypes.byref(n)))
        steps = np.zeros(n.value, dtype=np.int64)
        res = np.zeros(n.value)
        if n.value:
            check(lib().lbm_residual_history(self._h, _ptr(steps), _ptr(res), n.value, ctypes.byref(n)))
        return steps, res

    def residual(self):
        r = ctypes.c_double()
        sums = (ctypes.c_double * 5)()
        check(lib().lbm_residual(self._h, ctypes.byref(r), sums))
        return r.value, np.array(sums[:])

    # -- output
    def fields(self, out=None):
        """(rho, ux, uy) as (ny, nx) float64 arrays; ``out`` may supply them
        (C-contiguous float64, e.g. pinned host memory)."""
        if out is None:
            out = [np.empty((self.ny, self.nx)) for _ in range(3)]
        for a in out:
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.nx * self.ny
        check(lib().lbm_fields(self._h, *[_ptr(a) for a in out]))
        return tuple(out)

    def populations(self) -> np.ndarray:
        f = np.empty((9, self.ny, self.nx))
        check(lib().lbm_get_populations(self._h, _ptr(f)))
        return f

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        check(lib().lbm_set_populations(self._h, _ptr(f)))

    @property
    def steps(self) -> int:
        v = ctypes.c_long()
        check(lib().lbm_steps_done(self._h, ctypes.byref(v)))
        return v.value

    @property
    def kernel_launches(self) -> int:
        v = ctypes.c_long()
        check(lib().lbm_kernel_launches(self._h, ctypes.byref(v)))
        return v.value

    @property
    def guard_count(self) -> int:
        v = ctypes.c_long()
        check(lib().lbm_guard_count(self._h, ctypes.byref(v)))
        return v.value

    def drag(self) -> np.ndarray:
        """Momentum-exchange force on the solid cells (lattice momentum per step)."""
        F = np.zeros(2)
        check(lib().lbm_drag(self._h, _ptr(F)))
        return F

    def bounded_wait_selftest(self):
        """Run lbm_bounded_wait_selftest; returns (status, seconds waited) without
        raising (the expected status is ERR_CUDA)."""
        w = ctypes.c_double()
        st = lib().lbm_bounded_wait_selftest(self._h, ctypes.byref(w))
        return st, w.value

    def save(self, path: str):
        check(lib().lbm_save(self._h, os.fspath(path).encode()))

    def load(self, path: str):
        check(lib().lbm_load(self._h, os.fspath(path).encode()))


def residual_sums_noalloc(desc: PopulationDesc, f_dev: int, snap_ux_dev: int, snap_uy_dev: int, sums_dev: int,
                          stream: Optional[int] = None) -> None:
    """lbm_residual_sums_noalloc on caller-owned device buffers (raw pointers)."""
    check(lib().lbm_residual_sums_noalloc(ctypes.byref(desc), ctypes.c_void_p(f_dev), ctypes.c_void_p(snap_ux_dev),
                                          ctypes.c_void_p(snap_uy_dev), ctypes.c_void_p(sums_dev),
                                          ctypes.c_void_p(stream) if stream else None))


class Batch:
    """A batch of steady solves (``lbm_batch``); methods map onto the C ABI."""

    def __init__(self, hbm_budget_bytes: int, storage: int = STORAGE_F16, gi_mode: int = GI_FULL):
        self._h = ctypes.c_void_p()
        check(lib().lbm_batch_create(int(hbm_budget_bytes), int(storage), int(gi_mode), ctypes.byref(self._h)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().lbm_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: str, value: float):
        check(lib().lbm_batch_set_option(self._h, key.encode(), float(value)))

    def submit(self, nx, ny, nu, gamma, U=0.0, sides=None, solid=None, fx=0.0, fy=0.0, tol=1e-6,
               max_steps=1_000_000, check_every=0) -> int:
        r = Request()
        r.nx, r.ny, r.nu, r.gamma, r.U = int(nx), int(ny), float(nu), float(gamma), float(U)
        keep = None
        if sides is not None or solid is not None:
            if sides is None:
                sides = ((SIDE_WALL, 0, 0), (SIDE_WALL, 0, 0), (SIDE_WALL, 0, 0), (SIDE_MOVING_WALL, U, 0))
            b, keep = make_boundaries(sides, solid)
            r.bnd = b
            r.use_bnd = 1
        r.fx, r.fy, r.tol, r.max_steps = float(fx), float(fy), float(tol), int(max_steps)
        r.check_every = int(check_every)
        rid = ctypes.c_long()
        check(lib().lbm_batch_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        return rid.value

    def submit_case(self, case, tol=1e-6, max_steps=1_000_000, check_every=0) -> int:
        """Submit a ``workloads.Case``; a batch starts every domain at rest and
        takes a uniform body force only."""
        if case.force_x is not None or case.rho0 is not None or case.ux0 is not None:
            raise ValueError("a batch request takes no force field and no initial fields")
        return self.submit(case.nx, case.ny, case.nu, case.gamma, case.U, case.sides, case.solid, case.Fx,
                           case.Fy, tol, max_steps, check_every)

    def poll(self, rid: int):
        done = ctypes.c_int()
        res = Result()
        check(lib().lbm_batch_poll(self._h, int(rid), ctypes.byref(done), ctypes.byref(res)))
        return bool(done.value), res

    def fields(self, rid: int, nx: int, ny: int):
        out = [np.empty((ny, nx)) for _ in range(3)]
        check(lib().lbm_batch_fields(self._h, int(rid), *[_ptr(a) for a in out]))
        return tuple(out)

    def cancel(self, rid: int):
        check(lib().lbm_batch_cancel(self._h, int(rid)))

    def release(self, rid: int):
        check(lib().lbm_batch_release(self._h, int(rid)))

    def run(self, wall_seconds: float = 0.0):
        check(lib().lbm_batch_run(self._h, float(wall_seconds)))

    def start(self):
        check(lib().lbm_batch_start(self._h))

    def stop(self):
        check(lib().lbm_batch_stop(self._h))

    def stats(self) -> dict:
        a = (ctypes.c_double * 6)()
        check(lib().lbm_batch_stats(self._h, a))
        return {"cell_updates": a[0], "launches": int(a[1]), "ticks": int(a[2]), "running": int(a[3]),
                "queued": int(a[4]), "device_bytes": int(a[5])}


def solver_from_case(case, gi_mode: int = GI_FULL, storage: int = STORAGE_F32, **options) -> Solver:
    """Create a Solver for a ``workloads.Case`` (geometry, parameters, initial fields)."""
    s = Solver(case.nx, case.ny, case.nu, case.gamma, case.U, case.sides, case.solid)
    s.set_option("gi_mode", gi_mode)
    if storage != STORAGE_F32:
        s.set_option("storage", storage)
    if case.Fx:
        s.set_option("fx", case.Fx)
    if case.Fy:
        s.set_option("fy", case.Fy)
    for k, v in options.items():
        s.set_option(k, v)
    if case.force_x is not None:
        s.set_force_field(case.force_x, case.force_y)
    s.init_fields(case.rho0, case.ux0, case.uy0)
    return s
