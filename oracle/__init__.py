"""FP64 CPU oracle for the GI preconditioned cascaded central-moment LBM (D2Q9).

TEST INFRASTRUCTURE ONLY.  The plain C oracle in ``gi_oracle.c`` is the
reference the CUDA path is checked against; this module compiles it with gcc
(OpenMP, no fast-math, no FMA contraction) and wraps it with ctypes.  Only the
test suite, the smoke check and the CPU-baseline leg of the benchmark may import
it.  It imports nothing from the product package.

Parameters follow the paper's notation (arXiv 1806.10251): ``gamma`` is the
preconditioning parameter, ``nu`` the kinematic viscosity, and the shear rates
follow nu = (gamma/3)(1/omega - 1/2) (Eq. 49, Sec. 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgi_oracle.so")
_lock = threading.Lock()
_lib = None

GI_UNCORRECTED, GI_CUBIC_ONLY, GI_FULL = 0, 1, 2
FD_CENTRAL, FD_ISOTROPIC = 0, 1
SIDE_PERIODIC, SIDE_WALL, SIDE_MOVING_WALL, SIDE_INLET, SIDE_OUTLET = 0, 1, 2, 3, 4


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("omega", ctypes.c_double * 9),
        ("gi_mode", ctypes.c_int), ("fd_scheme", ctypes.c_int), ("guard", ctypes.c_int),
        ("side_kind", ctypes.c_int * 4),
        ("side_u", (ctypes.c_double * 2) * 4),
        ("rho0", ctypes.c_double),
        ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libgi_oracle.so`` (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "gi_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_set_force_field.argtypes = [ctypes.c_void_p, dp, dp]
            L.orc_init_equilibrium.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            L.orc_get_pops.argtypes = [ctypes.c_void_p, dp]
            L.orc_set_pops.argtypes = [ctypes.c_void_p, dp]
            L.orc_fields.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_used_fields.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_residual.restype = ctypes.c_double
            L.orc_residual.argtypes = [ctypes.c_void_p, dp]
            L.orc_steps_done.restype = ctypes.c_long
            L.orc_steps_done.argtypes = [ctypes.c_void_p]
            L.orc_guard_count.restype = ctypes.c_long
            L.orc_guard_count.argtypes = [ctypes.c_void_p]
            L.orc_drag.argtypes = [ctypes.c_void_p, dp]
            L.orc_density_gradient_field.argtypes = [ctypes.c_void_p] * 4
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_get_threads.restype = ctypes.c_int
            L.orc_lattice.argtypes = [ctypes.c_void_p] * 4
            L.orc_raw_moments.argtypes = [dp, dp]
            L.orc_pops_from_raw.argtypes = [dp, dp]
            L.orc_raw_equilibrium.argtypes = [ctypes.c_double] * 4 + [dp]
            L.orc_source_moments.argtypes = [ctypes.c_double] * 5 + [dp]
            L.orc_K_columns.argtypes = [dp]
            L.orc_gi_coefficients.argtypes = [ctypes.c_double] * 7 + [dp]
            L.orc_strain_rates.restype = ctypes.c_int
            L.orc_strain_rates.argtypes = [ctypes.c_double] * 10 + [ctypes.c_int, dp, dp]
            L.orc_collide_cell.restype = ctypes.c_int
            L.orc_collide_cell.argtypes = [ctypes.POINTER(OrcParams), dp, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, dp, dp, dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def omega_from_nu(nu: float, gamma: float) -> float:
    """Eq. 49 / Sec. 2: nu = (gamma/3)(1/omega - 1/2)  =>  omega = 1/(3 nu/gamma + 1/2)."""
    return 1.0 / (3.0 * nu / gamma + 0.5)


def make_params(nx, ny, gamma, omega, gi_mode=GI_FULL, fd=FD_CENTRAL, guard=False,
                sides=((SIDE_WALL, 0.0, 0.0),) * 4, Fx=0.0, Fy=0.0, rho0=1.0) -> OrcParams:
    p = OrcParams()
    p.nx, p.ny, p.gamma = int(nx), int(ny), float(gamma)
    for i in range(9):
        p.omega[i] = float(omega[i])
    p.gi_mode, p.fd_scheme, p.guard = int(gi_mode), int(fd), int(bool(guard))
    for s in range(4):
        kind, uw, vw = sides[s]
        p.side_kind[s] = int(kind)
        p.side_u[s][0] = float(uw)
        p.side_u[s][1] = float(vw)
    p.rho0 = float(rho0)
    p.Fx, p.Fy = float(Fx), float(Fy)
    return p


def omegas(nu: float, gamma: float, omega3=1.0, omega6=1.0, omega7=1.0, omega8=1.0):
    w = omega_from_nu(nu, gamma)
    return [0.0, 0.0, 0.0, omega3, w, w, omega6, omega7, omega8]


class Domain:
    """Whole-domain oracle.  Population arrays are (9, ny, nx) float64."""

    def __init__(self, nx, ny, nu, gamma, sides, gi_mode=GI_FULL, fd=FD_CENTRAL, guard=False,
                 solid=None, Fx=0.0, Fy=0.0, omega3=1.0, omega6=1.0, omega7=1.0, omega8=1.0):
        L = lib()
        self.nx, self.ny, self.gamma = int(nx), int(ny), float(gamma)
        self.params = make_params(nx, ny, gamma, omegas(nu, gamma, omega3, omega6, omega7, omega8),
                                  gi_mode, fd, guard, sides, Fx, Fy)
        self._solid = None
        if solid is not None:
            self._solid = np.ascontiguousarray(solid, dtype=np.uint8).reshape(ny, nx)
        ptr = self._solid.ctypes.data_as(ctypes.c_void_p) if self._solid is not None else None
        self._h = L.orc_create(ctypes.byref(self.params), ptr)
        if not self._h:
            raise MemoryError("orc_create failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_force_field(self, Fx, Fy):
        Fx = np.ascontiguousarray(Fx, dtype=np.float64).reshape(self.ny, self.nx)
        Fy = np.ascontiguousarray(Fy, dtype=np.float64).reshape(self.ny, self.nx)
        if lib().orc_set_force_field(self._h, _dp(Fx), _dp(Fy)) != 0:
            raise MemoryError("orc_set_force_field")

    def init_equilibrium(self, rho=None, ux=None, uy=None):
        args = []
        keep = []
        for a in (rho, ux, uy):
            if a is None:
                args.append(None)
            else:
                a = np.ascontiguousarray(np.broadcast_to(a, (self.ny, self.nx)), dtype=np.float64)
                keep.append(a)
                args.append(a.ctypes.data_as(ctypes.c_void_p))
        lib().orc_init_equilibrium(self._h, *args)

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    @property
    def steps(self):
        return lib().orc_steps_done(self._h)

    @property
    def guard_count(self):
        return lib().orc_guard_count(self._h)

    def pops(self):
        f = np.empty((9, self.ny, self.nx))
        lib().orc_get_pops(self._h, _dp(f))
        return f

    def density_gradient(self, rho):
        """The domain's density-gradient stencil applied to rho (ny, nx)."""
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ny, self.nx)
        gx, gy = np.empty((self.ny, self.nx)), np.empty((self.ny, self.nx))
        lib().orc_density_gradient_field(self._h, _dp(rho), _dp(gx), _dp(gy))
        return gx, gy

    def set_pops(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        lib().orc_set_pops(self._h, _dp(f))

    def fields(self):
        r, u, v = (np.empty((self.ny, self.nx)) for _ in range(3))
        lib().orc_fields(self._h, r.ctypes.data_as(ctypes.c_void_p), u.ctypes.data_as(ctypes.c_void_p),
                         v.ctypes.data_as(ctypes.c_void_p))
        return r, u, v

    def used_fields(self):
        r, u, v = (np.empty((self.ny, self.nx)) for _ in range(3))
        lib().orc_used_fields(self._h, r.ctypes.data_as(ctypes.c_void_p), u.ctypes.data_as(ctypes.c_void_p),
                              v.ctypes.data_as(ctypes.c_void_p))
        return r, u, v

    def residual(self):
        s = np.zeros(5)
        r = lib().orc_residual(self._h, _dp(s))
        return r, s

    def drag(self):
        """Momentum-exchange force on the solid cells (lattice momentum per step)."""
        F = np.zeros(2)
        lib().orc_drag(self._h, _dp(F))
        return F


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return lib().orc_get_threads()


# ---- per-cell wrappers for the pins ------------------------------------------
def lattice():
    ex, ey, opp = (np.zeros(9, dtype=np.int32) for _ in range(3))
    w = np.zeros(9)
    lib().orc_lattice(ex.ctypes.data_as(ctypes.c_void_p), ey.ctypes.data_as(ctypes.c_void_p),
                      w.ctypes.data_as(ctypes.c_void_p), opp.ctypes.data_as(ctypes.c_void_p))
    return ex, ey, w, opp


def raw_moments(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    k = np.zeros(9)
    lib().orc_raw_moments(_dp(f), _dp(k))
    return k


def pops_from_raw(k):
    k = np.ascontiguousarray(k, dtype=np.float64)
    f = np.zeros(9)
    lib().orc_pops_from_raw(_dp(k), _dp(f))
    return f


def raw_equilibrium(rho, ux, uy, gamma):
    k = np.zeros(9)
    lib().orc_raw_equilibrium(rho, ux, uy, gamma, _dp(k))
    return k


def source_moments(Fx, Fy, ux, uy, gamma):
    s = np.zeros(9)
    lib().orc_source_moments(Fx, Fy, ux, uy, gamma, _dp(s))
    return s


def K_columns():
    K = np.zeros((9, 9))
    lib().orc_K_columns(_dp(K))
    return K


def gi_coefficients(rho, ux, uy, gamma, w3, w4, w5):
    c = np.zeros(12)
    lib().orc_gi_coefficients(rho, ux, uy, gamma, w3, w4, w5, _dp(c))
    return c


def strain_rates(rho, ux, uy, gamma, w3, w4, m3, m4, drx, dry, guard=False):
    a = ctypes.c_double()
    b = ctypes.c_double()
    g = lib().orc_strain_rates(rho, ux, uy, gamma, w3, w4, m3, m4, drx, dry, int(guard),
                               ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value, g


def collide_cell(params: OrcParams, fbar, drx=0.0, dry=0.0, Fx=0.0, Fy=0.0):
    fbar = np.ascontiguousarray(fbar, dtype=np.float64)
    ft, gh, M = np.zeros(9), np.zeros(9), np.zeros(3)
    guarded = lib().orc_collide_cell(ctypes.byref(params), _dp(fbar), drx, dry, Fx, Fy,
                                     _dp(ft), _dp(gh), _dp(M))
    return ft, gh, M, guarded
