"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds only the input recipe -- geometry, parameters and initial
macroscopic fields -- and none of the method's arithmetic (no equilibria, no
relaxation rates, no moments).  Both the FP64 oracle and the CUDA library build
their own initial populations from the (rho, ux, uy) fields given here.

Sides are listed west, east, south, north as (kind, u_wall, v_wall) with kind
0 = periodic, 1 = stationary wall, 2 = moving wall, 3 = parabolic velocity inlet
(west side, u_wall = peak speed), 4 = convective outlet (east side, u_wall =
convection speed).  Arrays are (ny, nx), x fastest.
All random numbers come from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

PERIODIC, WALL, MOVING_WALL, INLET, OUTLET = 0, 1, 2, 3, 4


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    nu: float
    gamma: float
    sides: tuple
    U: float = 0.0                    # lid / reference velocity
    Fx: float = 0.0
    Fy: float = 0.0
    solid: Optional[np.ndarray] = None        # (ny, nx) uint8
    rho0: Optional[np.ndarray] = None         # initial fields; None = rest (rho 1, u 0)
    ux0: Optional[np.ndarray] = None
    uy0: Optional[np.ndarray] = None
    force_x: Optional[np.ndarray] = None      # (ny, nx) force field, overrides Fx/Fy
    force_y: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def cavity(n: int, Re: float, U: float = 0.1, gamma: float = 0.5, ny: Optional[int] = None) -> Case:
    """Lid-driven square cavity: three stationary walls, north lid moving at (U, 0),
    fluid at rest with rho = 1, nu = U n / Re."""
    ny = n if ny is None else ny
    nu = U * n / Re
    sides = ((WALL, 0.0, 0.0), (WALL, 0.0, 0.0), (WALL, 0.0, 0.0), (MOVING_WALL, U, 0.0))
    return Case(f"cavity{n}x{ny}_Re{Re:g}_g{gamma:g}", n, ny, nu, gamma, sides, U=U,
                meta={"Re": Re})


def periodic_sides():
    return ((PERIODIC, 0.0, 0.0),) * 4


def shear_wave(n: int, gamma: float, nu: float, U_frame: float = 0.1, amp: float = 0.05,
               ny: Optional[int] = None) -> Case:
    """Periodic shear wave u_x = U_frame + amp sin(2 pi y / ny), u_y = 0, rho = 1."""
    ny = n if ny is None else ny
    y = np.arange(ny, dtype=np.float64)[:, None]
    ux = np.broadcast_to(U_frame + amp * np.sin(2 * np.pi * y / ny), (ny, n)).copy()
    return Case(f"shearwave{n}x{ny}_g{gamma:g}", n, ny, nu, gamma, periodic_sides(), U=U_frame,
                rho0=np.ones((ny, n)), ux0=ux, uy0=np.zeros((ny, n)),
                meta={"amp": amp, "k": 2 * np.pi / ny})


def taylor_green(n: int, gamma: float, nu: float, u0: float = 0.02, U_frame: float = 0.0) -> Case:
    """Periodic Taylor-Green vortex in a frame moving at (U_frame, 0):
    u_x = U_frame - u0 cos(kx) sin(ky), u_y = u0 sin(kx) cos(ky), rho = 1."""
    k = 2 * np.pi / n
    x = np.arange(n, dtype=np.float64)[None, :]
    y = np.arange(n, dtype=np.float64)[:, None]
    ux = U_frame - u0 * np.cos(k * x) * np.sin(k * y)
    uy = u0 * np.sin(k * x) * np.cos(k * y)
    return Case(f"tgv{n}_g{gamma:g}_U{U_frame:g}", n, n, nu, gamma, periodic_sides(), U=U_frame,
                rho0=np.ones((n, n)), ux0=ux, uy0=uy, meta={"u0": u0, "k": k})


def random_periodic(nx: int, ny: int, gamma: float, nu: float, seed: int = 0,
                    du: float = 0.04, drho: float = 0.01, U_frame=(0.03, -0.02)) -> Case:
    """Periodic box with smooth random rho and u fields (a sum of a few seeded
    Fourier modes), so that every correction term of the collision is exercised."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]

    def field_(scale):
        out = np.zeros((ny, nx))
        for _ in range(4):
            kx, ky = rng.integers(1, 4, size=2)
            ph1, ph2 = rng.uniform(0, 2 * np.pi, size=2)
            a = rng.uniform(-1, 1)
            out += a * np.sin(2 * np.pi * kx * x / nx + ph1) * np.cos(2 * np.pi * ky * y / ny + ph2)
        return scale * out / 4

    rho = 1.0 + field_(drho)
    ux = U_frame[0] + field_(du)
    uy = U_frame[1] + field_(du)
    return Case(f"random{nx}x{ny}_s{seed}", nx, ny, nu, gamma, periodic_sides(),
                rho0=rho, ux0=ux, uy0=uy, meta={"seed": seed})


def random_cavity_state(n: int, ny: int, gamma: float, Re: float = 100.0, U: float = 0.1,
                        seed: int = 0, du: float = 0.03, drho: float = 0.005) -> Case:
    """Cavity geometry started from smooth random fields (exercises walls, lid and
    corrections from the first step on)."""
    base = cavity(n, Re, U, gamma, ny=ny)
    r = random_periodic(n, ny, gamma, base.nu, seed=seed, du=du, drho=drho, U_frame=(0.0, 0.0))
    base.rho0, base.ux0, base.uy0 = r.rho0, r.ux0, r.uy0
    base.name += f"_rand{seed}"
    return base


def channel_obstacle(nx: int = 8192, ny: int = 2048, D: int = 128, Re: float = 40.0,
                     U0: float = 0.05, gamma: float = 0.3, xc: Optional[int] = None) -> Case:
    """Channel periodic in x with stationary walls at y = -1/2 and ny - 1/2, driven by a
    uniform body force F_x = 8 nu U0 / H^2 (the Poiseuille centre-line speed U0 for
    H = ny), with a solid D x D square centred at (xc, ny/2); nu = U0 D / Re."""
    nu = U0 * D / Re
    H = float(ny)
    Fx = 8.0 * nu * U0 / (H * H)
    xc = nx // 8 if xc is None else xc
    yc = ny // 2
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[yc - D // 2: yc - D // 2 + D, xc - D // 2: xc - D // 2 + D] = 1
    sides = ((PERIODIC, 0.0, 0.0), (PERIODIC, 0.0, 0.0), (WALL, 0.0, 0.0), (WALL, 0.0, 0.0))
    return Case(f"channel{nx}x{ny}_D{D}_Re{Re:g}", nx, ny, nu, gamma, sides, U=U0, Fx=Fx,
                solid=solid, meta={"Re": Re, "D": D, "xc": xc})


def poiseuille(nx: int, ny: int, nu: float, gamma: float, Fx: float) -> Case:
    """Body-force-driven channel, periodic in x, stationary walls south and north."""
    sides = ((PERIODIC, 0.0, 0.0), (PERIODIC, 0.0, 0.0), (WALL, 0.0, 0.0), (WALL, 0.0, 0.0))
    return Case(f"poiseuille{nx}x{ny}", nx, ny, nu, gamma, sides, Fx=Fx)


def couette(nx: int, ny: int, nu: float, gamma: float, U: float) -> Case:
    """Periodic in x, stationary south wall, north wall moving at (U, 0)."""
    sides = ((PERIODIC, 0.0, 0.0), (PERIODIC, 0.0, 0.0), (WALL, 0.0, 0.0), (MOVING_WALL, U, 0.0))
    return Case(f"couette{nx}x{ny}", nx, ny, nu, gamma, sides, U=U)


def four_rolls_mill(n: int = 251, u0: float = 0.045, Re: float = 20.0, gamma: float = 0.3) -> Case:
    """Periodic box of side 2 pi resolved by n cells, force
    F = 2 nu u0 (sin x sin y, cos x cos y) in lattice units, nu from Re = u0 L / nu
    with L = n lattice units.  Analytic steady field u = u0 (sin x sin y, cos x cos y)."""
    h = 2 * np.pi / n
    xs = (np.arange(n) + 0.0) * h
    X = xs[None, :]
    Y = xs[:, None]
    nu = u0 * n / Re
    k = h  # d/dx in lattice units: the 2 pi box has n cells
    fx = 2.0 * nu * u0 * k * k * np.sin(X) * np.sin(Y)
    fy = 2.0 * nu * u0 * k * k * np.cos(X) * np.cos(Y)
    ua = u0 * np.sin(X) * np.sin(Y) * np.ones((n, n))
    va = u0 * np.cos(X) * np.cos(Y) * np.ones((n, n))
    return Case(f"fourrolls{n}_g{gamma:g}", n, n, nu, gamma, periodic_sides(), U=u0,
                force_x=fx, force_y=fy, meta={"ua": ua, "va": va, "Re": Re})


def hartmann(nx: int, ny: int, Ha: float, nu: float = 0.1, gamma: float = 0.1, Ma: float = 0.02) -> Case:
    """Hartmann flow (Sec. 6): a channel periodic in x between stationary walls at
    y = -1/2 and ny - 1/2 (half width L = ny/2, z = y + 1/2 - L), driven by a
    driving force F_b plus the Lorentz force B0 dB_x/dz of the induced field
    B_x(z) = (F_b L / B0)[sinh(Ha z/L)/sinh(Ha) - z/L], which together give the
    body force F_x(z) = F_b Ha cosh(Ha z/L) / sinh(Ha).  Analytic steady profile
    u_x(z) = (F_b L^2 / (Ha nu)) coth(Ha) [1 - cosh(Ha z/L) / cosh(Ha)]; F_b is
    set so that the centre-line speed is Ma c_s."""
    L = ny / 2.0
    z = np.arange(ny, dtype=np.float64) + 0.5 - L
    umax = Ma / np.sqrt(3.0)
    Fb = umax * Ha * nu / (L * L / np.tanh(Ha) * (1.0 - 1.0 / np.cosh(Ha)))
    fx = Fb * Ha * np.cosh(Ha * z / L) / np.sinh(Ha)
    ua = Fb * L * L / (Ha * nu) / np.tanh(Ha) * (1.0 - np.cosh(Ha * z / L) / np.cosh(Ha))
    sides = ((PERIODIC, 0.0, 0.0), (PERIODIC, 0.0, 0.0), (WALL, 0.0, 0.0), (WALL, 0.0, 0.0))
    return Case(f"hartmann{nx}x{ny}_Ha{Ha:g}", nx, ny, nu, gamma, sides, U=umax,
                force_x=np.broadcast_to(fx[:, None], (ny, nx)).copy(), force_y=np.zeros((ny, nx)),
                meta={"ua": ua, "Ha": Ha, "Fb": Fb})


def batch_cavities(count: int = 256, seed: int = 0, U: float = 0.1):
    """Independent cavities: side 64 + 32 k with k ~ U{0..30}, Re ~ U[100, 1000],
    gamma ~ U[0.2, 1.0]."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(0, 31, size=count)
    Res = rng.uniform(100.0, 1000.0, size=count)
    gammas = rng.uniform(0.2, 1.0, size=count)
    return [cavity(int(64 + 32 * k), float(Re), U, float(g)) for k, Re, g in zip(ks, Res, gammas)]


def poisson_requests(count: int = 2000, rate: float = 200.0, seed: int = 0, U: float = 0.1,
                     side_min: int = 128, side_max: int = 2048):
    """Poisson arrival stream of steady-solve requests: kind cavity or obstacle
    channel (p = 1/2), side H uniform on multiples of 32 in [side_min, side_max],
    Re ~ U[50, 1000], gamma ~ U[0.2, 1.0].  Returns a list of (t_arrival, Case)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for i in range(count):
        kind = rng.integers(0, 2)
        H = int(32 * rng.integers(side_min // 32, side_max // 32 + 1))
        Re = float(rng.uniform(50.0, 1000.0))
        g = float(rng.uniform(0.2, 1.0))
        if kind == 0:
            c = cavity(H, Re, U, g)
        else:
            c = channel_obstacle(nx=4 * H, ny=H, D=max(H // 16, 2), Re=Re, U0=U / 2, gamma=g,
                                 xc=H // 2)
        out.append((float(t[i]), c))
    return out


def open_channel(nx: int, ny: int, nu: float, gamma: float, U_max: float = 0.05) -> Case:
    """Channel between stationary walls at y = -1/2 and ny - 1/2 with a parabolic
    velocity inlet of peak U_max on the west side and a convective outlet
    (convection speed U_max) on the east side, fluid initially at rest."""
    sides = ((INLET, U_max, 0.0), (OUTLET, U_max, 0.0), (WALL, 0.0, 0.0), (WALL, 0.0, 0.0))
    return Case(f"openchannel{nx}x{ny}", nx, ny, nu, gamma, sides, U=U_max, meta={"U_max": U_max})


def square_cylinder(D: int = 10, Re: float = 20.0, U_max: float = 0.1, gamma: float = 0.5,
                    length: float = 50.0, height: float = 8.0, upstream: float = 12.5) -> Case:
    """Flow past a square cylinder in a channel (Sec. 6): channel length 50 D and
    height 8 D, cylinder of side D centred on the channel axis at 12.5 D from
    the inlet, parabolic inflow of peak U_max, convective outflow, stationary
    walls; nu = U_max D / Re.  The solid cells are the D x D block whose
    half-way surfaces lie at xc +- D/2, yc +- D/2 (xc, yc on cell faces)."""
    nx, ny = int(round(length * D)), int(round(height * D))
    nu = U_max * D / Re
    x0 = int(round(upstream * D - D / 2.0))
    y0 = ny // 2 - D // 2
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[y0:y0 + D, x0:x0 + D] = 1
    sides = ((INLET, U_max, 0.0), (OUTLET, U_max, 0.0), (WALL, 0.0, 0.0), (WALL, 0.0, 0.0))
    return Case(f"squarecyl_D{D}_Re{Re:g}_g{gamma:g}", nx, ny, nu, gamma, sides, U=U_max, solid=solid,
                meta={"Re": Re, "D": D, "x_front": x0 - 0.5, "x_rear": x0 + D - 0.5,
                      "y_axis": ny / 2.0 - 0.5, "U_max": U_max})


def periodic_obstacle(n: int = 48, D: int = 8, nu: float = 0.05, gamma: float = 0.5,
                      Fx: float = 2e-6) -> Case:
    """Fully periodic box with a square solid block of side D and a uniform body
    force F_x on the fluid (no walls: at steady state the force on the block
    balances the force on the fluid)."""
    solid = np.zeros((n, n), dtype=np.uint8)
    c0 = n // 2 - D // 2
    solid[c0:c0 + D, c0:c0 + D] = 1
    return Case(f"periodicobstacle{n}_D{D}", n, n, nu, gamma, periodic_sides(), Fx=Fx, solid=solid,
                meta={"D": D})
