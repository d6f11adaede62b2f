"""Steady periodic solutions of the preconditioned Navier-Stokes equations, by a
pseudo-spectral Newton solve.  Test infrastructure: an independent reference for
body-force-driven flows whose incompressible closed form is only the Ma -> 0
limit of what the scheme solves.

The equations are the macroscopic system that the Chapman-Enskog analysis of
Secs. 3-4 assigns to the GI corrected scheme (Eq. 1 with p* = gamma rho / 3,
Eqs. 42 and 48-49), at steady state and multiplied through by gamma:

    div(rho u) = 0,
    div(rho u u) + (gamma/3) grad rho = div(tau) + F,

with the viscous stress of the physical (underlined) terms of Eqs. 23-25,

    tau_xx = rho [nu3 div u + nu (d_x u_x - d_y u_y)],
    tau_yy = rho [nu3 div u - nu (d_x u_x - d_y u_y)],
    tau_xy = rho nu (d_x u_y + d_y u_x),

nu = (gamma/3)(1/omega_4 - 1/2) the shear and nu3 = (gamma/3)(1/omega_3 - 1/2)
the bulk viscosity (Eq. 49).  Everything is in lattice units on a periodic box
of n x n lattice spacings; the unknowns are rho, j = rho u on an M x M
collocation grid.  The system fixes rho and j only up to their means, so the
Newton residual carries mean(rho) - 1, mean(j_x) and mean(j_y) in its constant
modes (mass and momentum of a box that starts at rest with rho = 1 and is
driven by a force of zero mean).  No lattice Boltzmann arithmetic is used.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


class PeriodicSteadyNS:
    def __init__(self, n: int, M: int, nu: float, gamma: float, omega3: float = 1.0):
        self.n, self.M, self.nu, self.gamma = int(n), int(M), float(nu), float(gamma)
        self.nu3 = gamma / 3.0 * (1.0 / omega3 - 0.5)
        k = np.fft.fftfreq(M, d=n / M) * 2.0 * np.pi
        self.KX, self.KY = np.meshgrid(k, k)          # arrays [y, x]
        xs = np.arange(M) * n / M
        self.X, self.Y = np.meshgrid(xs, xs)          # lattice coordinates of the nodes

    def _dx(self, a):
        return np.real(np.fft.ifft2(1j * self.KX * np.fft.fft2(a, axes=(-2, -1)), axes=(-2, -1)))

    def _dy(self, a):
        return np.real(np.fft.ifft2(1j * self.KY * np.fft.fft2(a, axes=(-2, -1)), axes=(-2, -1)))

    def residual(self, z, Fx, Fy):
        """Residual of the steady system; z has shape (..., 3 M^2) (batched)."""
        M, g = self.M, self.gamma
        z = np.asarray(z)
        q = z.reshape(z.shape[:-1] + (3, M, M))
        rho, jx, jy = q[..., 0, :, :], q[..., 1, :, :], q[..., 2, :, :]
        ux, uy = jx / rho, jy / rho
        dx, dy = self._dx, self._dy
        div_u = dx(ux) + dy(uy)
        dev = dx(ux) - dy(uy)
        txx = rho * (self.nu3 * div_u + self.nu * dev)
        tyy = rho * (self.nu3 * div_u - self.nu * dev)
        txy = rho * self.nu * (dx(uy) + dy(ux))
        mean = lambda a: a.mean(axis=(-2, -1), keepdims=True)
        r_rho = -(dx(jx) + dy(jy)) + (mean(rho) - 1.0)
        r_jx = (-(dx(rho * ux * ux) + dy(rho * ux * uy)) - g / 3.0 * dx(rho)
                + dx(txx) + dy(txy) + Fx) + mean(jx)
        r_jy = (-(dx(rho * ux * uy) + dy(rho * uy * uy)) - g / 3.0 * dy(rho)
                + dx(txy) + dy(tyy) + Fy) + mean(jy)
        return np.stack([r_rho, r_jx, r_jy], axis=-3).reshape(z.shape)

    def solve(self, Fx, Fy, ux0, uy0, tol=1e-11, max_iter=12):
        """Newton iteration from (rho = 1, u0) with a central-difference Jacobian.
        Stops when the largest residual is below tol times the largest force.
        Returns rho, ux, uy on the collocation grid and the final residual norm."""
        M = self.M
        z = np.concatenate([np.ones(M * M), np.ravel(ux0), np.ravel(uy0)])
        scale = np.abs(Fx).max() + np.abs(Fy).max()
        for _ in range(max_iter):
            r = self.residual(z, Fx, Fy)
            if np.abs(r).max() <= tol * scale:
                break
            h = 1e-7 * np.maximum(1.0, np.abs(z))
            E = np.diag(h)
            J = ((self.residual(z[None, :] + E, Fx, Fy) - self.residual(z[None, :] - E, Fx, Fy))
                 / (2.0 * h[:, None])).T
            z = z - scipy.linalg.solve(J, r)
        r = self.residual(z, Fx, Fy)
        rho, jx, jy = z.reshape(3, M, M)
        return rho, jx / rho, jy / rho, float(np.abs(r).max())

    def to_lattice(self, a, n_nodes=None):
        """Fourier interpolation of a collocation-grid field onto the lattice
        nodes x, y = 0, 1, ..., n - 1 (array [y, x])."""
        n = self.n if n_nodes is None else n_nodes
        M = self.M
        A = np.fft.fft2(a) / (M * M)
        k = np.fft.fftfreq(M, d=1.0 / M)
        E = np.exp(2j * np.pi * np.outer(np.arange(n) / n, k))   # (n, M)
        return np.real(E @ A @ E.T)
