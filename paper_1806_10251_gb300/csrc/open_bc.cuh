// Open sides of a channel (Sec. 6, square cylinder): the parabolic velocity
// inlet (west), the convective outlet (east) and its ghost column, shared by
// the step kernels and the auxiliary kernels.
//
// Readings (the paper gives the inlet profile and the outlet equation only):
// the inlet is half-way bounce-back with the moving-wall term (rho0 = 1), the
// wall velocity taken where the link crosses the inlet plane; the outlet
// advances a ghost velocity by the convective equation and lets the
// populations with e_x = -1 enter from a ghost column holding the equilibrium
// at the reference density rho0 = 1 and that velocity plus the last column's
// non-equilibrium part.
#pragma once

#include "d2q9_collide.cuh"

namespace lbm {

// ---- open sides of a channel (Sec. 6, square cylinder) ---------------------

// Slot of direction a (one of 3, 6, 7: e_x = -1) in the outlet ghost column.
__device__ __forceinline__ int ghost_slot(int a) { return a == 3 ? 0 : (a == 6 ? 1 : 2); }

// Population a of a cell whose source (sx, sy) lies beyond the outx / outy
// side(s) of the domain: on a convective-outlet east side, the ghost column's
// incoming population; otherwise half-way bounce-back of the cell's opposite
// population own_opp with the moving-wall term 6 w_a rho0 (e_a . u_w), where a
// parabolic inlet (west side) takes u_w at the height where the link crosses
// the inlet plane.  A source beyond two sides (a corner) sees a stationary wall.
template <typename R>
__device__ __forceinline__ R boundary_value(const StepParams &p, const Consts<R> &c, int a, int ex, int ey, int sx,
                                            int sy, bool outx, bool outy, R own_opp)
{
    if (outx == outy) return own_opp;
    const int side = outx ? (sx < 0 ? 0 : 1) : (sy < 0 ? 2 : 3);
    if (side == 1 && p.outlet) {
        const int gy = !p.pery ? sy : (sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy));
        const long long gi = (long long)(2 + ghost_slot(a)) * p.ny + gy;
        return LBM_IN_BOUNDS(gi, 5LL * p.ny, p.error) ? static_cast<const R *>(p.ghost_in)[gi] : own_opp;
    }
    const R wa = a == 0 ? R(4.0 / 9.0) : (a <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0));
    R uw = c.wall6[side][0];
    if (side == 0 && p.inlet) {
        // 4 U_max t (H - t) / H^2 with t = y_cross + 1/2, y_cross = sy + e_y / 2
        const R t = R(sy) + R(0.5) * R(ey) + R(0.5);
        uw = uw * (c.inlet_k * t * (c.H - t));
    }
    return own_opp + wa * (R(ex) * uw + R(ey) * c.wall6[side][1]);
}

// Deviations f_eq - w of directions 3, 6, 7 of the preconditioned equilibrium
// (Eq. 15, fourth moment as the initialisation, through the inverse of Eq. 5)
// at rho = 1 + drho and u.
template <typename R>
__device__ __forceinline__ void west_equilibrium(const Consts<R> &c, R drho, R ux, R uy, R &e3, R &e6, R &e7)
{
    const R rho = R(1) + drho;
    const R third = R(1.0 / 3.0);
    const R ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const R q = (ux2 + uy2) * third + ux2 * uy2 * c.c4;
    const R x2y = ux2 * uy * c.ig2, xy2 = ux * uy2 * c.ig2;
    e3 = drho * R(1.0 / 9.0) + R(0.5) * rho * (R(-2.0 / 3.0) * ux + ux2 * c.ig + xy2 - q);
    e6 = drho * R(1.0 / 36.0) + R(0.25) * rho * (-uxy * c.ig + (uy - ux) * third + (x2y - xy2) + q);
    e7 = drho * R(1.0 / 36.0) + R(0.25) * rho * (uxy * c.ig - (ux + uy) * third - (x2y + xy2) + q);
}

// rho - 1 and u of a cell from its post-collision deviations g (rho u =
// sum g e - F/(2 gamma)).
template <typename R>
__device__ __forceinline__ void cell_state(const Consts<R> &c, const R (&g)[9], R Fx, R Fy, R &drho, R &ux, R &uy)
{
    R s = R(0), jx = R(0), jy = R(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        s += g[a];
        jx += R(cx(a)) * g[a];
        jy += R(cy(a)) * g[a];
    }
    const R rho = R(1) + s;
    drho = s;
    ux = (jx - Fx * c.half_ig) / rho;
    uy = (jy - Fy * c.half_ig) / rho;
}

// Outlet ghost row y from the last column's deviations g and state (drho, u)
// and the ghost velocity (ug, vg): the incoming populations are the
// equilibrium at rho0 = 1 and (ug, vg) plus the last column's
// non-equilibrium part.  ghost: [5][ny] (u_g, v_g, populations 3, 6, 7).
template <typename R>
__device__ __forceinline__ void outlet_row(const Consts<R> &c, int ny, int y, const R (&g)[9], R drho, R ux, R uy,
                                           R ug, R vg, R *ghost)
{
    R e3, e6, e7, r3, r6, r7;
    west_equilibrium(c, drho, ux, uy, e3, e6, e7);
    west_equilibrium(c, R(0), ug, vg, r3, r6, r7);
    ghost[y] = ug;
    ghost[ny + y] = vg;
    ghost[2 * ny + y] = r3 + (g[3] - e3);
    ghost[3 * ny + y] = r6 + (g[6] - e6);
    ghost[4 * ny + y] = r7 + (g[7] - e7);
}

// Convective outlet, row y, after the collision of the last column: advance
// the ghost velocity, u_g <- u_g + U (u - u_g) (d_t u + U d_x u = 0, explicit
// and upwind in lattice units), then the incoming populations.
template <typename R>
__device__ __forceinline__ void outlet_update(const StepParams &p, const Consts<R> &c, int y, const R (&g)[9], R Fx,
                                              R Fy)
{
    if (!LBM_IN_BOUNDS(y, p.ny, p.error)) return;
    R drho, ux, uy;
    cell_state(c, g, Fx, Fy, drho, ux, uy);
    const R *gin = static_cast<const R *>(p.ghost_in);
    const R ug = gin[y] + c.out_u * (ux - gin[y]);
    const R vg = gin[p.ny + y] + c.out_u * (uy - gin[p.ny + y]);
    outlet_row(c, p.ny, y, g, drho, ux, uy, ug, vg, static_cast<R *>(p.ghost_out));
}

}  // namespace lbm
