/*
 * gi_oracle.h -- FP64 CPU oracle for the Galilean-invariant preconditioned
 * cascaded central-moment lattice Boltzmann method on D2Q9
 * (Hajabdollahi & Premnath, arXiv 1806.10251).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or constant with the CUDA library, and it never
 * includes anything from the product package.
 *
 * Arithmetic is IEEE double throughout.  Layout of every population array is
 * f[alpha][y][x] with x fastest (index alpha*nx*ny + y*nx + x).
 *
 * Velocity ordering (the paper prints none; this ordering is a reading):
 *   0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
 *
 * Raw-moment vector order used by every function below (Eq. 3 / Eq. 6):
 *   k[0]=kappa_0, k[1]=kappa_x, k[2]=kappa_y, k[3]=kappa_xx, k[4]=kappa_yy,
 *   k[5]=kappa_xy, k[6]=kappa_xxy, k[7]=kappa_xyy, k[8]=kappa_xxyy
 *
 * Parity status of each part is stated beside it in the source file.
 */
#ifndef GI_ORACLE_H
#define GI_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_GI_UNCORRECTED = 0, ORC_GI_CUBIC_ONLY = 1, ORC_GI_FULL = 2 };
enum { ORC_FD_CENTRAL = 0, ORC_FD_ISOTROPIC = 1 };
/* Side kinds.  INLET (west side only): fully developed parabolic velocity
 * profile of peak side_u[WEST][0] across the channel, imposed by half-way
 * bounce-back with the moving-wall term.  OUTLET (east side only): convective
 * outflow d_t phi + U d_x phi = 0 with U = side_u[EAST][0] (Sec. 6, square
 * cylinder). */
enum { ORC_SIDE_PERIODIC = 0, ORC_SIDE_WALL = 1, ORC_SIDE_MOVING_WALL = 2, ORC_SIDE_INLET = 3,
       ORC_SIDE_OUTLET = 4 };
enum { ORC_WEST = 0, ORC_EAST = 1, ORC_SOUTH = 2, ORC_NORTH = 3 };

typedef struct {
    int nx, ny;
    double gamma;          /* preconditioning parameter, 0 < gamma <= 1     */
    double omega[9];       /* relaxation rates; omega[3..8] are used         */
    int gi_mode;           /* ORC_GI_*                                        */
    int fd_scheme;         /* ORC_FD_*                                        */
    int guard;             /* 1: apply the small-determinant guard of the     */
                           /*    strain-rate solve (a reading; see source)    */
    int side_kind[4];      /* ORC_SIDE_* for west, east, south, north         */
    double side_u[4][2];   /* wall velocity of each side                      */
    double rho0;           /* reference density in the moving-wall term (1)   */
    double Fx, Fy;         /* uniform body force (used when no force field)   */
} orc_params;

/* ---- per-cell building blocks (exposed so tests can pin them one by one) -- */
void orc_lattice(int ex[9], int ey[9], double w[9], int opp[9]);
void orc_raw_moments(const double f[9], double k[9]);
void orc_pops_from_raw(const double k[9], double f[9]);
void orc_raw_equilibrium(double rho, double ux, double uy, double gamma, double keq[9]);
void orc_source_moments(double Fx, double Fy, double ux, double uy, double gamma, double s[9]);
void orc_K_columns(double K[9][9]);          /* K[j][alpha] */
void orc_gi_coefficients(double rho, double ux, double uy, double gamma,
                         double omega3, double omega4, double omega5, double c[12]);
int  orc_strain_rates(double rho, double ux, double uy, double gamma,
                      double omega3, double omega4, double m3, double m4,
                      double drho_x, double drho_y, int guard,
                      double *dux_dx, double *duy_dy);
int  orc_collide_cell(const orc_params *p, const double fbar[9],
                      double drho_x, double drho_y, double Fx, double Fy,
                      double ftilde[9], double ghat[9], double M[3]);

/* ---- whole-domain oracle ------------------------------------------------ */
typedef struct orc_domain orc_domain;

orc_domain *orc_create(const orc_params *p, const uint8_t *solid /* nx*ny or NULL */);
void   orc_destroy(orc_domain *d);
int    orc_set_force_field(orc_domain *d, const double *Fx, const double *Fy);
void   orc_init_equilibrium(orc_domain *d, const double *rho, const double *ux, const double *uy);
void   orc_step(orc_domain *d, long n);
void   orc_density_gradient_field(orc_domain *d, const double *rho, double *gx, double *gy);
void   orc_get_pops(const orc_domain *d, double *f);
void   orc_set_pops(orc_domain *d, const double *f);
void   orc_fields(const orc_domain *d, double *rho, double *ux, double *uy);
void   orc_used_fields(const orc_domain *d, double *rho, double *ux, double *uy);
double orc_residual(orc_domain *d, double *sums /* 5: dU2, U2, mass, momx, momy */);
long   orc_steps_done(const orc_domain *d);
long   orc_guard_count(const orc_domain *d);
/* Momentum-exchange force on the solid cells (Sec. 6, square cylinder), in
 * lattice momentum per step, from the current post-collision state. */
void   orc_drag(const orc_domain *d, double force[2]);
void   orc_set_threads(int n);
int    orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
