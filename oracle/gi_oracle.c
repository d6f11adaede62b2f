/*
 * gi_oracle.c -- FP64 CPU oracle: Galilean-invariant preconditioned cascaded
 * central-moment LBM on D2Q9 (Hajabdollahi & Premnath, arXiv 1806.10251).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, written to be checked against the
 * paper by eye: every function follows one equation or section and says which.
 * No blocking, fusion or reordering beyond what the paper states.  It shares
 * nothing with the CUDA library.
 *
 * One time step, in the paper's order (Eq. 2a collide, Eq. 2b stream), written
 * in pull form: the stored state is the post-collision array f~; a step first
 * streams (Eq. 2b, pulling f~ from the upwind neighbour, half-way bounce-back at
 * walls), then collides every cell (Eq. 2a with the Sec. 5 kernel).
 *
 * Readings of the paper taken here (the paper is silent, garbled or
 * inconsistent at these points):
 *   - velocity ordering and weights (not printed): see gi_oracle.h; the weights
 *     follow from the rest-state equilibrium moments (Eq. 15);
 *   - collision matrix K (not printed, deferred to an earlier paper): rebuilt as
 *     the Gram-Schmidt orthogonalisation of the Eq. 5 monomials, scaled so that
 *     the factors omega3/12, omega4/4, omega5/4 of Eq. 4 and the cascade
 *     relations of Sec. 5 ("-4 g6", "-6 u_y g3", "-2 g3") hold;
 *   - omega3, omega6, omega7, omega8 (never given): caller-chosen, default 1;
 *   - raw equilibrium kappa_xxyy (Eq. 15 is inconsistent with the kernel's
 *     central target rho/9 when gamma != 1): initialisation uses the value that
 *     makes the central fourth moment equal rho/9;
 *   - Eq. 55b sign: the printed "+ c~1 R3" is "- c~1 R3" (solving Eqs. 51-52);
 *   - Eq. 47c/d: lambda^5 carries no factor rho (Eqs. 28a and 44c give none);
 *   - the Sec. 5 kernel drops the bars and the -1/2 sigma terms of Eq. 4 in
 *     g6..g8; they are kept here, reading sigma_xxy as sigma'_xxy;
 *   - velocity with forcing: rho u = sum fbar e + F/(2 gamma);
 *   - moving-wall term uses rho0 = 1; a link whose source lies beyond two sides
 *     (a corner) sees a stationary wall;
 *   - density gradient: central difference on the same step's post-streaming
 *     rho; a missing neighbour (wall side or solid) takes the cell's own rho;
 *   - open boundaries of the square-cylinder channel (Sec. 6 gives the inlet
 *     profile and the outlet equation only): the parabolic inlet is imposed
 *     by half-way bounce-back with the moving-wall term (rho0 = 1), the wall
 *     velocity taken at the point where the link crosses the inlet plane; the
 *     convective outlet equation d_t u + U d_x u = 0 advances the velocity u_g
 *     of a ghost column at x = nx, explicitly and upwind with unit lattice
 *     steps (u_g <- u_g + U (u(nx-1) - u_g) after every collision), and the
 *     populations that enter through the east side (e_x = -1) are the
 *     equilibrium (Eq. 15) at the reference density rho0 = 1 and u_g plus the
 *     non-equilibrium part f~ - f_eq of the last column (the reference density
 *     fixes the pressure level, which a velocity condition leaves free); u_g
 *     starts from the initial velocity of the last column; a link crossing two
 *     sides (a corner) sees a stationary wall;
 *   - momentum-exchange force: 2 e_a f~_a(x) summed over the links from fluid
 *     cells x to solid cells x + e_a (half-way bounce-back, stationary solid);
 *   - strain-rate guard (optional, off by default): if |D| < 0.1 |D0| the
 *     velocity-dependent parts P, Q, P~, Q~ are dropped for that cell.
 *     Parity unpinned against the paper (it is silent on the case); the
 *     trigger and the reduced solve are pinned to this reading by a property
 *     test.  It is counted, never silent.
 */
#include "gi_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D2Q9 lattice (reading: the paper prints no ordering). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

enum { K0 = 0, KX, KY, KXX, KYY, KXY, KXXY, KXYY, KXXYY };

void orc_lattice(int ex[9], int ey[9], double w[9], int opp[9])
{
    for (int a = 0; a < 9; ++a) {
        ex[a] = EX[a];
        ey[a] = EY[a];
        w[a] = W[a];
        opp[a] = OPP[a];
    }
}

/* Eq. 3: raw moments kappa'_{x^m y^n} = sum_alpha f_alpha e_x^m e_y^n. */
void orc_raw_moments(const double f[9], double k[9])
{
    for (int i = 0; i < 9; ++i) k[i] = 0.0;
    for (int a = 0; a < 9; ++a) {
        double x = EX[a], y = EY[a];
        k[K0] += f[a];
        k[KX] += f[a] * x;
        k[KY] += f[a] * y;
        k[KXX] += f[a] * x * x;
        k[KYY] += f[a] * y * y;
        k[KXY] += f[a] * x * y;
        k[KXXY] += f[a] * x * x * y;
        k[KXYY] += f[a] * x * y * y;
        k[KXXYY] += f[a] * x * x * y * y;
    }
}

/* Inverse of the Eq. 5/6 map (raw moments -> populations), solved by hand from
 * the monomial table of the ordering above. */
void orc_pops_from_raw(const double k[9], double f[9])
{
    f[0] = k[K0] - k[KXX] - k[KYY] + k[KXXYY];
    f[1] = 0.5 * (k[KX] + k[KXX] - k[KXYY] - k[KXXYY]);
    f[3] = 0.5 * (-k[KX] + k[KXX] + k[KXYY] - k[KXXYY]);
    f[2] = 0.5 * (k[KY] + k[KYY] - k[KXXY] - k[KXXYY]);
    f[4] = 0.5 * (-k[KY] + k[KYY] + k[KXXY] - k[KXXYY]);
    f[5] = 0.25 * (k[KXY] + k[KXXY] + k[KXYY] + k[KXXYY]);
    f[6] = 0.25 * (-k[KXY] + k[KXXY] - k[KXYY] + k[KXXYY]);
    f[7] = 0.25 * (k[KXY] - k[KXXY] - k[KXYY] + k[KXXYY]);
    f[8] = 0.25 * (-k[KXY] - k[KXXY] + k[KXYY] + k[KXXYY]);
}

/* Eq. 15 (preconditioned raw equilibria, boxed gamma^2 cubic terms).  The
 * fourth moment is the kernel-consistent value (central kappa_xxyy = rho/9);
 * at gamma = 1 it coincides with the printed rho/9 + rho(ux^2+uy^2)/3 + rho ux^2 uy^2. */
void orc_raw_equilibrium(double rho, double ux, double uy, double g, double keq[9])
{
    keq[K0] = rho;
    keq[KX] = rho * ux;
    keq[KY] = rho * uy;
    keq[KXX] = rho / 3.0 + rho * ux * ux / g;
    keq[KYY] = rho / 3.0 + rho * uy * uy / g;
    keq[KXY] = rho * ux * uy / g;
    keq[KXXY] = rho * uy / 3.0 + rho * ux * ux * uy / (g * g);
    keq[KXYY] = rho * ux / 3.0 + rho * ux * uy * uy / (g * g);
    keq[KXXYY] = rho / 9.0 + rho * (ux * ux + uy * uy) / 3.0
               + rho * ux * ux * uy * uy * (3.0 - 6.0 / g + 4.0 / (g * g));
}

/* Preconditioned source raw moments sigma' (the list after Eq. 15). */
void orc_source_moments(double Fx, double Fy, double ux, double uy, double g, double s[9])
{
    s[K0] = 0.0;
    s[KX] = Fx / g;
    s[KY] = Fy / g;
    s[KXX] = 2.0 * Fx * ux / (g * g);
    s[KYY] = 2.0 * Fy * uy / (g * g);
    s[KXY] = (Fx * uy + Fy * ux) / (g * g);
    s[KXXY] = Fy * ux * ux + 2.0 * Fx * ux * uy;
    s[KXYY] = Fx * uy * uy + 2.0 * Fy * uy * ux;
    s[KXXYY] = 2.0 * (Fx * ux * uy * uy + Fy * uy * ux * ux);
}

/* Orthogonal collision basis K (columns K_j, j = 0..8, as functions of alpha):
 * Gram-Schmidt of the Eq. 5 monomials, scaled to the Eq. 4 factors. */
void orc_K_columns(double K[9][9])
{
    for (int a = 0; a < 9; ++a) {
        double x = EX[a], y = EY[a];
        double x2 = x * x, y2 = y * y;
        K[0][a] = 1.0;
        K[1][a] = x;
        K[2][a] = y;
        K[3][a] = 3.0 * (x2 + y2) - 4.0;
        K[4][a] = x2 - y2;
        K[5][a] = x * y;
        K[6][a] = -3.0 * x2 * y + 2.0 * y;
        K[7][a] = -3.0 * x * y2 + 2.0 * x;
        K[8][a] = 9.0 * x2 * y2 - 6.0 * (x2 + y2) + 4.0;
    }
}

/* Eqs. 45-47: coefficients of the extended moment equilibria.
 * c = {th3x, th3y, la3x, la3y, th4x, th4y, la4x, la4y, th5x, th5y, la5x, la5y}.
 * A, B, C as defined after Eq. 53; lambda^5 without the factor rho (reading). */
void orc_gi_coefficients(double rho, double ux, double uy, double g,
                         double w3, double w4, double w5, double c[12])
{
    double A = 4.0 / (g * g) - 1.0 / g;
    double B = 1.0 / (g * g) - 1.0 / g;
    double C = 1.0 / g - 1.0;
    double k3 = 1.0 / w3 - 0.5, k4 = 1.0 / w4 - 0.5, k5 = 1.0 / w5 - 0.5;
    double ux2 = ux * ux, uy2 = uy * uy;
    /* Eq. 45 */
    c[0] = -k3 * rho * (A * ux2 + B * uy2);
    c[1] = -k3 * rho * (A * uy2 + B * ux2);
    c[2] = -2.0 / 3.0 * k3 * C * ux;
    c[3] = -2.0 / 3.0 * k3 * C * uy;
    /* Eq. 46 */
    c[4] = -k4 * rho * (A * ux2 - B * uy2);
    c[5] = k4 * rho * (-A * uy2 + B * ux2);
    c[6] = -2.0 / 3.0 * k4 * C * ux;
    c[7] = -2.0 / 3.0 * k4 * C * uy;
    /* Eq. 47 */
    c[8] = -k5 * rho * B * ux * uy;
    c[9] = -k5 * rho * B * ux * uy;
    c[10] = -1.0 / 3.0 * k5 * C * uy;
    c[11] = -1.0 / 3.0 * k5 * C * ux;
}

/* Eqs. 51-55: diagonal strain rates from the non-equilibrium moments m3, m4
 * and the density gradient.  Returns 1 when the guard replaced the
 * velocity-dependent parts (only if guard != 0), else 0. */
int orc_strain_rates(double rho, double ux, double uy, double g,
                     double w3, double w4, double m3, double m4,
                     double drx, double dry, int guard,
                     double *dux_dx, double *duy_dy)
{
    double A = 4.0 / (g * g) - 1.0 / g;
    double B = 1.0 / (g * g) - 1.0 / g;
    double C = 1.0 / g - 1.0;
    double ux2 = ux * ux, uy2 = uy * uy;
    double P = -0.5 * (A * ux2 + B * uy2);
    double Q = -0.5 * (A * uy2 + B * ux2);
    double Pt = -0.5 * (A * ux2 - B * uy2);
    double Qt = -0.5 * (A * uy2 - B * ux2);
    /* Eq. 53 */
    double c1 = (2.0 / (3.0 * w3) + P) * rho;
    double c2 = (2.0 / (3.0 * w3) + Q) * rho;
    double c1t = (2.0 / (3.0 * w4) + Pt) * rho;
    double c2t = (2.0 / (3.0 * w4) + Qt) * rho;
    double D = -c1 * c2t - c1t * c2;
    int guarded = 0;
    if (guard) {
        double D0 = -2.0 * (2.0 * rho / (3.0 * w3)) * (2.0 * rho / (3.0 * w4));
        if (fabs(D) < 0.1 * fabs(D0)) {
            c1 = c2 = 2.0 * rho / (3.0 * w3);
            c1t = c2t = 2.0 * rho / (3.0 * w4);
            D = -c1 * c2t - c1t * c2;
            guarded = 1;
        }
    }
    /* Eq. 54 */
    double e_rho = C / 3.0 * (ux * drx + uy * dry);
    double e_rho_t = C / 3.0 * (ux * drx - uy * dry);
    double R3 = m3 - e_rho, R4 = m4 - e_rho_t;
    /* Eq. 55a, and Eq. 55b with the sign of the c~1 term corrected */
    *dux_dx = (c2t * R3 + c2 * R4) / D;
    *duy_dy = -(c1 * R4 - c1t * R3) / D;
    return guarded;
}

/* Sec. 5 collision of one cell.  fbar are the post-streaming (transformed)
 * populations; returns the post-collision populations f~ = fbar + K g + S
 * (Eq. 2a).  Also returns ghat[9] and the corrections M[3] for tests. */
int orc_collide_cell(const orc_params *p, const double fbar[9],
                     double drx, double dry, double Fx, double Fy,
                     double ft[9], double gh[9], double M[3])
{
    const double g = p->gamma;
    const double w3 = p->omega[3], w4 = p->omega[4], w5 = p->omega[5];
    const double w6 = p->omega[6], w7 = p->omega[7], w8 = p->omega[8];

    /* Eq. 3 on fbar */
    double kb[9];
    orc_raw_moments(fbar, kb);
    /* conserved moments, velocity with the forcing shift */
    double rho = kb[K0];
    double ux = (kb[KX] + 0.5 * Fx / g) / rho;
    double uy = (kb[KY] + 0.5 * Fy / g) / rho;
    double ux2 = ux * ux, uy2 = uy * uy;

    double s[9];
    orc_source_moments(Fx, Fy, ux, uy, g, s);

    /* Extended equilibria (Eq. 33), from the strain rates (Eqs. 51-55). */
    double M3 = 0.0, M4 = 0.0, M5 = 0.0;
    int guarded = 0;
    if (p->gi_mode == ORC_GI_FULL) {
        /* moments of f = fbar + S/2 */
        double kxx = kb[KXX] + 0.5 * s[KXX];
        double kyy = kb[KYY] + 0.5 * s[KYY];
        double m3 = (kxx + kyy) - (2.0 / 3.0 * rho + rho * (ux2 + uy2) / g);
        double m4 = (kxx - kyy) - rho * (ux2 - uy2) / g;
        double dux, duy;
        guarded = orc_strain_rates(rho, ux, uy, g, w3, w4, m3, m4, drx, dry,
                                   p->guard, &dux, &duy);
        double c[12];
        orc_gi_coefficients(rho, ux, uy, g, w3, w4, w5, c);
        M3 = c[0] * dux + c[1] * duy + c[2] * drx + c[3] * dry;
        M4 = c[4] * dux - c[5] * duy + c[6] * drx - c[7] * dry;
        M5 = c[8] * dux + c[9] * duy + c[10] * drx + c[11] * dry;
    }
    /* third-order equilibrium factor: Eq. 4 uses 2, Sec. 5 uses 3/g - 1/g^2 */
    double c6 = (p->gi_mode == ORC_GI_UNCORRECTED) ? 2.0 : (3.0 / g - 1.0 / (g * g));

    double g3 = w3 / 12.0 * (2.0 / 3.0 * rho + rho * (ux2 + uy2) / g
                             - (kb[KXX] + kb[KYY]) - 0.5 * (s[KXX] + s[KYY]) + M3);
    double g4 = w4 / 4.0 * (rho * (ux2 - uy2) / g
                            - (kb[KXX] - kb[KYY]) - 0.5 * (s[KXX] - s[KYY]) + M4);
    double g5 = w5 / 4.0 * (rho * ux * uy / g - kb[KXY] - 0.5 * s[KXY] + M5);
    double g6 = w6 / 4.0 * (c6 * rho * ux2 * uy + kb[KXXY] - 2.0 * ux * kb[KXY]
                            - uy * kb[KXX] - 0.5 * s[KXXY])
              - 0.5 * uy * (3.0 * g3 + g4) - 2.0 * ux * g5;
    double g7 = w7 / 4.0 * (c6 * rho * ux * uy2 + kb[KXYY] - 2.0 * uy * kb[KXY]
                            - ux * kb[KYY] - 0.5 * s[KXYY])
              - 0.5 * ux * (3.0 * g3 - g4) - 2.0 * uy * g5;
    double g8 = w8 / 4.0 * (rho / 9.0 + 3.0 * rho * ux2 * uy2
                            - (kb[KXXYY] - 2.0 * ux * kb[KXYY] - 2.0 * uy * kb[KXXY]
                               + ux2 * kb[KYY] + uy2 * kb[KXX] + 4.0 * ux * uy * kb[KXY])
                            - 0.5 * s[KXXYY])
              - 2.0 * g3 - 0.5 * uy2 * (3.0 * g3 + g4) - 0.5 * ux2 * (3.0 * g3 - g4)
              - 4.0 * ux * uy * g5 - 2.0 * uy * g6 - 2.0 * ux * g7;

    double ghat[9] = {0.0, 0.0, 0.0, g3, g4, g5, g6, g7, g8};
    double K[9][9];
    orc_K_columns(K);
    double S[9];
    orc_pops_from_raw(s, S);
    for (int a = 0; a < 9; ++a) {
        double kg = 0.0;
        for (int j = 0; j < 9; ++j) kg += K[j][a] * ghat[j];
        ft[a] = fbar[a] + kg + S[a];
    }
    if (gh)
        for (int j = 0; j < 9; ++j) gh[j] = ghat[j];
    if (M) {
        M[0] = M3;
        M[1] = M4;
        M[2] = M5;
    }
    return guarded;
}

/* ------------------------------------------------------------------------- */
struct orc_domain {
    orc_params p;
    long N;
    double *f;      /* stored post-collision state f~, [9][ny][nx] */
    double *fbar;   /* scratch: post-streaming populations          */
    double *rho, *ux, *uy;      /* rho, u used by the last collision */
    double *uxs, *uys;          /* velocity snapshot for the residual */
    double *Fx, *Fy;            /* optional force field               */
    uint8_t *solid;
    double *ghost;              /* convective outlet at x = nx, [5][ny]: u_g, v_g and f~ of 3, 6, 7 */
    long steps;
    long guard_count;
};

static int g_threads = 0;
void orc_set_threads(int n) { g_threads = n; }
int orc_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

static double force_x(const orc_domain *d, long i) { return d->Fx ? d->Fx[i] : d->p.Fx; }
static double force_y(const orc_domain *d, long i) { return d->Fy ? d->Fy[i] : d->p.Fy; }
static int is_solid(const orc_domain *d, int x, int y)
{
    return d->solid ? d->solid[(long)y * d->p.nx + x] != 0 : 0;
}

/* ghost-column index of the directions with e_x = -1 (3, 6, 7); -1 otherwise */
static int ghost_index(int a) { return a == 3 ? 0 : (a == 6 ? 1 : (a == 7 ? 2 : -1)); }

/* Parabolic inlet profile (Sec. 6): u(y) = 4 U_max (y + 1/2)(H - y - 1/2) / H^2
 * between the walls at y = -1/2 and H - 1/2, H = ny. */
static double inlet_velocity(const orc_params *p, double y)
{
    const double H = p->ny, t = y + 0.5;
    return 4.0 * p->side_u[ORC_WEST][0] * t * (H - t) / (H * H);
}

/* Populations f_eq of the preconditioned equilibrium (Eq. 15, through the
 * inverse of Eq. 5). */
static void equilibrium_pops(double rho, double ux, double uy, double g, double feq[9])
{
    double keq[9];
    orc_raw_equilibrium(rho, ux, uy, g, keq);
    orc_pops_from_raw(keq, feq);
}

/* Velocity of a cell of the stored state (moments of f~ with the forcing
 * shift, as orc_fields). */
static void cell_velocity(const orc_domain *d, long i, double *rho, double *ux, double *uy);

/* Convective outlet, one ghost row: given its velocity u_g, the incoming
 * populations are f_eq(rho0, u_g) + (f~ - f_eq(rho, u)) of the last column. */
static void outlet_populations(orc_domain *d, int y)
{
    const int nx = d->p.nx, ny = d->p.ny;
    const long i = (long)y * nx + nx - 1;
    double rho, ux, uy, fe[9], fg[9];
    cell_velocity(d, i, &rho, &ux, &uy);
    equilibrium_pops(rho, ux, uy, d->p.gamma, fe);
    equilibrium_pops(d->p.rho0, d->ghost[y], d->ghost[ny + y], d->p.gamma, fg);
    for (int a = 3; a <= 7; ++a) {
        const int gi = ghost_index(a);
        if (gi < 0) continue;
        d->ghost[(2 + gi) * ny + y] = fg[a] + (d->f[a * d->N + i] - fe[a]);
    }
}

/* ghost velocity <- the last column's velocity, then the incoming populations */
static void outlet_seed(orc_domain *d)
{
    if (!d->ghost) return;
    const int nx = d->p.nx, ny = d->p.ny;
    for (int y = 0; y < ny; ++y) {
        const long i = (long)y * nx + nx - 1;
        double rho, ux, uy;
        cell_velocity(d, i, &rho, &ux, &uy);
        d->ghost[y] = ux;
        d->ghost[ny + y] = uy;
        outlet_populations(d, y);
    }
}

orc_domain *orc_create(const orc_params *p, const uint8_t *solid)
{
    if (p->nx < 3 || p->ny < 3) return NULL;
    orc_domain *d = (orc_domain *)calloc(1, sizeof(orc_domain));
    if (!d) return NULL;
    d->p = *p;
    d->N = (long)p->nx * p->ny;
    d->f = (double *)calloc(9 * d->N, sizeof(double));
    d->fbar = (double *)calloc(9 * d->N, sizeof(double));
    d->rho = (double *)calloc(d->N, sizeof(double));
    d->ux = (double *)calloc(d->N, sizeof(double));
    d->uy = (double *)calloc(d->N, sizeof(double));
    d->uxs = (double *)calloc(d->N, sizeof(double));
    d->uys = (double *)calloc(d->N, sizeof(double));
    if (solid) {
        d->solid = (uint8_t *)malloc(d->N);
        if (d->solid) memcpy(d->solid, solid, d->N);
    }
    const int outlet = p->side_kind[ORC_EAST] == ORC_SIDE_OUTLET;
    if (outlet) d->ghost = (double *)calloc(5 * (size_t)p->ny, sizeof(double));
    if (!d->f || !d->fbar || !d->rho || !d->ux || !d->uy || !d->uxs || !d->uys ||
        (solid && !d->solid) || (outlet && !d->ghost)) {
        orc_destroy(d);
        return NULL;
    }
    /* rest state */
    for (int a = 0; a < 9; ++a)
        for (long i = 0; i < d->N; ++i) d->f[a * d->N + i] = W[a];
    outlet_seed(d);
    return d;
}

void orc_destroy(orc_domain *d)
{
    if (!d) return;
    free(d->f); free(d->fbar); free(d->rho); free(d->ux); free(d->uy);
    free(d->uxs); free(d->uys); free(d->Fx); free(d->Fy); free(d->solid); free(d->ghost);
    free(d);
}

int orc_set_force_field(orc_domain *d, const double *Fx, const double *Fy)
{
    if (!d->Fx) d->Fx = (double *)calloc(d->N, sizeof(double));
    if (!d->Fy) d->Fy = (double *)calloc(d->N, sizeof(double));
    if (!d->Fx || !d->Fy) return -1;
    memcpy(d->Fx, Fx, d->N * sizeof(double));
    memcpy(d->Fy, Fy, d->N * sizeof(double));
    return 0;
}

/* Initial state: f~0 = f_eq(rho, u) - S/2, f_eq from Eq. 15 through the inverse
 * of Eq. 5 (so that the first streaming delivers fbar = f - S/2, Eq. 2). */
void orc_init_equilibrium(orc_domain *d, const double *rho, const double *ux, const double *uy)
{
    const double g = d->p.gamma;
    for (long i = 0; i < d->N; ++i) {
        double r = rho ? rho[i] : 1.0, u = ux ? ux[i] : 0.0, v = uy ? uy[i] : 0.0;
        double keq[9], feq[9], s[9], S[9];
        orc_raw_equilibrium(r, u, v, g, keq);
        orc_pops_from_raw(keq, feq);
        orc_source_moments(force_x(d, i), force_y(d, i), u, v, g, s);
        orc_pops_from_raw(s, S);
        for (int a = 0; a < 9; ++a) d->f[a * d->N + i] = feq[a] - 0.5 * S[a];
    }
    outlet_seed(d);
    d->steps = 0;
    double sums[5];
    orc_residual(d, sums); /* snapshot of the initial velocity */
}

/* Eq. 2b in pull form with half-way bounce-back (momentum-augmented); the
 * open sides of the square-cylinder channel as in the readings above. */
static void stream_cell(orc_domain *d, int x, int y, double fb[9])
{
    const orc_params *p = &d->p;
    const int nx = p->nx, ny = p->ny;
    const long N = d->N, i = (long)y * nx + x;
    const int perx = p->side_kind[ORC_WEST] == ORC_SIDE_PERIODIC;
    const int pery = p->side_kind[ORC_SOUTH] == ORC_SIDE_PERIODIC;
    for (int a = 0; a < 9; ++a) {
        int sx = x - EX[a], sy = y - EY[a];
        if (perx) sx = (sx + nx) % nx;
        if (pery) sy = (sy + ny) % ny;
        int outx = sx < 0 || sx >= nx;
        int outy = sy < 0 || sy >= ny;
        if (!outx && !outy && !is_solid(d, sx, sy)) {
            fb[a] = d->f[a * N + (long)sy * nx + sx];
            continue;
        }
        double uw = 0.0, vw = 0.0;
        if (outx != outy) {
            int side = outx ? (sx < 0 ? ORC_WEST : ORC_EAST) : (sy < 0 ? ORC_SOUTH : ORC_NORTH);
            if (p->side_kind[side] == ORC_SIDE_MOVING_WALL) {
                uw = p->side_u[side][0];
                vw = p->side_u[side][1];
            } else if (p->side_kind[side] == ORC_SIDE_INLET) {
                uw = inlet_velocity(p, 0.5 * (sy + y));  /* where the link crosses x = -1/2 */
            } else if (p->side_kind[side] == ORC_SIDE_OUTLET) {
                fb[a] = d->ghost[(2 + ghost_index(a)) * ny + sy];
                continue;
            }
        }
        fb[a] = d->f[OPP[a] * N + i] + 6.0 * W[a] * p->rho0 * (EX[a] * uw + EY[a] * vw);
    }
}

/* rho of a neighbour for the finite differences, with the ghost rule. */
static double rho_neighbour(const orc_domain *d, int x, int y, int dx, int dy)
{
    const orc_params *p = &d->p;
    int nx = p->nx, ny = p->ny;
    int sx = x + dx, sy = y + dy;
    if (p->side_kind[ORC_WEST] == ORC_SIDE_PERIODIC) sx = (sx + nx) % nx;
    if (p->side_kind[ORC_SOUTH] == ORC_SIDE_PERIODIC) sy = (sy + ny) % ny;
    if (sx < 0 || sx >= nx || sy < 0 || sy >= ny || is_solid(d, sx, sy))
        return d->rho[(long)y * nx + x];
    return d->rho[(long)sy * nx + sx];
}

static void density_gradient(const orc_domain *d, int x, int y, double *drx, double *dry)
{
    if (d->p.fd_scheme == ORC_FD_ISOTROPIC) {
        double gx = 0.0, gy = 0.0;
        for (int a = 1; a < 9; ++a) {
            double r = rho_neighbour(d, x, y, EX[a], EY[a]);
            gx += 3.0 * W[a] * EX[a] * r;
            gy += 3.0 * W[a] * EY[a] * r;
        }
        *drx = gx;
        *dry = gy;
    } else {
        *drx = 0.5 * (rho_neighbour(d, x, y, 1, 0) - rho_neighbour(d, x, y, -1, 0));
        *dry = 0.5 * (rho_neighbour(d, x, y, 0, 1) - rho_neighbour(d, x, y, 0, -1));
    }
}

/* The density-gradient stencil alone (Eq. 54's d_i rho; central differences or
 * the isotropic stencil, by the domain's fd_scheme, with the ghost rule of
 * rho_neighbour), applied to a given density field rho[ny][nx] so that it can
 * be checked against closed forms.  Overwrites the domain's post-streaming
 * density scratch (the next step recomputes it). */
void orc_density_gradient_field(orc_domain *d, const double *rho, double *gx, double *gy)
{
    memcpy(d->rho, rho, d->N * sizeof(double));
    for (int y = 0; y < d->p.ny; ++y)
        for (int x = 0; x < d->p.nx; ++x) {
            const long i = (long)y * d->p.nx + x;
            density_gradient(d, x, y, gx + i, gy + i);
        }
}

void orc_step(orc_domain *d, long n)
{
    const int nx = d->p.nx, ny = d->p.ny;
    const long N = d->N;
    const double g = d->p.gamma;
    int nt = orc_get_threads();
    (void)nt;
    for (long s = 0; s < n; ++s) {
        /* sweep 1: streaming and the macroscopic fields of every fluid cell */
#pragma omp parallel for schedule(static) num_threads(nt)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long i = (long)y * nx + x;
                if (is_solid(d, x, y)) continue;
                double fb[9];
                stream_cell(d, x, y, fb);
                double r = 0.0, jx = 0.0, jy = 0.0;
                for (int a = 0; a < 9; ++a) {
                    r += fb[a];
                    jx += fb[a] * EX[a];
                    jy += fb[a] * EY[a];
                    d->fbar[a * N + i] = fb[a];
                }
                d->rho[i] = r;
                d->ux[i] = (jx + 0.5 * force_x(d, i) / g) / r;
                d->uy[i] = (jy + 0.5 * force_y(d, i) / g) / r;
            }
        /* sweep 2: density gradient and collision */
        long guards = 0;
#pragma omp parallel for schedule(static) num_threads(nt) reduction(+ : guards)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long i = (long)y * nx + x;
                if (is_solid(d, x, y)) continue;
                double fb[9], ft[9], drx = 0.0, dry = 0.0;
                for (int a = 0; a < 9; ++a) fb[a] = d->fbar[a * N + i];
                if (d->p.gi_mode == ORC_GI_FULL) density_gradient(d, x, y, &drx, &dry);
                guards += orc_collide_cell(&d->p, fb, drx, dry, force_x(d, i),
                                           force_y(d, i), ft, NULL, NULL);
                for (int a = 0; a < 9; ++a) d->f[a * N + i] = ft[a];
            }
        d->guard_count += guards;
        /* convective outlet: advance the ghost velocity with the new last column */
        if (d->ghost) {
            const double U = d->p.side_u[ORC_EAST][0];
            for (int y = 0; y < ny; ++y) {
                if (is_solid(d, nx - 1, y)) continue;
                double rho, ux, uy;
                cell_velocity(d, (long)y * nx + nx - 1, &rho, &ux, &uy);
                d->ghost[y] += U * (ux - d->ghost[y]);
                d->ghost[ny + y] += U * (uy - d->ghost[ny + y]);
                outlet_populations(d, y);
            }
        }
        d->steps += 1;
    }
}

void orc_get_pops(const orc_domain *d, double *f) { memcpy(f, d->f, 9 * d->N * sizeof(double)); }
void orc_set_pops(orc_domain *d, const double *f)
{
    memcpy(d->f, f, 9 * d->N * sizeof(double));
    outlet_seed(d);
}
long orc_steps_done(const orc_domain *d) { return d->steps; }
long orc_guard_count(const orc_domain *d) { return d->guard_count; }

/* Momentum exchange (Sec. 6, square cylinder): the population f~_a(x) of a
 * fluid cell that heads into a solid cell x + e_a returns as f~_a(x) in the
 * opposite direction at the next streaming, handing the solid 2 e_a f~_a(x). */
void orc_drag(const orc_domain *d, double force[2])
{
    const orc_params *p = &d->p;
    const int nx = p->nx, ny = p->ny;
    const int perx = p->side_kind[ORC_WEST] == ORC_SIDE_PERIODIC;
    const int pery = p->side_kind[ORC_SOUTH] == ORC_SIDE_PERIODIC;
    double fx = 0.0, fy = 0.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (is_solid(d, x, y)) continue;
            for (int a = 1; a < 9; ++a) {
                int tx = x + EX[a], ty = y + EY[a];
                if (perx) tx = (tx + nx) % nx;
                if (pery) ty = (ty + ny) % ny;
                if (tx < 0 || tx >= nx || ty < 0 || ty >= ny || !is_solid(d, tx, ty)) continue;
                const double fa = d->f[a * d->N + (long)y * nx + x];
                fx += 2.0 * EX[a] * fa;
                fy += 2.0 * EY[a] * fa;
            }
        }
    force[0] = fx;
    force[1] = fy;
}

static void cell_velocity(const orc_domain *d, long i, double *rho, double *ux, double *uy)
{
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; ++a) {
        const double fa = d->f[a * d->N + i];
        r += fa;
        jx += fa * EX[a];
        jy += fa * EY[a];
    }
    *rho = r;
    *ux = (jx - 0.5 * force_x(d, i) / d->p.gamma) / r;
    *uy = (jy - 0.5 * force_y(d, i) / d->p.gamma) / r;
}

/* Observed fields: local moments of the stored post-collision array, with the
 * forcing shift, rho u = sum f~ e - F/(2 gamma).  Because the collision
 * conserves rho and changes rho u by exactly F/gamma, these equal the rho, u the
 * last collision used (up to rounding).  Solid cells report NaN. */
void orc_fields(const orc_domain *d, double *rho, double *ux, double *uy)
{
    const long N = d->N;
    const double g = d->p.gamma;
    for (long i = 0; i < N; ++i) {
        int x = (int)(i % d->p.nx), y = (int)(i / d->p.nx);
        if (is_solid(d, x, y)) {
            if (rho) rho[i] = NAN;
            if (ux) ux[i] = NAN;
            if (uy) uy[i] = NAN;
            continue;
        }
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int a = 0; a < 9; ++a) {
            double fa = d->f[a * N + i];
            r += fa;
            jx += fa * EX[a];
            jy += fa * EY[a];
        }
        if (rho) rho[i] = r;
        if (ux) ux[i] = (jx - 0.5 * force_x(d, i) / g) / r;
        if (uy) uy[i] = (jy - 0.5 * force_y(d, i) / g) / r;
    }
}

/* rho and u exactly as used by the last collision (sweep 1 of the last step). */
void orc_used_fields(const orc_domain *d, double *rho, double *ux, double *uy)
{
    if (rho) memcpy(rho, d->rho, d->N * sizeof(double));
    if (ux) memcpy(ux, d->ux, d->N * sizeof(double));
    if (uy) memcpy(uy, d->uy, d->N * sizeof(double));
}

/* Convergence residual (the paper plots histories but never defines one;
 * reading): r = ||u^n - u^snap||_2 / ||u^n||_2 over fluid cells, then the
 * snapshot is replaced by u^n.  sums = {sum|du|^2, sum|u|^2, sum rho,
 * sum rho ux, sum rho uy}.  r = 0 when both norms vanish. */
double orc_residual(orc_domain *d, double *sums)
{
    const long N = d->N;
    double *rho = (double *)malloc(N * sizeof(double));
    double *ux = (double *)malloc(N * sizeof(double));
    double *uy = (double *)malloc(N * sizeof(double));
    if (!rho || !ux || !uy) {
        free(rho); free(ux); free(uy);
        return NAN;
    }
    orc_fields(d, rho, ux, uy);
    double du2 = 0.0, u2 = 0.0, m = 0.0, jx = 0.0, jy = 0.0;
    for (long i = 0; i < N; ++i) {
        if (d->solid && d->solid[i]) continue;
        double a = ux[i] - d->uxs[i], b = uy[i] - d->uys[i];
        du2 += a * a + b * b;
        u2 += ux[i] * ux[i] + uy[i] * uy[i];
        m += rho[i];
        jx += rho[i] * ux[i];
        jy += rho[i] * uy[i];
        d->uxs[i] = ux[i];
        d->uys[i] = uy[i];
    }
    free(rho); free(ux); free(uy);
    if (sums) {
        sums[0] = du2; sums[1] = u2; sums[2] = m; sums[3] = jx; sums[4] = jy;
    }
    if (u2 == 0.0) return du2 == 0.0 ? 0.0 : INFINITY;
    return sqrt(du2 / u2);
}
