/*
 * FP64 CPU oracle of the consistent and conservative phase-field lattice
 * Boltzmann method of Zhan, Chai & Shi, "Consistent and conservative
 * phase-field based lattice Boltzmann method for incompressible two-phase
 * flows" (arXiv:2111.00847).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference against which the
 * CUDA path is checked.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline / reference leg may load it; the product never
 * links, calls or falls back to it.  It shares no source with the CUDA path:
 * its parameter struct, lattice tables and every formula are written here
 * again, from the paper.
 *
 * Style: plain C99, double precision, one whole-grid pass per sub-step of
 * the scheme, moments formed by dense 9x9 products with the transformation
 * matrix of Eq. (C.1), no fusion and no blocking.  Loops over nodes carry an
 * OpenMP "parallel for" (each pass writes only its own node) so that the
 * same code runs single- or multi-threaded with identical results.
 *
 * One time step t -> t+1 (Sec. 3 and App. C), in this order:
 *   1. phi = sum_i f_i                                    Eq. (22a)
 *   2. ghost values of phi next to walls (wetting, Eqs. (49)-(50))
 *   3. grad phi, lap phi by the isotropic stencils          Eqs. (C.9)-(C.10)
 *   4. chemical potential mu_phi                           Eq. (5)
 *      AC: lambda, n, D = grad phi - lambda n              Eqs. (7)-(8)
 *      CH: D = grad mu_phi (mu ghosts mirrored)            Eq. (6)
 *   5. rho(phi), grad rho, nu(phi)                         Eqs. (10)-(12)
 *   6. m^{phi C} = -(d rho/d phi) M_phi D                  Eq. (15)
 *      F = mu_phi grad phi + G                             Sec. 2, Eq. (9c)
 *   7. rho u = sum_i c_i g_i + F/2                         Eq. (22b)
 *      p from Eq. (39), second way of Remark 1
 *   8. explicit-Euler time derivatives from the stored history   App. C
 *   9. MRT collisions of f (Eq. (17)) and g (Eq. (40)) with the moment
 *      vectors of Eqs. (C.2)-(C.4) and the relaxation rules of Sec. 4
 *  10. streaming with half-way bounce-back (Sec. 4)
 *
 * Solid obstacles (optional, oracle_set_solid): a node marked solid takes no
 * part in the flow.  A link whose upstream node is solid reflects like a
 * wall link (half-way bounce-back, Sec. 4), and the stencils of step 3 see
 * at a solid node the neutral-wetting value of the field (mean over its fluid
 * neighbours, fill_pad).  Every per-node output at a solid node is zero.
 *
 * Parity notes (readings of points the paper leaves open) are stated where
 * they are used: the guard on n, the stable form of the wetting root, the
 * ghost value next to a wall, the initial populations and history.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Parameter block: same field order and types as the library's C-ABI. */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t version, nx, ny, precision;
    int32_t phase_model, flux_model, visc_law, gravity_mode;
    int32_t bc[4];             /* left, right, bottom, top: 0 periodic, 1 wall */
    int32_t diag_every, reserved;
    double phiA, phiB, rhoA, rhoB, muA, muB;
    double mobility, width, sigma, eta;
    double gx, gy, rho0;
    double theta_deg[4];
    double s_f[9], s_g[9];     /* NaN: the default rule of Sec. 4 */
    double n_delta;            /* regularisation of n in units of dphi / W; 0: 5e-3 */
} oracle_params;

enum { O_OK = 0, O_EINVAL = -1, O_ENOMEM = -2, O_EUNSTABLE = -4, O_EUNSUPPORTED = -5 };
enum { O_AC = 0, O_CH = 1 };
enum { O_PRESENT = 0, O_ORIGINAL = 1, O_CORRECTED = 2 };
enum { O_LINEAR_MU = 0, O_INVERSE_NU = 1 };
enum { O_G_CONST = 0, O_G_RHO = 1, O_G_RHO_MINUS_MEAN = 2 };
enum { O_PERIODIC = 0, O_WALL = 1 };
enum { O_LEFT = 0, O_RIGHT = 1, O_BOTTOM = 2, O_TOP = 3 };
enum {
    O_PHI = 0, O_UX = 1, O_UY = 2, O_P = 3, O_RHO = 4, O_FPOP = 5, O_GPOP = 6,
    O_HIST = 7, O_DIAG = 8, O_MU = 9, O_MCX = 10, O_MCY = 11
};
#define O_NDIAG 8

/* ------------------------------------------------------------------ */
/* D2Q9 lattice.  The velocity order is the one fixed by rows 3 and 5  */
/* (x and y momentum) of the matrix in Eq. (C.1).                      */
/* ------------------------------------------------------------------ */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double WI[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
#define CS2 (1.0 / 3.0)

/* Orthogonal transformation matrix, Eq. (C.1). */
static const double MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
};

/* M^{-1}: the rows of M are mutually orthogonal, so M^{-1} = M^T D^{-1}
 * with D = diag(|row_k|^2).  Filled once by minv_init(). */
static double MINV[9][9];
static int minv_ready = 0;

static void minv_init(void)
{
    if (minv_ready) return;
    for (int k = 0; k < 9; ++k) {
        double n2 = 0.0;
        for (int j = 0; j < 9; ++j) n2 += MM[k][j] * MM[k][j];
        for (int i = 0; i < 9; ++i) MINV[i][k] = MM[k][i] / n2;
    }
    minv_ready = 1;
}

/* ------------------------------------------------------------------ */
/* State                                                              */
/* ------------------------------------------------------------------ */
typedef struct {
    oracle_params P;
    int nx, ny;
    long N;
    long t;
    /* free-energy constants, Eq. (3), and density slope, Eq. (10) */
    double beta, kappa, dphi, drho_dphi, lam_coef, n_delta;
    /* rates: constant value, or NaN for the per-node default rule */
    double sf[9], sg[9];
    double Hc, Kc;            /* pressure-scheme constants, App. C */
    double cos_t[4];          /* cos(theta) per side */
    /* populations (post-stream, i.e. what each node sees at time t) */
    double *f[9], *g[9];
    double *fs[9], *gs[9];    /* post-collision scratch */
    double *hist[5];          /* chi(t-1): phi u, phi v, u.m, u mx - v my, u my + v mx */
    double *phi_prev;         /* phi(t-1), for d rho/dt in the S_m statistic */
    /* macroscopic work arrays (one pass each) */
    double *phi, *pad, *padmu, *gpx, *gpy, *lap, *mu, *Dx, *Dy, *lam, *nxv, *nyv;
    double *rho, *ux, *uy, *p, *mcx, *mcy, *Fx, *Fy, *s78;
    double *cur[5], *dt[5];
    double diag[O_NDIAG];
    unsigned char *solid;     /* NULL, or [ny][nx] with 1 at solid nodes */
    int wet_flag;
    char err[256];
} ostate;

static int g_threads = 0;

void oracle_set_threads(int n) { g_threads = n; }

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

static void set_threads(void)
{
#ifdef _OPENMP
    if (g_threads > 0) omp_set_num_threads(g_threads);
#endif
}

static double cos_deg(double th)
{
    /* exact zero for the neutral wall */
    return th == 90.0 ? 0.0 : cos(th * 3.14159265358979323846 / 180.0);
}

/* ------------------------------------------------------------------ */
/* Wetting boundary, Eqs. (49)-(50).                                   */
/* The wall order parameter phi_w solves a phi_w^2 + b phi_w + c = 0   */
/* with a = 4 cos(theta)/(W dphi), b = 8/3 - a (phiA + phiB),          */
/* c = a phiA phiB + phi_2/3 - 3 phi_1, phi_1 and phi_2 the first and  */
/* second fluid nodes (at 1/2 and 3/2 from the wall).  The root the    */
/* paper selects, (-b + sqrt(b^2 - 4ac))/(2a), is evaluated in the     */
/* algebraically identical form 2c / (-b - sqrt(b^2 - 4ac)), which has */
/* the a -> 0 limit -c/b (theta = 90 degrees) without cancellation.    */
/* A negative discriminant is clamped to zero and flagged.             */
/* The ghost value at -1/2 (the stencil point beyond the wall) is the  */
/* quadratic through (0, phi_w), (1/2, phi_1), (3/2, phi_2) -- the     */
/* same quadratic whose wall slope gives the coefficients of Eq. (50)  */
/* -- evaluated at -1/2:  ghost = 8/3 phi_w - 2 phi_1 + phi_2 / 3.      */
/* ------------------------------------------------------------------ */
static double wall_phi(const oracle_params *P, double phi1, double phi2, double cos_t, int *flag)
{
    const double a = 4.0 * cos_t / (P->width * (P->phiA - P->phiB));
    const double b = 8.0 / 3.0 - a * (P->phiA + P->phiB);
    const double c = a * P->phiA * P->phiB + phi2 / 3.0 - 3.0 * phi1;
    double disc = b * b - 4.0 * a * c;
    if (disc < 0.0) {
        disc = 0.0;
        if (flag) *flag = 1;
    }
    return 2.0 * c / (-b - sqrt(disc));
}

static double wall_ghost(const oracle_params *P, double phi1, double phi2, double cos_t, int *flag)
{
    const double phiw = wall_phi(P, phi1, phi2, cos_t, flag);
    return 8.0 / 3.0 * phiw - 2.0 * phi1 + phi2 / 3.0;
}

/* ------------------------------------------------------------------ */
/* Padded copy of a node field with one ghost layer.  Solid nodes      */
/* first (solid_value), then the x sides, then the y sides over the    */
/* extended x range (so corners take the y rule applied to the x       */
/* ghosts).  Periodic sides wrap; wall sides use the wetting ghost      */
/* (wetting != 0) or the mirror value (wetting == 0).                  */
/* ------------------------------------------------------------------ */
#define PADI(st, i, j) ((size_t)((j) + 1) * (size_t)((st)->nx + 2) + (size_t)((i) + 1))

/* Node index of (i, j) wrapped across periodic sides, or -1 beyond a wall. */
static long node_at(const ostate *st, int i, int j)
{
    if (i < 0 || i >= st->nx) {
        if (st->P.bc[O_LEFT] != O_PERIODIC) return -1;
        i = (i + st->nx) % st->nx;
    }
    if (j < 0 || j >= st->ny) {
        if (st->P.bc[O_BOTTOM] != O_PERIODIC) return -1;
        j = (j + st->ny) % st->ny;
    }
    return (long)j * st->nx + i;
}

/* Value a solid node (i, j) shows to the stencils.  The paper states the
 * wetting condition for plane walls only (Eqs. (49)-(50)); for obstacles the
 * reading is neutral wetting: the mean of the field over the fluid nodes
 * among the four axis neighbours, or, if there are none, over the fluid
 * diagonal neighbours (0 where no fluid node is adjacent: no fluid stencil
 * reaches it).  Next to a plane wall of solid nodes this is the mirror value,
 * the theta = 90 degrees ghost of Eq. (50). */
static double solid_value(const ostate *st, const double *a, int i, int j)
{
    for (int k0 = 1; k0 <= 5; k0 += 4) {
        double s = 0.0;
        int c = 0;
        for (int k = k0; k < k0 + 4; ++k) {
            const long q = node_at(st, i + CX[k], j + CY[k]);
            if (q >= 0 && !st->solid[q]) {
                s += a[q];
                ++c;
            }
        }
        if (c > 0) return s / c;
    }
    return 0.0;
}

static void fill_pad(ostate *st, const double *a, double *pad, int wetting)
{
    const int nx = st->nx, ny = st->ny;
    const oracle_params *P = &st->P;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const size_t n = (size_t)j * nx + i;
            pad[PADI(st, i, j)] = (st->solid && st->solid[n]) ? solid_value(st, a, i, j) : a[n];
        }
    for (int j = 0; j < ny; ++j) {
        const double c0 = pad[PADI(st, 0, j)], c1 = pad[PADI(st, 1, j)];
        const double e0 = pad[PADI(st, nx - 1, j)], e1 = pad[PADI(st, nx - 2, j)];
        if (P->bc[O_LEFT] == O_PERIODIC) {
            pad[PADI(st, -1, j)] = e0;
            pad[PADI(st, nx, j)] = c0;
        } else {
            pad[PADI(st, -1, j)] = wetting ? wall_ghost(P, c0, c1, st->cos_t[O_LEFT], &st->wet_flag) : c0;
            pad[PADI(st, nx, j)] = wetting ? wall_ghost(P, e0, e1, st->cos_t[O_RIGHT], &st->wet_flag) : e0;
        }
    }
    for (int i = -1; i <= nx; ++i) {
        if (P->bc[O_BOTTOM] == O_PERIODIC) {
            pad[PADI(st, i, -1)] = pad[PADI(st, i, ny - 1)];
            pad[PADI(st, i, ny)] = pad[PADI(st, i, 0)];
        } else {
            pad[PADI(st, i, -1)] = wetting ? wall_ghost(P, pad[PADI(st, i, 0)], pad[PADI(st, i, 1)], st->cos_t[O_BOTTOM], &st->wet_flag) : pad[PADI(st, i, 0)];
            pad[PADI(st, i, ny)] = wetting ? wall_ghost(P, pad[PADI(st, i, ny - 1)], pad[PADI(st, i, ny - 2)], st->cos_t[O_TOP], &st->wet_flag) : pad[PADI(st, i, ny - 1)];
        }
    }
}

/* Isotropic central schemes, Eqs. (C.9)-(C.10) with dt = 1:
 *   grad chi = sum_{i != 0} w_i c_i chi(x + c_i) / c_s^2
 *   lap chi  = sum_{i != 0} 2 w_i [chi(x + c_i) - chi(x)] / c_s^2        */
static void stencil(ostate *st, const double *pad, double *gx, double *gy, double *lap)
{
    const int nx = st->nx, ny = st->ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const double c0 = pad[PADI(st, i, j)];
            double sx = 0.0, sy = 0.0, sl = 0.0;
            for (int k = 1; k < 9; ++k) {
                const double v = pad[PADI(st, i + CX[k], j + CY[k])];
                sx += WI[k] * CX[k] * v;
                sy += WI[k] * CY[k] * v;
                sl += 2.0 * WI[k] * (v - c0);
            }
            const size_t n = (size_t)j * nx + i;
            if (gx) gx[n] = sx / CS2;
            if (gy) gy[n] = sy / CS2;
            if (lap) lap[n] = sl / CS2;
        }
}

/* ------------------------------------------------------------------ */
/* Node-level moment vectors of App. C (c = dx/dt = 1).               */
/* in[] layout (see oracle_node_moments):                              */
/*  0 phi 1 mu 2 u 3 v 4 p 5 rho 6 mcx 7 mcy 8 Fx 9 Fy 10 drho_x       */
/*  11 drho_y 12 lambda 13 nx 14 ny 15 dt(phi u) 16 dt(phi v)          */
/*  17 dt(u.m) 18 dt(u mx - v my) 19 dt(u my + v mx)                   */
/* ------------------------------------------------------------------ */
static void node_moments(const oracle_params *P, const double *in,
                         double mfeq[9], double mR[9], double mgeq[9], double mF[9])
{
    const double phi = in[0], mu = in[1], u = in[2], v = in[3], p = in[4], rho = in[5];
    const double mx = in[6], my = in[7], Fx = in[8], Fy = in[9], rx = in[10], ry = in[11];
    const double lam = in[12], nxn = in[13], nyn = in[14];
    const double dphiu = in[15], dphiv = in[16], dum = in[17], dA = in[18], dB = in[19];
    const double eta = P->eta, rho0 = P->rho0;

    /* phase field, Eq. (C.4) (AC) or Eq. (C.3) (CH) */
    const double chi = (P->phase_model == O_CH) ? mu : phi; /* the eta-term argument */
    mfeq[0] = phi;
    mfeq[1] = -4.0 * phi + 2.0 * eta * chi;
    mfeq[2] = 4.0 * phi - 3.0 * eta * chi;
    mfeq[3] = phi * u;
    mfeq[4] = -phi * u;
    mfeq[5] = phi * v;
    mfeq[6] = -phi * v;
    mfeq[7] = 0.0;
    mfeq[8] = 0.0;
    double Xx = dphiu, Xy = dphiv;
    if (P->phase_model == O_AC) {
        Xx += lam * nxn / 3.0;
        Xy += lam * nyn / 3.0;
    }
    mR[0] = mR[1] = mR[2] = 0.0;
    mR[3] = Xx;
    mR[4] = -Xx;
    mR[5] = Xy;
    mR[6] = -Xy;
    mR[7] = mR[8] = 0.0;

    /* hydrodynamics, Eq. (C.2) */
    const double uu = u * u + v * v;
    const double um = u * mx + v * my;
    mgeq[0] = rho0;
    mgeq[1] = -4.0 * rho0 + 6.0 * p + 3.0 * rho * uu + 3.0 * um;
    mgeq[2] = 4.0 * rho0 - 9.0 * p - 3.0 * rho * uu - 3.0 * um;
    mgeq[3] = rho * u;
    mgeq[4] = -rho * u;
    mgeq[5] = rho * v;
    mgeq[6] = -rho * v;
    mgeq[7] = u * mx - v * my + rho * (u * u - v * v);
    mgeq[8] = (u * my + v * mx + 2.0 * rho * u * v) / 2.0;

    const double ugr = u * rx + v * ry;
    const double uF = u * Fx + v * Fy;
    mF[0] = ugr;
    mF[1] = 3.0 * dum + 6.0 * uF;
    mF[2] = -ugr - 3.0 * dum - 6.0 * uF;
    mF[3] = Fx;
    mF[4] = -Fx;
    mF[5] = Fy;
    mF[6] = -Fy;
    mF[7] = 2.0 / 3.0 * (u * rx - v * ry) + 2.0 * (u * Fx - v * Fy) + dA;
    mF[8] = 1.0 / 3.0 * (u * ry + v * rx) + (2.0 * (u * Fy + v * Fx) + dB) / 2.0;
}

/* Steps 2-4 from st->phi: ghosts, stencils, mu_phi and the diffusion flux D. */
static void phase_pass(ostate *st)
{
    const oracle_params *P = &st->P;
    const long N = st->N;
    const double phiA = P->phiA, phiB = P->phiB;
    /* 2.-3. ghosts and stencils */
    fill_pad(st, st->phi, st->pad, 1);
    stencil(st, st->pad, st->gpx, st->gpy, st->lap);

    /* 4. chemical potential, Eq. (5) */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        const double ph = st->phi[n];
        st->mu[n] = 4.0 * st->beta * (ph - phiA) * (ph - phiB) * (ph - 0.5 * (phiA + phiB)) - st->kappa * st->lap[n];
    }
    if (P->phase_model == O_CH) {
        /* CH: D = grad mu_phi (Eq. (6)); mu ghosts take the mirror value */
        fill_pad(st, st->mu, st->padmu, 0);
        stencil(st, st->padmu, st->Dx, st->Dy, NULL);
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) st->lam[n] = st->nxv[n] = st->nyv[n] = 0.0;
    } else {
        /* AC: lambda = sqrt(2 beta/k)(phiA - phi)(phi - phiB) = 4 (phiA-phi)(phi-phiB)/(W dphi),
         * n = grad phi / |grad phi|, D = grad phi - lambda n  (Eqs. (7)-(8)).
         * n is undefined where grad phi = 0; reading:
         *   n = grad phi / (|grad phi|^4 + delta_n^4)^(1/4),
         *   delta_n = n_delta dphi / W,  n_delta = 5e-3 unless the parameter sets it.
         * It is the unit normal to within (delta_n / |grad phi|)^4 / 4 -- 2.5e-5
         * where |grad phi| = 10 delta_n -- and a smooth function of grad phi
         * everywhere.  Where |grad phi| is not far above delta_n (phi (1 - phi)
         * below about n_delta / 4 in a tanh profile) the sharpening flux is
         * weakened and the interface tails widen; with viscosity ratio 1000 a
         * tail of 1e-3 in phi doubles the light phase's viscosity, so the
         * layered Poiseuille error of Table 2 needs a small n_delta: 0.277 at
         * n_delta = 5e-3 against 1.03e-2 at 1e-5 (ratio 1000; Table 2:
         * 8.4e-3).  The slope of n in the bulk, about 1/delta_n, bounds how
         * strongly a round-off-level gradient -- where an overshoot
         * phi > phiA (or < phiB) makes lambda nonzero -- can steer the flux
         * (for lambda > |grad phi| the anti-diffusive rate is lambda/delta_n):
         * on a 64 x 256 RTI (Re 1000) a one-ulp perturbation of phi0 grows in
         * 2000 steps to 7e-15 with n_delta = 5e-3 but to 3e-3 with 3e-3; with
         * 1e-5, rounding-order differences between two FP64 implementations
         * reach 1e-8 within 100 steps of the dam break.  The default keeps
         * the step well conditioned and differentiable; flows whose
         * viscosity follows the tails closely (the layered channel) set the
         * small value. */
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            const double ph = st->phi[n];
            const double lam = st->lam_coef * (phiA - ph) * (ph - phiB);
            const double g2 = st->gpx[n] * st->gpx[n] + st->gpy[n] * st->gpy[n];
            const double d2 = st->n_delta * st->n_delta;
            const double gm = sqrt(sqrt(g2 * g2 + d2 * d2));
            const double nxn = st->gpx[n] / gm;
            const double nyn = st->gpy[n] / gm;
            st->lam[n] = lam;
            st->nxv[n] = nxn;
            st->nyv[n] = nyn;
            st->Dx[n] = st->gpx[n] - lam * nxn;
            st->Dy[n] = st->gpy[n] - lam * nyn;
        }
    }

}

/* Every per-node quantity of a solid node is zero (it carries no fluid). */
static void zero_solid(ostate *st)
{
    double *arrs[] = {st->phi, st->gpx, st->gpy, st->lap, st->mu, st->Dx, st->Dy, st->lam, st->nxv,
                      st->nyv, st->rho, st->ux, st->uy, st->p, st->mcx, st->mcy, st->Fx, st->Fy,
                      st->s78, st->cur[0], st->cur[1], st->cur[2], st->cur[3], st->cur[4],
                      st->dt[0], st->dt[1], st->dt[2], st->dt[3], st->dt[4]};
    for (long n = 0; n < st->N; ++n)
        if (st->solid[n])
            for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); ++k) arrs[k][n] = 0.0;
}

/* ------------------------------------------------------------------ */
/* Macroscopic pass at the current time t.  Fills phi, gradients, mu,  */
/* D, rho, m^{phi C}, F, u, p, the per-node viscous rate and the       */
/* explicit-Euler time derivatives against the stored history.         */
/* ------------------------------------------------------------------ */
static void macro_pass(ostate *st)
{
    const oracle_params *P = &st->P;
    const long N = st->N;
    const double phiA = P->phiA, phiB = P->phiB;

    /* 1. phi = sum_i f_i, Eq. (22a) */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double s = 0.0;
        for (int i = 0; i < 9; ++i) s += st->f[i][n];
        st->phi[n] = s;
    }
    phase_pass(st);

    /* 5.-8. */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        const double ph = st->phi[n];
        /* Eq. (10) */
        const double rho = st->drho_dphi * (ph - phiB) + P->rhoB;
        const double rx = st->drho_dphi * st->gpx[n], ry = st->drho_dphi * st->gpy[n];
        /* Eq. (11) or Eq. (12); s_g^{7,8} = 1/(nu/c_s^2 + 1/2) (Sec. 4) */
        double nu;
        const double frac = (ph - phiB) / (phiA - phiB);
        if (P->visc_law == O_LINEAR_MU) {
            nu = (frac * (P->muA - P->muB) + P->muB) / rho;
        } else {
            const double inuA = P->rhoA / P->muA, inuB = P->rhoB / P->muB;
            nu = 1.0 / (frac * (inuA - inuB) + inuB);
        }
        st->s78[n] = 1.0 / (nu / CS2 + 0.5);
        /* Eq. (15): consistent flux of the present model; m = rho u for the original one */
        double mx = 0.0, my = 0.0;
        if (P->flux_model == O_PRESENT) {
            mx = -st->drho_dphi * P->mobility * st->Dx[n];
            my = -st->drho_dphi * P->mobility * st->Dy[n];
        }
        /* body force G (Sec. 4.2, 4.4, 4.5) and total force F = mu grad phi + G */
        double Gs = 1.0;
        if (P->gravity_mode == O_G_RHO) Gs = rho;
        else if (P->gravity_mode == O_G_RHO_MINUS_MEAN) Gs = rho - 0.5 * (P->rhoA + P->rhoB);
        const double Fx = st->mu[n] * st->gpx[n] + Gs * P->gx;
        const double Fy = st->mu[n] * st->gpy[n] + Gs * P->gy;
        /* Eq. (22b) */
        double jx = 0.0, jy = 0.0, gsum = 0.0;
        for (int i = 0; i < 9; ++i) {
            jx += CX[i] * st->g[i][n];
            jy += CY[i] * st->g[i][n];
            if (i != 0) gsum += st->g[i][n];
        }
        const double u = (jx + 0.5 * Fx) / rho;
        const double v = (jy + 0.5 * Fy) / rho;
        /* time derivatives, explicit Euler against chi(t-1) (App. C) */
        const double c0 = ph * u, c1 = ph * v, c2 = u * mx + v * my;
        const double c3 = u * mx - v * my, c4 = u * my + v * mx;
        st->cur[0][n] = c0;
        st->cur[1][n] = c1;
        st->cur[2][n] = c2;
        st->cur[3][n] = c3;
        st->cur[4][n] = c4;
        for (int k = 0; k < 5; ++k) st->dt[k][n] = st->cur[k][n] - st->hist[k][n];
        /* Eq. (39), second way of Remark 1: J d dt p dropped,
         * dt(rho u.u) -> 2 F.u, dt(m.u) kept by explicit Euler;
         * s_0(phi,u) = -w_0 (rho u.u + m.u) / (2 c_s^2) from Eq. (20) at i = 0 */
        const double s0 = -WI[0] * (rho * (u * u + v * v) + c2) / (2.0 * CS2);
        const double p = CS2 / (1.0 - WI[0]) *
                         (gsum + (0.5 + st->Hc) * (u * rx + v * ry) + s0 +
                          st->Kc * (2.0 * (Fx * u + Fy * v) + st->dt[2][n]));
        st->rho[n] = rho;
        st->ux[n] = u;
        st->uy[n] = v;
        st->p[n] = p;
        st->mcx[n] = mx;
        st->mcy[n] = my;
        st->Fx[n] = Fx;
        st->Fy[n] = Fy;
    }
    if (st->solid) zero_solid(st);
}

static void gather_node_input(const ostate *st, long n, double in[20])
{
    const double drx = st->drho_dphi * st->gpx[n], dry = st->drho_dphi * st->gpy[n];
    in[0] = st->phi[n];
    in[1] = st->mu[n];
    in[2] = st->ux[n];
    in[3] = st->uy[n];
    in[4] = st->p[n];
    in[5] = st->rho[n];
    in[6] = st->mcx[n];
    in[7] = st->mcy[n];
    in[8] = st->Fx[n];
    in[9] = st->Fy[n];
    in[10] = drx;
    in[11] = dry;
    in[12] = st->lam[n];
    in[13] = st->nxv[n];
    in[14] = st->nyv[n];
    for (int k = 0; k < 5; ++k) in[15 + k] = st->dt[k][n];
}

/* MRT collisions, Eq. (17) (f) and Eq. (40) (g):
 *   x* = M^{-1} [ (I - S) m + S m^eq + (I - S/2) m_src ]                 */
static void collide(ostate *st)
{
    const long N = st->N;
    const oracle_params *P = &st->P;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (st->solid && st->solid[n]) {
            for (int i = 0; i < 9; ++i) st->fs[i][n] = st->gs[i][n] = 0.0;
            continue;
        }
        double in[20], mfeq[9], mR[9], mgeq[9], mF[9];
        gather_node_input(st, n, in);
        node_moments(P, in, mfeq, mR, mgeq, mF);
        double Sf[9], Sg[9];
        for (int k = 0; k < 9; ++k) {
            Sf[k] = isnan(st->sf[k]) ? 1.0 : st->sf[k];
            Sg[k] = isnan(st->sg[k]) ? 1.0 : st->sg[k];
        }
        /* default rules (Sec. 4): s_f^3 = s_f^5 = 1/(M_phi/(eta c_s^2) + 1/2),
         * s_g^7 = s_g^8 = 1/(nu/c_s^2 + 1/2) per node, all others 1 */
        const double sfm = 1.0 / (P->mobility / (P->eta * CS2) + 0.5);
        if (isnan(st->sf[3])) Sf[3] = sfm;
        if (isnan(st->sf[5])) Sf[5] = sfm;
        if (isnan(st->sg[7])) Sg[7] = st->s78[n];
        if (isnan(st->sg[8])) Sg[8] = st->s78[n];

        double m[9], ms[9];
        for (int k = 0; k < 9; ++k) {
            m[k] = 0.0;
            for (int j = 0; j < 9; ++j) m[k] += MM[k][j] * st->f[j][n];
        }
        for (int k = 0; k < 9; ++k) ms[k] = (1.0 - Sf[k]) * m[k] + Sf[k] * mfeq[k] + (1.0 - 0.5 * Sf[k]) * mR[k];
        for (int i = 0; i < 9; ++i) {
            double s = 0.0;
            for (int k = 0; k < 9; ++k) s += MINV[i][k] * ms[k];
            st->fs[i][n] = s;
        }
        for (int k = 0; k < 9; ++k) {
            m[k] = 0.0;
            for (int j = 0; j < 9; ++j) m[k] += MM[k][j] * st->g[j][n];
        }
        for (int k = 0; k < 9; ++k) ms[k] = (1.0 - Sg[k]) * m[k] + Sg[k] * mgeq[k] + (1.0 - 0.5 * Sg[k]) * mF[k];
        for (int i = 0; i < 9; ++i) {
            double s = 0.0;
            for (int k = 0; k < 9; ++k) s += MINV[i][k] * ms[k];
            st->gs[i][n] = s;
        }
    }
}

/* Streaming x_i(x + c_i, t+1) = x_i*(x, t), written as a pull; a link whose
 * upstream node x - c_i lies beyond a wall, or is a solid node, takes the
 * reflected population x_{opp(i)}*(x, t) (half-way bounce-back, Sec. 4).
 * Solid nodes hold no populations (zero). */
static void stream_pull(ostate *st, double *const *src, double *const *dst)
{
    const int nx = st->nx, ny = st->ny;
    const oracle_params *P = &st->P;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t n = (size_t)y * nx + x;
            if (st->solid && st->solid[n]) {
                for (int i = 0; i < 9; ++i) dst[i][n] = 0.0;
                continue;
            }
            for (int i = 0; i < 9; ++i) {
                int sx = x - CX[i], sy = y - CY[i];
                int wall = 0;
                if (sx < 0 || sx >= nx) {
                    if (P->bc[O_LEFT] == O_PERIODIC) sx = (sx + nx) % nx;
                    else wall = 1;
                }
                if (sy < 0 || sy >= ny) {
                    if (P->bc[O_BOTTOM] == O_PERIODIC) sy = (sy + ny) % ny;
                    else wall = 1;
                }
                if (!wall && st->solid && st->solid[(size_t)sy * nx + sx]) wall = 1;
                dst[i][n] = wall ? src[OPP[i]][n] : src[i][(size_t)sy * nx + sx];
            }
        }
}

/* ------------------------------------------------------------------ */
/* Diagnostics (Sec. 4.1, Eqs. (42)-(43)) at the current time t.       */
/*  D_u: rms of tr S, with S from the local scheme Eq. (35) using the   */
/*       viscous rate s_2 = s_g^7 of the node;                          */
/*  S_m: rms of d rho/dt + div(rho u + m^{phi C}), d rho/dt by explicit */
/*       Euler against phi(t-1), the divergence by Eq. (C.9).           */
/* Both are averaged over the fluid nodes not adjacent to a wall or a   */
/* solid node (their stencils would reach beyond the boundary); sums    */
/* and maxima run over the fluid nodes.  Requires macro_pass() first.   */
/* out: t, sum phi, D_u^rms, S_m^rms, max|u|, non-finite count,         */
/*      number of averaged nodes, 0                                     */
/* ------------------------------------------------------------------ */
static void diagnostics(ostate *st, double out[O_NDIAG])
{
    const int nx = st->nx, ny = st->ny;
    const oracle_params *P = &st->P;
    double sphi = 0.0, sdu = 0.0, ssm = 0.0, umax = 0.0, nbad = 0.0, nint = 0.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const long n = (long)y * nx + x;
            if (st->solid && st->solid[n]) continue;
            sphi += st->phi[n];
            const double um2 = st->ux[n] * st->ux[n] + st->uy[n] * st->uy[n];
            if (!isfinite(st->phi[n]) || !isfinite(um2)) nbad += 1.0;
            else if (sqrt(um2) > umax) umax = sqrt(um2);
            if ((P->bc[O_LEFT] == O_WALL && (x == 0 || x == nx - 1)) ||
                (P->bc[O_BOTTOM] == O_WALL && (y == 0 || y == ny - 1)))
                continue;
            if (st->solid) {
                int near = 0;
                for (int k = 1; k < 9; ++k) {
                    const long q = node_at(st, x + CX[k], y + CY[k]);
                    if (q >= 0 && st->solid[q]) near = 1;
                }
                if (near) continue;
            }
            /* tr S, Eq. (35): tr sum c c (g - g^eq) = [(m1-m1eq) + 4 (m0-m0eq)]/3,
             * tr M_2F = (mF1 + 4 mF0)/3 */
            double in[20], mfeq[9], mR[9], mgeq[9], mF[9], m[9];
            gather_node_input(st, n, in);
            node_moments(P, in, mfeq, mR, mgeq, mF);
            for (int k = 0; k < 2; ++k) {
                m[k] = 0.0;
                for (int j = 0; j < 9; ++j) m[k] += MM[k][j] * st->g[j][n];
            }
            const double s2 = isnan(st->sg[7]) ? st->s78[n] : st->sg[7];
            const double trneq = ((m[1] - mgeq[1]) + 4.0 * (m[0] - mgeq[0])) / 3.0;
            const double trM2F = (mF[1] + 4.0 * mF[0]) / 3.0;
            const double trS = -s2 / (2.0 * st->rho[n] * CS2) * (trneq + 0.5 * trM2F);
            /* S_m */
            double div = 0.0;
            for (int k = 1; k < 9; ++k) {
                int xn = x + CX[k], yn = y + CY[k];
                xn = (xn + nx) % nx;
                yn = (yn + ny) % ny;
                const long q = (long)yn * nx + xn;
                const double Jx = st->rho[q] * st->ux[q] + st->mcx[q];
                const double Jy = st->rho[q] * st->uy[q] + st->mcy[q];
                div += WI[k] * (CX[k] * Jx + CY[k] * Jy) / CS2;
            }
            const double drho_dt = st->drho_dphi * (st->phi[n] - st->phi_prev[n]);
            const double sm = drho_dt + div;
            sdu += trS * trS;
            ssm += sm * sm;
            nint += 1.0;
        }
    out[0] = (double)st->t;
    out[1] = sphi;
    out[2] = nint > 0 ? sqrt(sdu / nint) : 0.0;
    out[3] = nint > 0 ? sqrt(ssm / nint) : 0.0;
    out[4] = umax;
    out[5] = nbad;
    out[6] = nint;
    out[7] = 0.0;
}

/* ------------------------------------------------------------------ */
/* Public entry points                                                */
/* ------------------------------------------------------------------ */
static void *xalloc(size_t n) { return calloc(n ? n : 1, sizeof(double)); }

const char *oracle_last_error(const ostate *st) { return st ? st->err : "null handle"; }

void oracle_destroy(ostate *st)
{
    if (!st) return;
    for (int i = 0; i < 9; ++i) {
        free(st->f[i]); free(st->g[i]); free(st->fs[i]); free(st->gs[i]);
    }
    for (int k = 0; k < 5; ++k) { free(st->hist[k]); free(st->cur[k]); free(st->dt[k]); }
    double *arrs[] = {st->phi_prev, st->phi, st->pad, st->padmu, st->gpx, st->gpy, st->lap, st->mu,
                      st->Dx, st->Dy, st->lam, st->nxv, st->nyv, st->rho, st->ux, st->uy, st->p,
                      st->mcx, st->mcy, st->Fx, st->Fy, st->s78};
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); ++k) free(arrs[k]);
    free(st->solid);
    free(st);
}

static int validate(const oracle_params *P, char *err)
{
#define BAD(msg) do { snprintf(err, 256, "%s", msg); return O_EINVAL; } while (0)
    if (P->version != 1) BAD("params.version must be 1");
    if (P->nx < 3 || P->ny < 3) BAD("grid must be at least 3 x 3");
    if ((long)P->nx * (long)P->ny > (1L << 31) - 1) BAD("grid too large");
    if (P->phase_model != O_AC && P->phase_model != O_CH) BAD("phase_model");
    if (P->flux_model == O_CORRECTED) { snprintf(err, 256, "flux_model CORRECTED not implemented"); return O_EUNSUPPORTED; }
    if (P->flux_model != O_PRESENT && P->flux_model != O_ORIGINAL) BAD("flux_model");
    if (P->visc_law != O_LINEAR_MU && P->visc_law != O_INVERSE_NU) BAD("visc_law");
    if (P->gravity_mode < 0 || P->gravity_mode > 2) BAD("gravity_mode");
    if (P->bc[0] != P->bc[1] || P->bc[2] != P->bc[3]) BAD("opposite sides must share a boundary type");
    for (int s = 0; s < 4; ++s) {
        if (P->bc[s] != O_PERIODIC && P->bc[s] != O_WALL) BAD("bc");
        if (!(P->theta_deg[s] >= 0.0 && P->theta_deg[s] <= 180.0)) BAD("contact angle outside [0,180]");
    }
    if (!(P->phiA > P->phiB)) BAD("phiA must exceed phiB");
    if (!(P->rhoA > 0 && P->rhoB > 0 && P->muA > 0 && P->muB > 0)) BAD("densities and viscosities must be positive");
    if (!(P->width > 0 && P->sigma >= 0 && P->mobility >= 0 && P->eta > 0)) BAD("width, sigma, mobility, eta");
    if (!(P->n_delta >= 0.0 && P->n_delta < 1.0)) BAD("n_delta outside [0, 1)");
    for (int k = 0; k < 9; ++k) {
        if (!isnan(P->s_f[k]) && !(P->s_f[k] > 0 && P->s_f[k] < 2)) BAD("s_f outside (0,2)");
        if (!isnan(P->s_g[k]) && !(P->s_g[k] > 0 && P->s_g[k] < 2)) BAD("s_g outside (0,2)");
    }
    {
        const double amax = 4.0 / (P->width * (P->phiA - P->phiB));
        if (8.0 / 3.0 - amax * fabs(P->phiA + P->phiB) <= 0.0) BAD("interface too thin for the wetting root");
    }
    return O_OK;
#undef BAD
}

int oracle_create(const oracle_params *P, ostate **out)
{
    if (!P || !out) return O_EINVAL;
    *out = NULL;
    char err[256] = {0};
    int rc = validate(P, err);
    if (rc != O_OK) {
        fprintf(stderr, "oracle_create: %s\n", err);
        return rc;
    }
    minv_init();
    ostate *st = (ostate *)calloc(1, sizeof(ostate));
    if (!st) return O_ENOMEM;
    st->P = *P;
    st->nx = P->nx;
    st->ny = P->ny;
    st->N = (long)P->nx * P->ny;
    const long N = st->N;
    const size_t NP = (size_t)(P->nx + 2) * (P->ny + 2);
    int ok = 1;
    for (int i = 0; i < 9; ++i) {
        ok &= !!(st->f[i] = xalloc(N)); ok &= !!(st->g[i] = xalloc(N));
        ok &= !!(st->fs[i] = xalloc(N)); ok &= !!(st->gs[i] = xalloc(N));
    }
    for (int k = 0; k < 5; ++k) {
        ok &= !!(st->hist[k] = xalloc(N)); ok &= !!(st->cur[k] = xalloc(N)); ok &= !!(st->dt[k] = xalloc(N));
    }
    double **arrs[] = {&st->phi_prev, &st->phi, &st->gpx, &st->gpy, &st->lap, &st->mu, &st->Dx, &st->Dy,
                       &st->lam, &st->nxv, &st->nyv, &st->rho, &st->ux, &st->uy, &st->p, &st->mcx,
                       &st->mcy, &st->Fx, &st->Fy, &st->s78};
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); ++k) ok &= !!(*arrs[k] = xalloc(N));
    ok &= !!(st->pad = xalloc(NP));
    ok &= !!(st->padmu = xalloc(NP));
    if (!ok) { oracle_destroy(st); return O_ENOMEM; }

    /* Eq. (3) and Eq. (10) */
    st->dphi = P->phiA - P->phiB;
    st->beta = 12.0 * P->sigma / (P->width * pow(st->dphi, 4));
    st->kappa = 1.5 * P->sigma * P->width / (st->dphi * st->dphi);
    /* sqrt(2 beta/k) of Eq. (8); equal to 4/(W dphi) (Sec. 4.3) for any sigma > 0,
     * and given that value when sigma = 0 switches surface tension off */
    st->lam_coef = P->sigma > 0.0 ? sqrt(2.0 * st->beta / st->kappa) : 4.0 / (P->width * st->dphi);
    st->drho_dphi = (P->rhoA - P->rhoB) / st->dphi;
    st->n_delta = (P->n_delta > 0.0 ? P->n_delta : 5e-3) * st->dphi / P->width;
    for (int k = 0; k < 9; ++k) { st->sf[k] = P->s_f[k]; st->sg[k] = P->s_g[k]; }
    /* App. C (first matrix): H = (s_g^2 - s_g^0)/(9 s_g^0 s_g^2), K = 1/(3c^2) */
    {
        const double s0 = isnan(P->s_g[0]) ? 1.0 : P->s_g[0];
        const double s2 = isnan(P->s_g[2]) ? 1.0 : P->s_g[2];
        st->Hc = (s2 - s0) / (9.0 * s0 * s2);
        st->Kc = 1.0 / 3.0;
    }
    for (int s = 0; s < 4; ++s) st->cos_t[s] = cos_deg(P->theta_deg[s]);
    *out = st;
    return O_OK;
}

/* Initial state (the paper does not state one; this is the reading used
 * throughout): f = f^eq(phi0, u0), g = g^eq(p0, u0) with m^{phi C} from phi0,
 * then the history is set to the values the scheme computes from those
 * populations at t = 0, so every time derivative of the first step is zero. */
int oracle_init_fields(ostate *st, const double *phi0, const double *ux0, const double *uy0, const double *p0)
{
    if (!st || !phi0) return O_EINVAL;
    const long N = st->N;
    const oracle_params *P = &st->P;
    /* phi, grad phi, mu and D of the initial field */
    memcpy(st->phi, phi0, sizeof(double) * N);
    phase_pass(st);
    for (long n = 0; n < N; ++n) {
        const double ph = st->phi[n];
        const double rho = st->drho_dphi * (ph - P->phiB) + P->rhoB;
        double mx = 0.0, my = 0.0;
        if (P->flux_model == O_PRESENT) {
            mx = -st->drho_dphi * P->mobility * st->Dx[n];
            my = -st->drho_dphi * P->mobility * st->Dy[n];
        }
        double in[20] = {0};
        in[0] = ph;
        in[1] = st->mu[n];
        in[2] = ux0 ? ux0[n] : 0.0;
        in[3] = uy0 ? uy0[n] : 0.0;
        in[4] = p0 ? p0[n] : 0.0;
        in[5] = rho;
        in[6] = mx;
        in[7] = my;
        double mfeq[9], mR[9], mgeq[9], mF[9];
        node_moments(P, in, mfeq, mR, mgeq, mF);
        const int solid = st->solid && st->solid[n];
        for (int i = 0; i < 9; ++i) {
            double sf = 0.0, sg = 0.0;
            for (int k = 0; k < 9; ++k) { sf += MINV[i][k] * mfeq[k]; sg += MINV[i][k] * mgeq[k]; }
            st->f[i][n] = solid ? 0.0 : sf;
            st->g[i][n] = solid ? 0.0 : sg;
        }
    }
    for (int k = 0; k < 5; ++k) memset(st->hist[k], 0, sizeof(double) * N);
    macro_pass(st);
    for (int k = 0; k < 5; ++k) memcpy(st->hist[k], st->cur[k], sizeof(double) * N);
    memcpy(st->phi_prev, st->phi, sizeof(double) * N);
    st->t = 0;
    memset(st->diag, 0, sizeof(st->diag));
    return O_OK;
}

int oracle_step(ostate *st, int64_t nsteps)
{
    if (!st || nsteps < 0) return O_EINVAL;
    set_threads();
    for (int64_t s = 0; s < nsteps; ++s) {
        macro_pass(st);
        memcpy(st->phi_prev, st->phi, sizeof(double) * st->N);
        for (int k = 0; k < 5; ++k) memcpy(st->hist[k], st->cur[k], sizeof(double) * st->N);
        collide(st);
        stream_pull(st, st->fs, st->f);
        stream_pull(st, st->gs, st->g);
        st->t += 1;
        if (st->P.diag_every > 0 && st->t % st->P.diag_every == 0) {
            macro_pass(st);
            diagnostics(st, st->diag);
            if (st->diag[5] > 0 || st->diag[4] > 0.4) {
                snprintf(st->err, sizeof(st->err), "unstable at t=%ld (non-finite %g, max|u| %g)",
                         st->t, st->diag[5], st->diag[4]);
                return O_EUNSTABLE;
            }
        }
    }
    return O_OK;
}

int oracle_fields(ostate *st, int32_t which, double *out)
{
    if (!st || !out) return O_EINVAL;
    const long N = st->N;
    set_threads();
    switch (which) {
    case O_FPOP:
        for (int i = 0; i < 9; ++i) memcpy(out + (size_t)i * N, st->f[i], sizeof(double) * N);
        return O_OK;
    case O_GPOP:
        for (int i = 0; i < 9; ++i) memcpy(out + (size_t)i * N, st->g[i], sizeof(double) * N);
        return O_OK;
    case O_HIST:
        for (int k = 0; k < 5; ++k) memcpy(out + (size_t)k * N, st->hist[k], sizeof(double) * N);
        return O_OK;
    case O_DIAG:
        macro_pass(st);
        diagnostics(st, st->diag);
        memcpy(out, st->diag, sizeof(st->diag));
        return O_OK;
    default:
        break;
    }
    macro_pass(st);
    const double *src = NULL;
    switch (which) {
    case O_PHI: src = st->phi; break;
    case O_UX: src = st->ux; break;
    case O_UY: src = st->uy; break;
    case O_P: src = st->p; break;
    case O_RHO: src = st->rho; break;
    case O_MU: src = st->mu; break;
    case O_MCX: src = st->mcx; break;
    case O_MCY: src = st->mcy; break;
    default:
        snprintf(st->err, sizeof(st->err), "unknown field %d", which);
        return O_EINVAL;
    }
    memcpy(out, src, sizeof(double) * N);
    return O_OK;
}

/* Resume from stored populations / history (post-stream populations at t). */
int oracle_set_fields(ostate *st, int32_t which, const double *in)
{
    if (!st || !in) return O_EINVAL;
    const long N = st->N;
    switch (which) {
    case O_FPOP:
        for (int i = 0; i < 9; ++i) memcpy(st->f[i], in + (size_t)i * N, sizeof(double) * N);
        return O_OK;
    case O_GPOP:
        for (int i = 0; i < 9; ++i) memcpy(st->g[i], in + (size_t)i * N, sizeof(double) * N);
        return O_OK;
    case O_HIST:
        for (int k = 0; k < 5; ++k) memcpy(st->hist[k], in + (size_t)k * N, sizeof(double) * N);
        return O_OK;
    default:
        snprintf(st->err, sizeof(st->err), "field %d cannot be set", which);
        return O_EINVAL;
    }
}

long oracle_time(const ostate *st) { return st ? st->t : -1; }

/* Mark solid nodes (mask [ny][nx], nonzero = solid; NULL removes them).
 * Takes effect from the next call; set it before oracle_init_fields so that
 * the initial state already holds no populations at solid nodes. */
int oracle_set_solid(ostate *st, const uint8_t *mask)
{
    if (!st) return O_EINVAL;
    if (!mask) {
        free(st->solid);
        st->solid = NULL;
        return O_OK;
    }
    if (!st->solid) st->solid = (unsigned char *)malloc((size_t)st->N);
    if (!st->solid) return O_ENOMEM;
    for (long n = 0; n < st->N; ++n) st->solid[n] = mask[n] ? 1 : 0;
    return O_OK;
}

/* ------------------------------------------------------------------ */
/* Test hooks (node-level pieces, so tests can pin them to the paper). */
/* ------------------------------------------------------------------ */
void oracle_moment_matrix(double *M, double *Minv)
{
    minv_init();
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            if (M) M[i * 9 + j] = MM[i][j];
            if (Minv) Minv[i * 9 + j] = MINV[i][j];
        }
}

void oracle_lattice(int *cx, int *cy, double *w)
{
    for (int i = 0; i < 9; ++i) { cx[i] = CX[i]; cy[i] = CY[i]; w[i] = WI[i]; }
}

/* out[0:9] m_f^eq, out[9:18] m_R, out[18:27] m_g^eq, out[27:36] m_F */
int oracle_node_moments(const oracle_params *P, const double *in, double *out)
{
    if (!P || !in || !out) return O_EINVAL;
    node_moments(P, in, out, out + 9, out + 18, out + 27);
    return O_OK;
}

/* Isotropic gradient and Laplacian of a periodic nx x ny field. */
int oracle_grad_lap(int nx, int ny, const double *field, double *gx, double *gy, double *lap)
{
    if (nx < 3 || ny < 3) return O_EINVAL;
    ostate tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.nx = nx;
    tmp.ny = ny;
    tmp.P.bc[0] = tmp.P.bc[1] = tmp.P.bc[2] = tmp.P.bc[3] = O_PERIODIC;
    double *pad = (double *)xalloc((size_t)(nx + 2) * (ny + 2));
    if (!pad) return O_ENOMEM;
    fill_pad(&tmp, field, pad, 0);
    stencil(&tmp, pad, gx, gy, lap);
    free(pad);
    return O_OK;
}

/* The padded field (nx+2) x (ny+2), x fastest, node (i, j) at (i+1, j+1),
 * as the stencils of the last macro pass saw it: which = 0 phi (wetting
 * ghosts), 1 mu_phi (mirror ghosts; Cahn-Hilliard only). */
int oracle_padded(ostate *st, int32_t which, double *out)
{
    if (!st || !out || which < 0 || which > 1) return O_EINVAL;
    if (which == 1 && st->P.phase_model != O_CH) return O_EINVAL;
    memcpy(out, which ? st->padmu : st->pad, sizeof(double) * (size_t)(st->nx + 2) * (st->ny + 2));
    return O_OK;
}

/* Wall order parameter and ghost value for given phi_1, phi_2, theta. */
double oracle_wall_phi(const oracle_params *P, double phi1, double phi2, double theta_deg, double *ghost)
{
    int flag = 0;
    const double c = cos_deg(theta_deg);
    if (ghost) *ghost = wall_ghost(P, phi1, phi2, c, &flag);
    return wall_phi(P, phi1, phi2, c, &flag);
}
