/*
 * lpic_oracle.c -- plain, slow FP64 CPU oracle for the explicit electromagnetic
 * particle-in-cell timestep (the "unified pusher" loop of the lambdaPIC paper).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or constant with the
 * CUDA library; the two meet only through the seeded input generators.
 *
 * Every routine follows one passage of the paper (section / equation /
 * algorithm named in its comment) in the paper's order, in double precision,
 * with modular (periodic) indexing and no guard cells.  Readings where the
 * paper is silent:
 *   - one shape order per run for gather AND deposit (1 = CIC, 2 = TSC);
 *   - each field component is gathered with the full shape in every dimension
 *     at its own staggered node positions;
 *   - the deposit of step n follows the straight path from x^{n+1/2} to
 *     x^{n+1/2} + dt v^{n+1} (centred on t_{n+1}, Sec. 3.1); both E
 *     half-updates that meet at t_{n+1} use that current: the second half of
 *     step n and the first half of step n+1 (J = 0 before the first step);
 *     the first half advances E then B, the second B then E;
 *   - 2D3V J_z uses v_z^{n+1};
 *   - classic Boris with gamma taken from u-minus;
 *   - normalised units c = eps0 = 1;
 *   - absorbing x edges: first-order Mur condition on the tangential E at the
 *     edge nodes, applied in each half-step with tau = dt/2, with an incoming
 *     Gaussian/sin^2 laser in E_y at x-min; particles whose deposit end point
 *     x^{n+1/2} + dt v^{n+1} lies outside [2 dx, (nx-2) dx) deposit their
 *     last step and are removed.
 *
 * Layout (shared with nothing, stated here for the Python wrapper): every
 * field array is [nz][ny][fx] row-major, fx = nx for periodic x and nx+1 for
 * absorbing x.  Index i of a component stands for its staggered position:
 *   Ex (i+1/2, j, k)  Ey (i, j+1/2, k)  Ez (i, j, k+1/2)
 *   Bx (i, j+1/2, k+1/2)  By (i+1/2, j, k+1/2)  Bz (i+1/2, j+1/2, k)
 * J is co-located with E.  In 2D, nz = 1 and the k offsets are dropped.
 *
 * Parity status: every function here is pinned by a CPU test against a closed
 * form or an independent derivation (shape moments, linear-field gather,
 * Boris rotation angle / radius / E x B drift, per-particle continuity,
 * sequential-sub-move and path-integral re-derivations of the Esirkepov
 * weights, Villasenor-Buneman limit, the discrete Yee dispersion relation,
 * Gauss-law constancy, cold Langmuir frequency, Mur reflection, translation
 * invariance); the CPML layers by a conducting-cavity mode at the discrete
 * frequency (lossless layers), wave-packet absorption, decay of oblique
 * waves and the laser sheet's amplitude and one-sidedness.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int dim;                 /* 2 or 3 */
    int nx, ny, nz;          /* cells; nz = 1 in 2D */
    int fx;                  /* stored x extent: nx (periodic) or nx+1 (absorbing) */
    double dx, dy, dz, dt;
    int order;               /* 1 = CIC, 2 = TSC */
    int absorb_x;            /* 0 periodic x, 1 absorbing x */
    int laser;               /* 1: incoming laser at x-min (needs absorb_x) */
    double a0, w0, tau, omega, yc, zc;
    double *E[3], *B[3], *J[3];
    /* CPML absorbing layers instead of the Mur edge condition (cpml = 1):
     * pml_cells cells at each x end, grading exponent pml_m, sigma_max,
     * kappa_max, alpha_max; psi[0..3] = memory variables of the x derivatives
     * in the E_y, E_z, B_y, B_z updates ([nz][ny][fx], zero outside the
     * layers); the laser then enters as a current sheet on node plane
     * laser_plane. */
    int cpml, pml_cells, laser_plane;
    double pml_m, pml_sigma_max, pml_kappa_max, pml_alpha_max;
    double *psi[4];
} orc_grid;

typedef struct {
    double q, m;
    long n;
    double *x[3];            /* physical positions; x[2] unused in 2D */
    double *u[3];            /* u = gamma v / c */
    double *w;               /* macro-particle weight (physical particles) */
    int *alive;
} orc_species;

enum { ORC_OK = 0, ORC_EOUTSIDE = 1, ORC_EARG = 2 };

/* ---------------------------------------------------------------- indexing */

static long wrap(long i, long n) { long r = i % n; return r < 0 ? r + n : r; }

/* Linear index of node (i, j, k); periodic dimensions wrap, an absorbing x
 * index must already lie in [0, fx). Returns -1 when it does not. */
static long node(const orc_grid *g, long i, long j, long k)
{
    if (g->absorb_x) {
        if (i < 0 || i >= g->fx) return -1;
    } else {
        i = wrap(i, g->nx);
    }
    j = wrap(j, g->ny);
    k = (g->dim == 3) ? wrap(k, g->nz) : 0;
    return (k * g->ny + j) * (long)g->fx + i;
}

static double h(const orc_grid *g, int d) { return d == 0 ? g->dx : (d == 1 ? g->dy : g->dz); }

/* ------------------------------------------------------------ shape (Sec. 3.1)
 * Particle shape of order 1 (cloud-in-cell, the bilinear/trilinear weighting
 * of Sec. 3.1) or order 2 (the quadratic spline named for the deposit in
 * Sec. 3.1), as a function of the distance to a node in cell units. */
double orc_shape(int order, double d)
{
    d = fabs(d);
    if (order == 1) return d < 1.0 ? 1.0 - d : 0.0;
    if (d <= 0.5) return 0.75 - d * d;
    if (d < 1.5) return 0.5 * (1.5 - d) * (1.5 - d);
    return 0.0;
}

/* ----------------------------------------------------------- gather (Sec. 3.1)
 * Field at a particle: each component is weighted from its own staggered
 * node positions with the shape in every dimension. */
static const double STAG_E[3][3] = {{0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5}};
static const double STAG_B[3][3] = {{0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};

static double gather_component(const orc_grid *g, const double *F, const double off[3],
                               const double pos[3], int *outside)
{
    double xi[3], acc = 0.0;
    long lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        if (d < g->dim) {
            xi[d] = pos[d] / h(g, d) - off[d];
            lo[d] = (long)floor(xi[d]) - 2;
            hi[d] = (long)floor(xi[d]) + 2;
        } else {
            xi[d] = 0.0; lo[d] = 0; hi[d] = 0;
        }
    }
    for (long k = lo[2]; k <= hi[2]; ++k) {
        double sz = (g->dim == 3) ? orc_shape(g->order, (double)k - xi[2]) : 1.0;
        if (sz == 0.0) continue;
        for (long j = lo[1]; j <= hi[1]; ++j) {
            double sy = orc_shape(g->order, (double)j - xi[1]);
            if (sy == 0.0) continue;
            for (long i = lo[0]; i <= hi[0]; ++i) {
                double sx = orc_shape(g->order, (double)i - xi[0]);
                if (sx == 0.0) continue;
                long n = node(g, i, j, k);
                if (n < 0) { *outside = 1; continue; }
                acc += F[n] * sx * sy * sz;
            }
        }
    }
    return acc;
}

int orc_gather(const orc_grid *g, const double pos[3], double Ep[3], double Bp[3])
{
    int outside = 0;
    for (int c = 0; c < 3; ++c) {
        Ep[c] = gather_component(g, g->E[c], STAG_E[c], pos, &outside);
        Bp[c] = gather_component(g, g->B[c], STAG_B[c], pos, &outside);
    }
    return outside ? ORC_EOUTSIDE : ORC_OK;
}

/* ------------------------------------------------------------ Boris (Sec. 3.1)
 * Relativistic Boris momentum update on u = gamma v (c = 1): half electric
 * kick, magnetic rotation, half electric kick. */
void orc_boris(double q, double m, double dt, double u[3], const double E[3], const double B[3])
{
    const double k = q * dt / (2.0 * m);
    double um[3], t[3], s[3], up[3], uq[3];
    for (int c = 0; c < 3; ++c) um[c] = u[c] + k * E[c];
    const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int c = 0; c < 3; ++c) t[c] = k * B[c] / gm;
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int c = 0; c < 3; ++c) s[c] = 2.0 * t[c] / (1.0 + t2);
    /* u' = u- + u- x t */
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    /* u+ = u- + u' x s */
    uq[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
    uq[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
    uq[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
    for (int c = 0; c < 3; ++c) u[c] = uq[c] + k * E[c];
}

/* -------------------------------------------------------- Esirkepov (Sec. 3.1)
 * Charge-conserving current of one macro-particle of charge qw moving in a
 * straight line from x0 to x1 during dt (Esirkepov 2001, cited in Sec. 3.1).
 * Per dimension S0/S1 are the shapes at the old/new positions on integer
 * nodes of a window covering both supports, DS = S1 - S0, and
 *   3D: W_x = DS_x (S0_y S0_z + DS_y S0_z / 2 + S0_y DS_z / 2 + DS_y DS_z / 3)
 *       (and cyclically), J_x(i+1/2) - J_x(i-1/2) = -qw W_x / (dt dy dz);
 *   2D: W_x = DS_x (S0_y + DS_y / 2), W_y = DS_y (S0_x + DS_x / 2),
 *       W_z = S0_x S0_y + DS_x S0_y / 2 + S0_x DS_y / 2 + DS_x DS_y / 3,
 *       J_x steps by -qw W_x / (dt dy), J_y by -qw W_y / (dt dx),
 *       J_z = qw vz W_z / (dx dy).
 * J is the running sum from zero at the low edge of the window. */
#define WIN 7
int orc_deposit(orc_grid *g, double qw, const double x0[3], const double x1[3], double vz)
{
    double S0[3][WIN], S1[3][WIN], DS[3][WIN];
    long base[3];
    int nd = g->dim;
    int bad = 0;
    for (int d = 0; d < 3; ++d) {
        for (int a = 0; a < WIN; ++a) { S0[d][a] = 1.0; S1[d][a] = 1.0; DS[d][a] = 0.0; }
        base[d] = 0;
        if (d >= nd) continue;
        double xi0 = x0[d] / h(g, d), xi1 = x1[d] / h(g, d);
        base[d] = (long)floor(xi0 < xi1 ? xi0 : xi1) - 2;
        for (int a = 0; a < WIN; ++a) {
            S0[d][a] = orc_shape(g->order, (double)(base[d] + a) - xi0);
            S1[d][a] = orc_shape(g->order, (double)(base[d] + a) - xi1);
            DS[d][a] = S1[d][a] - S0[d][a];
        }
        /* the window must hold both supports: its last node carries no weight */
        if (S0[d][WIN - 1] != 0.0 || S1[d][WIN - 1] != 0.0) bad = 1;
    }
    if (bad) return ORC_EARG;

    if (nd == 3) {
        const double cx = -qw / (g->dt * g->dy * g->dz);
        const double cy = -qw / (g->dt * g->dx * g->dz);
        const double cz = -qw / (g->dt * g->dx * g->dy);
        for (int b = 0; b < WIN; ++b)
            for (int c = 0; c < WIN; ++c) {
                double run = 0.0;
                for (int a = 0; a < WIN; ++a) {
                    double W = DS[0][a] * (S0[1][b] * S0[2][c] + 0.5 * DS[1][b] * S0[2][c]
                                           + 0.5 * S0[1][b] * DS[2][c] + DS[1][b] * DS[2][c] / 3.0);
                    run += cx * W;
                    if (run != 0.0) {
                        long n = node(g, base[0] + a, base[1] + b, base[2] + c);
                        if (n < 0) return ORC_EOUTSIDE;
                        g->J[0][n] += run;
                    }
                }
            }
        for (int a = 0; a < WIN; ++a)
            for (int c = 0; c < WIN; ++c) {
                double run = 0.0;
                for (int b = 0; b < WIN; ++b) {
                    double W = DS[1][b] * (S0[0][a] * S0[2][c] + 0.5 * DS[0][a] * S0[2][c]
                                           + 0.5 * S0[0][a] * DS[2][c] + DS[0][a] * DS[2][c] / 3.0);
                    run += cy * W;
                    if (run != 0.0) {
                        long n = node(g, base[0] + a, base[1] + b, base[2] + c);
                        if (n < 0) return ORC_EOUTSIDE;
                        g->J[1][n] += run;
                    }
                }
            }
        for (int a = 0; a < WIN; ++a)
            for (int b = 0; b < WIN; ++b) {
                double run = 0.0;
                for (int c = 0; c < WIN; ++c) {
                    double W = DS[2][c] * (S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b]
                                           + 0.5 * S0[0][a] * DS[1][b] + DS[0][a] * DS[1][b] / 3.0);
                    run += cz * W;
                    if (run != 0.0) {
                        long n = node(g, base[0] + a, base[1] + b, base[2] + c);
                        if (n < 0) return ORC_EOUTSIDE;
                        g->J[2][n] += run;
                    }
                }
            }
        return ORC_OK;
    }

    /* 2D3V */
    const double cx = -qw / (g->dt * g->dy);
    const double cy = -qw / (g->dt * g->dx);
    const double cz = qw * vz / (g->dx * g->dy);
    for (int b = 0; b < WIN; ++b) {
        double run = 0.0;
        for (int a = 0; a < WIN; ++a) {
            run += cx * DS[0][a] * (S0[1][b] + 0.5 * DS[1][b]);
            if (run != 0.0) {
                long n = node(g, base[0] + a, base[1] + b, 0);
                if (n < 0) return ORC_EOUTSIDE;
                g->J[0][n] += run;
            }
        }
    }
    for (int a = 0; a < WIN; ++a) {
        double run = 0.0;
        for (int b = 0; b < WIN; ++b) {
            run += cy * DS[1][b] * (S0[0][a] + 0.5 * DS[0][a]);
            if (run != 0.0) {
                long n = node(g, base[0] + a, base[1] + b, 0);
                if (n < 0) return ORC_EOUTSIDE;
                g->J[1][n] += run;
            }
        }
    }
    for (int a = 0; a < WIN; ++a)
        for (int b = 0; b < WIN; ++b) {
            double W = S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b]
                     + 0.5 * S0[0][a] * DS[1][b] + DS[0][a] * DS[1][b] / 3.0;
            if (W != 0.0) {
                long n = node(g, base[0] + a, base[1] + b, 0);
                if (n < 0) return ORC_EOUTSIDE;
                g->J[2][n] += cz * W;
            }
        }
    return ORC_OK;
}

/* Charge density of one species on the integer nodes: rho = q w S S S / dV
 * (the charge that the Esirkepov current conserves, Sec. 3.1). Accumulates. */
int orc_rho(const orc_grid *g, const orc_species *sp, double *rho)
{
    const double dV = g->dx * g->dy * (g->dim == 3 ? g->dz : 1.0);
    for (long p = 0; p < sp->n; ++p) {
        if (!sp->alive[p]) continue;
        double xi[3] = {0, 0, 0};
        long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int d = 0; d < g->dim; ++d) {
            xi[d] = sp->x[d][p] / h(g, d);
            lo[d] = (long)floor(xi[d]) - 2;
            hi[d] = (long)floor(xi[d]) + 2;
        }
        for (long k = lo[2]; k <= hi[2]; ++k) {
            double sz = (g->dim == 3) ? orc_shape(g->order, (double)k - xi[2]) : 1.0;
            for (long j = lo[1]; j <= hi[1]; ++j) {
                double sy = orc_shape(g->order, (double)j - xi[1]);
                for (long i = lo[0]; i <= hi[0]; ++i) {
                    double s = orc_shape(g->order, (double)i - xi[0]) * sy * sz;
                    if (s == 0.0) continue;
                    long n = node(g, i, j, k);
                    if (n < 0) return ORC_EOUTSIDE;
                    rho[n] += sp->q * sp->w[p] * s / dV;
                }
            }
        }
    }
    return ORC_OK;
}

/* ---------------------------------------------------- Yee curls (Sec. 3.2, Eq. 1-4)
 * Standard first differences on the staggered grid.  curl B is evaluated at
 * the E positions, curl E at the B positions.  Returns 0 where a neighbour
 * would fall outside an absorbing x edge (those nodes are set by the edge
 * condition instead). */
static int curlB(const orc_grid *g, int c, long i, long j, long k, double *out)
{
    const int d3 = (g->dim == 3);
    long n = node(g, i, j, k);
    double v = 0.0;
    if (c == 0) {                       /* at (i+1/2, j, k) */
        v = (g->B[2][n] - g->B[2][node(g, i, j - 1, k)]) / g->dy;
        if (d3) v -= (g->B[1][n] - g->B[1][node(g, i, j, k - 1)]) / g->dz;
    } else if (c == 1) {                /* at (i, j+1/2, k) */
        long m = node(g, i - 1, j, k);
        if (m < 0) return 0;
        v = -(g->B[2][n] - g->B[2][m]) / g->dx;
        if (d3) v += (g->B[0][n] - g->B[0][node(g, i, j, k - 1)]) / g->dz;
    } else {                            /* at (i, j, k+1/2) */
        long m = node(g, i - 1, j, k);
        if (m < 0) return 0;
        v = (g->B[1][n] - g->B[1][m]) / g->dx - (g->B[0][n] - g->B[0][node(g, i, j - 1, k)]) / g->dy;
    }
    *out = v;
    return 1;
}

static int curlE(const orc_grid *g, int c, long i, long j, long k, double *out)
{
    const int d3 = (g->dim == 3);
    long n = node(g, i, j, k);
    double v = 0.0;
    if (c == 0) {                       /* at (i, j+1/2, k+1/2) */
        v = (g->E[2][node(g, i, j + 1, k)] - g->E[2][n]) / g->dy;
        if (d3) v -= (g->E[1][node(g, i, j, k + 1)] - g->E[1][n]) / g->dz;
    } else if (c == 1) {                /* at (i+1/2, j, k+1/2) */
        long m = node(g, i + 1, j, k);
        if (m < 0) return 0;
        v = -(g->E[2][m] - g->E[2][n]) / g->dx;
        if (d3) v += (g->E[0][node(g, i, j, k + 1)] - g->E[0][n]) / g->dz;
    } else {                            /* at (i+1/2, j+1/2, k) */
        long m = node(g, i + 1, j, k);
        if (m < 0) return 0;
        v = (g->E[1][m] - g->E[1][n]) / g->dx - (g->E[0][node(g, i, j + 1, k)] - g->E[0][n]) / g->dy;
    }
    *out = v;
    return 1;
}

/* Is index i of component c a real (stored, used) x position?  With absorbing
 * x the half-integer components (E_x, B_y, B_z, J_x) have nx entries and the
 * integer ones nx+1. */
static int half_x_E(int c) { return c == 0; }
static int half_x_B(int c) { return c != 0; }

/* Incoming laser, E_y polarised, travelling in +x from the x-min edge
 * (Sec. 4.2 describes a Gaussian spot with a sin^2 temporal envelope): */
double orc_laser_ey(const orc_grid *g, double x, double y, double z, double t)
{
    double s = t - x;                               /* retarded time, c = 1 */
    if (s <= 0.0 || s >= g->tau) return 0.0;
    double env = sin(M_PI * s / g->tau);
    env *= env;
    double r2 = (y - g->yc) * (y - g->yc);
    if (g->dim == 3) r2 += (z - g->zc) * (z - g->zc);
    return g->a0 * env * exp(-r2 / (g->w0 * g->w0)) * sin(g->omega * s);
}

/* ------------------------------------------------ CPML (Sec. 3.2 boundaries)
 * Convolutional PML on the x ends (Roden & Gedney's recursive convolution of
 * the stretched-coordinate PML of Berenger): inside a layer of L cells the x
 * derivative d/dx of a field update becomes (1/kappa) d/dx + psi, with the
 * memory variable psi <- b psi + a d/dx updated before the field, and
 * b = exp(-(sigma/kappa + alpha) tau), a = sigma (b - 1) / (sigma kappa +
 * kappa^2 alpha) for the update's time step tau (each half step here).  The
 * profiles over the depth d in [0, 1] into the layer (d = 0 at the inner
 * face): sigma = sigma_max d^m, kappa = 1 + (kappa_max - 1) d^m,
 * alpha = alpha_max (1 - d).  The outer faces x = 0 and x = nx dx are perfect
 * conductors (tangential E = 0). */
static double pml_depth(const orc_grid *g, double xc)   /* xc: position in cells */
{
    const double L = g->pml_cells;
    if (xc < L) return (L - xc) / L;
    if (xc > g->nx - L) return (xc - (g->nx - L)) / L;
    return 0.0;
}

static void pml_coef(const orc_grid *g, double xc, double tau, double *kinv, double *a, double *b)
{
    const double d = pml_depth(g, xc);
    const double dm = pow(d, g->pml_m);
    const double sigma = g->pml_sigma_max * dm;
    const double kappa = 1.0 + (g->pml_kappa_max - 1.0) * dm;
    const double alpha = d > 0.0 ? g->pml_alpha_max * (1.0 - d) : 0.0;
    *kinv = 1.0 / kappa;
    *b = exp(-(sigma / kappa + alpha) * tau);
    *a = sigma > 0.0 ? sigma * (*b - 1.0) / (sigma * kappa + kappa * kappa * alpha) : 0.0;
}

/* The CPML E half step: E_x as in the interior; E_y, E_z on nodes 1..nx-1
 * with the modified x derivative; nodes 0 and nx stay zero.  The laser sheet:
 * a surface current K_y = -2 E_inc(t) on node plane laser_plane radiates
 * E_y = E_inc into +x (and the same into -x, which the layer absorbs); it
 * enters the update as the volume current K_y / dx at the half step's centre
 * time. */
static void advance_E_cpml(orc_grid *g, double tau, double t_old)
{
    const long ny = g->ny, nz = (g->dim == 3) ? g->nz : 1, fx = g->fx, nx = g->nx;
    const long plane = ny * nz;
    const int d3 = g->dim == 3;
    for (int c = 0; c < 3; ++c) {
        double *newE = (double *)malloc(sizeof(double) * fx * plane);
        memcpy(newE, g->E[c], sizeof(double) * fx * plane);
        for (long k = 0; k < nz; ++k)
            for (long j = 0; j < ny; ++j)
                for (long i = 0; i < fx; ++i) {
                    if (half_x_E(c) && i == nx) continue;
                    if (!half_x_E(c) && (i == 0 || i == nx)) continue;
                    const long n = node(g, i, j, k);
                    double cb;
                    if (c == 0) {
                        if (!curlB(g, c, i, j, k, &cb)) continue;
                    } else {
                        double kinv, a, b;
                        pml_coef(g, (double)i, tau, &kinv, &a, &b);
                        if (c == 1) {   /* E_y: -dBz/dx + dBx/dz */
                            const double dbz = (g->B[2][n] - g->B[2][node(g, i - 1, j, k)]) / g->dx;
                            g->psi[0][n] = b * g->psi[0][n] + a * dbz;
                            cb = -(kinv * dbz + g->psi[0][n]);
                            if (d3) cb += (g->B[0][n] - g->B[0][node(g, i, j, k - 1)]) / g->dz;
                        } else {        /* E_z: dBy/dx - dBx/dy */
                            const double dby = (g->B[1][n] - g->B[1][node(g, i - 1, j, k)]) / g->dx;
                            g->psi[1][n] = b * g->psi[1][n] + a * dby;
                            cb = kinv * dby + g->psi[1][n]
                               - (g->B[0][n] - g->B[0][node(g, i, j - 1, k)]) / g->dy;
                        }
                    }
                    double jc = g->J[c][n];
                    if (c == 1 && g->laser && i == g->laser_plane) {
                        const double y = (j + 0.5) * g->dy, z = k * g->dz;
                        jc += -2.0 * orc_laser_ey(g, 0.0, y, z, t_old + 0.5 * tau) / g->dx;
                    }
                    newE[n] = g->E[c][n] + tau * (cb - jc);
                }
        memcpy(g->E[c], newE, sizeof(double) * fx * plane);
        free(newE);
    }
}

/* The CPML B half step: B_x as in the interior; B_y, B_z at i + 1/2 for
 * i = 0..nx-1 with the modified x derivative. */
static void advance_B_cpml(orc_grid *g, double tau)
{
    const long ny = g->ny, nz = (g->dim == 3) ? g->nz : 1, fx = g->fx, nx = g->nx;
    const long plane = ny * nz;
    const int d3 = g->dim == 3;
    for (int c = 0; c < 3; ++c) {
        double *newB = (double *)malloc(sizeof(double) * fx * plane);
        memcpy(newB, g->B[c], sizeof(double) * fx * plane);
        for (long k = 0; k < nz; ++k)
            for (long j = 0; j < ny; ++j)
                for (long i = 0; i < fx; ++i) {
                    if (half_x_B(c) && i == nx) continue;
                    const long n = node(g, i, j, k);
                    double ce;
                    if (c == 0) {
                        if (!curlE(g, c, i, j, k, &ce)) continue;
                    } else {
                        double kinv, a, b;
                        pml_coef(g, i + 0.5, tau, &kinv, &a, &b);
                        if (c == 1) {   /* B_y: dEx/dz - dEz/dx */
                            const double dez = (g->E[2][node(g, i + 1, j, k)] - g->E[2][n]) / g->dx;
                            g->psi[2][n] = b * g->psi[2][n] + a * dez;
                            ce = -(kinv * dez + g->psi[2][n]);
                            if (d3) ce += (g->E[0][node(g, i, j, k + 1)] - g->E[0][n]) / g->dz;
                        } else {        /* B_z: dEy/dx - dEx/dy */
                            const double dey = (g->E[1][node(g, i + 1, j, k)] - g->E[1][n]) / g->dx;
                            g->psi[3][n] = b * g->psi[3][n] + a * dey;
                            ce = kinv * dey + g->psi[3][n]
                               - (g->E[0][node(g, i, j + 1, k)] - g->E[0][n]) / g->dy;
                        }
                    }
                    newB[n] = g->B[c][n] - tau * ce;
                }
        memcpy(g->B[c], newB, sizeof(double) * fx * plane);
        free(newB);
    }
}

/* E += tau (curl B - J) at every E position; absorbing x edges of E_y and
 * E_z then follow the first-order Mur condition for an outgoing wave (with
 * the incoming laser added at x-min), or, with CPML, the x derivatives in the
 * layers are replaced as above, the outer faces stay at zero and the laser is
 * a current sheet.  tau = dt/2, t_old -> t_old + tau. */
static void advance_E(orc_grid *g, double tau, double t_old)
{
    if (g->absorb_x && g->cpml) {
        advance_E_cpml(g, tau, t_old);
        return;
    }
    const long ny = g->ny, nz = (g->dim == 3) ? g->nz : 1, fx = g->fx, nx = g->nx;
    const long plane = ny * nz;
    double *old = NULL;
    if (g->absorb_x) {
        /* old values of E_y, E_z on planes i = 0, 1, nx-1, nx */
        old = (double *)malloc(sizeof(double) * 2 * 4 * plane);
        for (int c = 1; c < 3; ++c)
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j) {
                    long q = k * ny + j;
                    double *o = old + ((c - 1) * 4) * plane;
                    o[0 * plane + q] = g->E[c][node(g, 0, j, k)];
                    o[1 * plane + q] = g->E[c][node(g, 1, j, k)];
                    o[2 * plane + q] = g->E[c][node(g, nx - 1, j, k)];
                    o[3 * plane + q] = g->E[c][node(g, nx, j, k)];
                }
    }
    /* curl B from B that this update does not change: compute into a copy */
    for (int c = 0; c < 3; ++c) {
        double *newE = (double *)malloc(sizeof(double) * fx * plane);
        memcpy(newE, g->E[c], sizeof(double) * fx * plane);
        for (long k = 0; k < nz; ++k)
            for (long j = 0; j < ny; ++j)
                for (long i = 0; i < fx; ++i) {
                    if (g->absorb_x) {
                        if (half_x_E(c) && i == nx) continue;
                        if (!half_x_E(c) && (i == 0 || i == nx)) continue;
                    }
                    double cb;
                    if (!curlB(g, c, i, j, k, &cb)) continue;
                    long n = node(g, i, j, k);
                    newE[n] = g->E[c][n] + tau * (cb - g->J[c][n]);
                }
        memcpy(g->E[c], newE, sizeof(double) * fx * plane);
        free(newE);
    }
    if (g->absorb_x) {
        const double c1 = (tau - g->dx) / (tau + g->dx);
        const double t_new = t_old + tau;
        for (int c = 1; c < 3; ++c) {
            const double *o = old + ((c - 1) * 4) * plane;
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j) {
                    long q = k * ny + j;
                    double inc0o = 0, inc1o = 0, inc0n = 0, inc1n = 0;
                    if (g->laser && c == 1) {
                        double y = (j + 0.5) * g->dy, z = k * g->dz;
                        inc0o = orc_laser_ey(g, 0.0, y, z, t_old);
                        inc1o = orc_laser_ey(g, g->dx, y, z, t_old);
                        inc0n = orc_laser_ey(g, 0.0, y, z, t_new);
                        inc1n = orc_laser_ey(g, g->dx, y, z, t_new);
                    }
                    double e1n = g->E[c][node(g, 1, j, k)];
                    g->E[c][node(g, 0, j, k)] = inc0n + (o[1 * plane + q] - inc1o)
                        + c1 * ((e1n - inc1n) - (o[0 * plane + q] - inc0o));
                    double eMn = g->E[c][node(g, nx - 1, j, k)];
                    g->E[c][node(g, nx, j, k)] = o[2 * plane + q] + c1 * (eMn - o[3 * plane + q]);
                }
        }
        free(old);
    }
}

/* B -= tau curl E at every B position (with CPML: the x derivatives of E_z and
 * E_y in the B_y and B_z updates replaced inside the layers). */
static void advance_B(orc_grid *g, double tau)
{
    if (g->absorb_x && g->cpml) {
        advance_B_cpml(g, tau);
        return;
    }
    const long ny = g->ny, nz = (g->dim == 3) ? g->nz : 1, fx = g->fx, nx = g->nx;
    const long plane = ny * nz;
    for (int c = 0; c < 3; ++c) {
        double *newB = (double *)malloc(sizeof(double) * fx * plane);
        memcpy(newB, g->B[c], sizeof(double) * fx * plane);
        for (long k = 0; k < nz; ++k)
            for (long j = 0; j < ny; ++j)
                for (long i = 0; i < fx; ++i) {
                    if (g->absorb_x && half_x_B(c) && i == nx) continue;
                    double ce;
                    if (!curlE(g, c, i, j, k, &ce)) continue;
                    long n = node(g, i, j, k);
                    newB[n] = g->B[c][n] - tau * ce;
                }
        memcpy(g->B[c], newB, sizeof(double) * fx * plane);
        free(newB);
    }
}

/* Maxwell half-step (Sec. 3.2 Eq. 3-4 split in two halves as in Algorithm 1):
 * which = 0: advance E then B from t to t + dt/2;
 * which = 1: advance B then E from t to t + dt/2. */
void orc_maxwell_half(orc_grid *g, int which, double t)
{
    const double tau = 0.5 * g->dt;
    if (which == 0) { advance_E(g, tau, t); advance_B(g, tau); }
    else            { advance_B(g, tau); advance_E(g, tau, t); }
}

/* ---------------------------------------------- particle loop (Algorithm 1)
 * One species: half position push x^n -> x^{n+1/2}, gather at x^{n+1/2},
 * Boris u^n -> u^{n+1}, half position push x^{n+1/2} -> x^{n+1}, and the
 * Esirkepov deposit into g->J (zeroed by the caller before the species loop).
 * Sec. 3.1 has the deposit trace the trajectory over one step centred on the
 * time at which the current is used; with the split field update of
 * Algorithm 1 that is t_{n+1}, so the path is the straight line from
 * x^{n+1/2} to x^{n+1/2} + dt v^{n+1} (whose end point is where the next
 * step's first half push will put the particle).  2D3V J_z uses v_z^{n+1}.
 * Periodic coordinates of x^{n+1} are wrapped; with absorbing x a particle
 * whose deposit end point leaves [2 dx, (nx-2) dx) is removed after its
 * deposit. */
/* Nonlinear Compton emission inside the particle loop (Algorithm 1 places
 * the QED events between the field interpolation and the momentum push), for
 * orc_push_species_qed below. */
typedef struct {
    double eps_ref;
    uint32_t seed_lo, seed_hi;
    long step;
    double *tau;     /* optical depth per particle index */
    double *ph;      /* photons [8][cap]: x0, x1, x2, u0, u1, u2, w, emitter index */
    long cap, *nph;
} orc_qed_push;

static int push_species_impl(orc_grid *g, orc_species *sp, const orc_qed_push *q);
static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
static double u01(uint32_t x);
double orc_chi_e(const double u[3], const double E[3], const double B[3], double eps_ref);
double orc_compton_rate(double chi, double gamma, double eps_ref);
double orc_compton_xi(double chi, double r);

int orc_push_species(orc_grid *g, orc_species *sp)
{
    return push_species_impl(g, sp, NULL);
}

/* The particle loop of Algorithm 1 with nonlinear Compton emission (Sec. 3.4)
 * between "interpolate E, B" and "push momenta": after the gather at
 * x^{n+1/2}, chi is formed from u^n and those fields, tau[p] decreases by
 * W(chi, gamma^n) dt, and when it reaches zero a photon of energy fraction
 * xi = F^-1(r1) (counter (p, step, 0, 0), word 0) is emitted along u^n with
 * the particle's weight, the particle recoils (u^n -> u^n (1 - k/|u^n|), k =
 * xi gamma^n) and tau restarts at -ln r2 (word 1); the Boris push, the move
 * and the deposit then use the recoiled momentum.  The photon leaves from
 * x^{n+1/2} at the speed of light: it is stored at its position at t_{n+1},
 * x^{n+1/2} + (dt/2) khat (periodic coordinates wrapped), with the emitter's
 * index in row 7.  More photons than cap: ORC_EARG. */
int orc_push_species_qed(orc_grid *g, orc_species *sp, double eps_ref, uint32_t seed_lo, uint32_t seed_hi,
                         long step, double *tau, double *ph, long cap, long *nph)
{
    if (sp->m == 0.0) return ORC_EARG;
    const orc_qed_push q = {eps_ref, seed_lo, seed_hi, step, tau, ph, cap, nph};
    return push_species_impl(g, sp, &q);
}

static int push_species_impl(orc_grid *g, orc_species *sp, const orc_qed_push *q)
{
    const double dt = g->dt;
    const double L[3] = {g->nx * g->dx, g->ny * g->dy, g->nz * g->dz};
    for (long p = 0; p < sp->n; ++p) {
        if (!sp->alive[p]) continue;
        double xm[3] = {0, 0, 0}, x1[3] = {0, 0, 0}, xe[3] = {0, 0, 0}, u[3], E[3], B[3];
        for (int c = 0; c < 3; ++c) u[c] = sp->u[c][p];
        /* a massless species (photons, m = 0, q = 0) moves at c along u */
        const int massless = sp->m == 0.0;
        const double uu0 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double g0 = massless ? sqrt(uu0) : sqrt(1.0 + uu0);
        for (int d = 0; d < g->dim; ++d) xm[d] = sp->x[d][p] + (g0 > 0 ? 0.5 * dt * u[d] / g0 : 0.0);
        if (orc_gather(g, xm, E, B) != ORC_OK) return ORC_EOUTSIDE;
        if (q) {
            const double chi = orc_chi_e(u, E, B, q->eps_ref);
            if (chi > 0.0) {
                q->tau[p] -= orc_compton_rate(chi, g0, q->eps_ref) * dt;
                if (q->tau[p] <= 0.0) {
                    if (*q->nph >= q->cap) return ORC_EARG;
                    const uint32_t ctr[4] = {(uint32_t)p, (uint32_t)q->step, 0u, 0u};
                    const uint32_t key[2] = {q->seed_lo, q->seed_hi};
                    uint32_t o[4];
                    philox4x32_10(ctr, key, o);
                    const double xi = orc_compton_xi(chi, u01(o[0]));
                    const double umag = sqrt(uu0);
                    const double k = xi * g0;
                    const long j = *q->nph;
                    for (int d = 0; d < 3; ++d) {
                        double xp = 0.0;
                        if (d < g->dim) {
                            xp = xm[d] + 0.5 * dt * u[d] / umag;
                            if (!(d == 0 && g->absorb_x)) {
                                if (xp >= L[d]) xp -= L[d];
                                else if (xp < 0.0) xp += L[d];
                            }
                        }
                        q->ph[d * q->cap + j] = xp;
                    }
                    for (int c = 0; c < 3; ++c) q->ph[(3 + c) * q->cap + j] = k * u[c] / umag;
                    q->ph[6 * q->cap + j] = sp->w[p];
                    q->ph[7 * q->cap + j] = (double)p;
                    *q->nph = j + 1;
                    for (int c = 0; c < 3; ++c) u[c] *= 1.0 - k / umag;
                    q->tau[p] = -log(u01(o[1]));
                }
            }
        }
        if (!massless) orc_boris(sp->q, sp->m, dt, u, E, B);
        const double uu1 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double g1 = massless ? (uu1 > 0 ? sqrt(uu1) : 1.0) : sqrt(1.0 + uu1);
        for (int d = 0; d < g->dim; ++d) {
            x1[d] = xm[d] + 0.5 * dt * u[d] / g1;
            xe[d] = xm[d] + dt * u[d] / g1;
        }
        int rc = orc_deposit(g, sp->q * sp->w[p], xm, xe, u[2] / g1);
        if (rc != ORC_OK) return rc;
        for (int d = 0; d < g->dim; ++d) {
            if (d == 0 && g->absorb_x) continue;
            if (x1[d] >= L[d]) x1[d] -= L[d];
            else if (x1[d] < 0.0) x1[d] += L[d];
        }
        if (g->absorb_x && (xe[0] < 2.0 * g->dx || xe[0] >= (g->nx - 2) * g->dx)) sp->alive[p] = 0;
        for (int d = 0; d < g->dim; ++d) sp->x[d][p] = x1[d];
        for (int c = 0; c < 3; ++c) sp->u[c][p] = u[c];
    }
    return ORC_OK;
}

static void zero_J(orc_grid *g)
{
    long cnt = (long)g->fx * g->ny * (g->dim == 3 ? g->nz : 1);
    for (int c = 0; c < 3; ++c) memset(g->J[c], 0, sizeof(double) * cnt);
}

/* One full timestep t -> t + dt (Algorithm 1 without QED, load balancing or
 * MPI): first Maxwell half with the current J, J zeroed, all species pushed
 * and deposited, second Maxwell half with the new J.  J is left holding this
 * step's deposit for the next step's first half. */
int orc_step(orc_grid *g, orc_species *sp, int nsp, double t)
{
    orc_maxwell_half(g, 0, t);
    zero_J(g);
    for (int s = 0; s < nsp; ++s) {
        int rc = orc_push_species(g, &sp[s]);
        if (rc != ORC_OK) return rc;
    }
    orc_maxwell_half(g, 1, t + 0.5 * g->dt);
    return ORC_OK;
}

/* ---------------------------------------------------- diagnostics (Sec. 4.1)
 * out[0] = kinetic energy sum w m (gamma - 1); out[1] = field energy
 * (1/2) sum (E^2 + B^2) dV over the stored positions; out[2] = total charge. */
void orc_energy(const orc_grid *g, const orc_species *sp, int nsp, double out[3])
{
    const double dV = g->dx * g->dy * (g->dim == 3 ? g->dz : 1.0);
    long cnt = (long)g->fx * g->ny * (g->dim == 3 ? g->nz : 1);
    double ek = 0.0, ef = 0.0, qt = 0.0;
    for (int s = 0; s < nsp; ++s)
        for (long p = 0; p < sp[s].n; ++p) {
            if (!sp[s].alive[p]) continue;
            double u2 = sp[s].u[0][p] * sp[s].u[0][p] + sp[s].u[1][p] * sp[s].u[1][p]
                      + sp[s].u[2][p] * sp[s].u[2][p];
            /* photons (m = 0) carry energy |u| m_e c^2 */
            ek += sp[s].m == 0.0 ? sp[s].w[p] * sqrt(u2) : sp[s].w[p] * sp[s].m * (sqrt(1.0 + u2) - 1.0);
            qt += sp[s].w[p] * sp[s].q;
        }
    for (int c = 0; c < 3; ++c)
        for (long n = 0; n < cnt; ++n)
            ef += 0.5 * (g->E[c][n] * g->E[c][n] + g->B[c][n] * g->B[c][n]) * dV;
    out[0] = ek; out[1] = ef; out[2] = qt;
}

/* Discrete divergence of E on the integer nodes (periodic grids only):
 * sum_d (E_d(i+1/2) - E_d(i-1/2)) / h_d. */
void orc_div_e(const orc_grid *g, double *out)
{
    const long ny = g->ny, nz = (g->dim == 3) ? g->nz : 1, nx = g->nx;
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long n = node(g, i, j, k);
                double v = (g->E[0][n] - g->E[0][node(g, i - 1, j, k)]) / g->dx
                         + (g->E[1][n] - g->E[1][node(g, i, j - 1, k)]) / g->dy;
                if (g->dim == 3) v += (g->E[2][n] - g->E[2][node(g, i, j, k - 1)]) / g->dz;
                out[n] = v;
            }
}

/* --------------------------------------------- QED: nonlinear Compton (Sec. 3.4)
 * Photon emission by electrons (and positrons) in the locally-constant-field
 * approximation, event-based Monte Carlo with an optical depth per particle
 * (Sec. 3.4 and its references).  Normalised units: eps_ref = hbar omega_ref /
 * (m c^2) for the unit frequency omega_ref; fields in m c omega_ref / e.
 *
 * chi_e = eps_ref gamma sqrt((E + beta x B)^2 - (beta . E)^2).
 * Emission spectrum per unit time and photon energy fraction xi:
 *   d2W / dt dxi = alpha / (eps_ref sqrt(3) pi gamma) S(xi, chi),
 *   S = (1 - xi + 1 / (1 - xi)) K_{2/3}(delta) - int_delta^inf K_{1/3}(s) ds,
 *   delta = 2 xi / (3 chi (1 - xi)),
 * with the modified Bessel functions from their integral representation
 * K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (and int_x^inf K_nu =
 * int_0^inf exp(-x cosh t) cosh(nu t) / cosh t dt), evaluated by the
 * trapezoid rule (the integrands decay double-exponentially).
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), counter (id, step,
 * kind, 0), key (seed_lo, seed_hi). */

static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0; c1 = lo1; c2 = hi0 ^ c3 ^ k1; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { philox4x32_10(ctr, key, out); }

/* uniform in (0, 1) from 32 random bits */
static double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

static double bessel_k_int(double nu, double x, int integrated)
{
    if (x <= 0.0) return INFINITY;
    const double h = 0.01;
    double tmax = acosh(fmax(1.0, 60.0 / x)) + 1.0;
    double sum = 0.5 * exp(-x) * (integrated ? 1.0 : 1.0);
    for (double t = h; t <= tmax; t += h) {
        const double ch = cosh(t);
        double v = exp(-x * ch) * cosh(nu * t);
        if (integrated) v /= ch;
        sum += v;
    }
    return sum * h;
}

double orc_bessel_k(double nu, double x) { return bessel_k_int(nu, x, 0); }
double orc_bessel_k_int(double nu, double x) { return bessel_k_int(nu, x, 1); }

double orc_compton_s(double xi, double chi)
{
    if (xi <= 0.0 || xi >= 1.0) return 0.0;
    const double delta = 2.0 * xi / (3.0 * chi * (1.0 - xi));
    if (delta > 700.0) return 0.0;
    return (1.0 - xi + 1.0 / (1.0 - xi)) * bessel_k_int(2.0 / 3.0, delta, 0) - bessel_k_int(1.0 / 3.0, delta, 1);
}

/* cumulative int_0^xi S dxi' on xi = y^3, y in [0, 1] (n intervals); cum[n] = total */
static void compton_cumulative(double chi, int n, double *cum)
{
    cum[0] = 0.0;
    double prev = 0.0;              /* S(y^3) 3 y^2 -> finite limit at y = 0 */
    {
        const double y = 1e-4;
        prev = orc_compton_s(y * y * y, chi) * 3.0 * y * y;
    }
    for (int k = 1; k <= n; ++k) {
        const double y = (double)k / n;
        const double f = (k == n) ? 0.0 : orc_compton_s(y * y * y, chi) * 3.0 * y * y;
        cum[k] = cum[k - 1] + 0.5 * (prev + f) / n;
        prev = f;
    }
}

/* total emission rate per unit time (units of omega_ref) */
double orc_compton_rate(double chi, double gamma, double eps_ref)
{
    const int n = 2000;
    double *cum = (double *)malloc(sizeof(double) * (n + 1));
    compton_cumulative(chi, n, cum);
    const double F = cum[n];
    free(cum);
    const double alpha = 1.0 / 137.035999084;
    return alpha / (eps_ref * sqrt(3.0) * M_PI * gamma) * F;
}

/* photon energy fraction with cumulative probability r */
double orc_compton_xi(double chi, double r)
{
    const int n = 2000;
    double *cum = (double *)malloc(sizeof(double) * (n + 1));
    compton_cumulative(chi, n, cum);
    const double target = r * cum[n];
    int k = 0;
    while (k < n && cum[k + 1] < target) ++k;
    const double f = (cum[k + 1] > cum[k]) ? (target - cum[k]) / (cum[k + 1] - cum[k]) : 0.0;
    const double y = (k + f) / n;
    free(cum);
    return y * y * y;
}

double orc_chi_e(const double u[3], const double E[3], const double B[3], double eps_ref)
{
    const double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double b[3] = {u[0] / gam, u[1] / gam, u[2] / gam};
    const double f[3] = {E[0] + b[1] * B[2] - b[2] * B[1], E[1] + b[2] * B[0] - b[0] * B[2],
                         E[2] + b[0] * B[1] - b[1] * B[0]};
    const double be = b[0] * E[0] + b[1] * E[1] + b[2] * E[2];
    const double q = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] - be * be;
    return eps_ref * gam * sqrt(q > 0.0 ? q : 0.0);
}

/* Initial optical depth of particle id: -ln u, counter (id, 0, 2, 0). */
double orc_qed_initial_tau(long id, uint32_t seed_lo, uint32_t seed_hi)
{
    const uint32_t ctr[4] = {(uint32_t)id, 0u, 2u, 0u}, key[2] = {seed_lo, seed_hi};
    uint32_t o[4];
    philox4x32_10(ctr, key, o);
    return -log(u01(o[0]));
}

/* After step n (fields, positions and momenta all at t_{n+1}): for every
 * alive particle of `e` the fields at its position x^{n+1} and its momentum
 * u^{n+1} give chi;
 * tau[p] decreases by W dt; when it reaches zero a photon of energy fraction
 * xi = F^-1(r1) (counter (id, step, 0, 0), first word) is emitted along the
 * particle's velocity with the particle's weight and position, the particle
 * recoils by the photon momentum, and tau restarts at -ln r2 (second word).
 * Photons go to ph[7][cap] (x0, x1, x2, u0, u1, u2, w) from *nph on. */
int orc_qed_compton(const orc_grid *g, orc_species *e, double eps_ref, uint32_t seed_lo, uint32_t seed_hi,
                    long step, double *tau, double *ph, long cap, long *nph)
{
    const double dt = g->dt;
    for (long p = 0; p < e->n; ++p) {
        if (!e->alive[p]) continue;
        double u[3] = {e->u[0][p], e->u[1][p], e->u[2][p]}, x[3] = {0, 0, 0}, E[3], B[3];
        const double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int d = 0; d < g->dim; ++d) x[d] = e->x[d][p];
        if (orc_gather(g, x, E, B) != ORC_OK) return ORC_EOUTSIDE;
        const double chi = orc_chi_e(u, E, B, eps_ref);
        if (chi <= 0.0) continue;
        tau[p] -= orc_compton_rate(chi, gam, eps_ref) * dt;
        if (tau[p] > 0.0) continue;
        const uint32_t ctr[4] = {(uint32_t)p, (uint32_t)step, 0u, 0u}, key[2] = {seed_lo, seed_hi};
        uint32_t o[4];
        philox4x32_10(ctr, key, o);
        const double xi = orc_compton_xi(chi, u01(o[0]));
        const double umag = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double k = xi * gam;                   /* photon energy = momentum (m c) */
        if (*nph < cap) {
            for (int d = 0; d < 3; ++d) ph[d * cap + *nph] = d < g->dim ? e->x[d][p] : 0.0;
            for (int c = 0; c < 3; ++c) ph[(3 + c) * cap + *nph] = k * u[c] / umag;
            ph[6 * cap + *nph] = e->w[p];
            *nph += 1;
        }
        for (int c = 0; c < 3; ++c) e->u[c][p] = u[c] * (1.0 - k / umag);
        tau[p] = -log(u01(o[1]));
    }
    return ORC_OK;
}

/* --------------------------------------- QED: Breit-Wheeler pairs (Sec. 3.4)
 * Pair creation by photons in the locally-constant-field approximation, by
 * the same event Monte Carlo.  Photon of momentum k (m c units, energy k m c^2)
 * along khat:
 *   chi_g = eps_ref k sqrt((E + khat x B)^2 - (khat . E)^2),
 *   dW / deta = alpha / (eps_ref sqrt(3) pi k) F(eta, chi_g),
 *   F = (eta / (1 - eta) + (1 - eta) / eta) K_{2/3}(z) + int_z^inf K_{1/3},
 *   z = 2 / (3 chi_g eta (1 - eta)),
 * eta = the electron's share of the photon energy (the spectrum is symmetric
 * in eta <-> 1 - eta).  The pair takes the photon's momentum: u_- = eta k,
 * u_+ = (1 - eta) k (vectors along khat); photons with k <= 2 (below the
 * pair threshold) never convert.  Counter (id, step, 1, 0) word 0 draws eta;
 * a photon's initial depth uses counter (id, 0, 3, 0). */

double orc_bw_f(double eta, double chi)
{
    if (eta <= 0.0 || eta >= 1.0) return 0.0;
    const double z = 2.0 / (3.0 * chi * eta * (1.0 - eta));
    if (z > 700.0) return 0.0;
    return (eta / (1.0 - eta) + (1.0 - eta) / eta) * bessel_k_int(2.0 / 3.0, z, 0) + bessel_k_int(1.0 / 3.0, z, 1);
}

/* cumulative int_0^eta F on the uniform grid eta_k = k / n */
static void bw_cumulative(double chi, int n, double *cum)
{
    cum[0] = 0.0;
    double prev = 0.0;
    for (int k = 1; k <= n; ++k) {
        const double f = orc_bw_f((double)k / n, chi);
        cum[k] = cum[k - 1] + 0.5 * (prev + f) / n;
        prev = f;
    }
}

double orc_bw_rate(double chi, double k, double eps_ref)
{
    if (chi <= 0.0 || k <= 2.0) return 0.0;
    const int n = 4000;
    double *cum = (double *)malloc(sizeof(double) * (n + 1));
    bw_cumulative(chi, n, cum);
    const double F = cum[n];
    free(cum);
    const double alpha = 1.0 / 137.035999084;
    return alpha / (eps_ref * sqrt(3.0) * M_PI * k) * F;
}

/* electron energy share with cumulative probability r */
double orc_bw_eta(double chi, double r)
{
    const int n = 4000;
    double *cum = (double *)malloc(sizeof(double) * (n + 1));
    bw_cumulative(chi, n, cum);
    const double target = r * cum[n];
    int k = 0;
    while (k < n && cum[k + 1] < target) ++k;
    const double f = (cum[k + 1] > cum[k]) ? (target - cum[k]) / (cum[k + 1] - cum[k]) : 0.0;
    free(cum);
    return (k + f) / n;
}

double orc_chi_g(const double k[3], const double E[3], const double B[3], double eps_ref)
{
    const double km = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    if (km <= 0.0) return 0.0;
    const double n[3] = {k[0] / km, k[1] / km, k[2] / km};
    const double f[3] = {E[0] + n[1] * B[2] - n[2] * B[1], E[1] + n[2] * B[0] - n[0] * B[2],
                         E[2] + n[0] * B[1] - n[1] * B[0]};
    const double ne = n[0] * E[0] + n[1] * E[1] + n[2] * E[2];
    const double q = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] - ne * ne;
    return eps_ref * km * sqrt(q > 0.0 ? q : 0.0);
}

double orc_qed_initial_tau_kind(long id, uint32_t kind, uint32_t seed_lo, uint32_t seed_hi)
{
    const uint32_t ctr[4] = {(uint32_t)id, 0u, kind, 0u}, key[2] = {seed_lo, seed_hi};
    uint32_t o[4];
    philox4x32_10(ctr, key, o);
    return -log(u01(o[0]));
}

/* After step n: for every alive photon of `ph` (index = id) the fields at its
 * position and its momentum give chi_g; tau[p] decreases by W dt and at zero
 * the photon is removed and an electron (eta) and a positron (1 - eta) are
 * written to pe[7][cap] and pp[7][cap] (x0, x1, x2, u0, u1, u2, w) from *npair
 * on (the same count for both). */
int orc_qed_bw(const orc_grid *g, orc_species *ph, double eps_ref, uint32_t seed_lo, uint32_t seed_hi,
               long step, double *tau, double *pe, double *pp, long cap, long *npair)
{
    const double dt = g->dt;
    for (long p = 0; p < ph->n; ++p) {
        if (!ph->alive[p]) continue;
        const double k[3] = {ph->u[0][p], ph->u[1][p], ph->u[2][p]};
        const double km = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        if (km <= 2.0) continue;
        double x[3] = {0, 0, 0}, E[3], B[3];
        for (int d = 0; d < g->dim; ++d) x[d] = ph->x[d][p];
        if (orc_gather(g, x, E, B) != ORC_OK) return ORC_EOUTSIDE;
        const double chi = orc_chi_g(k, E, B, eps_ref);
        if (chi <= 0.0) continue;
        tau[p] -= orc_bw_rate(chi, km, eps_ref) * dt;
        if (tau[p] > 0.0) continue;
        const uint32_t ctr[4] = {(uint32_t)p, (uint32_t)step, 1u, 0u}, key[2] = {seed_lo, seed_hi};
        uint32_t o[4];
        philox4x32_10(ctr, key, o);
        const double eta = orc_bw_eta(chi, u01(o[0]));
        if (*npair < cap) {
            for (int d = 0; d < 3; ++d) {
                const double xd = d < g->dim ? ph->x[d][p] : 0.0;
                pe[d * cap + *npair] = xd;
                pp[d * cap + *npair] = xd;
            }
            for (int c = 0; c < 3; ++c) {
                pe[(3 + c) * cap + *npair] = eta * k[c];
                pp[(3 + c) * cap + *npair] = (1.0 - eta) * k[c];
            }
            pe[6 * cap + *npair] = ph->w[p];
            pp[6 * cap + *npair] = ph->w[p];
            *npair += 1;
        }
        ph->alive[p] = 0;
    }
    return ORC_OK;
}
