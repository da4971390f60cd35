/*
 * kgs_oracle.c -- plain serial FP64 oracle of the iterative DVM scheme
 * (arXiv 1810.00348, Sections 2-4).  TEST INFRASTRUCTURE ONLY: loaded by the
 * tests, the smoke check and the CPU-baseline leg of the benchmark, never by
 * the product path.
 *
 * The code follows the paper's equations in the paper's order, one discrete
 * velocity at a time (the velocity-space memory reduction of Section 2.2):
 *   Eq. (2)  Shakhov equilibrium f^S from the lagged macros,
 *   Eq. (6)  outer iteration with f^S and tau lagged at step n,
 *   Eq. (7)  first-order upwind implicit update, swept along the
 *            characteristic direction of each velocity (optionally the
 *            second-order upwind difference that Section 6 names as the
 *            next step),
 *   Eq. (5)  quadrature moments,
 *   Eq. (8)  diffuse-wall emission with the lagged wall density,
 *   Eq. (9)  wall density from the non-penetration condition,
 *   Sec. 3.4 global density rescaling for closed cavities,
 *   Eq. (10) reference viscosity from the Knudsen number,
 *   Sec. 4.1 convergence monitor (relative L2 change of rho, rho U, rho E).
 * Readings of silent or garbled passages are listed where they are used.
 * The serial loop over velocities is the default; an optional mode sweeps
 * contiguous velocity ranges concurrently and adds their private sums in
 * range order (kgso_set_threads), for comparisons at full workload sizes.
 *
 * Parity status: every function here is pinned by the CPU tests (closed-form
 * quadrature moments, dense linear solves of the sweep of either order, the
 * convergence order of both on a relaxation problem with a closed-form
 * solution, rest state, mass, mirror symmetry, free-molecular linear system,
 * BGK limit).
 */
#include "kgs_oracle.h"

#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define R_GAS 0.5 /* nondimensional gas constant: velocity unit sqrt(2 R T0) */

struct kgso_state {
    kgso_problem p;
    int ncell, nvel;
    double *dx, *dy, *dz;
    double *xi_x, *xi_y, *xi_z, *w_x, *w_y, *w_z;
    unsigned char *solid;
    double *mac;    /* [8][ncell] macros at step n                */
    double *rho_w;  /* [6][ncell] wall density per wall face       */
    double *f;      /* [ncell] distribution of one velocity        */
    double mu_ref;
    double M0;      /* initial total mass                          */
    double out_flux_unit[7][6]; /* discrete-mode normaliser, per wall kind and face */
    int threads;    /* velocity ranges swept concurrently (1: plain serial loop) */
};

/* ------------------------------------------------------------------------ */
/* grid helpers                                                             */

static int cell_index(const kgso_state *s, int i, int j, int k)
{
    return i + s->p.nx * (j + s->p.ny * k);
}

static void cell_ijk(const kgso_state *s, int c, int *i, int *j, int *k)
{
    *i = c % s->p.nx;
    *j = (c / s->p.nx) % s->p.ny;
    *k = c / (s->p.nx * s->p.ny);
}

static int is_solid(const kgso_state *s, int c)
{
    return s->solid != NULL && s->solid[c] != 0;
}

static void velocity(const kgso_state *s, int a, double xi[3], double *w)
{
    int ix = a % s->p.nvx;
    int iy = (a / s->p.nvx) % s->p.nvy;
    int iz = a / (s->p.nvx * s->p.nvy);
    xi[0] = s->xi_x[ix];
    xi[1] = s->xi_y[iy];
    xi[2] = s->xi_z[iz];
    *w = s->w_x[ix] * s->w_y[iy] * s->w_z[iz];
}

/* Neighbour of cell c through face f (0..5 = -x,+x,-y,+y,-z,+z):
 * returns the neighbour index, -1 outside the domain, -2 if solid. */
static int neighbour(const kgso_state *s, int c, int face)
{
    int i, j, k;
    cell_ijk(s, c, &i, &j, &k);
    int d = face / 2, step = (face % 2) ? 1 : -1;
    if (d == 0) i += step;
    if (d == 1) j += step;
    if (d == 2) k += step;
    if (i < 0 || j < 0 || k < 0 || i >= s->p.nx || j >= s->p.ny || k >= s->p.nz) return -1;
    int n = cell_index(s, i, j, k);
    return is_solid(s, n) ? -2 : n;
}

/* wall kind of a wall face: 0..5 = domain side, 6 = solid surface */
static int wall_kind(const kgso_state *s, int c, int face)
{
    return neighbour(s, c, face) == -1 ? face : 6;
}

static void wall_params(const kgso_state *s, int kind, double U[3], double *T)
{
    if (kind < 6) {
        U[0] = s->p.U_w[kind][0];
        U[1] = s->p.U_w[kind][1];
        U[2] = s->p.U_w[kind][2];
        *T = s->p.T_w[kind];
    } else {
        U[0] = U[1] = U[2] = 0.0;
        *T = s->p.T_solid;
    }
}

/* face f is a wall face (domain wall or solid surface) of fluid cell c */
static int is_wall_face(const kgso_state *s, int c, int face)
{
    int n = neighbour(s, c, face);
    if (n == -2) return 1;
    if (n == -1) return s->p.face_type[face] == KGSO_FACE_WALL;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* physics                                                                  */

/* Maxwellian of Eq. (2) / Eq. (8): rho (2 pi R T)^{-3/2} exp(-|xi-U|^2 / (2 R T)) */
static double maxwellian(double rho, const double U[3], double T, const double xi[3])
{
    double c2 = 0.0;
    for (int d = 0; d < 3; d++) c2 += (xi[d] - U[d]) * (xi[d] - U[d]);
    return rho / pow(2.0 * M_PI * R_GAS * T, 1.5) * exp(-c2 / (2.0 * R_GAS * T));
}

/* Shakhov equilibrium, Eq. (2), at macros m = (rho, U, T, q). */
static double shakhov(const kgso_state *s, const double m[8], const double xi[3])
{
    double rho = m[0], T = m[4];
    const double U[3] = {m[1], m[2], m[3]};
    double c[3], c2 = 0.0, cq = 0.0;
    for (int d = 0; d < 3; d++) {
        c[d] = xi[d] - U[d];
        c2 += c[d] * c[d];
        cq += c[d] * m[5 + d];
    }
    double p = rho * R_GAS * T;
    double fM = maxwellian(rho, U, T, xi);
    return fM * (1.0 + (1.0 - s->p.Pr) * cq / (5.0 * p * R_GAS * T) * (c2 / (R_GAS * T) - 5.0));
}

/* Eq. (10): mu_ref = 15 sqrt(pi) p_ref lambda_ref / ((5-2w)(7-2w) sqrt(2 R T_ref)),
 * with T_ref = 1, p_ref = rho_ref R T_ref = R, lambda_ref = Kn (length unit 1).
 * Reading: the reference state is the initial uniform state (Section 4.1,
 * "based on the initial constant pressure"). */
static double mu_reference(double Kn, double omega)
{
    double p_ref = 1.0 * R_GAS * 1.0;
    return 15.0 * sqrt(M_PI) * p_ref * Kn / ((5.0 - 2.0 * omega) * (7.0 - 2.0 * omega) * sqrt(2.0 * R_GAS * 1.0));
}

/* Inverse relaxation time: tau = mu/p (Section 2.1), mu = mu_ref T^omega (Section 4). */
static double inv_tau(const kgso_state *s, const double m[8])
{
    double rho = m[0], T = m[4];
    double mu = s->mu_ref * pow(T, s->p.omega);
    double p = rho * R_GAS * T;
    return p / mu;
}

static void cell_macros(const kgso_state *s, int c, double m[8])
{
    for (int q = 0; q < 8; q++) m[q] = s->mac[(size_t)q * s->ncell + c];
}

/* ------------------------------------------------------------------------ */
/* boundary conditions, Section 3.4                                         */

double kgso_ghost(const kgso_state *s, int c, int face, int a)
{
    double xi[3], w, U[3], T;
    velocity(s, a, xi, &w);
    int n = neighbour(s, c, face);
    if (n >= 0) return 0.0;
    if (n == -1 && s->p.face_type[face] == KGSO_FACE_INFLOW) {
        /* free stream: equilibrium of the free-stream state */
        return maxwellian(s->p.rho_in, s->p.U_in, s->p.T_in, xi);
    }
    /* diffuse wall, Eq. (8).  Reading: Eq. (8) omits the wall velocity; the
     * moving lid of Section 4.1 needs it, so the Maxwellian is centred on U_w. */
    wall_params(s, wall_kind(s, c, face), U, &T);
    return s->rho_w[(size_t)face * s->ncell + c] * maxwellian(1.0, U, T, xi);
}

/* Incoming flux onto the wall at face `face` of cell c from distribution value
 * f of velocity xi:  w |xi.n| f  when xi.n < 0 (n points from the wall into the
 * gas), else 0.  Eq. (9), with the quadrature weight that the printed
 * equation leaves out. */
static double incoming_flux(int face, const double xi[3], double w, double f)
{
    int d = face / 2;
    double n = (face % 2) ? -1.0 : 1.0; /* wall on the minus side: n = +e_d */
    double xn = xi[d] * n;
    return xn < 0.0 ? w * (-xn) * f : 0.0;
}

/* rho_w from the incoming flux F, Eq. (9).  Analytic mode is the printed
 * formula, sqrt(2 pi / (R T_w)) F.  Discrete mode (reading) divides by the
 * discrete outgoing flux of the unit wall Maxwellian, so that the discrete
 * mass flux through the wall is zero. */
static double wall_density(const kgso_state *s, int kind, int face, double F)
{
    double U[3], T;
    wall_params(s, kind, U, &T);
    if (s->p.wall_mode == KGSO_WALL_ANALYTIC) return sqrt(2.0 * M_PI / (R_GAS * T)) * F;
    return F / s->out_flux_unit[kind][face];
}

static void compute_out_flux_unit(kgso_state *s)
{
    for (int kind = 0; kind < 7; kind++) {
        double U[3], T;
        wall_params(s, kind, U, &T);
        for (int face = 0; face < 6; face++) {
            int d = face / 2;
            double n = (face % 2) ? -1.0 : 1.0;
            double sum = 0.0;
            for (int a = 0; a < s->nvel; a++) {
                double xi[3], w;
                velocity(s, a, xi, &w);
                double xn = xi[d] * n;
                if (xn > 0.0) sum += w * xn * maxwellian(1.0, U, T, xi);
            }
            s->out_flux_unit[kind][face] = sum;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. (7): the upwind sweep of one discrete velocity                       */

void kgso_sweep(const kgso_state *s, int a, double *f)
{
    const kgso_problem *p = &s->p;
    double xi[3], w;
    velocity(s, a, xi, &w);
    /* Sweep along the characteristic: increasing index where xi_d >= 0,
     * decreasing where xi_d < 0 (Algorithm 1's eight sweep directions). */
    int i0 = xi[0] >= 0.0 ? 0 : p->nx - 1, di = xi[0] >= 0.0 ? 1 : -1;
    int j0 = xi[1] >= 0.0 ? 0 : p->ny - 1, dj = xi[1] >= 0.0 ? 1 : -1;
    int k0 = xi[2] >= 0.0 ? 0 : p->nz - 1, dk = xi[2] >= 0.0 ? 1 : -1;
    const double *width[3] = {s->dx, s->dy, s->dz};

    for (int kk = 0; kk < p->nz; kk++) {
        int k = k0 + dk * kk;
        for (int jj = 0; jj < p->ny; jj++) {
            int j = j0 + dj * jj;
            for (int ii = 0; ii < p->nx; ii++) {
                int i = i0 + di * ii;
                int c = cell_index(s, i, j, k);
                if (is_solid(s, c)) {
                    f[c] = 0.0;
                    continue;
                }
                double m[8];
                cell_macros(s, c, m);
                double rtau = inv_tau(s, m);
                double fS = shakhov(s, m, xi);
                /* Eq. (7) solved for f_{i,j,k}:
                 *   sum_d |xi_d|/dx_d (f - f_up,d) = -(f - f^S)/tau                */
                double num = rtau * fS, den = rtau;
                int ijk[3] = {i, j, k};
                for (int d = 0; d < 3; d++) {
                    if (xi[d] == 0.0) continue; /* no transport along d */
                    double coef = fabs(xi[d]) / width[d][ijk[d]];
                    int face = 2 * d + (xi[d] > 0.0 ? 0 : 1); /* upwind side */
                    int n = neighbour(s, c, face);
                    int n2 = n >= 0 ? neighbour(s, n, face) : -1;
                    if (p->order == 2 && n2 >= 0) {
                        /* Second-order upwind (reading of Section 6, no
                         * limiter): |xi_d| (3 f_c - 4 f_n + f_n2) / (2 dx_d). */
                        num += coef * (2.0 * f[n] - 0.5 * f[n2]);
                        den += 1.5 * coef;
                        continue;
                    }
                    double up = n >= 0 ? f[n] : kgso_ghost(s, c, face, a);
                    num += coef * up;
                    den += coef;
                }
                f[c] = num / den;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. (5) moments                                                          */

void kgso_moments(const kgso_state *s, const double *f, double out[8])
{
    double rho = 0.0, mom[3] = {0.0, 0.0, 0.0}, rhoE = 0.0, q[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < s->nvel; a++) {
        double xi[3], w;
        velocity(s, a, xi, &w);
        rho += w * f[a];
        for (int d = 0; d < 3; d++) mom[d] += w * xi[d] * f[a];
        rhoE += 0.5 * w * (xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]) * f[a];
    }
    double U[3] = {mom[0] / rho, mom[1] / rho, mom[2] / rho};
    double U2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    /* rho E = rho U^2/2 + C_v T with C_v = (3/2) R per unit mass (Section 2.1) */
    double T = (rhoE - 0.5 * rho * U2) / (1.5 * rho * R_GAS);
    for (int a = 0; a < s->nvel; a++) {
        double xi[3], w, c[3];
        velocity(s, a, xi, &w);
        for (int d = 0; d < 3; d++) c[d] = xi[d] - U[d];
        double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        for (int d = 0; d < 3; d++) q[d] += 0.5 * w * c[d] * c2 * f[a];
    }
    out[0] = rho;
    out[1] = U[0];
    out[2] = U[1];
    out[3] = U[2];
    out[4] = T;
    out[5] = q[0];
    out[6] = q[1];
    out[7] = q[2];
}

void kgso_equilibrium(const kgso_state *s, const double mac[8], double *out)
{
    for (int a = 0; a < s->nvel; a++) {
        double xi[3], w;
        velocity(s, a, xi, &w);
        out[a] = shakhov(s, mac, xi);
    }
}

/* ------------------------------------------------------------------------ */
/* state                                                                    */

static double *copy_array(const double *src, int n)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(d, src, sizeof(double) * (size_t)n);
    return d;
}

double kgso_total_mass(const kgso_state *s)
{
    double M = 0.0;
    for (int c = 0; c < s->ncell; c++) {
        if (is_solid(s, c)) continue;
        int i, j, k;
        cell_ijk(s, c, &i, &j, &k);
        M += s->mac[c] * s->dx[i] * s->dy[j] * s->dz[k];
    }
    return M;
}

double kgso_mu_ref(const kgso_state *s) { return s->mu_ref; }

/* Wall densities from the incoming flux of a distribution known per velocity
 * through a callback-free route: the caller accumulates F[6][ncell]. */
static void rho_w_from_flux(kgso_state *s, const double *F)
{
    for (int face = 0; face < 6; face++)
        for (int c = 0; c < s->ncell; c++) {
            size_t idx = (size_t)face * s->ncell + c;
            if (!is_solid(s, c) && is_wall_face(s, c, face))
                s->rho_w[idx] = wall_density(s, wall_kind(s, c, face), face, F[idx]);
            else
                s->rho_w[idx] = 0.0;
        }
}

kgso_state *kgso_create(const kgso_problem *p, const double *macros0)
{
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nvx < 1 || p->nvy < 1 || p->nvz < 1) return NULL;
    if (p->order < 0 || p->order > 2) return NULL;
    if (p->order == 2) {
        /* the three-point difference assumes equal widths along each axis */
        const double *w[3] = {p->dx, p->dy, p->dz};
        const int n[3] = {p->nx, p->ny, p->nz};
        for (int d = 0; d < 3; d++)
            for (int q = 1; q < n[d]; q++)
                if (w[d][q] != w[d][0]) return NULL;
    }
    kgso_state *s = (kgso_state *)calloc(1, sizeof(kgso_state));
    s->p = *p;
    if (s->p.order == 0) s->p.order = 1;
    s->threads = 1;
    s->ncell = p->nx * p->ny * p->nz;
    s->nvel = p->nvx * p->nvy * p->nvz;
    s->dx = copy_array(p->dx, p->nx);
    s->dy = copy_array(p->dy, p->ny);
    s->dz = copy_array(p->dz, p->nz);
    s->xi_x = copy_array(p->xi_x, p->nvx);
    s->xi_y = copy_array(p->xi_y, p->nvy);
    s->xi_z = copy_array(p->xi_z, p->nvz);
    s->w_x = copy_array(p->w_x, p->nvx);
    s->w_y = copy_array(p->w_y, p->nvy);
    s->w_z = copy_array(p->w_z, p->nvz);
    s->p.dx = s->dx; s->p.dy = s->dy; s->p.dz = s->dz;
    s->p.xi_x = s->xi_x; s->p.xi_y = s->xi_y; s->p.xi_z = s->xi_z;
    s->p.w_x = s->w_x; s->p.w_y = s->w_y; s->p.w_z = s->w_z;
    if (p->solid) {
        s->solid = (unsigned char *)malloc((size_t)s->ncell);
        memcpy(s->solid, p->solid, (size_t)s->ncell);
        s->p.solid = s->solid;
    }
    s->mac = (double *)calloc((size_t)8 * s->ncell, sizeof(double));
    s->rho_w = (double *)calloc((size_t)6 * s->ncell, sizeof(double));
    s->f = (double *)calloc((size_t)s->ncell, sizeof(double));
    s->mu_ref = mu_reference(p->Kn, p->omega);

    int any_inflow = 0;
    for (int face = 0; face < 6; face++) any_inflow |= p->face_type[face] == KGSO_FACE_INFLOW;
    for (int c = 0; c < s->ncell; c++) {
        double m[8];
        if (macros0) {
            for (int q = 0; q < 8; q++) m[q] = macros0[(size_t)q * s->ncell + c];
        } else if (any_inflow) {
            double init[8] = {p->rho_in, p->U_in[0], p->U_in[1], p->U_in[2], p->T_in, 0, 0, 0};
            memcpy(m, init, sizeof m);
        } else {
            double init[8] = {1.0, 0, 0, 0, 1.0, 0, 0, 0};
            memcpy(m, init, sizeof m);
        }
        if (is_solid(s, c)) memset(m, 0, sizeof m);
        for (int q = 0; q < 8; q++) s->mac[(size_t)q * s->ncell + c] = m[q];
    }
    s->M0 = kgso_total_mass(s);
    compute_out_flux_unit(s);

    /* Reading: rho_w^0 comes from f^0 = f^{S,0}, the equilibrium of the
     * initial macros (Section 2.2 starts the iteration from it). */
    double *F = (double *)calloc((size_t)6 * s->ncell, sizeof(double));
    for (int c = 0; c < s->ncell; c++) {
        if (is_solid(s, c)) continue;
        double m[8];
        cell_macros(s, c, m);
        for (int face = 0; face < 6; face++) {
            if (!is_wall_face(s, c, face)) continue;
            double sum = 0.0;
            for (int a = 0; a < s->nvel; a++) {
                double xi[3], w;
                velocity(s, a, xi, &w);
                sum += incoming_flux(face, xi, w, shakhov(s, m, xi));
            }
            F[(size_t)face * s->ncell + c] = sum;
        }
    }
    rho_w_from_flux(s, F);
    free(F);
    return s;
}

void kgso_destroy(kgso_state *s)
{
    if (!s) return;
    free(s->dx); free(s->dy); free(s->dz);
    free(s->xi_x); free(s->xi_y); free(s->xi_z);
    free(s->w_x); free(s->w_y); free(s->w_z);
    free(s->solid); free(s->mac); free(s->rho_w); free(s->f);
    free(s);
}

void kgso_get_macros(const kgso_state *s, double *out)
{
    memcpy(out, s->mac, sizeof(double) * (size_t)8 * s->ncell);
}

void kgso_get_rho_w(const kgso_state *s, double *out)
{
    memcpy(out, s->rho_w, sizeof(double) * (size_t)6 * s->ncell);
}

void kgso_set_rho_w(kgso_state *s, const double *in)
{
    memcpy(s->rho_w, in, sizeof(double) * (size_t)6 * s->ncell);
}

/* ------------------------------------------------------------------------ */
/* one outer iteration, Eq. (6) + Algorithm 1                               */

/* Sums of one outer iteration's first pass over velocities [a0, a1): each
 * velocity is swept into f with the lagged f^{S,n}, tau^n and rho_w^n and
 * added to rho, rho U, rho E (Eq. (5)) and to the incoming wall fluxes of
 * Eq. (9). */
static void pass1(const kgso_state *s, int a0, int a1, double *f, double *rho, double *mom, double *rhoE, double *F)
{
    const int nc = s->ncell;
    for (int a = a0; a < a1; a++) {
        double xi[3], w;
        velocity(s, a, xi, &w);
        kgso_sweep(s, a, f);
        double xi2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
        for (int c = 0; c < nc; c++) {
            if (is_solid(s, c)) continue;
            double fc = f[c];
            rho[c] += w * fc;
            for (int d = 0; d < 3; d++) mom[(size_t)d * nc + c] += w * xi[d] * fc;
            rhoE[c] += 0.5 * w * xi2 * fc;
            for (int face = 0; face < 6; face++)
                if (is_wall_face(s, c, face)) F[(size_t)face * nc + c] += incoming_flux(face, xi, w, fc);
        }
    }
}

/* Second pass over velocities [a0, a1): q = 1/2 sum w c |c|^2 f with
 * c = xi - U^{n+1} (Eq. (5)), from the same sweeps. */
static void pass2(const kgso_state *s, int a0, int a1, double *f, const double *U, double *q)
{
    const int nc = s->ncell;
    for (int a = a0; a < a1; a++) {
        double xi[3], w;
        velocity(s, a, xi, &w);
        kgso_sweep(s, a, f);
        for (int c = 0; c < nc; c++) {
            if (is_solid(s, c)) continue;
            double cc[3], c2 = 0.0;
            for (int d = 0; d < 3; d++) {
                cc[d] = xi[d] - U[(size_t)d * nc + c];
                c2 += cc[d] * cc[d];
            }
            for (int d = 0; d < 3; d++) q[(size_t)d * nc + c] += 0.5 * w * cc[d] * c2 * f[c];
        }
    }
}

void kgso_set_threads(kgso_state *s, int n) { s->threads = n > 1 ? n : 1; }

/* The two passes of an outer iteration over one velocity range [a0, a1),
 * added into caller-owned sums (rho [nc], mom [3][nc], rhoE [nc], F [6][nc];
 * q [3][nc] about the given U [3][nc]): the unit of a velocity-space
 * partition whose ranges are summed afterwards. */
void kgso_pass1_range(const kgso_state *s, int a0, int a1, double *rho, double *mom, double *rhoE, double *F)
{
    double *f = (double *)calloc((size_t)s->ncell, sizeof(double));
    pass1(s, a0, a1, f, rho, mom, rhoE, F);
    free(f);
}

void kgso_pass2_range(const kgso_state *s, int a0, int a1, const double *U, double *q)
{
    double *f = (double *)calloc((size_t)s->ncell, sizeof(double));
    pass2(s, a0, a1, f, U, q);
    free(f);
}

int kgso_parallel(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

double kgso_iterate(kgso_state *s)
{
    const int nc = s->ncell;
    double *rho = (double *)calloc((size_t)nc, sizeof(double));
    double *mom = (double *)calloc((size_t)3 * nc, sizeof(double));
    double *rhoE = (double *)calloc((size_t)nc, sizeof(double));
    double *q = (double *)calloc((size_t)3 * nc, sizeof(double));
    double *F = (double *)calloc((size_t)6 * nc, sizeof(double));
    double *U = (double *)calloc((size_t)3 * nc, sizeof(double));
    double *newmac = (double *)calloc((size_t)8 * nc, sizeof(double));

    /* Pass 1: each velocity in turn is swept with the lagged f^{S,n}, tau^n and
     * rho_w^n, and its contribution is added to rho, rho U, rho E (Eq. (5))
     * and to the incoming wall fluxes of Eq. (9). */
    if (s->threads <= 1) {
        pass1(s, 0, s->nvel, s->f, rho, mom, rhoE, F);
    } else {
        /* optional: contiguous velocity ranges with private sums, added up in
         * range order afterwards */
        const int T = s->threads;
        double *f_t = (double *)calloc((size_t)T * nc, sizeof(double));
        double *acc = (double *)calloc((size_t)T * 11 * nc, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static, 1)
#endif
        for (int t = 0; t < T; t++) {
            double *a_t = acc + (size_t)t * 11 * nc;
            pass1(s, (int)((long long)s->nvel * t / T), (int)((long long)s->nvel * (t + 1) / T), f_t + (size_t)t * nc,
                  a_t, a_t + nc, a_t + 4 * (size_t)nc, a_t + 5 * (size_t)nc);
        }
        for (int t = 0; t < T; t++) {
            const double *a_t = acc + (size_t)t * 11 * nc;
            for (size_t i = 0; i < (size_t)nc; i++) rho[i] += a_t[i];
            for (size_t i = 0; i < (size_t)3 * nc; i++) mom[i] += a_t[nc + i];
            for (size_t i = 0; i < (size_t)nc; i++) rhoE[i] += a_t[4 * (size_t)nc + i];
            for (size_t i = 0; i < (size_t)6 * nc; i++) F[i] += a_t[5 * (size_t)nc + i];
        }
        free(acc);
        free(f_t);
    }
    for (int c = 0; c < nc; c++) {
        if (is_solid(s, c)) continue;
        for (int d = 0; d < 3; d++) U[(size_t)d * nc + c] = mom[(size_t)d * nc + c] / rho[c];
    }
    /* Pass 2: the heat flux of Eq. (5) needs the new U, so every velocity is
     * swept again (the sweep is deterministic) and q = 1/2 sum w c c^2 f is
     * accumulated with c = xi - U^{n+1}.  Option: the peculiar velocity taken
     * about the lagged U^n instead (Algorithm 3 accumulates its eight moments
     * in one pass, before the new U is known); the two agree at the fixed
     * point. */
    const double *Uq = U;
    double *Ulag = NULL;
    if (s->p.q_lagged) {
        Ulag = copy_array(s->mac + nc, 3 * nc);
        Uq = Ulag;
    }
    if (s->threads <= 1) {
        pass2(s, 0, s->nvel, s->f, Uq, q);
    } else {
        const int T = s->threads;
        double *f_t = (double *)calloc((size_t)T * nc, sizeof(double));
        double *acc = (double *)calloc((size_t)T * 3 * nc, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static, 1)
#endif
        for (int t = 0; t < T; t++)
            pass2(s, (int)((long long)s->nvel * t / T), (int)((long long)s->nvel * (t + 1) / T), f_t + (size_t)t * nc,
                  Uq, acc + (size_t)t * 3 * nc);
        for (int t = 0; t < T; t++)
            for (size_t i = 0; i < (size_t)3 * nc; i++) q[i] += acc[(size_t)t * 3 * nc + i];
        free(acc);
        free(f_t);
    }
    free(Ulag);

    int bad = 0;
    for (int c = 0; c < nc; c++) {
        if (is_solid(s, c)) continue;
        double u0 = U[c], u1 = U[(size_t)nc + c], u2 = U[(size_t)2 * nc + c];
        double T = (rhoE[c] - 0.5 * rho[c] * (u0 * u0 + u1 * u1 + u2 * u2)) / (1.5 * rho[c] * R_GAS);
        newmac[c] = rho[c];
        newmac[(size_t)1 * nc + c] = u0;
        newmac[(size_t)2 * nc + c] = u1;
        newmac[(size_t)3 * nc + c] = u2;
        newmac[(size_t)4 * nc + c] = T;
        for (int d = 0; d < 3; d++) newmac[(size_t)(5 + d) * nc + c] = q[(size_t)d * nc + c];
        if (!(rho[c] > 0.0) || !(T > 0.0) || !isfinite(u0) || !isfinite(u1) || !isfinite(u2)) bad = 1;
    }

    /* Wall densities for the next sweep, from the flux of f^{n+1} (Eq. (9)). */
    double *old_rho_w = copy_array(s->rho_w, 6 * nc);
    rho_w_from_flux(s, F);

    /* Section 3.4: for internal flows the whole density field is rescaled so
     * that the total mass stays at its initial value.  Reading: scaling the
     * density field at fixed U and T scales f, hence q and rho_w, by the same
     * factor. */
    if (s->p.mass_rescale) {
        double M = 0.0;
        for (int c = 0; c < nc; c++) {
            if (is_solid(s, c)) continue;
            int i, j, k;
            cell_ijk(s, c, &i, &j, &k);
            M += newmac[c] * s->dx[i] * s->dy[j] * s->dz[k];
        }
        double scale = s->M0 / M;
        for (int c = 0; c < nc; c++) {
            if (is_solid(s, c)) continue;
            newmac[c] *= scale;
            for (int d = 0; d < 3; d++) newmac[(size_t)(5 + d) * nc + c] *= scale;
        }
        for (int idx = 0; idx < 6 * nc; idx++) s->rho_w[idx] *= scale;
    }
    free(old_rho_w);

    /* Section 4.1 convergence monitor.  Reading: the largest, over rho, the
     * three momentum components and rho E, of ||phi^{n+1}-phi^n||_2 /
     * ||phi^{n+1}||_2 over fluid cells, the denominator floored at
     * 1e-8 ||rho^{n+1}||_2 so that a field at rest does not divide by zero. */
    double dn[5] = {0}, nn[5] = {0};
    for (int c = 0; c < nc; c++) {
        if (is_solid(s, c)) continue;
        double phi_new[5], phi_old[5];
        for (int t = 0; t < 2; t++) {
            const double *m = t ? s->mac : newmac;
            double r = m[c], ux = m[(size_t)nc + c], uy = m[(size_t)2 * nc + c], uz = m[(size_t)3 * nc + c],
                   T = m[(size_t)4 * nc + c];
            double *phi = t ? phi_old : phi_new;
            phi[0] = r;
            phi[1] = r * ux;
            phi[2] = r * uy;
            phi[3] = r * uz;
            phi[4] = 0.5 * r * (ux * ux + uy * uy + uz * uz) + 1.5 * r * R_GAS * T;
        }
        for (int t = 0; t < 5; t++) {
            double dd = phi_new[t] - phi_old[t];
            dn[t] += dd * dd;
            nn[t] += phi_new[t] * phi_new[t];
        }
    }
    double res = 0.0;
    double floor_ = 1e-8 * sqrt(nn[0]);
    for (int t = 0; t < 5; t++) {
        double den = sqrt(nn[t]);
        if (den < floor_) den = floor_;
        double r = sqrt(dn[t]) / den;
        if (r > res) res = r;
    }

    memcpy(s->mac, newmac, sizeof(double) * (size_t)8 * nc);
    free(rho); free(mom); free(rhoE); free(q); free(F); free(U); free(newmac);
    if (bad) return -1.0;
    return res;
}
