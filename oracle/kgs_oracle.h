/*
 * kgs_oracle.h -- plain serial FP64 CPU oracle for the iterative DVM scheme of
 * Zhu, Wang, Chen, Guo & Zhang, "GPU acceleration of an iterative scheme for
 * gas-kinetic model equations with memory reduction techniques" (arXiv 1810.00348).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA solver it checks.
 *
 * Units (the paper is silent; reading used throughout): lengths in the cavity
 * side L, velocities in sqrt(2 R T0), temperature in T0, density in rho0, so
 * that the gas constant is R = 1/2 and p = rho R T.
 *
 * Layout: cell c = i + nx*(j + ny*k); discrete velocity a = ix + nvx*(iy + nvy*iz)
 * with xi_a = (xi_x[ix], xi_y[iy], xi_z[iz]) and weight w_a = w_x[ix] w_y[iy] w_z[iz].
 * Macroscopic fields are [8][ncell]: rho, Ux, Uy, Uz, T, qx, qy, qz.
 * Wall densities are stored per cell face, [6][ncell], face order
 * -x, +x, -y, +y, -z, +z (the face of cell c on that side).
 */
#ifndef KGS_ORACLE_H
#define KGS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { KGSO_FACE_WALL = 0, KGSO_FACE_INFLOW = 1 };
enum { KGSO_WALL_DISCRETE = 0, KGSO_WALL_ANALYTIC = 1 };

typedef struct {
    int nx, ny, nz;
    const double *dx, *dy, *dz;          /* cell widths, lengths nx, ny, nz        */
    const unsigned char *solid;          /* ncell flags (1 = solid) or NULL        */
    int nvx, nvy, nvz;
    const double *xi_x, *xi_y, *xi_z;    /* velocity nodes per axis                */
    const double *w_x, *w_y, *w_z;       /* quadrature weights per axis            */
    double Kn, Pr, omega;                /* Kn = +inf gives tau^-1 = 0             */
    int face_type[6];                    /* domain side -x,+x,-y,+y,-z,+z          */
    double T_w[6];                       /* diffuse wall temperature per side      */
    double U_w[6][3];                    /* diffuse wall velocity per side         */
    double rho_in, U_in[3], T_in;        /* free stream (inflow sides)             */
    double T_solid;                      /* temperature of solid-cell surfaces     */
    int wall_mode;                       /* KGSO_WALL_DISCRETE / KGSO_WALL_ANALYTIC */
    int mass_rescale;                    /* 1: keep total mass fixed (Section 3.4) */
    int q_lagged;                        /* 1: heat flux about the lagged U^n      */
    int order;                           /* upwind order of the sweep: 1 (Eq. (7), also 0) or 2 */
} kgso_problem;

typedef struct kgso_state kgso_state;

/* Create a solver state.  macros0 is [8][ncell] or NULL (uniform: the free
 * stream if any side is an inflow, else rho=1, U=0, T=1, q=0).  The wall
 * densities start from the flux of the initial equilibrium.  Returns NULL on
 * invalid input. */
kgso_state *kgso_create(const kgso_problem *p, const double *macros0);
void kgso_destroy(kgso_state *s);

/* One outer iteration n -> n+1.  Returns the residual (>= 0), or a negative
 * number if the new state is not physical (NaN, rho <= 0 or T <= 0). */
double kgso_iterate(kgso_state *s);

/* Optional: sweep n contiguous velocity ranges concurrently (OpenMP when the
 * library was built with it), each with private sums that are added in range
 * order; 1 (the default) is the plain serial loop.  kgso_parallel() tells
 * whether the build runs the ranges on several threads. */
void kgso_set_threads(kgso_state *s, int n);
int kgso_parallel(void);

/* One outer iteration's two passes over velocities [a0, a1) only, added into
 * caller-owned sums: rho [nc], mom [3][nc], rhoE [nc], wall fluxes F [6][nc];
 * then q [3][nc] about U [3][nc] (Eq. (5)).  A velocity-space partition sums
 * these over its ranges (the paper's MPI_Allreduce). */
void kgso_pass1_range(const kgso_state *s, int a0, int a1, double *rho, double *mom, double *rhoE, double *F);
void kgso_pass2_range(const kgso_state *s, int a0, int a1, const double *U, double *q);

void kgso_get_macros(const kgso_state *s, double *out);    /* [8][ncell] */
void kgso_get_rho_w(const kgso_state *s, double *out);     /* [6][ncell] */
void kgso_set_rho_w(kgso_state *s, const double *in);      /* [6][ncell] */
double kgso_total_mass(const kgso_state *s);
double kgso_mu_ref(const kgso_state *s);

/* f^S of Eq. (2) at one state for every discrete velocity (out[nvel]). */
void kgso_equilibrium(const kgso_state *s, const double mac[8], double *out);

/* Eq. (5) moments of one cell's distribution f[nvel] -> rho,Ux,Uy,Uz,T,qx,qy,qz. */
void kgso_moments(const kgso_state *s, const double *f, double out[8]);

/* The upwind sweep of Eq. (7) for one discrete velocity a, using the state's
 * current macros (for f^S and tau) and wall densities.  out[ncell]; solid cells
 * are set to 0.  With order 2 the derivative along an axis is the three-point
 * backward difference wherever both upwind neighbours are fluid cells (uniform
 * cell widths per axis only; kgso_create rejects other grids). */
void kgso_sweep(const kgso_state *s, int a, double *out);

/* The ghost value seen by cell c through its face `face` for velocity a
 * (diffuse wall or free stream).  Returns 0 for an interior face. */
double kgso_ghost(const kgso_state *s, int c, int face, int a);

#ifdef __cplusplus
}
#endif
#endif
