/*
 * kgs.h -- C ABI of the GB300 (sm_103a) solver for the steady Shakhov / BGK
 * model equation by the memory-reduced iterative discrete velocity method of
 * Zhu, Wang, Chen, Guo & Zhang (arXiv 1810.00348).
 *
 * One outer iteration (Eq. (6)) does, for every discrete velocity, the
 * first-order upwind implicit sweep of Eq. (7) with the Shakhov equilibrium
 * of Eq. (2) evaluated from the lagged macroscopic fields, adds the velocity's
 * contribution to the quadrature moments of Eq. (5) and to the incoming wall
 * fluxes of Eq. (9), and then closes with the macroscopic update, the wall
 * densities, the global mass rescaling of Section 3.4 and the convergence
 * monitor of Section 4.1.  The full phase-space distribution is never stored
 * (Section 2.2 and Section 3.2 memory reduction): only one XY slice per
 * in-flight velocity and the block faces between sweep stages.
 *
 * Units: lengths in the cavity side, velocities in sqrt(2 R T0), temperature
 * in T0, density in rho0; the gas constant is R = 1/2 and p = rho R T.
 *
 * Layouts (all FP64 unless stated):
 *   cell c = i + nx*(j + ny*k);
 *   macroscopic fields  [8][nz][ny][nx]: rho, Ux, Uy, Uz, T, qx, qy, qz;
 *   wall densities      [6][nz][ny][nx]: one value per cell face, sides
 *                       -x, +x, -y, +y, -z, +z (0 where the face is not a wall);
 *   discrete velocities a = ix + nvx*(iy + nvy*iz), xi_a = (xi_x[ix],
 *                       xi_y[iy], xi_z[iz]), weight w_x[ix] w_y[iy] w_z[iz].
 *
 * Ownership: every input array is copied during the call that receives it;
 * the caller keeps ownership.  Output arrays are caller-owned and must hold
 * the stated number of elements.  The library allocates (cudaMalloc) and
 * frees all of its device memory itself and launches on the stream given in
 * kgs_opts (NULL = the legacy default stream) of the device that is current
 * at kgs_setup.  Set-up calls (kgs_setup, kgs_batch_setup, kgs_net_create,
 * kgs_net_set_params) copy their tables on the legacy default stream and
 * wait for those copies before they return or launch, so a non-blocking
 * stream needs no ordering by the caller; they may also wait for work the
 * caller queued on the legacy default stream.  One context must not be used
 * by two host threads at once;
 * distinct contexts are independent.  Results are deterministic: every
 * reduction runs in a fixed order.
 *
 * Errors: functions return KGS_OK (0) or a negative KGS_E* code;
 * kgs_iterate returns KGS_NOTCONVERGED (> 0) when its iteration budget ends
 * above the tolerance.  kgs_strerror() gives a message.  After KGS_ECUDA the
 * context should be destroyed.
 */
#ifndef KGS_H
#define KGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KGS_OK 0
#define KGS_NOTCONVERGED 1
#define KGS_EINVAL (-1)     /* invalid argument                                   */
#define KGS_ENOMEM (-2)     /* device or host allocation failed                    */
#define KGS_ECUDA (-3)      /* a CUDA call failed                                  */
#define KGS_EDIVERGED (-4)  /* NaN, rho <= 0 or T <= 0 after an iteration          */
#define KGS_ETIMEOUT (-5)   /* a bounded device wait expired                       */
#define KGS_EFORMAT (-6)    /* checkpoint buffer does not match this context       */

enum { KGS_FACE_WALL = 0, KGS_FACE_INFLOW = 1 };
enum { KGS_FP64 = 0, KGS_MIXED = 1 };
enum { KGS_WALL_DISCRETE = 0, KGS_WALL_ANALYTIC = 1 };

typedef struct kgs_ctx kgs_ctx;

/* Physical grid: nx*ny*nz Cartesian cells with widths dx[nx], dy[ny], dz[nz]
 * (Eq. (7) uses the width of the cell being updated). */
typedef struct {
    int nx, ny, nz;
    const double *dx, *dy, *dz;
} kgs_grid;

/* Tensor-product velocity grid with its quadrature weights (Eq. (4), Eq. (5)).
 * Nodes need not be uniform; a node at exactly 0 has no upwind dependence
 * along that axis. */
typedef struct {
    int nvx, nvy, nvz;
    const double *xi_x, *xi_y, *xi_z;
    const double *w_x, *w_y, *w_z;
} kgs_vgrid;

/* Gas model: Knudsen number (Kn = +inf gives the free-molecular limit
 * 1/tau = 0), Prandtl number (Pr = 2/3 Shakhov, Pr = 1 BGK), viscosity index
 * omega of mu = mu_ref T^omega, mu_ref from Kn by Eq. (10) with the initial
 * uniform state as reference (T_ref = 1, p_ref = 1/2). */
typedef struct {
    double Kn, Pr, omega;
} kgs_gas;

/* Boundaries (Section 3.4).  type[s] for domain side s (-x,+x,-y,+y,-z,+z):
 * KGS_FACE_WALL = diffuse wall at T_w[s] moving at U_w[s] (Eq. (8), centred
 * on the wall velocity), KGS_FACE_INFLOW = free-stream equilibrium
 * (rho_in, U_in, T_in).  Faces between fluid and solid cells are diffuse
 * walls at rest at T_solid. */
typedef struct {
    int type[6];
    double T_w[6];
    double U_w[6][3];
    double rho_in, U_in[3], T_in;
    double T_solid;
} kgs_bc;

/* Options.
 *   precision    KGS_FP64: every step in FP64.  KGS_MIXED: equilibrium and
 *                sweep in FP32, moment sums FP32 within a slice then FP64,
 *                closure in FP64.
 *   wall_norm    KGS_WALL_DISCRETE: rho_w = incoming flux / discrete outgoing
 *                flux of the unit wall Maxwellian (zero discrete mass flux).
 *                KGS_WALL_ANALYTIC: rho_w = sqrt(2 pi/(R T_w)) * incoming flux,
 *                the printed Eq. (9) with the quadrature weights.
 *   mass_rescale 1: rescale rho, q and rho_w each iteration so that the total
 *                mass stays at its initial value (closed cavities, Section 3.4).
 *   max_iters, tol  used by kgs_iterate(n_iters <= 0): iterate until the
 *                residual is below tol or max_iters iterations have run.
 *   v_per_cta    discrete velocities per thread block: 0 (default for the
 *                precision, 256 for KGS_MIXED, 128 for KGS_FP64), 128, or 256
 *                (KGS_MIXED only); block_z cells per sweep block along z
 *                (0 = default, 32).
 *   stream       cudaStream_t to launch on (NULL = legacy default stream).
 *   q_lagged     0: heat flux of Eq. (5) about the new velocity U^{n+1}
 *                (default).  1: about the lagged velocity U^n, the single-pass
 *                form of Algorithm 3's eight moments; the two agree at the
 *                fixed point.
 *   vz_begin, vz_end  velocity-space partition: the context sweeps only the
 *                velocity planes iz in [vz_begin, vz_end) (0, 0 = all).  Its
 *                per-cell sums (kgs_sweep_sums) are then partial; the wall
 *                normalisation and the initial wall densities still use the
 *                whole velocity grid.
 *   order        upwind order of the sweep: 1 (or 0) is Eq. (7).  2 is the
 *                second-order upwind difference that Section 6 names as the
 *                next step, read as the three-point backward difference
 *                (3 f_i - 4 f_{i-1} + f_{i-2}) / (2 dx) along each axis without
 *                a limiter, used where both upwind cells are in the domain
 *                (the first two cells from each side keep Eq. (7)).  Order 2
 *                needs equal cell widths along each axis, no solid cells and
 *                no free-stream sides, holds two slices and two face planes
 *                per direction, and sweeps 128 velocities per thread block
 *                (KGS_EINVAL otherwise).
 *   dev_source   KGS_MIXED, order 1: 1 evaluates the FP32 sweep's source
 *                rtau (f^S - M_ref) from the small per-cell differences of the
 *                exponents of f^S and of the reference Maxwellian at rest
 *                (a 2^x - 1 series near the reference state), so that its
 *                rounding scales with the deviation from M_ref rather than
 *                with f: about 5 times lower residual floor of the mixed
 *                iteration, at about 1.2 times the sweep time.  Needs equal
 *                cell widths along each axis and no free-stream sides
 *                (KGS_EINVAL otherwise).  The order-2 FP32 sweep always uses
 *                this form; kgs_solve and kgs_batch_solve use it in their
 *                mixed phase wherever it applies. */
typedef struct {
    int precision;
    int wall_norm;
    int mass_rescale;
    int max_iters;
    double tol;
    int v_per_cta;
    int block_z;
    void *stream;
    int q_lagged;
    int vz_begin, vz_end;
    int order;
    int dev_source;
} kgs_opts;

/* Sizes and counters of a context. */
typedef struct {
    int nx, ny, nz, nvx, nvy, nvz;
    long long n_fluid;          /* fluid cells                                     */
    long long phase_points;     /* n_fluid * nvel: updates per outer iteration     */
    int iteration;              /* outer iterations done since setup / load        */
    int n_stages;               /* wavefront stages of the sweep (all in one launch) */
    int v_per_cta, block_z, precision;
    size_t device_bytes;        /* device memory held by the context               */
    double last_residual;
} kgs_info_t;

/* Build a context: copy the grids, mask and parameters to the device,
 * precompute per-velocity tables and start from the uniform state (the free
 * stream if any side is an inflow, else rho = 1, U = 0, T = 1, q = 0), with
 * wall densities from the flux of that state's equilibrium.
 * solid: nx*ny*nz bytes, 1 = solid cell, or NULL.
 * Errors: KGS_EINVAL (sizes < 1, non-positive widths or weights, Pr or omega
 * out of range, Kn = +inf together with a zero velocity node on every axis),
 * KGS_ENOMEM, KGS_ECUDA. */
int kgs_setup(kgs_ctx **out, const kgs_grid *grid, const uint8_t *solid, const kgs_vgrid *vgrid,
              const kgs_gas *gas, const kgs_bc *bc, const kgs_opts *opts);

/* Replace the macroscopic fields (host [8][nz][ny][nx]; NULL = the uniform
 * state of kgs_setup) and recompute the wall densities from the flux of the
 * new equilibrium (Section 2.2: the iteration starts from f^{S,0}).  Resets
 * the iteration counter and the reference mass used by mass_rescale. */
int kgs_set_initial(kgs_ctx *ctx, const double *macros);

/* Run outer iterations.  n_iters > 0: exactly n_iters iterations.
 * n_iters <= 0: until residual < opts.tol or opts.max_iters iterations.
 * *done (may be NULL) receives the number of iterations run, *residual
 * (may be NULL) the last residual (Section 4.1 reading: the largest relative
 * L2 change of rho, rho Ux, rho Uy, rho Uz, rho E over fluid cells, each
 * denominator floored at 1e-8 ||rho||_2).
 * Each iteration is one persistent sweep launch over the context's work items
 * (octant, velocity group, 8x8xblock_z block) in wavefront order; a thread
 * block waits with a bounded poll for the three upwind blocks of its item.
 * Returns KGS_OK, KGS_NOTCONVERGED (n_iters <= 0 only), KGS_EDIVERGED
 * (the state is left at the offending iterate), KGS_ETIMEOUT (a bounded wait
 * gave up; the iteration's results are discarded), KGS_ECUDA. */
int kgs_iterate(kgs_ctx *ctx, int n_iters, int *done, double *residual);

/* Copy the current macroscopic fields to host memory out[8*nz*ny*nx]
 * (solid cells hold 0).  Synchronises the context's stream. */
int kgs_moments(kgs_ctx *ctx, double *out);

/* Same, into device memory out_dev[8*nz*ny*nx] on the context's device;
 * asynchronous on the context's stream. */
int kgs_moments_device(kgs_ctx *ctx, double *out_dev);

/* Wall densities, host out[6*nz*ny*nx] (see the layout above). */
int kgs_rho_w(kgs_ctx *ctx, double *out);

/* Overwrite the wall densities (host in[6*nz*ny*nx]); entries of faces that
 * are not walls are ignored. */
int kgs_set_rho_w(kgs_ctx *ctx, const double *in);

/* Checkpoint.  The whole solver state is the macroscopic fields, the wall
 * densities, the reference mass and the iteration counter (the distribution
 * is never stored).  kgs_save with buf = NULL sets *len to the size needed;
 * otherwise it writes *len bytes.  kgs_load restores a buffer written by a
 * context of the same sizes (KGS_EFORMAT otherwise); iterating after a load
 * reproduces an uninterrupted run bit for bit. */
int kgs_save(kgs_ctx *ctx, void *buf, size_t *len);
int kgs_load(kgs_ctx *ctx, const void *buf, size_t len);

int kgs_info(kgs_ctx *ctx, kgs_info_t *out);

/* Sweep-kernel timing for roofline reports: when enabled, CUDA events are
 * recorded on the context's stream around every sweep launch; kgs_profile
 * returns the summed device time (ms) and the number of sweep launches since
 * the last reset, and resets the counters.  Synchronises the stream. */
int kgs_set_profiling(kgs_ctx *ctx, int enable);
int kgs_profile(kgs_ctx *ctx, double *sweep_ms, long long *sweep_launches, long long *kernel_launches);

/* ---- velocity-space partition ----
 * Within an outer iteration the velocities are independent (Eq. (6) lags
 * f^S, tau and rho_w), so the sweep splits over velocity ranges whose moment
 * sums are added before the closure: the paper's MPI CPU twin sums its
 * ranges with MPI_Allreduce (Section 5).  Each part is a context made with
 * kgs_opts.vz_begin / vz_end on the same problem and state.
 *
 * kgs_sweep_sums: the coefficient, sweep and moment kernels of one outer
 * iteration over this context's velocities, without the closure; writes the
 * per-cell sums to sums_dev[19][nz][ny][nx] (device, FP64, caller-owned): the
 * 13 sums about the lagged velocity U^n (as rounded to the sweep precision)
 * -- S0, S1 x y z, S2 xx yy zz xy xz yz, S3 x y z, with S_a = sum w f c^a,
 * c = xi - U^n and S3_i = sum w f c_i |c|^2 -- then the incoming flux onto
 * the wall on each side -x, +x, -y, +y, -z, +z (Eq. (9)).  The state does not
 * change.  Synchronises the context's stream.
 *
 * kgs_close_sums: the closure of the outer iteration from sums_dev (device,
 * the element-wise sum of every part's kgs_sweep_sums, same layout):
 * macroscopic fields of Eq. (5), wall densities of Eq. (9), mass rescale and
 * residual as kgs_iterate; advances the state by one iteration.  *residual
 * (may be NULL) receives the residual.  Returns KGS_OK, KGS_EDIVERGED,
 * KGS_ECUDA. */
int kgs_sweep_sums(kgs_ctx *ctx, double *sums_dev);
int kgs_close_sums(kgs_ctx *ctx, const double *sums_dev, double *residual);

void kgs_destroy(kgs_ctx *ctx);
const char *kgs_strerror(int code);

/* ---- batches of independent problems ----
 * Many instances (e.g. cavities of uneven grid and velocity sizes) advanced
 * together.  Each outer iteration of the batch is one persistent sweep launch
 * over the work items of every active instance (instance, octant, velocity
 * group, block, in wavefront-stage order; a thread block waits, with a
 * bounded spin, for the three upwind blocks of its item), wrapped with the
 * per-instance coefficient and closure kernels and replayed as a CUDA graph.
 * Iterates exactly like kgs_iterate on each instance (same arithmetic, same
 * results). */
typedef struct kgs_batch kgs_batch;

typedef struct {
    kgs_grid grid;
    const uint8_t *solid;     /* nx*ny*nz bytes or NULL */
    kgs_vgrid vgrid;
    kgs_gas gas;
    kgs_bc bc;
    int wall_norm;            /* KGS_WALL_DISCRETE / KGS_WALL_ANALYTIC */
    int mass_rescale;
    int q_lagged;             /* as kgs_opts.q_lagged */
} kgs_problem;

/* Sweep shape (velocities per thread block, block depth along z) of one
 * problem, chosen by timing a few outer iterations of each candidate on the
 * current device; cached per problem shape in the process and, when the
 * environment variable KGS_AUTOTUNE_CACHE names a file, in that file.
 * Allocates and frees a context per candidate. */
int kgs_autotune(const kgs_problem *prob, int precision, int *v_per_cta, int *block_z);

/* Build a batch of n instances (inputs copied; each instance starts from the
 * uniform state like kgs_setup).  opts: precision, tol, max_iters, stream;
 * v_per_cta = block_z = 0 asks kgs_autotune for the shape of the largest
 * instance, which then applies to all; wall_norm, mass_rescale and q_lagged
 * come from each kgs_problem.  Errors as kgs_setup. */
int kgs_batch_setup(kgs_batch **out, int n, const kgs_problem *probs, const kgs_opts *opts);

/* n_iters > 0: exactly n_iters outer iterations of every instance.
 * n_iters <= 0: iterate until every instance is below opts.tol (instances
 * retire from the work list as they converge) or max_iters iterations.
 * iters_done[n], residuals[n] (host, may be NULL): iterations run in this
 * call and last residual, per instance.  Returns KGS_OK, KGS_NOTCONVERGED,
 * KGS_EDIVERGED, KGS_ETIMEOUT (a bounded wait gave up; the batch state is
 * undefined), KGS_ECUDA. */
int kgs_batch_iterate(kgs_batch *b, int n_iters, int *iters_done, double *residuals);

/* Per-instance access: macroscopic fields to host (as kgs_moments), a new
 * initial state (as kgs_set_initial; the instance rejoins the work list),
 * sizes and counters (as kgs_info). */
int kgs_batch_moments(kgs_batch *b, int i, double *out);
int kgs_batch_set_initial(kgs_batch *b, int i, const double *macros);
int kgs_batch_info(kgs_batch *b, int i, kgs_info_t *out);

/* Summed device time (ms) of the persistent sweep launches, their number and
 * the number of kernel launches since the last call; resets the counters. */
int kgs_batch_profile(kgs_batch *b, double *sweep_ms, long long *sweeps, long long *kernel_launches);

/* Solve every instance to opts.tol as kgs_solve does one problem: a mixed
 * batch iterates each instance in chunks of 5 until its residual reaches
 * opts.tol or stops falling (the same rule as kgs_solve), and the instance
 * then retires from the mixed work list; an FP64 batch continues every
 * instance from its mixed state (macros, wall densities, mass target) until
 * its residual is below opts.tol, retiring instances as they converge.  An
 * instance may run at most opts.max_iters iterations in all (at least one in
 * FP64).  opts.precision is ignored; v_per_cta / block_z shape the mixed
 * batch (0: autotuned), the FP64 batch takes 128 velocities per thread block
 * and opts.block_z (0: 32).  *out receives the FP64 batch holding the
 * results (kgs_batch_moments, kgs_batch_info; destroy with
 * kgs_batch_destroy).  iters_mixed[n], iters_fp64[n], residuals[n] (host,
 * may be NULL): iterations per phase and final residual of each instance.
 * Returns KGS_OK, KGS_NOTCONVERGED (some instance ended above tol; *out is
 * still set), or the errors of kgs_batch_setup / kgs_batch_iterate (*out =
 * NULL). */
int kgs_batch_solve(kgs_batch **out, int n, const kgs_problem *probs, const kgs_opts *opts, int *iters_mixed,
                    int *iters_fp64, double *residuals);

/* Failure-detection controls (for tests): spin_limit = polls (about 100 ns
 * each) before a wait for an upwind block gives up (default 2e7, about 2 s);
 * unpublished_item >= 0 makes that work item of the list never announce its
 * completion, so the items that depend on it time out and the next
 * kgs_batch_iterate returns KGS_ETIMEOUT; -1 restores normal operation.  No
 * device fault is raised: the waiting thread blocks record the error and
 * return, and the batch stays usable after kgs_batch_set_initial. */
int kgs_batch_fault(kgs_batch *b, long long spin_limit, int unpublished_item);
void kgs_batch_destroy(kgs_batch *b);

/* ---- solve to a tolerance: mixed precision, then FP64 ----
 * The FP32 form of the iteration settles into rounding noise around its
 * fixed point, so its residual stops falling at a floor (about 3e-5 on the
 * cavity's spanwise momentum, about 1e-6 with the deviation-form source the
 * mixed phase uses on wall-bounded uniform grids).  kgs_solve runs mixed
 * iterations in chunks of 5 while the residual keeps falling (below 0.9 x its
 * best value within twenty chunks while it is above 1e-3, within six chunks
 * down to 3e-6, within two chunks below: at small Kn the residual falls with
 * bumps of about 25 iterations), then continues
 * in FP64 from the mixed state (macros, wall
 * densities and mass target carried over as by kgs_save / kgs_load) until
 * the residual is below tol or max_iters iterations ran in all.
 * initial: host [8][nz][ny][nx] or NULL (uniform state).  macros_out: host,
 * caller-owned, [8][nz][ny][nx], may be NULL.  iters_mixed, iters_fp64,
 * residual: host, may be NULL.  Allocates two contexts on `stream` for the
 * duration of the call.  Returns KGS_OK, KGS_NOTCONVERGED, or the errors of
 * kgs_setup / kgs_iterate. */
int kgs_solve(const kgs_problem *prob, const double *initial, double tol, int max_iters, double *macros_out,
              int *iters_mixed, int *iters_fp64, double *residual, void *stream);

/* ---- learned initial guess ----
 * The paper starts every solve from a uniform state and notes that the
 * iteration converges slowly at small Knudsen number (Section 4.1); this
 * library adds a learned starting field.  A stack of 3x3x3 convolutions
 * (zero padding, bias, ReLU between layers) maps 11 channels per cell --
 * log Kn, 10 U_lid, the solid flag and the normalised trilinear upsampling of
 * a coarse-grid solution -- to a normalised correction of the 8 macroscopic
 * fields over that upsampling.  Normalisation of field c (order rho, Ux, Uy,
 * Uz, T, qx, qy, qz): n_c = s_c (m_c - r_c) with r = (1,0,0,0,1,0,0,0) and
 * s = (10,10,10,10,50,100,100,100); corrections are scaled by s_c alone.
 *
 * Tensors are device arrays, channels last: x[B][D][H][W][C] with D = nz,
 * H = ny, W = nx.  Weights and stored activations are bfloat16, products
 * accumulate in FP32 on the tensor cores; the master parameters and Adam
 * moments are FP32.  Channel counts are at most 112.  A network is bound to
 * the device current at creation and works on `stream` (NULL = legacy
 * default stream); calls are ordered on that stream and kgs_net_forward,
 * kgs_net_train_step and the functions that return host values synchronise
 * it.  The convolutions run on the tensor cores with bounded waits; a wait
 * that gives up makes kgs_net_forward / kgs_net_train_step return
 * KGS_ETIMEOUT (no parameter update is made).  Parameter layout on the host (get/set):
 * per layer W[27][Cout][Cin] (tap t = (kz*3 + ky)*3 + kx reads the input at
 * offset (kz-1, ky-1, kx-1)) followed by b[Cout], FP32. */
typedef struct kgs_net kgs_net;

/* channels[n_layers + 1]: input, hidden..., output.  Weights He-normal from
 * a splitmix64 stream seeded by `seed` (the last layer scaled by 0.1), biases
 * zero.  KGS_EINVAL for a channel count outside [1, 112]. */
int kgs_net_create(kgs_net **out, int n_layers, const int *channels, unsigned long long seed, void *stream);
/* Parameter counts without and with the padding of channels to 16. */
int kgs_net_num_params(kgs_net *net, long long *real, long long *padded);
/* what = 0: parameters, 1: gradients of the last kgs_net_train_step; host. */
int kgs_net_get(kgs_net *net, int what, float *host);
/* Replace the parameters (host) and reset the optimiser state. */
int kgs_net_set_params(kgs_net *net, const float *host);
/* y[B][D][H][W][Cout] (FP32, device) for x[B][D][H][W][Cin] (FP32, device). */
int kgs_net_forward(kgs_net *net, const float *x, int B, int D, int H, int W, float *y);
/* One training step on the mean squared error over the voxels with
 * mask != 0 (mask: device bytes [B][D][H][W], NULL = all) and the output
 * channels, target[B][D][H][W][Cout] (FP32, device): forward, backward,
 * then Adam (beta 0.9 / 0.999, eps 1e-8) with step lr; lr <= 0 computes the
 * gradients only.  *loss (host, may be NULL) receives the loss of the
 * parameters before the update. */
int kgs_net_train_step(kgs_net *net, const float *x, const float *target, const uint8_t *mask, int B, int D, int H,
                       int W, float lr, float *loss);
void kgs_net_destroy(kgs_net *net);

/* Features of one instance: coarse[8][nzc][nyc][nxc] (device FP64, a
 * solution on a grid of equal-width cells covering the same box) is
 * upsampled trilinearly between cell centres (clamped at the outer centres)
 * to up[8][nz][ny][nx] (device FP64); x[nz][ny][nx][11] (device FP32)
 * receives (log kn, 10 u_lid, solid flag, normalised up).  solid: device
 * bytes [nz][ny][nx] or NULL. */
int kgs_surrogate_features(int nx, int ny, int nz, int nxc, int nyc, int nzc, const double *coarse,
                           const uint8_t *solid, double kn, double u_lid, float *x, double *up, void *stream);
/* Training target[ncell][8] = s_c (fine - up) (device; fine, up [8][ncell]). */
int kgs_surrogate_target(long long ncell, const double *fine, const double *up, float *target, void *stream);
/* Initial guess macros[8][ncell] = up + y / s_c (device), y[ncell][8] the
 * network output; *n_bad (host) receives the number of cells whose guess is
 * not a physical state (non-finite, rho <= 0 or T <= 0): a caller rejects
 * such a guess and starts from the uniform state.  Synchronises `stream`. */
int kgs_surrogate_apply(long long ncell, const double *up, const float *y, double *macros, int *n_bad, void *stream);

/* ---- iteration without device allocation ----
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory themselves or through this library:
 * code running inside a framework whose pool owns all device memory, code on
 * a latency-critical path that cannot afford cudaMalloc's implicit
 * synchronisation, or code that must never allocate after start-up.
 *
 * One outer iteration of the problem described by the same structs as
 * kgs_setup, from the state (macros_in [8][nz][ny][nx], rho_w_in
 * [6][nz][ny][nx], device, FP64) to (macros_out, rho_w_out, device, FP64,
 * caller-owned, distinct from the inputs), on `stream` (cudaStream_t, NULL =
 * legacy default stream) of the current device.  M0 > 0 multiplies the new
 * density, heat flux and wall densities by one common factor so that the
 * total mass (sum of density times cell volume over the fluid cells) equals
 * M0; M0 <= 0 leaves them unscaled.  precision and wall_norm as in kgs_opts;
 * the velocities per thread block and the block depth take their defaults.
 * *residual (host, may be NULL) receives the step's convergence measure: the
 * largest relative L2 change between input and output of the density, the
 * three momentum components and the total energy density over the fluid
 * cells, as kgs_iterate reports it.
 *
 * The call copies small tables from host memory, launches the iteration and
 * reads the residual back, then blocks the host until the iteration has
 * finished on the GPU.  Those copies and that wait cannot be recorded in a
 * CUDA graph: the call must never be made while `stream` (or the device) is
 * being captured.
 *
 * No cudaMalloc, cudaFree or other allocating routine is called: every
 * intermediate buffer lives in one file-scope device array of
 * KGS_NOALLOC_SCRATCH_BYTES bytes that every GPU loading this library holds
 * until the process exits.  Problems whose buffers do not fit are rejected
 * with KGS_EINVAL (roughly: face planes (nx ny + ny nz + nz nx) * nvel and
 * moment partials 8 * 16 * ncell * ceil(nvel_octant / 128) words must fit).
 * The first call on a device looks up the array's device address (once per
 * device).  All calls share the array and each call overwrites it: calls
 * that overlap on the GPU (concurrent streams or host threads) race and must
 * be serialised by the caller.
 * Returns KGS_OK, KGS_EDIVERGED (outputs hold the offending iterate),
 * KGS_EINVAL, KGS_ECUDA. */
#define KGS_NOALLOC_SCRATCH_BYTES (64u << 20)
int kgs_iterate_noalloc(const kgs_grid *grid, const uint8_t *solid, const kgs_vgrid *vgrid, const kgs_gas *gas,
                        const kgs_bc *bc, int precision, int wall_norm, double M0, const double *macros_in,
                        const double *rho_w_in, double *macros_out, double *rho_w_out, double *residual,
                        void *stream);

#ifdef __cplusplus
}
#endif
#endif
