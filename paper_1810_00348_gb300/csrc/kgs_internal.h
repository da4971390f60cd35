// kgs_internal.h -- device-side data layouts and launch interfaces shared by
// the CUDA translation units of libkgs.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kgs {

// Spatial sweep block: BX x BY cells in the XY plane (compile time), a
// run-time number of cells along z.  The XY slice of every in-flight velocity
// stays in shared memory while the block marches along z (Section 3.2's slice
// marching, one slice updated in place).
constexpr int BX = 8;
constexpr int BY = 8;
constexpr int SLICE = BX * BY;
constexpr int NT = 128;          // threads per sweep CTA
constexpr int NCOEF = 16;        // per-cell coefficient record
constexpr int NPART = 16;        // per-cell partial: 13 moment sums + 3 wall fluxes

// Per-cell coefficient record (computed from the lagged FP64 macros each
// iteration, stored in the sweep precision).  U^n below is the lagged velocity
// as rounded to the sweep precision: the centre of c = xi - U^n for the
// moments.  The equilibrium is evaluated from s = |xi|^2 - 2 U^n . xi, which
// is |c|^2 - |U^n|^2; the |U^n|^2 terms are folded into the constants below.
enum {
    C_M2UX = 0, C_M2UY, C_M2UZ,  // -2 U^n (exactly twice the centre, negated)
    C_KAPPA,                // (1/tau) rho (2 pi R T)^{-3/2} exp(-|U^n|^2 / (2RT)); FP32: its base-2 logarithm
    C_NEXP,                 // exponent scale: -1/(2RT) (FP64) or -log2(e)/(2RT) (FP32)
    C_RT1,                  // 1/(R T)
    C_RTAU,                 // 1/tau
    C_FLAGS,                // cell flags (below), their bits stored in the value (flag_value)
    C_QX, C_QY, C_QZ,       // q' = (1 - Pr) q / (5 p R T)
    C_RDX, C_RDY, C_RDZ,    // 1/dx_i, 1/dy_j, 1/dz_k (FP32 second-order sweep, uniform grid:
                            // C_RDX, C_RDY hold the exponent terms of its deviation source)
    C_SHK0,                 // |U^n|^2 / (R T) - 5, so that |c|^2/(RT) - 5 = s/(RT) + C_SHK0
    C_MUQ                   // -U^n . q'
};

// Cell flags.
constexpr int F_SOLID = 1;               // the cell itself is solid
constexpr int F_SOLID_SIDE = 2;          // << s: the neighbour on side s is solid
constexpr int F_WALL_SIDE = 1 << 7;      // << s: face on side s is a diffuse wall

// Partial-sum slots per (velocity group, cell): the 13 sums about U^n
// (S0, S1xyz, S2 xx yy zz xy xz yz, S3xyz) and the incoming flux onto the
// wall ahead of the octant along x, y, z.
enum {
    P_S0 = 0, P_S1X, P_S1Y, P_S1Z, P_S2XX, P_S2YY, P_S2ZZ, P_S2XY, P_S2XZ, P_S2YZ,
    P_S3X, P_S3Y, P_S3Z, P_FX, P_FY, P_FZ
};

// Per-cell sums of one outer iteration as the closure reads them ([NSUM][ncell],
// FP64): the 13 sums about U^n in the P_* order, then the incoming flux onto
// the wall on each domain side s (-x, +x, -y, +y, -z, +z) at slot SUM_F0 + s.
constexpr int SUM_F0 = 13;
constexpr int NSUM = 19;
// Ordered accumulators of the persistent sweep: [nacc][ncell][acc_slots] (FP64,
// or float-float pairs (hi, lo) for the FP32 path).  ACC_COMPACT slots: the
// 13 sums, then one incoming flux per axis -- the flux onto the only wall a
// cell has along that axis -- the layout of an item's partials, so that an
// item adds its record element-wise.  ACC_SPLIT slots: the 13 sums, then one
// flux per side (slot SUM_F0 + side), for problems where some cell has walls
// on both sides along an axis.
constexpr int ACC_COMPACT = 16;
constexpr int ACC_SPLIT = 20;
constexpr int NACC_MAX = 8;  // accumulators per instance, at most

// Reference Maxwellian of the FP32 sweep, which carries g = f - M_ref rather
// than f: the moments of the FP32 table values of M_ref over the swept
// velocities, raw[a][b][c] = sum w M_ref xi_x^a xi_y^b xi_z^c (a + b + c <= 3,
// index ref_index), and their incoming flux onto each domain side.  All zero
// for the FP64 path, which carries f itself.
constexpr int NREF = 20;
__host__ __device__ constexpr int ref_index(int a, int b, int c)
{
    // a + b + c = n occupies [n (n+1) (n+2) / 6, ...), ordered by (b + c, c)
    return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}
struct RefMoments {
    double raw[NREF];
    double flux[6];
};

// Wall-Maxwellian table rows: 0..5 domain side, 6 solid surface, 7 free stream.
constexpr int MT_SOLID = 6;
constexpr int MT_INFLOW = 7;
constexpr int MT_ROWS = 8;

struct SweepArgs {
    int nx, ny, nz, bz;           // grid, block extent along z
    int nbx, nby, nbz;            // blocks per axis
    const int4 *work;             // per CTA row: octant, reflected block coords
    const int *oct_vstart;        // [8] first sorted velocity of each octant
    const int *oct_vcount;        // [8] velocities per octant
    const int *oct_vgbase;        // [8] first global velocity-group index
    int Nv;                       // all velocities
    int vg_size;                  // velocities per CTA
    const void *vel;              // Real[Nv][4]: xi_x, xi_y, xi_z, w (octant-sorted)
    const void *velm;             // Real[Nv][8]: w_x, w_y w_z, the low parts of xi_x, xi_y, xi_z
                                  // (xi = hi + lo with hi = the value in vel), M_ref (FP32
                                  // path; 0 for FP64), the rounding error of M_ref (FP32
                                  // path), 1 unused
    int oct_nx[8];                // x nodes in each octant (length of its velocity x-lines)
    int nxo_max;                  // max over octants of oct_nx
    int any_solid;                // the problem has solid cells
    const uint8_t *blk_plain;     // [nbz][nby][nbx]: 1 = no solid cell and no solid neighbour in the block (or NULL)
    const void *coef;             // Real[ncell][NCOEF]
    const double *rho_w;          // [6][ncell]
    const void *mtab;             // Real[MT_ROWS][Nv]: unit wall Maxwellians, free stream
    int side_inflow[6];           // domain side s is a free-stream boundary
    void *FX, *FY, *FZ;           // face planes: [nz*ny][Nv], [nz*nx][Nv], [ny*nx][Nv]
    int order;                    // upwind order of the sweep (1: Eq. (7), 2: three-point differences)
    void *FX2, *FY2, *FZ2;        // order 2: the planes one cell further upwind (same shapes)
    void *part;                   // staged sweep: [n_vg][ncell][NPART], double (FP64 path) or
                                  // float2 (s, c) with value s - c (FP32 path, Kahan pair)
    void *acc;                    // persistent sweep: [nacc][ncell][acc_slots] ordered accumulators
    int nacc;                     // accumulators: velocity group g of an octant adds into g % nacc
    int acc_slots;                // ACC_COMPACT or ACC_SPLIT
    int *tok;                     // persistent sweep: [nacc][nbz][nby][nbx] chain tokens
    unsigned long long ncell;
    int line16;                   // every octant has x-lines of 16 nodes (specialised moment loop)
    int uniform;                  // equal cell widths along each axis: a_d is per velocity
    double rd0[3];                // 1/dx, 1/dy, 1/dz of a uniform grid
};

// Persistent sweep over the work items of many instances (one launch per
// outer iteration): item = (instance, octant << 24 | velocity group of the
// octant, reflected block coordinates bx | by << 10 | bz << 20, global
// velocity-group index within the instance), list ordered by stage.
struct BatchSweepArgs {
    const SweepArgs *inst;        // [n_inst] per-instance arguments (device)
    const int4 *items;
    int n_items;
    int *counter;                 // claim counter, zero at launch
    int *flags;                   // completion flags, zero at launch
    const int *flag_off;          // [n_inst] first flag of each instance
    const int *pos;               // [n_items] place of each item in its accumulator chain
    void *scratch;                // [grid][bz * SLICE][NPART] per-CTA moment partials
    unsigned long long scratch_stride;  // bytes of one CTA's scratch, sweep_scratch_bytes(bz)
    int *error;                   // set to 1 when a bounded wait gives up
    long long spin_limit;         // polls before a wait gives up
    int skip_publish;             // fault injection: this item never sets its flag (-1: none)
};
// Bytes of one CTA's scratch partials for blocks bz cells deep (both precisions
// store 8 bytes per slot).
inline size_t sweep_scratch_bytes(int bz) { return (size_t)bz * SLICE * NPART * 8; }

// Cell flags travel in the coefficient array as the bit pattern of a Real
// (no conversion instruction on either side).
__host__ __device__ inline float flag_value_f(int f)
{
    union {
        int i;
        float v;
    } u;
    u.i = f;
    return u.v;
}
__host__ __device__ inline double flag_value_d(int f)
{
    union {
        long long i;
        double v;
    } u;
    u.i = f;
    return u.v;
}
template <typename Real>
__host__ __device__ inline Real flag_value(int f);
template <>
__host__ __device__ inline float flag_value<float>(int f)
{
    return flag_value_f(f);
}
template <>
__host__ __device__ inline double flag_value<double>(int f)
{
    return flag_value_d(f);
}
__device__ __forceinline__ int flag_bits(float v) { return __float_as_int(v); }
__device__ __forceinline__ int flag_bits(double v) { return (int)__double_as_longlong(v); }

// order: upwind order of the sweep; order 2 exists for tv = 1 on uniform
// grids only.  dev: the first-order FP32 sweep with the deviation-form source
// (uniform grids).  Other combinations: 0 CTAs per SM / cudaErrorInvalidValue.
cudaError_t launch_sweep_persistent(int precision, int tv, int line16, int uniform, const BatchSweepArgs &b, int nxo_max,
                                    int grid, cudaStream_t s, int order = 1, int dev = 0);
// Resident CTAs per SM of the persistent kernel (also sets its shared-memory limit).
int sweep_persistent_occupancy(int precision, int tv, int line16, int uniform, size_t smem, int order = 1,
                               int dev = 0);

// Sweep launch (one wavefront stage, order 1).  precision: 0 FP64, 1 FP32.
cudaError_t launch_sweep(int precision, int tv, const SweepArgs &a, int n_items, int max_vg, cudaStream_t s);
size_t sweep_smem_bytes(int precision, int tv, int line16, int nxo_max, int order = 1);

// Per-cell sums of the staged sweep's per-group partials (fixed group order).
struct PartSumArgs {
    unsigned long long ncell;
    int n_vg;
    const int *vg_oct;            // [n_vg] octant of each velocity group
    const void *part;             // [n_vg][ncell][NPART], see SweepArgs::part
    int precision;
    const uint8_t *solid;         // [ncell] or NULL
    double *sums;                 // [NSUM][ncell]
    const void *coef;             // sweep-precision coefficients (U centre)
    const int8_t *wall_kind;      // [6][ncell]
    RefMoments ref;               // moments of the reference Maxwellian, added to every cell
};

struct ClosureArgs {
    int nx, ny, nz;
    unsigned long long ncell;
    const double *sums;           // [NSUM][ncell]
    const void *coef;             // sweep-precision coefficients (U centre)
    int precision;
    int q_lagged;                 // 1: q = S3 / 2 about the lagged U^n (no shift)
    double *mac_new;              // [8][ncell] step n+1 (before rescale)
    double *rho_w_new;            // [6][ncell]
    const int8_t *wall_kind;      // [6][ncell]: -1 not a wall, 0..6 wall kind
    const double *wall_norm;      // [7][6] rho_w = F * wall_norm[kind][side]
    const double *dx, *dy, *dz;
    const uint8_t *solid;         // [ncell] or NULL
    double *blk_mass;             // [close_blocks(ncell)]
};

// dev_src (FP32 only): the C_RDX / C_RDY slots carry the exponent terms of
// the second-order sweep's deviation source instead of 1/dx, 1/dy.
cudaError_t launch_coef(int precision, const double *mac, const uint8_t *solid, const uint8_t *cell_flags_side,
                        const double *rdx, const double *rdy, const double *rdz, int nx, int ny, int nz,
                        double mu_ref, double omega, double Pr, void *coef, cudaStream_t s, int dev_src = 0);
// Cells per block of the closure kernel; blk_mass holds close_blocks(ncell)
// values.
constexpr int CLOSE_CELLS = 32;
inline size_t close_blocks(size_t ncell) { return (ncell + CLOSE_CELLS - 1) / CLOSE_CELLS; }
cudaError_t launch_part_sums(const PartSumArgs &a, cudaStream_t s);
// Per-cell sums of the persistent sweep's ordered accumulators (fixed order).
struct AccSumArgs {
    int precision;
    const void *acc;
    int nacc;
    int acc_slots;
    unsigned long long ncell;
    const uint8_t *solid;         // [ncell] or NULL
    double *sums;                 // [NSUM][ncell]
    const void *coef;             // sweep-precision coefficients (U centre)
    const int8_t *wall_kind;      // [6][ncell]
    RefMoments ref;
};
cudaError_t launch_acc_sums(const AccSumArgs &a, cudaStream_t s);
cudaError_t launch_closure(const ClosureArgs &a, cudaStream_t s);
cudaError_t launch_finalize_mass(const double *blk_mass, int n_blocks, double M0, int rescale, double *scale,
                                 cudaStream_t s);
cudaError_t launch_scale_residual(double *mac_new, double *rho_w_new, const double *mac, const uint8_t *solid,
                                  unsigned long long ncell, const double *scale, double *blk_res, int *blk_bad,
                                  int n_blocks, cudaStream_t s);
cudaError_t launch_finalize_residual(const double *blk_res, const int *blk_bad, int n_blocks, double *out2,
                                     cudaStream_t s);
cudaError_t launch_wall_flux_init(const double *mac, const int8_t *wall_kind, const double *wall_norm,
                                  const double *axis64, int nvx, int nvy, int nvz, unsigned long long ncell, double R,
                                  double Pr,
                                  double *rho_w, cudaStream_t s);
cudaError_t launch_fill(double *p, unsigned long long n, double v, cudaStream_t s);

}  // namespace kgs
