// kgs_tables.h -- host-side tables of one problem (octant-sorted velocity
// tables, wall Maxwellians and normalisers, face flags, wavefront stages),
// built once from the public ABI structs and uploaded by the contexts.
// Not part of the public ABI.
#pragma once

#include <vector>

#include "../../include/kgs.h"
#include "kgs_internal.h"

namespace kgs {

constexpr double R_GAS = 0.5;  // velocity unit sqrt(2 R T0)

struct HostTables {
    int nx = 0, ny = 0, nz = 0, nvx = 0, nvy = 0, nvz = 0, Nv = 0;  // Nv: velocities swept by this context
    int vz0 = 0, vz1 = 0;                    // swept velocity planes iz in [vz0, vz1)
    int order = 1;                           // upwind order of the sweep (1 or 2)
    bool dev = false;                        // FP32 deviation-form source (order 2, or the option)
    size_t ncell = 0;
    long long n_fluid = 0;
    int precision = KGS_FP64, wall_norm_mode = KGS_WALL_DISCRETE;
    int tv = 1, vg_size = NT, bz = 16;
    double mu_ref = 0.0, omega = 0.81, Pr = 2.0 / 3.0;
    bool any_solid = false, any_inflow = false;
    int side_inflow[6] = {0};
    kgs_bc bc{};
    // velocities sorted by octant (bit d set: xi_d >= 0), ix fastest
    int oct_vstart[8] = {0}, oct_vcount[8] = {0}, oct_vgbase[8] = {0}, oct_nx[8] = {0};
    int n_vg = 0, max_vg = 0, nxo_max = 1;
    int nacc = 1;                            // ordered accumulators of the persistent sweep
    int acc_slots = ACC_COMPACT;             // ACC_SPLIT if a cell has walls on both sides along an axis
    std::vector<int> vg_oct;                 // octant of each velocity group
    std::vector<double> vel64;               // [Nv][4] xi_x, xi_y, xi_z, w
    std::vector<double> axis64;              // 1D nodes and weights: xi_x, xi_y, xi_z, w_x, w_y, w_z
    std::vector<double> velm64;              // [Nv][8] w_x, w_y w_z, 0 ...
    std::vector<float> velm32;               // [Nv][8] w_x, w_y w_z, low parts of xi
    std::vector<double> mt;                  // [MT_ROWS][Nv] wall Maxwellians, free stream
    RefMoments ref{};                        // FP32 sweep: moments of the reference Maxwellian
    std::vector<double> wall_norm;           // [7][6] rho_w = F * wall_norm[kind][side]
    std::vector<int8_t> wall_kind;           // [6][ncell]
    std::vector<uint8_t> side_flags;         // [2][ncell]: solid-neighbour bits, wall-face bits
    std::vector<uint8_t> solid;              // [ncell] or empty
    std::vector<double> dx, dy, dz, rdx, rdy, rdz;
    // wavefront stages over 8 x 8 x bz blocks
    int nbx = 0, nby = 0, nbz = 0;
    std::vector<int> stage_off, stage_n;
    std::vector<int4> work;
    std::vector<uint8_t> blk_plain;          // [nbz][nby][nbx], problems with solid cells only
    size_t real_bytes() const { return precision == KGS_FP64 ? sizeof(double) : sizeof(float); }
    // Equal cell widths along each axis: the sweep then takes the upwind
    // coefficients a_d = abs(xi_d) / dx_d per velocity (sets a.uniform, a.rd0).
    void set_uniformity(SweepArgs &a) const
    {
        auto same = [](const std::vector<double> &v) {
            for (double x : v)
                if (x != v[0]) return false;
            return !v.empty();
        };
        a.uniform = same(rdx) && same(rdy) && same(rdz) ? 1 : 0;
        a.rd0[0] = rdx.empty() ? 0.0 : rdx[0];
        a.rd0[1] = rdy.empty() ? 0.0 : rdy[0];
        a.rd0[2] = rdz.empty() ? 0.0 : rdz[0];
    }
};

// Argument checks of kgs_setup (KGS_OK or KGS_EINVAL).
// vz_begin, vz_end: the velocity planes iz in [vz_begin, vz_end) of a
// velocity-space partition (0, 0: all of them).  order: upwind order of the
// sweep (0 or 1: Eq. (7); 2: three-point differences, which need equal widths
// along each axis, no solid cells and 128 velocities per thread block).
int validate_problem(const kgs_grid *grid, const uint8_t *solid, const kgs_vgrid *vg, const kgs_gas *gas,
                     const kgs_bc *bc, int precision, int wall_norm, int v_per_cta, int block_z, int vz_begin = 0,
                     int vz_end = 0, int order = 1, int dev_source = 0);

// The deviation-form FP32 source applies: equal widths along each axis and
// no free-stream side (the reference Maxwellian is the rest state).
bool dev_source_applies(const kgs_grid *grid, const kgs_bc *bc);

// Build every host table of a validated problem.
void build_tables(HostTables &t, const kgs_grid *grid, const uint8_t *solid, const kgs_vgrid *vg,
                  const kgs_gas *gas, const kgs_bc *bc, int precision, int wall_norm, int v_per_cta, int block_z,
                  int vz_begin = 0, int vz_end = 0, int order = 1, int dev_source = 0);

}  // namespace kgs
