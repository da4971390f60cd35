// kgs_tables.cu -- host-side problem tables (see kgs_tables.h).
#include "kgs_tables.h"

#include <algorithm>
#include <cmath>

namespace kgs {

namespace {

double maxwellian(double rho, const double U[3], double T, const double xi[3])
{
    double c2 = 0.0;
    for (int d = 0; d < 3; d++) c2 += (xi[d] - U[d]) * (xi[d] - U[d]);
    return rho / std::pow(2.0 * M_PI * R_GAS * T, 1.5) * std::exp(-c2 / (2.0 * R_GAS * T));
}

}  // namespace

bool dev_source_applies(const kgs_grid *grid, const kgs_bc *bc)
{
    for (int s = 0; s < 6; s++)
        if (bc->type[s] == KGS_FACE_INFLOW) return false;
    const double *w[3] = {grid->dx, grid->dy, grid->dz};
    const int n[3] = {grid->nx, grid->ny, grid->nz};
    for (int d = 0; d < 3; d++)
        for (int i = 1; i < n[d]; i++)
            if (w[d][i] != w[d][0]) return false;
    return true;
}

int validate_problem(const kgs_grid *grid, const uint8_t *solid, const kgs_vgrid *vg, const kgs_gas *gas,
                     const kgs_bc *bc, int precision, int wall_norm, int v_per_cta, int block_z, int vz_begin,
                     int vz_end, int order, int dev_source)
{
    if (!grid || !vg || !gas || !bc) return KGS_EINVAL;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !grid->dx || !grid->dy || !grid->dz) return KGS_EINVAL;
    if (vg->nvx < 1 || vg->nvy < 1 || vg->nvz < 1) return KGS_EINVAL;
    if (!vg->xi_x || !vg->xi_y || !vg->xi_z || !vg->w_x || !vg->w_y || !vg->w_z) return KGS_EINVAL;
    if (!(gas->Kn > 0.0) || !(gas->Pr > 0.0) || !(gas->omega >= 0.0 && gas->omega <= 1.5)) return KGS_EINVAL;
    if (precision != KGS_FP64 && precision != KGS_MIXED) return KGS_EINVAL;
    if (wall_norm != KGS_WALL_DISCRETE && wall_norm != KGS_WALL_ANALYTIC) return KGS_EINVAL;
    if (v_per_cta != 0 && v_per_cta != 128 && v_per_cta != 256) return KGS_EINVAL;
    if (precision == KGS_FP64 && v_per_cta == 256) return KGS_EINVAL;
    if (block_z < 0) return KGS_EINVAL;
    if (!(vz_begin == 0 && vz_end == 0) && !(vz_begin >= 0 && vz_begin < vz_end && vz_end <= vg->nvz))
        return KGS_EINVAL;
    const long long ncell = (long long)grid->nx * grid->ny * grid->nz;
    const long long nv = (long long)vg->nvx * vg->nvy * vg->nvz;
    if (ncell > (1LL << 31) || nv > (1LL << 24)) return KGS_EINVAL;
    for (int i = 0; i < grid->nx; i++) if (!(grid->dx[i] > 0.0)) return KGS_EINVAL;
    for (int i = 0; i < grid->ny; i++) if (!(grid->dy[i] > 0.0)) return KGS_EINVAL;
    for (int i = 0; i < grid->nz; i++) if (!(grid->dz[i] > 0.0)) return KGS_EINVAL;
    for (int i = 0; i < vg->nvx; i++) if (!(vg->w_x[i] > 0.0) || !std::isfinite(vg->xi_x[i])) return KGS_EINVAL;
    for (int i = 0; i < vg->nvy; i++) if (!(vg->w_y[i] > 0.0) || !std::isfinite(vg->xi_y[i])) return KGS_EINVAL;
    for (int i = 0; i < vg->nvz; i++) if (!(vg->w_z[i] > 0.0) || !std::isfinite(vg->xi_z[i])) return KGS_EINVAL;
    bool any_inflow = false, any_solid = false;
    for (int s = 0; s < 6; s++) {
        if (bc->type[s] != KGS_FACE_WALL && bc->type[s] != KGS_FACE_INFLOW) return KGS_EINVAL;
        if (bc->type[s] == KGS_FACE_WALL && !(bc->T_w[s] > 0.0)) return KGS_EINVAL;
        any_inflow |= bc->type[s] == KGS_FACE_INFLOW;
    }
    if (any_inflow && (!(bc->rho_in > 0.0) || !(bc->T_in > 0.0))) return KGS_EINVAL;
    if (solid)
        for (long long i = 0; i < ncell; i++) any_solid |= solid[i] != 0;
    if (any_solid && !(bc->T_solid > 0.0)) return KGS_EINVAL;
    if (order < 0 || order > 2 || dev_source < 0 || dev_source > 1) return KGS_EINVAL;
    if (dev_source && (precision != KGS_MIXED || !dev_source_applies(grid, bc))) return KGS_EINVAL;
    if (order == 2) {
        // the three-point difference assumes equal widths along each axis;
        // the kernel's second-order variant has no solid-cell path and keeps
        // two slices of 128 velocities in shared memory;
        // reference state at rest: no free-stream sides (the FP32 form's
        // deviation source is written about rho = 1, U = 0, T = 1)
        if (any_solid || any_inflow || v_per_cta == 256) return KGS_EINVAL;
        const double *w[3] = {grid->dx, grid->dy, grid->dz};
        const int n[3] = {grid->nx, grid->ny, grid->nz};
        for (int d = 0; d < 3; d++)
            for (int i = 1; i < n[d]; i++)
                if (w[d][i] != w[d][0]) return KGS_EINVAL;
    }
    if (std::isinf(gas->Kn)) {
        // free-molecular limit: a velocity with all components zero has no
        // equation (0 = 0); such grids are rejected
        bool zx = false, zy = false, zz = false;
        for (int i = 0; i < vg->nvx; i++) zx |= vg->xi_x[i] == 0.0;
        for (int i = 0; i < vg->nvy; i++) zy |= vg->xi_y[i] == 0.0;
        for (int i = 0; i < vg->nvz; i++) zz |= vg->xi_z[i] == 0.0;
        if (zx && zy && zz) return KGS_EINVAL;
    }
    return KGS_OK;
}

void build_tables(HostTables &t, const kgs_grid *grid, const uint8_t *solid, const kgs_vgrid *vg,
                  const kgs_gas *gas, const kgs_bc *bc, int precision, int wall_norm, int v_per_cta, int block_z,
                  int vz_begin, int vz_end, int order, int dev_source)
{
    t.nx = grid->nx;
    t.ny = grid->ny;
    t.nz = grid->nz;
    t.ncell = (size_t)t.nx * t.ny * t.nz;
    t.nvx = vg->nvx;
    t.nvy = vg->nvy;
    t.nvz = vg->nvz;
    t.vz0 = vz_end > 0 ? vz_begin : 0;
    t.vz1 = vz_end > 0 ? vz_end : t.nvz;
    t.Nv = t.nvx * t.nvy * (t.vz1 - t.vz0);
    t.precision = precision;
    t.wall_norm_mode = wall_norm;
    // defaults measured on the 64^3 x 32^3 cavity: two velocities per thread
    // and 32-cell-deep blocks for the FP32 sweep
    t.order = order == 2 ? 2 : 1;
    t.dev = precision == KGS_MIXED && (t.order == 2 || dev_source != 0);
    t.tv = (precision == KGS_FP64 || t.order == 2) ? 1 : (v_per_cta == 128 ? 1 : 2);
    t.vg_size = NT * t.tv;
    t.bz = block_z > 0 ? block_z : 32;
    t.omega = gas->omega;
    t.Pr = gas->Pr;
    // Eq. (10) with T_ref = 1, p_ref = rho_ref R T_ref = 1/2, lambda_ref = Kn
    t.mu_ref = 15.0 * std::sqrt(M_PI) * (R_GAS * 1.0) * gas->Kn /
               ((5.0 - 2.0 * gas->omega) * (7.0 - 2.0 * gas->omega) * std::sqrt(2.0 * R_GAS * 1.0));
    t.bc = *bc;
    t.any_inflow = false;
    for (int s = 0; s < 6; s++) {
        t.side_inflow[s] = bc->type[s] == KGS_FACE_INFLOW;
        t.any_inflow |= t.side_inflow[s] != 0;
    }
    t.any_solid = false;
    if (solid)
        for (size_t i = 0; i < t.ncell; i++) t.any_solid |= solid[i] != 0;
    if (t.any_solid) t.solid.assign(solid, solid + t.ncell);
    const size_t n = t.ncell;
    const int nx = t.nx, ny = t.ny, nz = t.nz;
    t.dx.assign(grid->dx, grid->dx + nx);
    t.dy.assign(grid->dy, grid->dy + ny);
    t.dz.assign(grid->dz, grid->dz + nz);
    t.rdx.resize(nx);
    t.rdy.resize(ny);
    t.rdz.resize(nz);
    for (int i = 0; i < nx; i++) t.rdx[i] = 1.0 / t.dx[i];
    for (int i = 0; i < ny; i++) t.rdy[i] = 1.0 / t.dy[i];
    for (int i = 0; i < nz; i++) t.rdz[i] = 1.0 / t.dz[i];

    // ---- velocities sorted by octant (bit d set: xi_d >= 0), ix fastest ----
    std::vector<int> vsorted;
    vsorted.reserve(t.Nv);
    auto oct_of = [&](int ix, int iy, int iz) {
        return (vg->xi_x[ix] >= 0.0 ? 1 : 0) | (vg->xi_y[iy] >= 0.0 ? 2 : 0) | (vg->xi_z[iz] >= 0.0 ? 4 : 0);
    };
    for (int o = 0; o < 8; o++) {
        t.oct_vstart[o] = (int)vsorted.size();
        for (int iz = t.vz0; iz < t.vz1; iz++)
            for (int iy = 0; iy < t.nvy; iy++)
                for (int ix = 0; ix < t.nvx; ix++)
                    if (oct_of(ix, iy, iz) == o) vsorted.push_back(ix + t.nvx * (iy + t.nvy * iz));
        t.oct_vcount[o] = (int)vsorted.size() - t.oct_vstart[o];
        int cnt = 0;
        for (int ix = 0; ix < t.nvx; ix++) cnt += ((vg->xi_x[ix] >= 0.0 ? 1 : 0) == (o & 1));
        t.oct_nx[o] = cnt;
        t.nxo_max = std::max(t.nxo_max, cnt);
    }
    t.axis64.clear();
    t.axis64.insert(t.axis64.end(), vg->xi_x, vg->xi_x + t.nvx);
    t.axis64.insert(t.axis64.end(), vg->xi_y, vg->xi_y + t.nvy);
    t.axis64.insert(t.axis64.end(), vg->xi_z, vg->xi_z + t.nvz);
    t.axis64.insert(t.axis64.end(), vg->w_x, vg->w_x + t.nvx);
    t.axis64.insert(t.axis64.end(), vg->w_y, vg->w_y + t.nvy);
    t.axis64.insert(t.axis64.end(), vg->w_z, vg->w_z + t.nvz);
    t.vel64.assign((size_t)t.Nv * 4, 0.0);
    t.velm64.assign((size_t)t.Nv * 8, 0.0);
    t.velm32.assign((size_t)t.Nv * 8, 0.f);
    for (int g = 0; g < t.Nv; g++) {
        const int a = vsorted[g];
        const int ix = a % t.nvx, iy = (a / t.nvx) % t.nvy, iz = a / (t.nvx * t.nvy);
        t.vel64[g * 4 + 0] = vg->xi_x[ix];
        t.vel64[g * 4 + 1] = vg->xi_y[iy];
        t.vel64[g * 4 + 2] = vg->xi_z[iz];
        t.vel64[g * 4 + 3] = vg->w_x[ix] * vg->w_y[iy] * vg->w_z[iz];
        // moment-phase factors: w_x, w_y w_z and, for the FP32 path, the low
        // parts of the nodes (xi = (float)xi + lo)
        t.velm64[g * 8 + 0] = vg->w_x[ix];
        t.velm64[g * 8 + 1] = vg->w_y[iy] * vg->w_z[iz];
        t.velm32[g * 8 + 0] = (float)vg->w_x[ix];
        t.velm32[g * 8 + 1] = (float)(vg->w_y[iy] * vg->w_z[iz]);
        for (int d = 0; d < 3; d++) {
            const double x = t.vel64[g * 4 + d];
            t.velm32[g * 8 + 2 + d] = (float)(x - (double)(float)x);
        }
    }
    t.vg_oct.clear();
    t.max_vg = 0;
    for (int o = 0; o < 8; o++) {
        t.oct_vgbase[o] = (int)t.vg_oct.size();
        const int ng = (t.oct_vcount[o] + t.vg_size - 1) / t.vg_size;
        for (int g = 0; g < ng; g++) t.vg_oct.push_back(o);
        t.max_vg = std::max(t.max_vg, ng);
    }
    t.n_vg = (int)t.vg_oct.size();
    // accumulators: velocity group g of an octant adds into g % nacc, and
    // every accumulator must receive a group of every block, so nacc is at
    // most the smallest group count of a non-empty octant
    t.nacc = NACC_MAX;
    for (int o = 0; o < 8; o++)
        if (t.oct_vcount[o] > 0) t.nacc = std::min(t.nacc, (t.oct_vcount[o] + t.vg_size - 1) / t.vg_size);

    // ---- wall tables: kinds 0..5 domain sides, 6 solid surfaces ----
    double wallU[7][3], wallT[7];
    for (int s = 0; s < 6; s++) {
        for (int d = 0; d < 3; d++) wallU[s][d] = bc->U_w[s][d];
        wallT[s] = bc->type[s] == KGS_FACE_WALL ? bc->T_w[s] : 1.0;
    }
    wallU[6][0] = wallU[6][1] = wallU[6][2] = 0.0;
    wallT[6] = t.any_solid ? bc->T_solid : 1.0;
    t.wall_norm.assign(7 * 6, 0.0);
    for (int k = 0; k < 7; k++)
        for (int s = 0; s < 6; s++) {
            if (wall_norm == KGS_WALL_ANALYTIC) {
                t.wall_norm[k * 6 + s] = std::sqrt(2.0 * M_PI / (R_GAS * wallT[k]));
                continue;
            }
            // discrete outgoing flux of the unit wall Maxwellian, over every
            // velocity of the grid (also when this context sweeps a part)
            const int d = s / 2;
            const double nrm = (s % 2) ? -1.0 : 1.0;
            double D = 0.0;
            for (int iz = 0; iz < t.nvz; iz++)
                for (int iy = 0; iy < t.nvy; iy++)
                    for (int ix = 0; ix < t.nvx; ix++) {
                        const double v[3] = {vg->xi_x[ix], vg->xi_y[iy], vg->xi_z[iz]};
                        const double xn = v[d] * nrm;
                        if (xn > 0.0)
                            D += vg->w_x[ix] * vg->w_y[iy] * vg->w_z[iz] * xn * maxwellian(1.0, wallU[k], wallT[k], v);
                    }
            t.wall_norm[k * 6 + s] = D > 0.0 ? 1.0 / D : 0.0;
        }
    // FP32 sweep: the reference Maxwellian is the uniform state the solve
    // starts from (the free stream if a side is an inflow, else rho = 1,
    // U = 0, T = 1); its FP32 values go into the velocity table and the
    // moments of exactly those values, in FP64, into t.ref.  On the inflow
    // faces the reference equals the ghost, so their deviation is zero.
    t.ref = RefMoments{};
    if (precision == KGS_MIXED) {
        double refU[3] = {0.0, 0.0, 0.0}, refT = 1.0, refRho = 1.0;
        if (t.any_inflow) {
            refRho = bc->rho_in;
            refT = bc->T_in;
            for (int d = 0; d < 3; d++) refU[d] = bc->U_in[d];
        }
        for (int g = 0; g < t.Nv; g++) {
            const double *v = &t.vel64[g * 4];
            const double m64 = maxwellian(refRho, refU, refT, v);
            const float m32 = (float)m64;
            t.velm32[g * 8 + 5] = m32;
            t.velm32[g * 8 + 6] = (float)(m64 - (double)m32);  // its rounding error (second-order sweep)
            const double wm = v[3] * (double)m32;
            for (int a = 0; a <= 3; a++)
                for (int b = 0; a + b <= 3; b++)
                    for (int c = 0; a + b + c <= 3; c++)
                        t.ref.raw[ref_index(a, b, c)] += wm * std::pow(v[0], a) * std::pow(v[1], b) * std::pow(v[2], c);
            for (int side = 0; side < 6; side++) {
                const double xn = v[side / 2] * ((side % 2) ? -1.0 : 1.0);  // normal from the wall into the gas
                if (xn < 0.0) t.ref.flux[side] += wm * (-xn);
            }
        }
    }
    t.mt.assign((size_t)MT_ROWS * t.Nv, 0.0);
    for (int g = 0; g < t.Nv; g++) {
        const double *v = &t.vel64[g * 4];
        for (int k = 0; k < 7; k++) t.mt[(size_t)k * t.Nv + g] = maxwellian(1.0, wallU[k], wallT[k], v);
        t.mt[(size_t)MT_INFLOW * t.Nv + g] = t.any_inflow ? maxwellian(bc->rho_in, bc->U_in, bc->T_in, v) : 0.0;
    }
    // ---- per (side, cell): wall kind and flags ----
    t.wall_kind.assign(6 * n, -1);
    t.side_flags.assign(2 * n, 0);
    t.n_fluid = 0;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const size_t cidx = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
                if (t.any_solid && solid[cidx]) continue;
                t.n_fluid++;
                for (int s = 0; s < 6; s++) {
                    int ii = i, jj = j, kk = k;
                    const int step = (s % 2) ? 1 : -1;
                    if (s / 2 == 0) ii += step;
                    if (s / 2 == 1) jj += step;
                    if (s / 2 == 2) kk += step;
                    const bool outside = ii < 0 || jj < 0 || kk < 0 || ii >= nx || jj >= ny || kk >= nz;
                    if (outside) {
                        if (bc->type[s] == KGS_FACE_WALL) {
                            t.wall_kind[s * n + cidx] = (int8_t)s;
                            t.side_flags[n + cidx] |= (uint8_t)(1 << s);
                        }
                    } else {
                        const size_t nb = (size_t)ii + (size_t)nx * ((size_t)jj + (size_t)ny * kk);
                        if (t.any_solid && solid[nb]) {
                            t.wall_kind[s * n + cidx] = 6;
                            t.side_flags[cidx] |= (uint8_t)(1 << s);
                            t.side_flags[n + cidx] |= (uint8_t)(1 << s);
                        }
                    }
                }
            }

    // accumulator layout: one flux slot per axis unless some cell has walls
    // on both of its sides along an axis
    t.acc_slots = ACC_COMPACT;
    for (size_t c = 0; c < n && t.acc_slots == ACC_COMPACT; c++)
        for (int d = 0; d < 3; d++)
            if (t.wall_kind[(2 * d) * n + c] >= 0 && t.wall_kind[(2 * d + 1) * n + c] >= 0) t.acc_slots = ACC_SPLIT;

    // ---- wavefront stages over blocks ----
    t.nbx = (nx + BX - 1) / BX;
    t.nby = (ny + BY - 1) / BY;
    t.nbz = (nz + t.bz - 1) / t.bz;
    // blocks without solid cells and without solid neighbours
    t.blk_plain.clear();
    if (t.any_solid) {
        t.blk_plain.assign((size_t)t.nbx * t.nby * t.nbz, 1);
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    const size_t c = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
                    if (t.solid[c] || (t.side_flags[c] & 63))
                        t.blk_plain[((size_t)(k / t.bz) * t.nby + j / BY) * t.nbx + i / BX] = 0;
                }
    }
    const int n_stages = t.nbx + t.nby + t.nbz - 2;
    std::vector<std::vector<int4>> stages(n_stages);
    for (int o = 0; o < 8; o++) {
        if (t.oct_vcount[o] == 0) continue;
        for (int bzr = 0; bzr < t.nbz; bzr++)
            for (int byr = 0; byr < t.nby; byr++)
                for (int bxr = 0; bxr < t.nbx; bxr++) stages[bxr + byr + bzr].push_back(make_int4(o, bxr, byr, bzr));
    }
    t.work.clear();
    t.stage_off.clear();
    t.stage_n.clear();
    for (int s = 0; s < n_stages; s++) {
        t.stage_off.push_back((int)t.work.size());
        t.stage_n.push_back((int)stages[s].size());
        t.work.insert(t.work.end(), stages[s].begin(), stages[s].end());
    }
}

}  // namespace kgs
