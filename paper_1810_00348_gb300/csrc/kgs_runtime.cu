// kgs_runtime.cu -- host runtime of libkgs: the C ABI of include/kgs.h.
//
// A context owns the device state of one problem: the lagged FP64
// macroscopic fields and wall densities (the whole solver state, Section 2.2:
// the distribution is never stored), per-cell coefficients in the sweep
// precision, octant-sorted velocity tables, the three face planes that carry
// block faces between sweep stages, and the per-(velocity group, cell)
// moment partials.  kgs_iterate launches, per outer iteration, the
// coefficient kernel, one sweep launch per wavefront stage and four small
// FP64 closure kernels, then reads back 16 bytes (residual and divergence
// flag).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/kgs.h"
#include "kgs_internal.h"

using namespace kgs;

namespace {

constexpr double R_GAS = 0.5;
constexpr uint32_t CKPT_MAGIC = 0x4b475331u;  // "KGS1"

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct kgs_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    int nx = 0, ny = 0, nz = 0, nvx = 0, nvy = 0, nvz = 0;
    size_t ncell = 0;
    int Nv = 0;
    long long n_fluid = 0;
    int precision = KGS_FP64;
    int wall_norm_mode = KGS_WALL_DISCRETE;
    int mass_rescale = 0;
    int max_iters = 1000;
    double tol = 1e-8;
    int tv = 1, vg_size = NT, bz = 16;
    double mu_ref = 0.0, omega = 0.81, Pr = 2.0 / 3.0;
    double M0 = 0.0;
    int iteration = 0;
    double last_residual = -1.0;
    int nbx = 0, nby = 0, nbz = 0;
    int oct_vstart[8] = {0}, oct_vcount[8] = {0}, oct_vgbase[8] = {0}, oct_nx[8] = {0};
    int n_vg = 0, max_vg = 0;
    int side_inflow[6] = {0};
    bool any_inflow = false;
    kgs_bc bc{};
    std::vector<int> stage_off, stage_n;
    std::vector<double> dx, dy, dz;
    std::vector<uint8_t> solid_h;
    // device buffers
    double *mac = nullptr, *mac_new = nullptr, *rho_w = nullptr, *rho_w_new = nullptr;
    void *coef = nullptr, *vel = nullptr, *velw = nullptr, *mtab = nullptr, *FX = nullptr, *FY = nullptr, *FZ = nullptr;
    double *vel64 = nullptr, *part = nullptr, *rdx = nullptr, *rdy = nullptr, *rdz = nullptr;
    double *ddx = nullptr, *ddy = nullptr, *ddz = nullptr;
    uint8_t *solid = nullptr, *side_flags = nullptr;
    int8_t *wall_kind = nullptr;
    double *wall_norm = nullptr;
    int4 *work = nullptr;
    int *d_vstart = nullptr, *d_vcount = nullptr, *d_vgbase = nullptr, *d_vg_oct = nullptr;
    double *blk_mass = nullptr, *blk_res = nullptr, *scale = nullptr, *resid = nullptr;
    int *blk_bad = nullptr;
    double *h_resid = nullptr;  // pinned
    int n_red_blocks = 0;
    size_t device_bytes = 0;
    std::vector<void *> allocs;
    // profiling
    int profiling = 0;
    std::vector<cudaEvent_t> ev;
    double sweep_ms = 0.0;
    long long sweep_launches = 0, kernel_launches = 0;
};

namespace {

int cuda_err(cudaError_t e)
{
    if (e == cudaSuccess) return KGS_OK;
    if (e == cudaErrorMemoryAllocation) return KGS_ENOMEM;
    return KGS_ECUDA;
}

#define KGS_CHECK(call)                      \
    do {                                     \
        cudaError_t e_ = (call);             \
        if (e_ != cudaSuccess) return cuda_err(e_); \
    } while (0)

int dalloc(kgs_ctx *c, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_err(e);
    }
    c->allocs.push_back(*p);
    c->device_bytes += bytes;
    return KGS_OK;
}

template <typename T>
int dalloc_t(kgs_ctx *c, T **p, size_t n)
{
    void *q = nullptr;
    int rc = dalloc(c, &q, n * sizeof(T));
    *p = static_cast<T *>(q);
    return rc;
}

template <typename T>
int upload(kgs_ctx *c, T **p, const std::vector<T> &h)
{
    int rc = dalloc_t(c, p, h.size());
    if (rc) return rc;
    return cuda_err(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
}

double maxwellian(double rho, const double U[3], double T, const double xi[3])
{
    double c2 = 0.0;
    for (int d = 0; d < 3; d++) c2 += (xi[d] - U[d]) * (xi[d] - U[d]);
    return rho / std::pow(2.0 * M_PI * R_GAS * T, 1.5) * std::exp(-c2 / (2.0 * R_GAS * T));
}

void free_all(kgs_ctx *c)
{
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    if (c->h_resid) cudaFreeHost(c->h_resid);
    c->h_resid = nullptr;
}

// Upload macros (or the uniform state), set M0 and the wall densities from
// the flux of the initial equilibrium.
int initial_state(kgs_ctx *c, const double *macros, const kgs_bc *bc_uniform)
{
    const size_t n = c->ncell;
    std::vector<double> m(8 * n);
    if (macros) {
        std::memcpy(m.data(), macros, sizeof(double) * 8 * n);
    } else {
        double u[8] = {1.0, 0, 0, 0, 1.0, 0, 0, 0};
        if (bc_uniform) {
            u[0] = bc_uniform->rho_in;
            u[1] = bc_uniform->U_in[0];
            u[2] = bc_uniform->U_in[1];
            u[3] = bc_uniform->U_in[2];
            u[4] = bc_uniform->T_in;
        }
        for (int q = 0; q < 8; q++)
            for (size_t i = 0; i < n; i++) m[q * n + i] = u[q];
    }
    double M0 = 0.0;
    for (size_t i = 0; i < n; i++) {
        if (!c->solid_h.empty() && c->solid_h[i]) {
            for (int q = 0; q < 8; q++) m[q * n + i] = 0.0;
            continue;
        }
        if (!(m[i] > 0.0) || !(m[4 * n + i] > 0.0)) return KGS_EINVAL;
        const size_t ii = i % c->nx, jj = (i / c->nx) % c->ny, kk = i / ((size_t)c->nx * c->ny);
        M0 += m[i] * c->dx[ii] * c->dy[jj] * c->dz[kk];
    }
    c->M0 = M0;
    KGS_CHECK(cudaMemcpyAsync(c->mac, m.data(), sizeof(double) * 8 * n, cudaMemcpyHostToDevice, c->stream));
    KGS_CHECK(launch_wall_flux_init(c->mac, c->wall_kind, c->wall_norm, c->vel64, c->Nv, n, R_GAS, c->Pr, c->rho_w,
                                    c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    c->iteration = 0;
    c->last_residual = -1.0;
    return KGS_OK;
}

int run_iteration(kgs_ctx *c, double *residual, int *bad)
{
    cudaStream_t st = c->stream;
    KGS_CHECK(launch_coef(c->precision, c->mac, c->solid, c->side_flags, c->rdx, c->rdy, c->rdz, c->nx, c->ny, c->nz,
                          c->mu_ref, c->omega, c->Pr, c->coef, st));
    SweepArgs a;
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    a.bz = c->bz;
    a.nbx = c->nbx;
    a.nby = c->nby;
    a.nbz = c->nbz;
    a.oct_vstart = c->d_vstart;
    a.oct_vcount = c->d_vcount;
    a.oct_vgbase = c->d_vgbase;
    a.Nv = c->Nv;
    a.vg_size = c->vg_size;
    a.vel = c->vel;
    a.velw = c->velw;
    for (int o = 0; o < 8; o++) a.oct_nx[o] = c->oct_nx[o] > 0 ? c->oct_nx[o] : 1;
    a.coef = c->coef;
    a.rho_w = c->rho_w;
    a.mtab = c->mtab;
    for (int s = 0; s < 6; s++) a.side_inflow[s] = c->side_inflow[s];
    a.FX = c->FX;
    a.FY = c->FY;
    a.FZ = c->FZ;
    a.part = c->part;
    a.ncell = c->ncell;
    const int ns = (int)c->stage_n.size();
    for (int s = 0; s < ns; s++) {
        a.work = c->work + c->stage_off[s];
        if (c->profiling) KGS_CHECK(cudaEventRecord(c->ev[2 * s], st));
        KGS_CHECK(launch_sweep(c->precision, c->tv, a, c->stage_n[s], c->max_vg, st));
        if (c->profiling) KGS_CHECK(cudaEventRecord(c->ev[2 * s + 1], st));
    }
    CloseArgs ca;
    ca.nx = c->nx;
    ca.ny = c->ny;
    ca.nz = c->nz;
    ca.ncell = c->ncell;
    ca.n_vg = c->n_vg;
    ca.vg_oct = c->d_vg_oct;
    ca.part = c->part;
    ca.coef = c->coef;
    ca.precision = c->precision;
    ca.mac = c->mac;
    ca.mac_new = c->mac_new;
    ca.rho_w_new = c->rho_w_new;
    ca.wall_kind = c->wall_kind;
    ca.wall_norm = c->wall_norm;
    ca.dx = c->ddx;
    ca.dy = c->ddy;
    ca.dz = c->ddz;
    ca.solid = c->solid;
    ca.blk_mass = c->blk_mass;
    KGS_CHECK(launch_close(ca, c->n_red_blocks, st));
    KGS_CHECK(launch_finalize_mass(c->blk_mass, c->n_red_blocks, c->M0, c->mass_rescale, c->scale, st));
    KGS_CHECK(launch_scale_residual(c->mac_new, c->rho_w_new, c->mac, c->solid, c->ncell, c->scale, c->blk_res,
                                    c->blk_bad, c->n_red_blocks, st));
    KGS_CHECK(launch_finalize_residual(c->blk_res, c->blk_bad, c->n_red_blocks, c->resid, st));
    KGS_CHECK(cudaMemcpyAsync(c->h_resid, c->resid, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    KGS_CHECK(cudaStreamSynchronize(st));
    c->kernel_launches += 5 + ns;
    c->sweep_launches += ns;
    if (c->profiling) {
        for (int s = 0; s < ns; s++) {
            float ms = 0.f;
            KGS_CHECK(cudaEventElapsedTime(&ms, c->ev[2 * s], c->ev[2 * s + 1]));
            c->sweep_ms += ms;
        }
    }
    std::swap(c->mac, c->mac_new);
    std::swap(c->rho_w, c->rho_w_new);
    c->iteration++;
    *residual = c->h_resid[0];
    *bad = c->h_resid[1] != 0.0;
    c->last_residual = *residual;
    return KGS_OK;
}

}  // namespace

extern "C" {

const char *kgs_strerror(int code)
{
    switch (code) {
    case KGS_OK: return "ok";
    case KGS_NOTCONVERGED: return "iteration budget ended above the tolerance";
    case KGS_EINVAL: return "invalid argument";
    case KGS_ENOMEM: return "out of memory";
    case KGS_ECUDA: return "CUDA error";
    case KGS_EDIVERGED: return "iteration diverged (NaN, rho <= 0 or T <= 0)";
    case KGS_ETIMEOUT: return "a bounded device wait expired";
    case KGS_EFORMAT: return "checkpoint does not match this context";
    default: return "unknown error code";
    }
}

int kgs_setup(kgs_ctx **out, const kgs_grid *grid, const uint8_t *solid, const kgs_vgrid *vg, const kgs_gas *gas,
              const kgs_bc *bc, const kgs_opts *opts)
{
    if (!out || !grid || !vg || !gas || !bc || !opts) return KGS_EINVAL;
    *out = nullptr;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !grid->dx || !grid->dy || !grid->dz) return KGS_EINVAL;
    if (vg->nvx < 1 || vg->nvy < 1 || vg->nvz < 1) return KGS_EINVAL;
    if (!vg->xi_x || !vg->xi_y || !vg->xi_z || !vg->w_x || !vg->w_y || !vg->w_z) return KGS_EINVAL;
    if (!(gas->Kn > 0.0) || !(gas->Pr > 0.0) || !(gas->omega >= 0.0 && gas->omega <= 1.5)) return KGS_EINVAL;
    if (opts->precision != KGS_FP64 && opts->precision != KGS_MIXED) return KGS_EINVAL;
    if (opts->wall_norm != KGS_WALL_DISCRETE && opts->wall_norm != KGS_WALL_ANALYTIC) return KGS_EINVAL;
    if (opts->v_per_cta != 0 && opts->v_per_cta != 128 && opts->v_per_cta != 256) return KGS_EINVAL;
    if (opts->precision == KGS_FP64 && opts->v_per_cta == 256) return KGS_EINVAL;
    if (opts->block_z < 0) return KGS_EINVAL;
    const long long ncell_ll = (long long)grid->nx * grid->ny * grid->nz;
    const long long nv_ll = (long long)vg->nvx * vg->nvy * vg->nvz;
    if (ncell_ll > (1LL << 31) || nv_ll > (1LL << 24)) return KGS_EINVAL;
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
        for (long long i = 0; i < ncell_ll; i++) any_solid |= solid[i] != 0;
    if (any_solid && !(bc->T_solid > 0.0)) return KGS_EINVAL;
    if (std::isinf(gas->Kn)) {
        // free-molecular limit: a velocity with all components zero has no
        // equation (0 = 0); reject such grids
        bool zx = false, zy = false, zz = false;
        for (int i = 0; i < vg->nvx; i++) zx |= vg->xi_x[i] == 0.0;
        for (int i = 0; i < vg->nvy; i++) zy |= vg->xi_y[i] == 0.0;
        for (int i = 0; i < vg->nvz; i++) zz |= vg->xi_z[i] == 0.0;
        if (zx && zy && zz) return KGS_EINVAL;
    }

    kgs_ctx *c = new (std::nothrow) kgs_ctx();
    if (!c) return KGS_ENOMEM;
    auto fail = [&](int rc) {
        free_all(c);
        delete c;
        return rc;
    };
    if (cudaGetDevice(&c->dev) != cudaSuccess) return fail(KGS_ECUDA);
    c->stream = static_cast<cudaStream_t>(opts->stream);
    c->nx = grid->nx;
    c->ny = grid->ny;
    c->nz = grid->nz;
    c->ncell = (size_t)ncell_ll;
    c->nvx = vg->nvx;
    c->nvy = vg->nvy;
    c->nvz = vg->nvz;
    c->Nv = (int)nv_ll;
    c->precision = opts->precision;
    c->wall_norm_mode = opts->wall_norm;
    c->mass_rescale = opts->mass_rescale ? 1 : 0;
    c->max_iters = opts->max_iters > 0 ? opts->max_iters : 1000;
    c->tol = opts->tol > 0.0 ? opts->tol : 1e-8;
    c->tv = (opts->precision == KGS_FP64) ? 1 : (opts->v_per_cta == 256 ? 2 : 1);
    c->vg_size = NT * c->tv;
    c->bz = opts->block_z > 0 ? opts->block_z : 16;
    c->omega = gas->omega;
    c->Pr = gas->Pr;
    // Eq. (10) with T_ref = 1, p_ref = rho_ref R T_ref = 1/2, lambda_ref = Kn
    c->mu_ref = 15.0 * std::sqrt(M_PI) * (R_GAS * 1.0) * gas->Kn /
                ((5.0 - 2.0 * gas->omega) * (7.0 - 2.0 * gas->omega) * std::sqrt(2.0 * R_GAS * 1.0));
    c->dx.assign(grid->dx, grid->dx + c->nx);
    c->dy.assign(grid->dy, grid->dy + c->ny);
    c->dz.assign(grid->dz, grid->dz + c->nz);
    if (any_solid) c->solid_h.assign(solid, solid + c->ncell);
    for (int s = 0; s < 6; s++) c->side_inflow[s] = bc->type[s] == KGS_FACE_INFLOW;
    c->any_inflow = any_inflow;
    c->bc = *bc;
    const size_t n = c->ncell;
    const int nx = c->nx, ny = c->ny, nz = c->nz;

    // ---- velocities sorted by octant (bit d set: xi_d >= 0), ix fastest ----
    std::vector<int> order;
    order.reserve(c->Nv);
    auto oct_of = [&](int ix, int iy, int iz) {
        return (vg->xi_x[ix] >= 0.0 ? 1 : 0) | (vg->xi_y[iy] >= 0.0 ? 2 : 0) | (vg->xi_z[iz] >= 0.0 ? 4 : 0);
    };
    for (int o = 0; o < 8; o++) {
        c->oct_vstart[o] = (int)order.size();
        for (int iz = 0; iz < c->nvz; iz++)
            for (int iy = 0; iy < c->nvy; iy++)
                for (int ix = 0; ix < c->nvx; ix++)
                    if (oct_of(ix, iy, iz) == o) order.push_back(ix + c->nvx * (iy + c->nvy * iz));
        c->oct_vcount[o] = (int)order.size() - c->oct_vstart[o];
    }
    for (int o = 0; o < 8; o++) {
        int cnt = 0;
        for (int ix = 0; ix < c->nvx; ix++) cnt += ((vg->xi_x[ix] >= 0.0 ? 1 : 0) == (o & 1));
        c->oct_nx[o] = cnt;
    }
    std::vector<double> vel64((size_t)c->Nv * 4), velw64((size_t)c->Nv * 2);
    for (int g = 0; g < c->Nv; g++) {
        const int a = order[g];
        const int ix = a % c->nvx, iy = (a / c->nvx) % c->nvy, iz = a / (c->nvx * c->nvy);
        vel64[g * 4 + 0] = vg->xi_x[ix];
        vel64[g * 4 + 1] = vg->xi_y[iy];
        vel64[g * 4 + 2] = vg->xi_z[iz];
        vel64[g * 4 + 3] = vg->w_x[ix] * vg->w_y[iy] * vg->w_z[iz];
        velw64[g * 2 + 0] = vg->w_x[ix];
        velw64[g * 2 + 1] = vg->w_y[iy] * vg->w_z[iz];
    }
    std::vector<int> vg_oct;
    for (int o = 0; o < 8; o++) {
        c->oct_vgbase[o] = (int)vg_oct.size();
        const int ng = (c->oct_vcount[o] + c->vg_size - 1) / c->vg_size;
        for (int g = 0; g < ng; g++) vg_oct.push_back(o);
        c->max_vg = std::max(c->max_vg, ng);
    }
    c->n_vg = (int)vg_oct.size();

    // ---- wall tables ----
    double wallU[7][3], wallT[7];
    for (int s = 0; s < 6; s++) {
        for (int d = 0; d < 3; d++) wallU[s][d] = bc->U_w[s][d];
        wallT[s] = bc->type[s] == KGS_FACE_WALL ? bc->T_w[s] : 1.0;
    }
    wallU[6][0] = wallU[6][1] = wallU[6][2] = 0.0;
    wallT[6] = any_solid ? bc->T_solid : 1.0;
    std::vector<double> wall_norm(7 * 6);
    for (int k = 0; k < 7; k++)
        for (int s = 0; s < 6; s++) {
            if (c->wall_norm_mode == KGS_WALL_ANALYTIC) {
                wall_norm[k * 6 + s] = std::sqrt(2.0 * M_PI / (R_GAS * wallT[k]));
                continue;
            }
            // discrete outgoing flux of the unit wall Maxwellian
            const int d = s / 2;
            const double nrm = (s % 2) ? -1.0 : 1.0;
            double D = 0.0;
            for (int g = 0; g < c->Nv; g++) {
                const double *v = &vel64[g * 4];
                const double xn = v[d] * nrm;
                if (xn > 0.0) D += v[3] * xn * maxwellian(1.0, wallU[k], wallT[k], v);
            }
            wall_norm[k * 6 + s] = D > 0.0 ? 1.0 / D : 0.0;
        }
    std::vector<double> mt((size_t)MT_ROWS * c->Nv);
    for (int g = 0; g < c->Nv; g++) {
        const double *v = &vel64[g * 4];
        for (int k = 0; k < 7; k++) mt[(size_t)k * c->Nv + g] = maxwellian(1.0, wallU[k], wallT[k], v);
        mt[(size_t)MT_INFLOW * c->Nv + g] = any_inflow ? maxwellian(bc->rho_in, bc->U_in, bc->T_in, v) : 0.0;
    }
    // per (side, cell): wall kind and flags
    std::vector<int8_t> wall_kind(6 * n, -1);
    std::vector<uint8_t> side_flags(2 * n, 0);
    long long n_fluid = 0;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const size_t cidx = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
                if (any_solid && solid[cidx]) continue;
                n_fluid++;
                for (int s = 0; s < 6; s++) {
                    int ii = i, jj = j, kk = k;
                    const int step = (s % 2) ? 1 : -1;
                    if (s / 2 == 0) ii += step;
                    if (s / 2 == 1) jj += step;
                    if (s / 2 == 2) kk += step;
                    const bool outside = ii < 0 || jj < 0 || kk < 0 || ii >= nx || jj >= ny || kk >= nz;
                    if (outside) {
                        if (bc->type[s] == KGS_FACE_WALL) {
                            wall_kind[s * n + cidx] = (int8_t)s;
                            side_flags[n + cidx] |= (uint8_t)(1 << s);
                        }
                    } else {
                        const size_t nb = (size_t)ii + (size_t)nx * ((size_t)jj + (size_t)ny * kk);
                        if (any_solid && solid[nb]) {
                            wall_kind[s * n + cidx] = 6;
                            side_flags[cidx] |= (uint8_t)(1 << s);
                            side_flags[n + cidx] |= (uint8_t)(1 << s);
                        }
                    }
                }
            }
    c->n_fluid = n_fluid;

    // ---- wavefront stages over blocks ----
    c->nbx = (nx + BX - 1) / BX;
    c->nby = (ny + BY - 1) / BY;
    c->nbz = (nz + c->bz - 1) / c->bz;
    const int n_stages = c->nbx + c->nby + c->nbz - 2;
    std::vector<std::vector<int4>> stages(n_stages);
    for (int o = 0; o < 8; o++) {
        if (c->oct_vcount[o] == 0) continue;
        for (int bzr = 0; bzr < c->nbz; bzr++)
            for (int byr = 0; byr < c->nby; byr++)
                for (int bxr = 0; bxr < c->nbx; bxr++) stages[bxr + byr + bzr].push_back(make_int4(o, bxr, byr, bzr));
    }
    std::vector<int4> work;
    for (int s = 0; s < n_stages; s++) {
        c->stage_off.push_back((int)work.size());
        c->stage_n.push_back((int)stages[s].size());
        work.insert(work.end(), stages[s].begin(), stages[s].end());
    }

    // ---- device allocations ----
    int rc = KGS_OK;
    const size_t rsz = c->precision == KGS_FP64 ? sizeof(double) : sizeof(float);
    std::vector<double> rdx(nx), rdy(ny), rdz(nz);
    for (int i = 0; i < nx; i++) rdx[i] = 1.0 / c->dx[i];
    for (int i = 0; i < ny; i++) rdy[i] = 1.0 / c->dy[i];
    for (int i = 0; i < nz; i++) rdz[i] = 1.0 / c->dz[i];
    c->n_red_blocks = (int)((n + 255) / 256);
    if ((rc = dalloc_t(c, &c->mac, 8 * n)) || (rc = dalloc_t(c, &c->mac_new, 8 * n)) ||
        (rc = dalloc_t(c, &c->rho_w, 6 * n)) || (rc = dalloc_t(c, &c->rho_w_new, 6 * n)) ||
        (rc = dalloc(c, &c->coef, n * NCOEF * rsz)) || (rc = upload(c, &c->vel64, vel64)) ||
        (rc = dalloc(c, &c->vel, (size_t)c->Nv * 4 * rsz)) || (rc = dalloc(c, &c->velw, (size_t)c->Nv * 2 * rsz)) || (rc = dalloc(c, &c->mtab, mt.size() * rsz)) ||
        (rc = dalloc(c, &c->FX, (size_t)nz * ny * c->Nv * rsz)) ||
        (rc = dalloc(c, &c->FY, (size_t)nz * nx * c->Nv * rsz)) ||
        (rc = dalloc(c, &c->FZ, (size_t)ny * nx * c->Nv * rsz)) ||
        (rc = dalloc_t(c, &c->part, (size_t)c->n_vg * NPART * n)) || (rc = upload(c, &c->rdx, rdx)) ||
        (rc = upload(c, &c->rdy, rdy)) || (rc = upload(c, &c->rdz, rdz)) || (rc = upload(c, &c->ddx, c->dx)) ||
        (rc = upload(c, &c->ddy, c->dy)) || (rc = upload(c, &c->ddz, c->dz)) ||
        (rc = upload(c, &c->side_flags, side_flags)) || (rc = upload(c, &c->wall_kind, wall_kind)) ||
        (rc = upload(c, &c->wall_norm, wall_norm)) || (rc = upload(c, &c->work, work)) ||
        (rc = upload(c, &c->d_vstart, std::vector<int>(c->oct_vstart, c->oct_vstart + 8))) ||
        (rc = upload(c, &c->d_vcount, std::vector<int>(c->oct_vcount, c->oct_vcount + 8))) ||
        (rc = upload(c, &c->d_vgbase, std::vector<int>(c->oct_vgbase, c->oct_vgbase + 8))) ||
        (rc = upload(c, &c->d_vg_oct, vg_oct)) || (rc = dalloc_t(c, &c->blk_mass, c->n_red_blocks)) ||
        (rc = dalloc_t(c, &c->blk_res, (size_t)c->n_red_blocks * 10)) ||
        (rc = dalloc_t(c, &c->blk_bad, c->n_red_blocks)) || (rc = dalloc_t(c, &c->scale, 2)) ||
        (rc = dalloc_t(c, &c->resid, 2)))
        return fail(rc);
    if (any_solid) {
        if ((rc = upload(c, &c->solid, c->solid_h))) return fail(rc);
    }
    if (c->precision == KGS_FP64) {
        if (cudaMemcpy(c->vel, vel64.data(), vel64.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->velw, velw64.data(), velw64.size() * sizeof(double), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(c->mtab, mt.data(), mt.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(KGS_ECUDA);
    } else {
        std::vector<float> v32(vel64.begin(), vel64.end()), m32(mt.begin(), mt.end());
        std::vector<float> w32(velw64.begin(), velw64.end());
        if (cudaMemcpy(c->vel, v32.data(), v32.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->velw, w32.data(), w32.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->mtab, m32.data(), m32.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(KGS_ECUDA);
    }
    if (cudaMemset(c->FX, 0, (size_t)nz * ny * c->Nv * rsz) != cudaSuccess ||
        cudaMemset(c->FY, 0, (size_t)nz * nx * c->Nv * rsz) != cudaSuccess ||
        cudaMemset(c->FZ, 0, (size_t)ny * nx * c->Nv * rsz) != cudaSuccess ||
        cudaMemset(c->coef, 0, n * NCOEF * rsz) != cudaSuccess)
        return fail(KGS_ECUDA);
    if (cudaMallocHost(&c->h_resid, 2 * sizeof(double)) != cudaSuccess) return fail(KGS_ENOMEM);
    c->ev.resize(2 * (size_t)n_stages);
    for (auto &e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(KGS_ECUDA);
    if ((rc = initial_state(c, nullptr, any_inflow ? bc : nullptr))) return fail(rc);
    *out = c;
    return KGS_OK;
}

int kgs_set_initial(kgs_ctx *c, const double *macros)
{
    if (!c) return KGS_EINVAL;
    if (cudaSetDevice(c->dev) != cudaSuccess) return KGS_ECUDA;
    return initial_state(c, macros, c->any_inflow ? &c->bc : nullptr);
}

int kgs_iterate(kgs_ctx *c, int n_iters, int *done, double *residual)
{
    if (!c) return KGS_EINVAL;
    if (cudaSetDevice(c->dev) != cudaSuccess) return KGS_ECUDA;
    int count = 0, bad = 0, rc = KGS_OK;
    double r = c->last_residual;
    const bool until = n_iters <= 0;
    const int limit = until ? c->max_iters : n_iters;
    while (count < limit) {
        rc = run_iteration(c, &r, &bad);
        if (rc) break;
        count++;
        if (bad) {
            rc = KGS_EDIVERGED;
            break;
        }
        if (until && r < c->tol) break;
    }
    if (rc == KGS_OK && until && !(r < c->tol)) rc = KGS_NOTCONVERGED;
    if (done) *done = count;
    if (residual) *residual = r;
    return rc;
}

int kgs_moments(kgs_ctx *c, double *out)
{
    if (!c || !out) return KGS_EINVAL;
    KGS_CHECK(cudaMemcpyAsync(out, c->mac, sizeof(double) * 8 * c->ncell, cudaMemcpyDeviceToHost, c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    return KGS_OK;
}

int kgs_moments_device(kgs_ctx *c, double *out_dev)
{
    if (!c || !out_dev) return KGS_EINVAL;
    KGS_CHECK(cudaMemcpyAsync(out_dev, c->mac, sizeof(double) * 8 * c->ncell, cudaMemcpyDeviceToDevice, c->stream));
    return KGS_OK;
}

int kgs_rho_w(kgs_ctx *c, double *out)
{
    if (!c || !out) return KGS_EINVAL;
    KGS_CHECK(cudaMemcpyAsync(out, c->rho_w, sizeof(double) * 6 * c->ncell, cudaMemcpyDeviceToHost, c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    return KGS_OK;
}

int kgs_set_rho_w(kgs_ctx *c, const double *in)
{
    if (!c || !in) return KGS_EINVAL;
    KGS_CHECK(cudaMemcpyAsync(c->rho_w, in, sizeof(double) * 6 * c->ncell, cudaMemcpyHostToDevice, c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    return KGS_OK;
}

namespace {
struct CkptHeader {
    uint32_t magic;
    int32_t nx, ny, nz, Nv, iteration;
    double M0, last_residual;
};
}  // namespace

int kgs_save(kgs_ctx *c, void *buf, size_t *len)
{
    if (!c || !len) return KGS_EINVAL;
    const size_t need = sizeof(CkptHeader) + sizeof(double) * 14 * c->ncell;
    if (!buf) {
        *len = need;
        return KGS_OK;
    }
    if (*len < need) return KGS_EINVAL;
    CkptHeader h{CKPT_MAGIC, c->nx, c->ny, c->nz, c->Nv, c->iteration, c->M0, c->last_residual};
    std::memcpy(buf, &h, sizeof h);
    double *body = reinterpret_cast<double *>(static_cast<char *>(buf) + sizeof h);
    KGS_CHECK(cudaMemcpyAsync(body, c->mac, sizeof(double) * 8 * c->ncell, cudaMemcpyDeviceToHost, c->stream));
    KGS_CHECK(cudaMemcpyAsync(body + 8 * c->ncell, c->rho_w, sizeof(double) * 6 * c->ncell, cudaMemcpyDeviceToHost,
                              c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    *len = need;
    return KGS_OK;
}

int kgs_load(kgs_ctx *c, const void *buf, size_t len)
{
    if (!c || !buf) return KGS_EINVAL;
    const size_t need = sizeof(CkptHeader) + sizeof(double) * 14 * c->ncell;
    if (len != need) return KGS_EFORMAT;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.magic != CKPT_MAGIC || h.nx != c->nx || h.ny != c->ny || h.nz != c->nz || h.Nv != c->Nv)
        return KGS_EFORMAT;
    const double *body = reinterpret_cast<const double *>(static_cast<const char *>(buf) + sizeof h);
    KGS_CHECK(cudaMemcpyAsync(c->mac, body, sizeof(double) * 8 * c->ncell, cudaMemcpyHostToDevice, c->stream));
    KGS_CHECK(cudaMemcpyAsync(c->rho_w, body + 8 * c->ncell, sizeof(double) * 6 * c->ncell, cudaMemcpyHostToDevice,
                              c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    c->iteration = h.iteration;
    c->M0 = h.M0;
    c->last_residual = h.last_residual;
    return KGS_OK;
}

int kgs_info(kgs_ctx *c, kgs_info_t *o)
{
    if (!c || !o) return KGS_EINVAL;
    o->nx = c->nx;
    o->ny = c->ny;
    o->nz = c->nz;
    o->nvx = c->nvx;
    o->nvy = c->nvy;
    o->nvz = c->nvz;
    o->n_fluid = c->n_fluid;
    o->phase_points = c->n_fluid * (long long)c->Nv;
    o->iteration = c->iteration;
    o->n_stages = (int)c->stage_n.size();
    o->v_per_cta = c->vg_size;
    o->block_z = c->bz;
    o->precision = c->precision;
    o->device_bytes = c->device_bytes;
    o->last_residual = c->last_residual;
    return KGS_OK;
}

int kgs_set_profiling(kgs_ctx *c, int enable)
{
    if (!c) return KGS_EINVAL;
    c->profiling = enable ? 1 : 0;
    return KGS_OK;
}

int kgs_profile(kgs_ctx *c, double *sweep_ms, long long *sweep_launches, long long *kernel_launches)
{
    if (!c) return KGS_EINVAL;
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    if (sweep_ms) *sweep_ms = c->sweep_ms;
    if (sweep_launches) *sweep_launches = c->sweep_launches;
    if (kernel_launches) *kernel_launches = c->kernel_launches;
    c->sweep_ms = 0.0;
    c->sweep_launches = 0;
    c->kernel_launches = 0;
    return KGS_OK;
}

void kgs_destroy(kgs_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->dev);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
