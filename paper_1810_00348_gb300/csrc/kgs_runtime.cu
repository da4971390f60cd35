// kgs_runtime.cu -- host runtime of libkgs: the C ABI of include/kgs.h.
//
// A context owns the device state of one problem: the lagged FP64
// macroscopic fields and wall densities (the whole solver state, Section 2.2:
// the distribution is never stored), per-cell coefficients in the sweep
// precision, octant-sorted velocity tables, the three face planes that carry
// block faces between sweep stages, the ordered per-cell moment accumulators
// with the work list, chain places and per-CTA scratch of the persistent
// sweep, and the per-cell sums.  kgs_iterate launches, per outer iteration,
// the coefficient kernel, one persistent sweep launch, the sums kernel and
// four small FP64 closure kernels, then reads back 24 bytes (residual,
// divergence flag and the wait-error word).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "kgs_ctx.h"

using namespace kgs;

namespace {
constexpr uint32_t CKPT_MAGIC = 0x4b475331u;  // "KGS1"
}

int kgs::cuda_err(cudaError_t e)
{
    if (e == cudaSuccess) return KGS_OK;
    if (e == cudaErrorMemoryAllocation) return KGS_ENOMEM;
    return KGS_ECUDA;
}

namespace {

#define KGS_CHECK(call)                             \
    do {                                            \
        cudaError_t e_ = (call);                    \
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

// Upload a FP64 host table into a device buffer of the sweep precision.
int upload_real(kgs_ctx *c, void **p, const std::vector<double> &h)
{
    const size_t rsz = c->t.real_bytes();
    int rc = dalloc(c, p, h.size() * rsz);
    if (rc) return rc;
    if (rsz == sizeof(double)) return cuda_err(cudaMemcpy(*p, h.data(), h.size() * rsz, cudaMemcpyHostToDevice));
    std::vector<float> f(h.begin(), h.end());
    return cuda_err(cudaMemcpy(*p, f.data(), f.size() * rsz, cudaMemcpyHostToDevice));
}

void free_all(kgs_ctx *c)
{
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    if (c->h_resid) cudaFreeHost(c->h_resid);
    c->h_resid = nullptr;
    if (c->h_args) cudaFreeHost(c->h_args);
    c->h_args = nullptr;
}

// Upload macros (or the uniform state), set M0 and the wall densities from
// the flux of the initial equilibrium.
int initial_state(kgs_ctx *c, const double *macros)
{
    const HostTables &t = c->t;
    const size_t n = t.ncell;
    std::vector<double> m(8 * n);
    if (macros) {
        std::memcpy(m.data(), macros, sizeof(double) * 8 * n);
    } else {
        double u[8] = {1.0, 0, 0, 0, 1.0, 0, 0, 0};
        if (t.any_inflow) {
            u[0] = t.bc.rho_in;
            u[1] = t.bc.U_in[0];
            u[2] = t.bc.U_in[1];
            u[3] = t.bc.U_in[2];
            u[4] = t.bc.T_in;
        }
        for (int q = 0; q < 8; q++)
            for (size_t i = 0; i < n; i++) m[q * n + i] = u[q];
    }
    double M0 = 0.0;
    for (size_t i = 0; i < n; i++) {
        if (t.any_solid && t.solid[i]) {
            for (int q = 0; q < 8; q++) m[q * n + i] = 0.0;
            continue;
        }
        if (!(m[i] > 0.0) || !(m[4 * n + i] > 0.0)) return KGS_EINVAL;
        const size_t ii = i % t.nx, jj = (i / t.nx) % t.ny, kk = i / ((size_t)t.nx * t.ny);
        M0 += m[i] * t.dx[ii] * t.dy[jj] * t.dz[kk];
    }
    c->M0 = M0;
    KGS_CHECK(cudaMemcpyAsync(c->mac, m.data(), sizeof(double) * 8 * n, cudaMemcpyHostToDevice, c->stream));
    KGS_CHECK(launch_wall_flux_init(c->mac, c->wall_kind, c->wall_norm, c->axis64, t.nvx, t.nvy, t.nvz, n, R_GAS, t.Pr,
                                    c->rho_w,
                                    c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    c->iteration = 0;
    c->last_residual = -1.0;
    return KGS_OK;
}

}  // namespace

SweepArgs kgs::ctx_sweep_args(const kgs_ctx *c)
{
    const HostTables &t = c->t;
    SweepArgs a{};
    a.nx = t.nx;
    a.ny = t.ny;
    a.nz = t.nz;
    a.bz = t.bz;
    a.nbx = t.nbx;
    a.nby = t.nby;
    a.nbz = t.nbz;
    a.work = c->work;
    a.oct_vstart = c->d_vstart;
    a.oct_vcount = c->d_vcount;
    a.oct_vgbase = c->d_vgbase;
    a.Nv = t.Nv;
    a.vg_size = t.vg_size;
    a.vel = c->vel;
    a.velm = c->velm;
    a.nxo_max = t.nxo_max;
    for (int o = 0; o < 8; o++) a.oct_nx[o] = t.oct_nx[o] > 0 ? t.oct_nx[o] : 1;
    a.any_solid = t.any_solid ? 1 : 0;
    a.blk_plain = c->blk_plain;
    a.coef = c->coef;
    a.rho_w = c->rho_w;
    a.mtab = c->mtab;
    for (int s = 0; s < 6; s++) a.side_inflow[s] = t.side_inflow[s];
    a.FX = c->FX;
    a.FY = c->FY;
    a.FZ = c->FZ;
    a.order = t.order;
    a.FX2 = c->FX2;
    a.FY2 = c->FY2;
    a.FZ2 = c->FZ2;
    a.part = c->part;
    a.acc = c->acc;
    a.nacc = t.nacc;
    a.acc_slots = t.acc_slots;
    a.tok = c->p_tok;
    a.ncell = t.ncell;
    a.line16 = 1;
    for (int o = 0; o < 8; o++)
        if (t.oct_vcount[o] > 0 && t.oct_nx[o] != 16) a.line16 = 0;
    t.set_uniformity(a);
    return a;
}

int kgs::ctx_launch_coef(kgs_ctx *c)
{
    const HostTables &t = c->t;
    KGS_CHECK(launch_coef(t.precision, c->mac, c->solid, c->side_flags, c->rdx, c->rdy, c->rdz, t.nx, t.ny, t.nz,
                          t.mu_ref, t.omega, t.Pr, c->coef, c->stream, t.dev ? 1 : 0));
    c->kernel_launches += 1;
    return KGS_OK;
}

int kgs::ctx_launch_stages(kgs_ctx *c)
{
    const HostTables &t = c->t;
    cudaStream_t st = c->stream;
    SweepArgs a = ctx_sweep_args(c);
    if (c->persist) {
        // the previous iteration has completed (run_iteration synchronises),
        // so the pinned staging copy is free to be rewritten
        *c->h_args = a;
        KGS_CHECK(cudaMemcpyAsync(c->p_args, c->h_args, sizeof(SweepArgs), cudaMemcpyHostToDevice, st));
        KGS_CHECK(cudaMemsetAsync(c->p_counter, 0, sizeof(int), st));
        KGS_CHECK(cudaMemsetAsync(c->p_flags, 0, c->p_n_flags * sizeof(int), st));
        KGS_CHECK(cudaMemsetAsync(c->p_tok, 0, ctx_n_tokens(t) * sizeof(int), st));
        BatchSweepArgs ba;
        ba.inst = c->p_args;
        ba.items = c->p_items;
        ba.n_items = c->persist_items;
        ba.counter = c->p_counter;
        ba.flags = c->p_flags;
        ba.flag_off = c->p_flag_off;
        ba.pos = c->p_pos;
        ba.scratch = c->p_scratch;
        ba.scratch_stride = c->scratch_stride;
        ba.error = reinterpret_cast<int *>(c->resid + 2);
        ba.spin_limit = c->spin_limit;
        ba.skip_publish = -1;
        if (c->profiling) KGS_CHECK(cudaEventRecord(c->ev[0], st));
        KGS_CHECK(
            launch_sweep_persistent(t.precision, t.tv, a.line16, a.uniform, ba, t.nxo_max, c->persist_grid, st,
                                    t.order, t.dev && t.order == 1));
        if (c->profiling) KGS_CHECK(cudaEventRecord(c->ev[1], st));
        c->kernel_launches += 1;
        c->sweep_launches += 1;
        return KGS_OK;
    }
    const int ns = (int)t.stage_n.size();
    for (int s = 0; s < ns; s++) {
        a.work = c->work + t.stage_off[s];
        if (c->profiling) KGS_CHECK(cudaEventRecord(c->ev[2 * s], st));
        KGS_CHECK(launch_sweep(t.precision, t.tv, a, t.stage_n[s], t.max_vg, st));
        if (c->profiling) KGS_CHECK(cudaEventRecord(c->ev[2 * s + 1], st));
    }
    c->kernel_launches += ns;
    c->sweep_launches += ns;
    return KGS_OK;
}

void kgs::ctx_stage_items(const HostTables &t, int inst, int stage, std::vector<int4> &out)
{
    for (int o = 0; o < 8; o++) {
        const int ng = (t.oct_vcount[o] + t.vg_size - 1) / t.vg_size;
        for (int vg = 0; vg < ng; vg++)
            for (int bzr = 0; bzr < t.nbz; bzr++)
                for (int byr = 0; byr < t.nby; byr++) {
                    const int bxr = stage - bzr - byr;
                    if (bxr < 0 || bxr >= t.nbx) continue;
                    out.push_back(make_int4(inst, (o << 24) | vg, bxr | (byr << 10) | (bzr << 20), t.oct_vgbase[o] + vg));
                }
    }
}

void kgs::chain_positions(const std::vector<int4> &items, const std::vector<const HostTables *> &tabs,
                          std::vector<int> &pos)
{
    std::vector<std::vector<int>> count(tabs.size());
    for (size_t i = 0; i < tabs.size(); i++) count[i].assign(ctx_n_tokens(*tabs[i]), 0);
    pos.resize(items.size());
    for (size_t it = 0; it < items.size(); it++) {
        const int4 w = items[it];
        const HostTables &t = *tabs[w.x];
        const int o = w.y >> 24, vg = w.y & 0xffffff;
        const int bxr = w.z & 1023, byr = (w.z >> 10) & 1023, bzr = (w.z >> 20) & 1023;
        const int bx = (o & 1) ? bxr : t.nbx - 1 - bxr;
        const int by = (o & 2) ? byr : t.nby - 1 - byr;
        const int bz = (o & 4) ? bzr : t.nbz - 1 - bzr;
        const size_t key = (((size_t)(vg % t.nacc) * t.nbz + bz) * t.nby + by) * t.nbx + bx;
        pos[it] = count[w.x][key]++;
    }
}

int kgs::ctx_alloc_acc(kgs_ctx *c)
{
    const HostTables &t = c->t;
    const size_t bytes = (size_t)t.nacc * t.ncell * t.acc_slots * 8;
    int rc = dalloc(c, &c->acc, bytes);
    if (rc) return rc;
    // every slot read by the sums is stored by the first item of its chain in
    // every iteration; all-ones bytes (NaN in both precisions) make any slot
    // that is not show up in the results at once
    KGS_CHECK(cudaMemset(c->acc, 0xff, bytes));
    c->use_acc = 1;
    return KGS_OK;
}

int kgs::ctx_persist_init(kgs_ctx *c)
{
    const HostTables &t = c->t;
    int sms = 0;
    KGS_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
    const SweepArgs a = ctx_sweep_args(c);
    const int per_sm = sweep_persistent_occupancy(t.precision, t.tv, a.line16, a.uniform,
                                                  sweep_smem_bytes(t.precision, t.tv, a.line16, t.nxo_max, t.order),
                                                  t.order, t.dev && t.order == 1);
    // the second-order sweep and the deviation-form source exist only in the
    // persistent kernel
    if (per_sm < 1 && (t.order == 2 || t.dev)) return KGS_EINVAL;
    if (per_sm < 1) {
        // the launch per stage, with per-group partials
        return dalloc(c, &c->part, (size_t)t.n_vg * NPART * t.ncell * 8);
    }
    std::vector<int4> items;
    for (int s = 0; s < (int)t.stage_n.size(); s++) ctx_stage_items(t, 0, s, items);
    std::vector<int> pos;
    chain_positions(items, std::vector<const HostTables *>(1, &t), pos);
    int rc;
    c->p_n_flags = (size_t)t.n_vg * t.nbx * t.nby * t.nbz;
    c->persist_grid = sms * per_sm;
    c->scratch_stride = sweep_scratch_bytes(t.bz);
    if ((rc = upload(c, &c->p_items, items)) || (rc = upload(c, &c->p_pos, pos)) ||
        (rc = dalloc_t(c, &c->p_counter, 1)) || (rc = dalloc_t(c, &c->p_flags, c->p_n_flags)) ||
        (rc = dalloc_t(c, &c->p_tok, ctx_n_tokens(t))) ||
        (rc = upload(c, &c->p_flag_off, std::vector<int>(1, 0))) || (rc = dalloc_t(c, &c->p_args, 1)) ||
        (rc = dalloc(c, &c->p_scratch, (size_t)c->persist_grid * c->scratch_stride)) || (rc = ctx_alloc_acc(c)))
        return rc;
    KGS_CHECK(cudaMallocHost(&c->h_args, sizeof(SweepArgs)));
    c->persist_items = (int)items.size();
    c->persist = 1;
    return KGS_OK;
}

int kgs::ctx_launch_sums(kgs_ctx *c)
{
    const HostTables &t = c->t;
    if (c->use_acc) {
        AccSumArgs aa;
        aa.precision = t.precision;
        aa.acc = c->acc;
        aa.nacc = t.nacc;
        aa.acc_slots = t.acc_slots;
        aa.ncell = t.ncell;
        aa.solid = c->solid;
        aa.sums = c->sums;
        aa.coef = c->coef;
        aa.wall_kind = c->wall_kind;
        aa.ref = t.ref;
        KGS_CHECK(launch_acc_sums(aa, c->stream));
    } else {
        PartSumArgs pa;
        pa.ncell = t.ncell;
        pa.n_vg = t.n_vg;
        pa.vg_oct = c->d_vg_oct;
        pa.part = c->part;
        pa.precision = t.precision;
        pa.solid = c->solid;
        pa.sums = c->sums;
        pa.coef = c->coef;
        pa.wall_kind = c->wall_kind;
        pa.ref = t.ref;
        KGS_CHECK(launch_part_sums(pa, c->stream));
    }
    c->kernel_launches += 1;
    return KGS_OK;
}

int kgs::ctx_launch_closure(kgs_ctx *c, double *resid_dev, const double *sums)
{
    const HostTables &t = c->t;
    cudaStream_t st = c->stream;
    ClosureArgs ca;
    ca.nx = t.nx;
    ca.ny = t.ny;
    ca.nz = t.nz;
    ca.ncell = t.ncell;
    ca.sums = sums ? sums : c->sums;
    ca.coef = c->coef;
    ca.precision = t.precision;
    ca.q_lagged = c->q_lagged;
    ca.mac_new = c->mac_new;
    ca.rho_w_new = c->rho_w_new;
    ca.wall_kind = c->wall_kind;
    ca.wall_norm = c->wall_norm;
    ca.dx = c->ddx;
    ca.dy = c->ddy;
    ca.dz = c->ddz;
    ca.solid = c->solid;
    ca.blk_mass = c->blk_mass;
    KGS_CHECK(launch_closure(ca, st));
    KGS_CHECK(launch_finalize_mass(c->blk_mass, (int)close_blocks(t.ncell), c->M0, c->mass_rescale, c->scale, st));
    KGS_CHECK(launch_scale_residual(c->mac_new, c->rho_w_new, c->mac, c->solid, t.ncell, c->scale, c->blk_res,
                                    c->blk_bad, c->n_red_blocks, st));
    KGS_CHECK(launch_finalize_residual(c->blk_res, c->blk_bad, c->n_red_blocks, resid_dev, st));
    c->kernel_launches += 4;
    return KGS_OK;
}

void kgs::ctx_finish(kgs_ctx *c, double residual)
{
    std::swap(c->mac, c->mac_new);
    std::swap(c->rho_w, c->rho_w_new);
    c->iteration++;
    c->last_residual = residual;
}

namespace {

int run_iteration(kgs_ctx *c, double *residual, int *bad)
{
    int rc;
    if ((rc = ctx_launch_coef(c)) || (rc = ctx_launch_stages(c)) || (rc = ctx_launch_sums(c)) ||
        (rc = ctx_launch_closure(c, c->resid, nullptr)))
        return rc;
    KGS_CHECK(cudaMemcpyAsync(c->h_resid, c->resid, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    if (c->persist && *reinterpret_cast<const int *>(c->h_resid + 2) != 0) {
        // a bounded wait of the persistent sweep gave up: clear the word and
        // report; the iteration's results are not used
        KGS_CHECK(cudaMemsetAsync(c->resid + 2, 0, sizeof(double), c->stream));
        KGS_CHECK(cudaStreamSynchronize(c->stream));
        return KGS_ETIMEOUT;
    }
    if (c->profiling) {
        const size_t n_pairs = c->persist ? 1 : c->t.stage_n.size();
        for (size_t s = 0; s < n_pairs; s++) {
            float ms = 0.f;
            KGS_CHECK(cudaEventElapsedTime(&ms, c->ev[2 * s], c->ev[2 * s + 1]));
            c->sweep_ms += ms;
        }
    }
    *residual = c->h_resid[0];
    *bad = c->h_resid[1] != 0.0;
    ctx_finish(c, *residual);
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
    if (!out || !opts) return KGS_EINVAL;
    *out = nullptr;
    int rc = validate_problem(grid, solid, vg, gas, bc, opts->precision, opts->wall_norm, opts->v_per_cta,
                              opts->block_z, opts->vz_begin, opts->vz_end, opts->order, opts->dev_source);
    if (rc) return rc;
    (void)cudaGetLastError();  // launches below check their own status
    if ((rc = ctx_create(out, grid, solid, vg, gas, bc, opts))) return rc;
    rc = ctx_persist_init(*out);
    // the persistent sweep's tables and the accumulator fill went to the
    // legacy default stream as well
    if (!rc && cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) rc = KGS_ECUDA;
    if (rc) {
        kgs_destroy(*out);
        *out = nullptr;
    }
    return rc;
}

}  // extern "C"

void kgs::ctx_free(kgs_ctx *c) { free_all(c); }

int kgs::ctx_create(kgs_ctx **out, const kgs_grid *grid, const uint8_t *solid, const kgs_vgrid *vg, const kgs_gas *gas,
                    const kgs_bc *bc, const kgs_opts *opts)
{
    int rc = KGS_OK;
    kgs_ctx *c = new (std::nothrow) kgs_ctx();
    if (!c) return KGS_ENOMEM;
    auto fail = [&](int code) {
        free_all(c);
        delete c;
        return code;
    };
    if (cudaGetDevice(&c->dev) != cudaSuccess) return fail(KGS_ECUDA);
    c->stream = static_cast<cudaStream_t>(opts->stream);
    c->mass_rescale = opts->mass_rescale ? 1 : 0;
    c->max_iters = opts->max_iters > 0 ? opts->max_iters : 1000;
    c->tol = opts->tol > 0.0 ? opts->tol : 1e-8;
    HostTables &t = c->t;
    build_tables(t, grid, solid, vg, gas, bc, opts->precision, opts->wall_norm, opts->v_per_cta, opts->block_z,
                 opts->vz_begin, opts->vz_end, opts->order, opts->dev_source);
    c->q_lagged = opts->q_lagged ? 1 : 0;
    const size_t n = t.ncell;
    const size_t rsz = t.real_bytes();
    c->n_red_blocks = (int)((n + 255) / 256);
    if ((rc = dalloc_t(c, &c->mac, 8 * n)) || (rc = dalloc_t(c, &c->mac_new, 8 * n)) ||
        (rc = dalloc_t(c, &c->rho_w, 6 * n)) || (rc = dalloc_t(c, &c->rho_w_new, 6 * n)) ||
        (rc = dalloc(c, &c->coef, n * NCOEF * rsz)) || (rc = upload(c, &c->vel64, t.vel64)) || (rc = upload(c, &c->axis64, t.axis64)) ||
        (rc = upload_real(c, &c->vel, t.vel64)) || (rc = upload_real(c, &c->mtab, t.mt)) ||
        (rc = dalloc(c, &c->FX, (size_t)t.nz * t.ny * t.Nv * rsz)) ||
        (rc = dalloc(c, &c->FY, (size_t)t.nz * t.nx * t.Nv * rsz)) ||
        (rc = dalloc(c, &c->FZ, (size_t)t.ny * t.nx * t.Nv * rsz)) ||
        (rc = dalloc_t(c, &c->sums, (size_t)NSUM * n)) || (rc = upload(c, &c->rdx, t.rdx)) ||
        (rc = upload(c, &c->rdy, t.rdy)) || (rc = upload(c, &c->rdz, t.rdz)) || (rc = upload(c, &c->ddx, t.dx)) ||
        (rc = upload(c, &c->ddy, t.dy)) || (rc = upload(c, &c->ddz, t.dz)) ||
        (rc = upload(c, &c->side_flags, t.side_flags)) || (rc = upload(c, &c->wall_kind, t.wall_kind)) ||
        (rc = upload(c, &c->wall_norm, t.wall_norm)) || (rc = upload(c, &c->work, t.work)) ||
        (rc = upload(c, &c->d_vstart, std::vector<int>(t.oct_vstart, t.oct_vstart + 8))) ||
        (rc = upload(c, &c->d_vcount, std::vector<int>(t.oct_vcount, t.oct_vcount + 8))) ||
        (rc = upload(c, &c->d_vgbase, std::vector<int>(t.oct_vgbase, t.oct_vgbase + 8))) ||
        (rc = upload(c, &c->d_vg_oct, t.vg_oct)) || (rc = dalloc_t(c, &c->blk_mass, close_blocks(n))) ||
        (rc = dalloc_t(c, &c->blk_res, (size_t)c->n_red_blocks * 10)) ||
        (rc = dalloc_t(c, &c->blk_bad, c->n_red_blocks)) || (rc = dalloc_t(c, &c->scale, 2)) ||
        (rc = dalloc_t(c, &c->resid, 3)))
        return fail(rc);
    if (t.precision == KGS_FP64) {
        if ((rc = upload(c, reinterpret_cast<double **>(&c->velm), t.velm64))) return fail(rc);
    } else {
        if ((rc = upload(c, reinterpret_cast<float **>(&c->velm), t.velm32))) return fail(rc);
    }
    if (t.any_solid && ((rc = upload(c, &c->solid, t.solid)) || (rc = upload(c, &c->blk_plain, t.blk_plain))))
        return fail(rc);
    if (t.order == 2 && ((rc = dalloc(c, &c->FX2, (size_t)t.nz * t.ny * t.Nv * rsz)) ||
                         (rc = dalloc(c, &c->FY2, (size_t)t.nz * t.nx * t.Nv * rsz)) ||
                         (rc = dalloc(c, &c->FZ2, (size_t)t.ny * t.nx * t.Nv * rsz))))
        return fail(rc);
    if (cudaMemset(c->FX, 0, (size_t)t.nz * t.ny * t.Nv * rsz) != cudaSuccess ||
        cudaMemset(c->FY, 0, (size_t)t.nz * t.nx * t.Nv * rsz) != cudaSuccess ||
        cudaMemset(c->FZ, 0, (size_t)t.ny * t.nx * t.Nv * rsz) != cudaSuccess ||
        cudaMemset(c->coef, 0, n * NCOEF * rsz) != cudaSuccess)
        return fail(KGS_ECUDA);
    if (t.order == 2 && (cudaMemset(c->FX2, 0, (size_t)t.nz * t.ny * t.Nv * rsz) != cudaSuccess ||
                         cudaMemset(c->FY2, 0, (size_t)t.nz * t.nx * t.Nv * rsz) != cudaSuccess ||
                         cudaMemset(c->FZ2, 0, (size_t)t.ny * t.nx * t.Nv * rsz) != cudaSuccess))
        return fail(KGS_ECUDA);
    if (cudaMallocHost(&c->h_resid, 3 * sizeof(double)) != cudaSuccess) return fail(KGS_ENOMEM);
    if (cudaMemset(c->resid, 0, 3 * sizeof(double)) != cudaSuccess) return fail(KGS_ECUDA);
    c->ev.resize(2 * t.stage_n.size());
    for (auto &e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(KGS_ECUDA);
    // the uploads and memsets above ran on the legacy default stream, which a
    // non-blocking stream of the caller does not wait for: complete them
    // before the first kernel on c->stream reads the tables
    if (cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) return fail(KGS_ECUDA);
    if ((rc = initial_state(c, nullptr))) return fail(rc);
    *out = c;
    return KGS_OK;
}

extern "C" {

int kgs_set_initial(kgs_ctx *c, const double *macros)
{
    if (!c) return KGS_EINVAL;
    if (cudaSetDevice(c->dev) != cudaSuccess) return KGS_ECUDA;
    (void)cudaGetLastError();  // launches below check their own status
    return initial_state(c, macros);
}

int kgs_iterate(kgs_ctx *c, int n_iters, int *done, double *residual)
{
    if (!c) return KGS_EINVAL;
    if (cudaSetDevice(c->dev) != cudaSuccess) return KGS_ECUDA;
    (void)cudaGetLastError();  // launches below check their own status
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

int kgs_sweep_sums(kgs_ctx *c, double *sums_dev)
{
    if (!c || !sums_dev) return KGS_EINVAL;
    if (cudaSetDevice(c->dev) != cudaSuccess) return KGS_ECUDA;
    (void)cudaGetLastError();  // launches below check their own status
    int rc;
    if ((rc = ctx_launch_coef(c)) || (rc = ctx_launch_stages(c)) || (rc = ctx_launch_sums(c))) return rc;
    KGS_CHECK(cudaMemcpyAsync(sums_dev, c->sums, sizeof(double) * NSUM * c->t.ncell, cudaMemcpyDeviceToDevice,
                              c->stream));
    KGS_CHECK(cudaMemcpyAsync(c->h_resid, c->resid, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    if (c->persist && *reinterpret_cast<const int *>(c->h_resid + 2) != 0) {
        KGS_CHECK(cudaMemsetAsync(c->resid + 2, 0, sizeof(double), c->stream));
        KGS_CHECK(cudaStreamSynchronize(c->stream));
        return KGS_ETIMEOUT;
    }
    return KGS_OK;
}

int kgs_close_sums(kgs_ctx *c, const double *sums_dev, double *residual)
{
    if (!c || !sums_dev) return KGS_EINVAL;
    if (cudaSetDevice(c->dev) != cudaSuccess) return KGS_ECUDA;
    (void)cudaGetLastError();
    // the closure takes the lagged velocity centre from the coefficients of
    // this iteration, which kgs_sweep_sums computed
    int rc;
    if ((rc = ctx_launch_closure(c, c->resid, sums_dev))) return rc;
    KGS_CHECK(cudaMemcpyAsync(c->h_resid, c->resid, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    const double r = c->h_resid[0];
    const bool bad = c->h_resid[1] != 0.0;
    ctx_finish(c, r);
    if (residual) *residual = r;
    return bad ? KGS_EDIVERGED : KGS_OK;
}

int kgs_moments(kgs_ctx *c, double *out)
{
    if (!c || !out) return KGS_EINVAL;
    KGS_CHECK(cudaSetDevice(c->dev));
    KGS_CHECK(cudaMemcpyAsync(out, c->mac, sizeof(double) * 8 * c->t.ncell, cudaMemcpyDeviceToHost, c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    return KGS_OK;
}

int kgs_moments_device(kgs_ctx *c, double *out_dev)
{
    if (!c || !out_dev) return KGS_EINVAL;
    KGS_CHECK(cudaSetDevice(c->dev));
    KGS_CHECK(
        cudaMemcpyAsync(out_dev, c->mac, sizeof(double) * 8 * c->t.ncell, cudaMemcpyDeviceToDevice, c->stream));
    return KGS_OK;
}

int kgs_rho_w(kgs_ctx *c, double *out)
{
    if (!c || !out) return KGS_EINVAL;
    KGS_CHECK(cudaSetDevice(c->dev));
    KGS_CHECK(cudaMemcpyAsync(out, c->rho_w, sizeof(double) * 6 * c->t.ncell, cudaMemcpyDeviceToHost, c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    return KGS_OK;
}

int kgs_set_rho_w(kgs_ctx *c, const double *in)
{
    if (!c || !in) return KGS_EINVAL;
    KGS_CHECK(cudaSetDevice(c->dev));
    KGS_CHECK(cudaMemcpyAsync(c->rho_w, in, sizeof(double) * 6 * c->t.ncell, cudaMemcpyHostToDevice, c->stream));
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
    const size_t n = c->t.ncell;
    const size_t need = sizeof(CkptHeader) + sizeof(double) * 14 * n;
    if (!buf) {
        *len = need;
        return KGS_OK;
    }
    if (*len < need) return KGS_EINVAL;
    KGS_CHECK(cudaSetDevice(c->dev));
    CkptHeader h{CKPT_MAGIC, c->t.nx, c->t.ny, c->t.nz, c->t.Nv, c->iteration, c->M0, c->last_residual};
    std::memcpy(buf, &h, sizeof h);
    double *body = reinterpret_cast<double *>(static_cast<char *>(buf) + sizeof h);
    KGS_CHECK(cudaMemcpyAsync(body, c->mac, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost, c->stream));
    KGS_CHECK(cudaMemcpyAsync(body + 8 * n, c->rho_w, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    *len = need;
    return KGS_OK;
}

int kgs_load(kgs_ctx *c, const void *buf, size_t len)
{
    if (!c || !buf) return KGS_EINVAL;
    const size_t n = c->t.ncell;
    const size_t need = sizeof(CkptHeader) + sizeof(double) * 14 * n;
    if (len != need) return KGS_EFORMAT;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.magic != CKPT_MAGIC || h.nx != c->t.nx || h.ny != c->t.ny || h.nz != c->t.nz || h.Nv != c->t.Nv)
        return KGS_EFORMAT;
    const double *body = reinterpret_cast<const double *>(static_cast<const char *>(buf) + sizeof h);
    KGS_CHECK(cudaSetDevice(c->dev));
    KGS_CHECK(cudaMemcpyAsync(c->mac, body, sizeof(double) * 8 * n, cudaMemcpyHostToDevice, c->stream));
    KGS_CHECK(cudaMemcpyAsync(c->rho_w, body + 8 * n, sizeof(double) * 6 * n, cudaMemcpyHostToDevice, c->stream));
    KGS_CHECK(cudaStreamSynchronize(c->stream));
    c->iteration = h.iteration;
    c->M0 = h.M0;
    c->last_residual = h.last_residual;
    return KGS_OK;
}

int kgs_info(kgs_ctx *c, kgs_info_t *o)
{
    if (!c || !o) return KGS_EINVAL;
    const HostTables &t = c->t;
    o->nx = t.nx;
    o->ny = t.ny;
    o->nz = t.nz;
    o->nvx = t.nvx;
    o->nvy = t.nvy;
    o->nvz = t.nvz;
    o->n_fluid = t.n_fluid;
    o->phase_points = t.n_fluid * (long long)t.Nv;
    o->iteration = c->iteration;
    o->n_stages = (int)t.stage_n.size();
    o->v_per_cta = t.vg_size;
    o->block_z = t.bz;
    o->precision = t.precision;
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
