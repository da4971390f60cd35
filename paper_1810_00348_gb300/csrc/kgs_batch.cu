// kgs_batch.cu -- many independent problem instances (e.g. cavities of
// uneven sizes) advanced together: one persistent sweep launch per outer
// iteration for all instances, the per-instance coefficient and closure
// kernels around it, the whole iteration captured in a CUDA graph and
// replayed.  Instances that reach the tolerance retire from the work list.
//
// Each instance is an ordinary context (kgs_ctx) created on the batch's
// stream; the batch adds the persistent work list, the completion flags and
// the graphs.  Work items are (instance, octant, velocity group, block) in
// stage order; a CTA of the persistent kernel waits (bounded) for the three
// upwind blocks of its item before sweeping it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "kgs_ctx.h"

using namespace kgs;

struct kgs_batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;  // graphs cannot be captured on the legacy default stream
    int n = 0;
    std::vector<kgs_ctx *> ctx;
    int precision = KGS_MIXED, tv = 2, bz = 32, line16 = 0, uniform = 0, nxo_max = 1;
    int dev_src = 0;  // deviation-form FP32 source (kgs_opts.dev_source)
    int max_iters = 1000;
    double tol = 1e-8;
    std::vector<char> active;
    std::vector<int> done;  // iterations per instance since setup / set_initial
    // persistent sweep
    SweepArgs *d_args[2] = {nullptr, nullptr};
    int4 *d_items = nullptr;
    size_t items_cap = 0;
    int n_items = 0;
    int *d_counter = nullptr, *d_flags = nullptr, *d_flag_off = nullptr, *d_error = nullptr;
    size_t n_flags = 0;
    int *d_pos = nullptr;               // place of each item in its accumulator chain
    size_t pos_cap = 0;
    int *d_tok = nullptr;               // chain tokens of all instances
    size_t n_tok = 0;
    std::vector<size_t> tok_off;        // first token of each instance
    void *d_scratch = nullptr;          // per-CTA moment partials
    size_t scratch_stride = 0;
    double *d_resid = nullptr;  // [2 n] + error word
    double *h_resid = nullptr;  // pinned copy
    int grid = 0;
    long long spin_limit = 20000000;  // ~2 s of polling at 100 ns per poll
    int skip_publish = -1;             // fault injection (kgs_batch_fault)
    // graphs: [0] with the current buffers, [1] with the swapped buffers
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    bool dirty = true;
    int next = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double sweep_ms = 0.0;
    long long sweeps = 0, kernel_launches = 0;
};

namespace {

#define KGS_CHECK(call)                             \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_err(e_); \
    } while (0)

void swap_state(kgs_ctx *c)
{
    std::swap(c->mac, c->mac_new);
    std::swap(c->rho_w, c->rho_w_new);
}

void destroy_graphs(kgs_batch *b)
{
    for (auto &e : b->exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
}

// Work list of the active instances in stage order.
int build_items(kgs_batch *b)
{
    std::vector<int4> items;
    int max_stage = 0;
    for (int i = 0; i < b->n; i++)
        if (b->active[i]) max_stage = std::max(max_stage, (int)b->ctx[i]->t.stage_n.size());
    for (int s = 0; s < max_stage; s++)
        for (int i = 0; i < b->n; i++)
            if (b->active[i]) ctx_stage_items(b->ctx[i]->t, i, s, items);
    b->n_items = (int)items.size();
    if (items.size() > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        KGS_CHECK(cudaMalloc(&b->d_items, items.size() * sizeof(int4)));
        b->items_cap = items.size();
    }
    std::vector<const HostTables *> tabs(b->n);
    for (int i = 0; i < b->n; i++) tabs[i] = &b->ctx[i]->t;
    std::vector<int> pos;
    chain_positions(items, tabs, pos);
    if (pos.size() > b->pos_cap) {
        if (b->d_pos) cudaFree(b->d_pos);
        b->d_pos = nullptr;
        KGS_CHECK(cudaMalloc(&b->d_pos, pos.size() * sizeof(int)));
        b->pos_cap = pos.size();
    }
    if (!items.empty()) {
        KGS_CHECK(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
        KGS_CHECK(cudaMemcpy(b->d_pos, pos.data(), pos.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    return KGS_OK;
}

int upload_args(kgs_batch *b, int which)
{
    std::vector<SweepArgs> args(b->n);
    for (int i = 0; i < b->n; i++) {
        args[i] = ctx_sweep_args(b->ctx[i]);
        args[i].tok = b->d_tok + b->tok_off[i];
    }
    KGS_CHECK(cudaMemcpy(b->d_args[which], args.data(), args.size() * sizeof(SweepArgs), cudaMemcpyHostToDevice));
    return KGS_OK;
}

// Enqueue one outer iteration of every active instance (no host sync).
int enqueue_iteration(kgs_batch *b, int which)
{
    int rc;
    cudaStream_t st = b->stream;
    for (int i = 0; i < b->n; i++)
        if (b->active[i] && (rc = ctx_launch_coef(b->ctx[i]))) return rc;
    KGS_CHECK(cudaMemsetAsync(b->d_counter, 0, sizeof(int), st));
    KGS_CHECK(cudaMemsetAsync(b->d_flags, 0, b->n_flags * sizeof(int), st));
    KGS_CHECK(cudaMemsetAsync(b->d_error, 0, sizeof(int), st));
    KGS_CHECK(cudaMemsetAsync(b->d_tok, 0, b->n_tok * sizeof(int), st));
    BatchSweepArgs ba;
    ba.inst = b->d_args[which];
    ba.items = b->d_items;
    ba.n_items = b->n_items;
    ba.counter = b->d_counter;
    ba.flags = b->d_flags;
    ba.flag_off = b->d_flag_off;
    ba.pos = b->d_pos;
    ba.scratch = b->d_scratch;
    ba.scratch_stride = b->scratch_stride;
    ba.error = b->d_error;
    ba.spin_limit = b->spin_limit;
    ba.skip_publish = b->skip_publish;
    // external records: inside a capture a plain record only orders streams
    KGS_CHECK(cudaEventRecordWithFlags(b->ev[0], st, cudaEventRecordExternal));
    KGS_CHECK(launch_sweep_persistent(b->precision, b->tv, b->line16, b->uniform, ba, b->nxo_max, b->grid, st, 1,
                                      b->dev_src));
    KGS_CHECK(cudaEventRecordWithFlags(b->ev[1], st, cudaEventRecordExternal));
    for (int i = 0; i < b->n; i++)
        if (b->active[i] &&
            ((rc = ctx_launch_sums(b->ctx[i])) || (rc = ctx_launch_closure(b->ctx[i], b->d_resid + 2 * i, nullptr))))
            return rc;
    KGS_CHECK(cudaMemcpyAsync(b->h_resid, b->d_resid, (2 * b->n + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
    return KGS_OK;
}

// Capture the two graphs (current buffers, swapped buffers).
int rebuild(kgs_batch *b)
{
    int rc;
    destroy_graphs(b);
    if ((rc = build_items(b))) return rc;
    for (int which = 0; which < 2; which++) {
        if ((rc = upload_args(b, which))) return rc;
        cudaGraph_t g = nullptr;
        KGS_CHECK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_iteration(b, which);
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        KGS_CHECK(e);
        e = cudaGraphInstantiate(&b->exec[which], g, 0);
        cudaGraphDestroy(g);
        KGS_CHECK(e);
        for (int i = 0; i < b->n; i++) swap_state(b->ctx[i]);
    }
    // The work list, chain places and arguments (and, before the first
    // rebuild, the set-up tables) were copied on the legacy default stream;
    // the graphs run on the batch's stream, which need not wait for it.
    KGS_CHECK(cudaStreamSynchronize(cudaStreamLegacy));
    // two swaps: every instance is back on its current buffers
    b->next = 0;
    b->dirty = false;
    return KGS_OK;
}

void free_batch(kgs_batch *b)
{
    destroy_graphs(b);
    for (kgs_ctx *c : b->ctx)
        if (c) {
            ctx_free(c);
            delete c;
        }
    b->ctx.clear();
    // d_error lives inside d_resid
    void *bufs[] = {b->d_args[0], b->d_args[1], b->d_items, b->d_counter, b->d_flags, b->d_flag_off, b->d_resid,
                    b->d_pos, b->d_tok, b->d_scratch};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (b->h_resid) cudaFreeHost(b->h_resid);
    for (auto &e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

// One outer iteration of the active instances (graph replay).  count and
// last receive, per instance, the iterations run and the last residual;
// retire: instances below the tolerance leave the work list.  Returns false
// when nothing is active or an error (rc) stops the run.
bool batch_step(kgs_batch *b, bool retire, std::vector<int> &count, std::vector<double> &last, int &rc)
{
    bool any = false;
    for (int i = 0; i < b->n; i++) any |= b->active[i] != 0;
    if (!any) return false;
    if (b->dirty && (rc = rebuild(b))) return false;
    const int which = b->next;
    cudaError_t e = cudaGraphLaunch(b->exec[which], b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        rc = cuda_err(e);
        return false;
    }
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
    if (e != cudaSuccess) {
        rc = cuda_err(e);
        return false;
    }
    b->sweep_ms += ms;
    b->sweeps++;
    const int *err = reinterpret_cast<const int *>(b->h_resid + 2 * b->n);
    if (*err) {
        rc = KGS_ETIMEOUT;
        return false;
    }
    bool bad = false, retired = false;
    for (int i = 0; i < b->n; i++) {
        if (!b->active[i]) continue;
        const double r = b->h_resid[2 * i];
        bad |= b->h_resid[2 * i + 1] != 0.0;
        ctx_finish(b->ctx[i], r);
        b->kernel_launches += 6;  // coefficients, sums, four closure kernels
        count[i]++;
        b->done[i]++;
        last[i] = r;
        if (retire && r < b->tol) {
            b->active[i] = 0;
            retired = true;
        }
    }
    b->kernel_launches += 1;
    b->next = 1 - which;
    if (retired) b->dirty = true;
    if (bad) {
        rc = KGS_EDIVERGED;
        return false;
    }
    return true;
}

}  // namespace

extern "C" {

int kgs_batch_setup(kgs_batch **out, int n, const kgs_problem *probs, const kgs_opts *opts)
{
    if (!out || n < 1 || !probs || !opts) return KGS_EINVAL;
    *out = nullptr;
    if (opts->order == 2) return KGS_EINVAL;  // batches sweep at first order
    int vpc = opts->v_per_cta, bz = opts->block_z;
    if (vpc == 0 && bz == 0) {
        // shapes of the largest instance, picked by the autotuner
        int big = 0;
        long long best = -1;
        for (int i = 0; i < n; i++) {
            const long long pp = (long long)probs[i].grid.nx * probs[i].grid.ny * probs[i].grid.nz *
                                 probs[i].vgrid.nvx * probs[i].vgrid.nvy * probs[i].vgrid.nvz;
            if (pp > best) best = pp, big = i;
        }
        int rc = kgs_autotune(&probs[big], opts->precision, &vpc, &bz);
        if (rc) return rc;
    }
    for (int i = 0; i < n; i++) {
        const kgs_problem &p = probs[i];
        int rc = validate_problem(&p.grid, p.solid, &p.vgrid, &p.gas, &p.bc, opts->precision, p.wall_norm, vpc, bz,
                                  0, 0, 1, opts->dev_source);
        if (rc) return rc;
    }
    (void)cudaGetLastError();  // launches below check their own status
    kgs_batch *b = new (std::nothrow) kgs_batch();
    if (!b) return KGS_ENOMEM;
    auto fail = [&](int rc) {
        free_batch(b);
        delete b;
        return rc;
    };
    if (cudaGetDevice(&b->dev) != cudaSuccess) return fail(KGS_ECUDA);
    b->stream = static_cast<cudaStream_t>(opts->stream);
    if (!b->stream) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(KGS_ECUDA);
        b->own_stream = true;
    }
    b->n = n;
    b->precision = opts->precision;
    b->dev_src = opts->dev_source ? 1 : 0;
    b->max_iters = opts->max_iters > 0 ? opts->max_iters : 1000;
    b->tol = opts->tol > 0.0 ? opts->tol : 1e-8;
    b->ctx.assign(n, nullptr);
    b->active.assign(n, 1);
    b->done.assign(n, 0);
    std::vector<int> flag_off(n);
    b->line16 = 1;
    b->uniform = 1;
    for (int i = 0; i < n; i++) {
        const kgs_problem &p = probs[i];
        kgs_opts o = *opts;
        o.stream = b->stream;
        o.wall_norm = p.wall_norm;
        o.mass_rescale = p.mass_rescale;
        o.q_lagged = p.q_lagged;
        o.order = 1;
        o.dev_source = opts->dev_source;
        o.v_per_cta = vpc;
        o.block_z = bz;
        int rc = ctx_create(&b->ctx[i], &p.grid, p.solid, &p.vgrid, &p.gas, &p.bc, &o);
        if (rc || (rc = ctx_alloc_acc(b->ctx[i]))) return fail(rc);
        const HostTables &t = b->ctx[i]->t;
        b->tok_off.push_back(b->n_tok);
        b->n_tok += ctx_n_tokens(t);
        b->tv = t.tv;
        b->bz = t.bz;
        b->nxo_max = std::max(b->nxo_max, t.nxo_max);
        for (int q = 0; q < 8; q++)
            if (t.oct_vcount[q] > 0 && t.oct_nx[q] != 16) b->line16 = 0;
        if (!ctx_sweep_args(b->ctx[i]).uniform) b->uniform = 0;
        flag_off[i] = (int)b->n_flags;
        b->n_flags += (size_t)t.n_vg * t.nbx * t.nby * t.nbz;
    }
    // every instance must see the same shared-memory layout
    for (int i = 0; i < n; i++) b->ctx[i]->t.nxo_max = b->nxo_max;
    if (cudaMalloc(&b->d_args[0], n * sizeof(SweepArgs)) != cudaSuccess ||
        cudaMalloc(&b->d_args[1], n * sizeof(SweepArgs)) != cudaSuccess ||
        cudaMalloc(&b->d_counter, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_flags, std::max<size_t>(b->n_flags, 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_flag_off, n * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_resid, (2 * n + 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->d_tok, b->n_tok * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&b->h_resid, (2 * n + 1) * sizeof(double)) != cudaSuccess)
        return fail(KGS_ENOMEM);
    // the error word shares the residual buffer so one copy brings both back
    b->d_error = reinterpret_cast<int *>(b->d_resid + 2 * n);
    if (cudaMemcpy(b->d_flag_off, flag_off.data(), n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_resid, 0, (2 * n + 1) * sizeof(double)) != cudaSuccess ||
        cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess)
        return fail(KGS_ECUDA);
    // persistent grid: as many CTAs as fit on the device at once
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev) != cudaSuccess) return fail(KGS_ECUDA);
    const size_t smem = sweep_smem_bytes(b->precision, b->tv, b->line16, b->nxo_max);
    per_sm = sweep_persistent_occupancy(b->precision, b->tv, b->line16, b->uniform, smem, 1, b->dev_src);
    if (per_sm < 1) return fail(KGS_ECUDA);
    b->grid = sms * per_sm;
    b->scratch_stride = sweep_scratch_bytes(b->bz);
    if (cudaMalloc(&b->d_scratch, (size_t)b->grid * b->scratch_stride) != cudaSuccess) return fail(KGS_ENOMEM);
    *out = b;
    return KGS_OK;
}

int kgs_batch_iterate(kgs_batch *b, int n_iters, int *iters_done, double *residuals)
{
    if (!b) return KGS_EINVAL;
    if (cudaSetDevice(b->dev) != cudaSuccess) return KGS_ECUDA;
    (void)cudaGetLastError();  // launches below check their own status
    const bool until = n_iters <= 0;
    const int limit = until ? b->max_iters : n_iters;
    std::vector<int> count(b->n, 0);
    std::vector<double> last(b->n, -1.0);
    for (int i = 0; i < b->n; i++) last[i] = b->ctx[i]->last_residual;
    if (!until) {
        // a fixed number of iterations runs every instance, retired or not
        for (int i = 0; i < b->n; i++)
            if (!b->active[i]) {
                b->active[i] = 1;
                b->dirty = true;
            }
    }
    int rc = KGS_OK;
    for (int k = 0; k < limit; k++)
        if (!batch_step(b, until, count, last, rc)) break;
    if (rc == KGS_OK && until)
        for (int i = 0; i < b->n; i++)
            if (!(last[i] >= 0.0 && last[i] < b->tol)) rc = KGS_NOTCONVERGED;
    if (iters_done)
        for (int i = 0; i < b->n; i++) iters_done[i] = count[i];
    if (residuals)
        for (int i = 0; i < b->n; i++) residuals[i] = last[i];
    return rc;
}

int kgs_batch_solve(kgs_batch **out, int n, const kgs_problem *probs, const kgs_opts *opts, int *iters_mixed,
                    int *iters_fp64, double *residuals)
{
    if (!out || n < 1 || !probs || !opts || !(opts->tol > 0.0)) return KGS_EINVAL;
    *out = nullptr;
    const int budget = opts->max_iters > 0 ? opts->max_iters : 1000;
    kgs_batch *m = nullptr, *d = nullptr;
    auto finish = [&](int code) {
        if (m) kgs_batch_destroy(m);
        if (code != KGS_OK && code != KGS_NOTCONVERGED && d) {
            kgs_batch_destroy(d);
            d = nullptr;
        }
        *out = d;
        return code;
    };
    // mixed phase: every instance runs until it reaches tol or stops making
    // progress (the rule of kgs_solve, per instance), then retires
    kgs_opts om = *opts;
    om.precision = KGS_MIXED;
    // the deviation-form source (lower residual floor) where every instance allows it
    om.dev_source = 1;
    for (int i = 0; i < n; i++)
        if (!dev_source_applies(&probs[i].grid, &probs[i].bc)) om.dev_source = 0;
    int rc = kgs_batch_setup(&m, n, probs, &om);
    if (rc) return finish(rc);
    if (cudaSetDevice(m->dev) != cudaSuccess) return finish(KGS_ECUDA);
    std::vector<int> nm(n, 0), nd(n, 0);
    std::vector<SolveSwitch> sw(n);
    std::vector<double> last(n, -1.0);
    for (;;) {
        bool any = false;
        for (int i = 0; i < n; i++) any |= m->active[i] != 0;
        if (!any) break;
        std::vector<int> count(n, 0);
        for (int k = 0; k < SOLVE_CHUNK; k++)
            if (!batch_step(m, false, count, last, rc)) break;
        if (rc) return finish(rc);
        for (int i = 0; i < n; i++) {
            if (!m->active[i]) continue;
            nm[i] += count[i];
            const double r = last[i];
            const bool retire = r < opts->tol || nm[i] >= budget || sw[i].stalled_after(r);
            if (retire) {
                m->active[i] = 0;
                m->dirty = true;
            }
        }
    }
    // FP64 phase from each mixed state (macros, wall densities, mass target)
    kgs_opts od = *opts;
    od.precision = KGS_FP64;
    od.dev_source = 0;
    od.v_per_cta = 128;
    od.block_z = opts->block_z > 0 ? opts->block_z : 32;
    if ((rc = kgs_batch_setup(&d, n, probs, &od))) return finish(rc);
    std::vector<unsigned char> state;
    for (int i = 0; i < n; i++) {
        size_t len = 0;
        if ((rc = kgs_save(m->ctx[i], nullptr, &len))) return finish(rc);
        state.resize(len);
        if ((rc = kgs_save(m->ctx[i], state.data(), &len)) || (rc = kgs_load(d->ctx[i], state.data(), len)))
            return finish(rc);
        // every instance with budget left runs at least one FP64 iteration
        // (it confirms the tolerance), at most max(1, budget - mixed iterations)
        d->active[i] = nm[i] < budget;
    }
    d->dirty = true;
    std::vector<int> count(n, 0);
    std::vector<double> dl(last);
    for (;;) {
        if (!batch_step(d, true, count, dl, rc)) break;
        for (int i = 0; i < n; i++)
            if (d->active[i] && count[i] >= std::max(1, budget - nm[i])) {
                d->active[i] = 0;
                d->dirty = true;
            }
    }
    if (rc) return finish(rc);
    int status = KGS_OK;
    for (int i = 0; i < n; i++) {
        if (iters_mixed) iters_mixed[i] = nm[i];
        if (iters_fp64) iters_fp64[i] = count[i];
        if (residuals) residuals[i] = dl[i];
        if (!(dl[i] >= 0.0 && dl[i] < opts->tol)) status = KGS_NOTCONVERGED;
    }
    return finish(status);
}

int kgs_batch_moments(kgs_batch *b, int i, double *out)
{
    if (!b || i < 0 || i >= b->n) return KGS_EINVAL;
    return kgs_moments(b->ctx[i], out);
}

int kgs_batch_set_initial(kgs_batch *b, int i, const double *macros)
{
    if (!b || i < 0 || i >= b->n) return KGS_EINVAL;
    const int rc = kgs_set_initial(b->ctx[i], macros);
    b->active[i] = 1;
    b->done[i] = 0;
    b->dirty = true;  // the reference mass is a launch parameter of the graphs
    return rc;
}

int kgs_batch_info(kgs_batch *b, int i, kgs_info_t *out)
{
    if (!b || i < 0 || i >= b->n) return KGS_EINVAL;
    return kgs_info(b->ctx[i], out);
}

int kgs_batch_profile(kgs_batch *b, double *sweep_ms, long long *sweeps, long long *kernel_launches)
{
    if (!b) return KGS_EINVAL;
    if (sweep_ms) *sweep_ms = b->sweep_ms;
    if (sweeps) *sweeps = b->sweeps;
    if (kernel_launches) *kernel_launches = b->kernel_launches;
    b->sweep_ms = 0.0;
    b->sweeps = 0;
    b->kernel_launches = 0;
    return KGS_OK;
}

int kgs_batch_fault(kgs_batch *b, long long spin_limit, int unpublished_item)
{
    if (!b || spin_limit < 1) return KGS_EINVAL;
    b->spin_limit = spin_limit;
    b->skip_publish = unpublished_item;
    b->dirty = true;  // both are launch parameters of the graphs
    return KGS_OK;
}

void kgs_batch_destroy(kgs_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->dev);
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
}

}  // extern "C"
