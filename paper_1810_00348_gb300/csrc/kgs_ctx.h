// kgs_ctx.h -- the context of one problem instance and the phases of one
// outer iteration, shared by the single-instance ABI (kgs_runtime.cu) and the
// batched ABI (kgs_batch.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "kgs_switch.h"
#include "kgs_tables.h"

struct kgs_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    kgs::HostTables t;
    int mass_rescale = 0;
    int q_lagged = 0;       // heat flux about the lagged velocity (closure option)
    int max_iters = 1000;
    double tol = 1e-8;
    double M0 = 0.0;
    int iteration = 0;
    double last_residual = -1.0;
    int n_red_blocks = 0;
    // device buffers
    double *mac = nullptr, *mac_new = nullptr, *rho_w = nullptr, *rho_w_new = nullptr;
    void *coef = nullptr, *vel = nullptr, *velm = nullptr, *mtab = nullptr, *FX = nullptr, *FY = nullptr,
         *FZ = nullptr;
    void *FX2 = nullptr, *FY2 = nullptr, *FZ2 = nullptr;  // second face planes of the order-2 sweep
    void *part = nullptr;   // staged sweep only: per-(group, cell) partials
    void *acc = nullptr;    // persistent sweep: ordered accumulators [nacc][ncell][acc_slots]
    int use_acc = 0;        // the sweep runs persistent and adds into acc
    double *sums = nullptr; // [NSUM][ncell] per-cell sums of the iteration (FP64)
    double *vel64 = nullptr, *axis64 = nullptr, *rdx = nullptr, *rdy = nullptr, *rdz = nullptr;
    double *ddx = nullptr, *ddy = nullptr, *ddz = nullptr;
    uint8_t *solid = nullptr, *side_flags = nullptr, *blk_plain = nullptr;
    int8_t *wall_kind = nullptr;
    double *wall_norm = nullptr;
    int4 *work = nullptr;
    int *d_vstart = nullptr, *d_vcount = nullptr, *d_vgbase = nullptr, *d_vg_oct = nullptr;
    double *blk_mass = nullptr, *blk_res = nullptr, *scale = nullptr, *resid = nullptr;
    int *blk_bad = nullptr;
    double *h_resid = nullptr;  // pinned: residual, divergence flag, wait-error word
    // persistent sweep of a standalone context: one launch per iteration over
    // the work items in stage order; a CTA waits (bounded) for the three
    // upwind blocks of its item.  Not set up for the instances of a batch.
    int persist = 0;
    int persist_grid = 0, persist_items = 0;
    int4 *p_items = nullptr;
    int *p_counter = nullptr, *p_flags = nullptr, *p_flag_off = nullptr;
    size_t p_n_flags = 0;
    int *p_pos = nullptr;             // place of each item in its accumulator chain
    int *p_tok = nullptr;             // chain tokens [nacc][nbz][nby][nbx]
    void *p_scratch = nullptr;        // per-CTA moment partials
    size_t scratch_stride = 0;
    kgs::SweepArgs *p_args = nullptr, *h_args = nullptr;  // device copy, pinned host staging
    long long spin_limit = 20000000;  // polls of ~100 ns before a wait gives up
    size_t device_bytes = 0;
    std::vector<void *> allocs;
    // profiling
    int profiling = 0;
    std::vector<cudaEvent_t> ev;
    double sweep_ms = 0.0;
    long long sweep_launches = 0, kernel_launches = 0;
};


namespace kgs {

int cuda_err(cudaError_t e);

// Build a context on the current device and `stream` (validated inputs).
int ctx_create(kgs_ctx **out, const kgs_grid *grid, const uint8_t *solid, const kgs_vgrid *vg, const kgs_gas *gas,
               const kgs_bc *bc, const kgs_opts *opts);
void ctx_free(kgs_ctx *c);
SweepArgs ctx_sweep_args(const kgs_ctx *c);
// Work items of instance `inst` at wavefront stage `stage`, appended in the
// order the persistent sweep claims them: (inst, octant << 24 | group,
// reflected block coordinates packed 10 bits each, global group index).
void ctx_stage_items(const HostTables &t, int inst, int stage, std::vector<int4> &out);
// Set up the persistent sweep of a standalone context (items, flags, chain
// tokens, scratch, grid), or the staged sweep's partials if the persistent
// kernel cannot be resident.
int ctx_persist_init(kgs_ctx *c);
// Ordered accumulators of a context whose sweep runs persistent.
int ctx_alloc_acc(kgs_ctx *c);
// Chain tokens per (accumulator, block) of one instance.
inline size_t ctx_n_tokens(const HostTables &t) { return (size_t)t.nacc * t.nbx * t.nby * t.nbz; }
// Place of every item of a stage-ordered work list in its accumulator chain
// (items of one (instance, accumulator, block), in list order).
void chain_positions(const std::vector<int4> &items, const std::vector<const HostTables *> &tabs,
                     std::vector<int> &pos);
// Phases of one outer iteration (asynchronous on the context's stream).
int ctx_launch_coef(kgs_ctx *c);
int ctx_launch_stages(kgs_ctx *c);
// Per-cell sums of the swept velocities into c->sums.
int ctx_launch_sums(kgs_ctx *c);
// Closure from the per-cell sums (sums = NULL: c->sums) into the new buffers;
// the residual and divergence flag go to resid_dev[0..1] (device).
int ctx_launch_closure(kgs_ctx *c, double *resid_dev, const double *sums);
// After the iteration's work has completed: swap the state buffers.
void ctx_finish(kgs_ctx *c, double residual);

}  // namespace kgs
