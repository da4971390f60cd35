// kgs_autotune.cu -- picks the sweep shape (velocities per thread block and
// block depth along z) of a problem by timing a few outer iterations of each
// candidate on the device, and caches the choice per problem shape (in the
// process, and in the file named by KGS_AUTOTUNE_CACHE when it is set).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

#include "kgs_ctx.h"

using namespace kgs;

namespace {

std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, int>> g_tune_cache;

std::string shape_key(const kgs_problem *p, int precision)
{
    bool any_solid = false;
    if (p->solid) {
        const long long n = (long long)p->grid.nx * p->grid.ny * p->grid.nz;
        for (long long i = 0; i < n && !any_solid; i++) any_solid = p->solid[i] != 0;
    }
    char buf[160];
    std::snprintf(buf, sizeof buf, "p%d_c%dx%dx%d_v%dx%dx%d_s%d", precision, p->grid.nx, p->grid.ny, p->grid.nz,
                  p->vgrid.nvx, p->vgrid.nvy, p->vgrid.nvz, any_solid ? 1 : 0);
    return buf;
}

bool file_lookup(const std::string &key, int *vpc, int *bz)
{
    const char *path = std::getenv("KGS_AUTOTUNE_CACHE");
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char k[160];
    int a = 0, b = 0;
    double ms = 0;
    bool found = false;
    while (std::fscanf(f, "%159s %d %d %lf", k, &a, &b, &ms) == 4)
        if (key == k) {
            *vpc = a;
            *bz = b;
            found = true;
        }
    std::fclose(f);
    return found;
}

void file_store(const std::string &key, int vpc, int bz, double ms)
{
    const char *path = std::getenv("KGS_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %.6f\n", key.c_str(), vpc, bz, ms);
    std::fclose(f);
}

// Mean device time (ms) of one outer iteration with the given shape, after
// one untimed iteration.
int time_shape(const kgs_problem *p, int precision, int vpc, int bz, double *ms)
{
    kgs_opts o{};
    o.precision = precision;
    o.wall_norm = p->wall_norm;
    o.mass_rescale = p->mass_rescale;
    o.v_per_cta = vpc;
    o.block_z = bz;
    kgs_ctx *c = nullptr;
    int rc = ctx_create(&c, &p->grid, p->solid, &p->vgrid, &p->gas, &p->bc, &o);
    if (rc) return rc;
    if ((rc = ctx_persist_init(c))) {  // time the sweep that contexts and batches run
        ctx_free(c);
        delete c;
        return rc;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int timed = 2;
    auto one = [&]() -> int {
        int r;
        if ((r = ctx_launch_coef(c)) || (r = ctx_launch_stages(c)) || (r = ctx_launch_sums(c)) ||
            (r = ctx_launch_closure(c, c->resid, nullptr)))
            return r;
        std::swap(c->mac, c->mac_new);
        std::swap(c->rho_w, c->rho_w_new);
        return KGS_OK;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = KGS_ECUDA;
    if (!rc) rc = one();
    if (!rc && cudaEventRecord(e0, c->stream) != cudaSuccess) rc = KGS_ECUDA;
    for (int k = 0; k < timed && !rc; k++) rc = one();
    if (!rc && cudaEventRecord(e1, c->stream) != cudaSuccess) rc = KGS_ECUDA;
    if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = KGS_ECUDA;
    float t = 0.f;
    if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = KGS_ECUDA;
    *ms = t / timed;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(c->stream);
    ctx_free(c);
    delete c;
    return rc;
}

}  // namespace

extern "C" int kgs_autotune(const kgs_problem *p, int precision, int *v_per_cta, int *block_z)
{
    if (!p || !v_per_cta || !block_z) return KGS_EINVAL;
    int rc = validate_problem(&p->grid, p->solid, &p->vgrid, &p->gas, &p->bc, precision, p->wall_norm, 0, 0);
    if (rc) return rc;
    (void)cudaGetLastError();  // launches below check their own status
    const std::string key = shape_key(p, precision);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
        *v_per_cta = it->second.first;
        *block_z = it->second.second;
        return KGS_OK;
    }
    int vpc = 0, bz = 0;
    if (file_lookup(key, &vpc, &bz)) {
        g_tune_cache[key] = {vpc, bz};
        *v_per_cta = vpc;
        *block_z = bz;
        return KGS_OK;
    }
    const int vpcs_mixed[] = {128, 256}, vpcs_fp64[] = {128};
    const int bzs[] = {8, 16, 32};
    const int *vpcs = precision == KGS_FP64 ? vpcs_fp64 : vpcs_mixed;
    const int nv = precision == KGS_FP64 ? 1 : 2;
    double best = 1e300;
    for (int a = 0; a < nv; a++)
        for (int bzi : bzs) {
            if (bzi > 2 * p->grid.nz && bzi != bzs[0]) continue;  // deeper than the grid: same as a smaller one
            double ms = 0.0;
            rc = time_shape(p, precision, vpcs[a], bzi, &ms);
            if (rc) return rc;
            if (ms < best) {
                best = ms;
                vpc = vpcs[a];
                bz = bzi;
            }
        }
    g_tune_cache[key] = {vpc, bz};
    file_store(key, vpc, bz, best);
    *v_per_cta = vpc;
    *block_z = bz;
    return KGS_OK;
}
