// kgs_noalloc.cu -- kgs_iterate_noalloc: one outer iteration of a small
// problem without any device memory allocation (declared in include/kgs.h).
//
// Some callers cannot allocate device memory: code that runs inside a host
// framework that owns every byte of the device through its own pool, code
// on a latency-critical path where cudaMalloc's implicit synchronisation is
// not acceptable, or code that must be set up once and then never allocate.
// They pass their own device buffers for the inputs and outputs; every
// intermediate buffer of the iteration (coefficients, velocity and wall
// tables, block faces, moment partials, reduction scratch) is carved out of
// one file-scope __device__ array of fixed size, which every GPU that loads
// the library holds until the process exits.
//
// The host code never dereferences the array's name (in host code it is
// only a stand-in for the symbol): its device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call made on the device, and cached.  Every call shares the array and
// leaves its contents behind, so the parts that must start at zero are
// cleared on each call, and calls that overlap on the GPU (other streams,
// other host threads) race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "kgs_tables.h"

using namespace kgs;

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[KGS_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mutex;
void *g_scratch_addr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device).
int scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return KGS_EINVAL;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return KGS_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return KGS_OK;
}

// Byte offsets of the buffers inside the scratch array, 256-byte aligned.
struct Carve {
    size_t used = 0;
    size_t take(size_t bytes)
    {
        const size_t off = used;
        used += (bytes + 255) & ~size_t(255);
        return off;
    }
};

}  // namespace

extern "C" int kgs_iterate_noalloc(const kgs_grid *grid, const uint8_t *solid, const kgs_vgrid *vgrid,
                                   const kgs_gas *gas, const kgs_bc *bc, int precision, int wall_norm,
                                   double M0, const double *macros_in, const double *rho_w_in,
                                   double *macros_out, double *rho_w_out, double *residual, void *stream)
{
    if (!macros_in || !rho_w_in || !macros_out || !rho_w_out) return KGS_EINVAL;
    if (macros_out == macros_in || rho_w_out == rho_w_in) return KGS_EINVAL;
    int rc = validate_problem(grid, solid, vgrid, gas, bc, precision, wall_norm, 0, 0);
    if (rc) return rc;
    HostTables t;
    build_tables(t, grid, solid, vgrid, gas, bc, precision, wall_norm, 0, 0);
    const size_t n = t.ncell, rsz = t.real_bytes();
    const int n_red = (int)((n + 255) / 256);

    Carve cv;
    const size_t o_coef = cv.take(n * NCOEF * rsz);
    const size_t o_vel = cv.take(t.vel64.size() * rsz);
    const size_t o_velm = cv.take((size_t)t.Nv * 8 * rsz);
    const size_t o_mt = cv.take(t.mt.size() * rsz);
    const size_t fx_bytes = (size_t)t.nz * t.ny * t.Nv * rsz, fy_bytes = (size_t)t.nz * t.nx * t.Nv * rsz,
                 fz_bytes = (size_t)t.ny * t.nx * t.Nv * rsz;
    const size_t o_fx = cv.take(fx_bytes), o_fy = cv.take(fy_bytes), o_fz = cv.take(fz_bytes);
    const size_t o_part = cv.take((size_t)t.n_vg * NPART * n * 8);
    const size_t o_sums = cv.take((size_t)NSUM * n * sizeof(double));
    const size_t o_rdx = cv.take(t.nx * sizeof(double)), o_rdy = cv.take(t.ny * sizeof(double)),
                 o_rdz = cv.take(t.nz * sizeof(double));
    const size_t o_dx = cv.take(t.nx * sizeof(double)), o_dy = cv.take(t.ny * sizeof(double)),
                 o_dz = cv.take(t.nz * sizeof(double));
    const size_t o_flags = cv.take(t.side_flags.size()), o_kind = cv.take(t.wall_kind.size());
    const size_t o_norm = cv.take(t.wall_norm.size() * sizeof(double));
    const size_t o_work = cv.take(t.work.size() * sizeof(int4));
    const size_t o_oct = cv.take(3 * 8 * sizeof(int));
    const size_t o_vgoct = cv.take(t.vg_oct.size() * sizeof(int));
    const size_t o_solid = cv.take(t.any_solid ? n : 0);
    const size_t o_bmass = cv.take(close_blocks(n) * sizeof(double)), o_bres = cv.take((size_t)n_red * 10 * sizeof(double)),
                 o_bbad = cv.take(n_red * sizeof(int)), o_scale = cv.take(2 * sizeof(double)),
                 o_resid = cv.take(2 * sizeof(double));
    if (cv.used > (size_t)KGS_NOALLOC_SCRATCH_BYTES) return KGS_EINVAL;  // too large for the fixed array

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KGS_ECUDA;
    (void)cudaGetLastError();  // launches below check their own status
    void *base = nullptr;
    if ((rc = scratch_address(dev, &base))) return rc;
    unsigned char *b = static_cast<unsigned char *>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto put = [&](size_t off, const void *src, size_t bytes) -> bool {
        return bytes == 0 || cudaMemcpyAsync(b + off, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
    };
    auto put_real = [&](size_t off, const std::vector<double> &h) -> bool {
        if (rsz == sizeof(double)) return put(off, h.data(), h.size() * sizeof(double));
        std::vector<float> f(h.begin(), h.end());
        // pageable source: the copy is staged before cudaMemcpyAsync returns
        return put(off, f.data(), f.size() * sizeof(float));
    };
    int oct[24];
    for (int o = 0; o < 8; o++) {
        oct[o] = t.oct_vstart[o];
        oct[8 + o] = t.oct_vcount[o];
        oct[16 + o] = t.oct_vgbase[o];
    }
    bool ok = put_real(o_vel, t.vel64) &&
              put_real(o_mt, t.mt) &&
              (rsz == sizeof(double) ? put(o_velm, t.velm64.data(), t.velm64.size() * sizeof(double))
                                     : put(o_velm, t.velm32.data(), t.velm32.size() * sizeof(float))) &&
              put(o_rdx, t.rdx.data(), t.nx * sizeof(double)) && put(o_rdy, t.rdy.data(), t.ny * sizeof(double)) &&
              put(o_rdz, t.rdz.data(), t.nz * sizeof(double)) && put(o_dx, t.dx.data(), t.nx * sizeof(double)) &&
              put(o_dy, t.dy.data(), t.ny * sizeof(double)) && put(o_dz, t.dz.data(), t.nz * sizeof(double)) &&
              put(o_flags, t.side_flags.data(), t.side_flags.size()) &&
              put(o_kind, t.wall_kind.data(), t.wall_kind.size()) &&
              put(o_norm, t.wall_norm.data(), t.wall_norm.size() * sizeof(double)) &&
              put(o_work, t.work.data(), t.work.size() * sizeof(int4)) && put(o_oct, oct, sizeof oct) &&
              put(o_vgoct, t.vg_oct.data(), t.vg_oct.size() * sizeof(int)) &&
              (!t.any_solid || put(o_solid, t.solid.data(), n));
    if (!ok) return KGS_ECUDA;
    // what the previous call left behind: face planes and coefficients start at zero
    if (cudaMemsetAsync(b + o_fx, 0, fx_bytes, st) != cudaSuccess ||
        cudaMemsetAsync(b + o_fy, 0, fy_bytes, st) != cudaSuccess ||
        cudaMemsetAsync(b + o_fz, 0, fz_bytes, st) != cudaSuccess ||
        cudaMemsetAsync(b + o_coef, 0, n * NCOEF * rsz, st) != cudaSuccess)
        return KGS_ECUDA;

    const uint8_t *d_solid = t.any_solid ? b + o_solid : nullptr;
    void *coef = b + o_coef;
    if (launch_coef(t.precision, macros_in, d_solid, b + o_flags, reinterpret_cast<double *>(b + o_rdx),
                    reinterpret_cast<double *>(b + o_rdy), reinterpret_cast<double *>(b + o_rdz), t.nx, t.ny, t.nz,
                    t.mu_ref, t.omega, t.Pr, coef, st) != cudaSuccess)
        return KGS_ECUDA;
    SweepArgs a{};
    a.nx = t.nx;
    a.ny = t.ny;
    a.nz = t.nz;
    a.bz = t.bz;
    a.nbx = t.nbx;
    a.nby = t.nby;
    a.nbz = t.nbz;
    const int *d_oct = reinterpret_cast<const int *>(b + o_oct);
    a.oct_vstart = d_oct;
    a.oct_vcount = d_oct + 8;
    a.oct_vgbase = d_oct + 16;
    a.Nv = t.Nv;
    a.vg_size = t.vg_size;
    a.vel = b + o_vel;
    a.velm = b + o_velm;
    a.nxo_max = t.nxo_max;
    a.line16 = 1;
    for (int o = 0; o < 8; o++) {
        a.oct_nx[o] = t.oct_nx[o] > 0 ? t.oct_nx[o] : 1;
        if (t.oct_vcount[o] > 0 && t.oct_nx[o] != 16) a.line16 = 0;
    }
    a.any_solid = t.any_solid ? 1 : 0;
    t.set_uniformity(a);
    a.coef = coef;
    a.rho_w = rho_w_in;
    a.mtab = b + o_mt;
    for (int s = 0; s < 6; s++) a.side_inflow[s] = t.side_inflow[s];
    a.FX = b + o_fx;
    a.FY = b + o_fy;
    a.FZ = b + o_fz;
    a.part = b + o_part;
    a.ncell = n;
    const int4 *d_work = reinterpret_cast<const int4 *>(b + o_work);
    for (size_t s = 0; s < t.stage_n.size(); s++) {
        a.work = d_work + t.stage_off[s];
        if (launch_sweep(t.precision, t.tv, a, t.stage_n[s], t.max_vg, st) != cudaSuccess) return KGS_ECUDA;
    }
    PartSumArgs pa;
    pa.ncell = n;
    pa.n_vg = t.n_vg;
    pa.vg_oct = reinterpret_cast<const int *>(b + o_vgoct);
    pa.part = b + o_part;
    pa.precision = t.precision;
    pa.solid = d_solid;
    pa.sums = reinterpret_cast<double *>(b + o_sums);
    pa.coef = coef;
    pa.wall_kind = reinterpret_cast<const int8_t *>(b + o_kind);
    pa.ref = t.ref;
    ClosureArgs ca;
    ca.nx = t.nx;
    ca.ny = t.ny;
    ca.nz = t.nz;
    ca.ncell = n;
    ca.sums = pa.sums;
    ca.coef = coef;
    ca.precision = t.precision;
    ca.q_lagged = 0;
    ca.mac_new = macros_out;
    ca.rho_w_new = rho_w_out;
    ca.wall_kind = reinterpret_cast<const int8_t *>(b + o_kind);
    ca.wall_norm = reinterpret_cast<const double *>(b + o_norm);
    ca.dx = reinterpret_cast<const double *>(b + o_dx);
    ca.dy = reinterpret_cast<const double *>(b + o_dy);
    ca.dz = reinterpret_cast<const double *>(b + o_dz);
    ca.solid = d_solid;
    ca.blk_mass = reinterpret_cast<double *>(b + o_bmass);
    double *d_scale = reinterpret_cast<double *>(b + o_scale);
    double *d_resid = reinterpret_cast<double *>(b + o_resid);
    if (launch_part_sums(pa, st) != cudaSuccess || launch_closure(ca, st) != cudaSuccess ||
        launch_finalize_mass(ca.blk_mass, (int)close_blocks(n), M0, M0 > 0.0 ? 1 : 0, d_scale, st) != cudaSuccess ||
        launch_scale_residual(macros_out, rho_w_out, macros_in, d_solid, n, d_scale,
                              reinterpret_cast<double *>(b + o_bres), reinterpret_cast<int *>(b + o_bbad), n_red,
                              st) != cudaSuccess ||
        launch_finalize_residual(reinterpret_cast<double *>(b + o_bres), reinterpret_cast<int *>(b + o_bbad),
                                 n_red, d_resid, st) != cudaSuccess)
        return KGS_ECUDA;
    double h[2] = {0.0, 0.0};
    // pageable destination: returns once the values are on the host
    if (cudaMemcpyAsync(h, d_resid, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return KGS_ECUDA;
    if (residual) *residual = h[0];
    return h[1] != 0.0 ? KGS_EDIVERGED : KGS_OK;
}
