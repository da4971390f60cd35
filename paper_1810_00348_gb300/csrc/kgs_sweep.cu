// kgs_sweep.cu -- the fused equilibrium + upwind implicit sweep + moment
// kernel of one outer iteration (arXiv 1810.00348, Eqs. (2), (5), (7), (9)).
//
// Work decomposition.  The physical grid is cut into blocks of BX x BY x bz
// cells.  For the velocities of octant o (signs of xi_x, xi_y, xi_z) a block
// depends only on its three upwind neighbour blocks, so the blocks are swept
// in diagonal stages (block coordinates reflected so that the sweep runs
// towards +x, +y, +z): stage s holds every block whose reflected coordinates
// sum to s, for all eight octants at once.  A work item is (octant, block,
// group of vg_size velocities of that octant).  The persistent kernel claims
// items in stage order and waits (bounded) for the completion flags of the
// item's three upwind blocks, so one launch covers the whole sweep; the
// kernel with one launch per stage serves the entry point that allocates no
// device memory (no flags needed).  Velocities
// are independent within an outer iteration (Eq. (6) lags f^S, tau and
// rho_w), which is what lets all octants and all velocity groups run
// concurrently.
//
// Inside a CTA each thread owns TV velocities of the group and marches the
// block slice by slice along z.  The XY slice of every velocity of the group
// lives in shared memory and is updated in place (Section 3.2: the value of
// slice k-1 at (i, j) is read once, by the update of (i, j, k), just before
// it is overwritten), with a halo row and column holding the values that
// enter the slice from the upwind neighbour blocks or the domain boundary.
// Within a slice a thread visits the cells by anti-diagonals i + j = d: the
// cells of one diagonal are independent and their upwind values (i-1, j),
// (i, j-1) were written on the previous diagonal.  Each update is the
// pointwise solution of Eq. (7):
//     f = (f^S/tau + sum_d a_d f_up,d) / (1/tau + sum_d a_d),  a_d = |xi_d|/dx_d,
// with the Shakhov equilibrium f^S of Eq. (2) computed on the fly from the
// lagged coefficients of the cell.
//
// After each slice the threads switch to a cell-per-thread layout and sum
// the slice's moments over the group's velocities: the 13 sums about the
// lagged velocity U^n and the incoming wall fluxes of Eq. (9).  Along an
// x-line of the tensor-product velocity grid only c_x changes, so a thread
// accumulates P_a = sum w_x c_x^a f (a = 0..3) and folds them with the line's
// c_y, c_z and w_y w_z at the end of the line.  In FP32 the factors c_d =
// xi_d - U_d are carried as float pairs (hi + lo, with first-order
// corrections): their rounding would otherwise repeat identically on every
// line and add up coherently in the heat flux.  The line folds go into
// Kahan-compensated sums.  The per-(group, cell) partial (FP64, or an FP32
// Kahan pair) goes to a per-CTA scratch block in the persistent kernel, which
// then adds it, in the fixed order of an accumulator chain, into one of a few
// per-cell accumulators (no atomics, no buffer that grows with the phase
// space); the staged kernel writes per-group partials for a fixed-order
// reduction kernel.  The FP32 sweep carries the deviation g = f - M_ref from
// a per-velocity reference Maxwellian, whose moments are added in FP64 when
// the sums are formed.  Block faces between stages go through three face
// planes in global memory indexed by the cell position on the face: a block
// reads the plane entries written by its upwind neighbour in the previous
// stage before overwriting them with its own outflow.
#include <map>
#include <mutex>
#include <utility>

#include "kgs_internal.h"

namespace kgs {
namespace {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 2^x - 1 with a relative error near FP32 rounding also for small x: for
// |x| < 1/4 the Taylor series of e^y - 1 in y = x ln 2 up to y^6 (the first
// omitted term is below 6e-9 of the sum), else the hardware 2^x minus 1
// (no cancellation beyond three bits there).
__device__ __forceinline__ float exp2m1(float x)
{
    const float y = x * 0.693147180559945309f;
    float p = fmaf(y, 1.f / 720.f, 1.f / 120.f);
    p = fmaf(p, y, 1.f / 24.f);
    p = fmaf(p, y, 1.f / 6.f);
    p = fmaf(p, y, 0.5f);
    const float small = fmaf(y * y, p, y);
    return fabsf(x) < 0.25f ? small : ex2_approx(x) - 1.f;
}

// exp of the scaled exponent: FP64 uses exp(), FP32 the hardware 2^x with the
// log2(e) factor already folded into the coefficient C_NEXP.
__device__ __forceinline__ double eq_exp(double x) { return exp(x); }
__device__ __forceinline__ float eq_exp(float x) { return ex2_approx(x); }
// FP64 implicit update: the reciprocal of the denominator from the hardware approximation
// refined by two Newton-Raphson steps r <- r + r (1 - den r) (quadratic
// convergence, about 1 ulp), then one product; den = 1/tau + sum a_d > 0.
__device__ __forceinline__ double implicit_div(double num, double den)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(den));
    r = fma(r, fma(-den, r, 1.0), r);
    r = fma(r, fma(-den, r, 1.0), r);
    return num * r;
}

__host__ __device__ constexpr size_t align16(size_t n) { return (n + 15) & ~size_t(15); }

// a - b = s + e exactly (Knuth's two-sum on a + (-b)).
template <typename Real>
__device__ __forceinline__ void two_diff(Real a, Real b, Real &s, Real &e)
{
    s = a - b;
    const Real bv = s - a;
    const Real av = s - bv;
    e = (a - av) - (b + bv);
}

// Running sum for the per-thread moment accumulation.  FP32 sums carry a
// Kahan compensation term (the value is sum - comp); FP64 sums are plain.
template <typename Real>
struct RunSum;
template <>
struct RunSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <>
struct RunSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

constexpr int VT = 8;  // moment-phase velocity table entries per velocity

// Four consecutive coefficients of a cell (one 16-byte shared load for FP32,
// two for FP64).
template <typename Real>
struct Quad {
    Real x, y, z, w;
};
__device__ __forceinline__ Quad<float> load_quad(const float *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Quad<double> load_quad(const double *p)
{
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
    return {a.x, a.y, b.x, b.y};
}

template <typename Real, int TV, int ORDER = 1>
struct SmemLayout {
    static constexpr int VG = NT * TV;
    static constexpr int CS = VG + 1;  // odd cell stride: conflict-free per-cell reads
    static constexpr int H = ORDER;    // halo width: the upwind cells a stencil reaches
    static constexpr int PX = BX + H;  // slice positions per row, halo included
    static constexpr size_t slice_bytes = align16(sizeof(Real) * (BY + H) * PX * CS);
    // order 2: slice k-2 at the block's own cells
    static constexpr size_t slice2_bytes = ORDER == 2 ? align16(sizeof(Real) * BY * BX * CS) : 0;
    static constexpr size_t coef_bytes = align16(sizeof(Real) * SLICE * NCOEF);
    static constexpr size_t vt_bytes = align16(sizeof(Real) * VG * VT);
    static constexpr size_t red_bytes = sizeof(double) * NPART * SLICE;
    // The halo rows of the slice (H rows of PX cell positions) are not read
    // during the moment phase, so the reduction buffer of the two velocity
    // halves lives there when it fits (it does for 256 FP32 or 128 FP64
    // velocities); a barrier at the end of the slice keeps the next slice's
    // halo from overwriting it early.
    static constexpr bool red_in_halo = sizeof(Real) * H * PX * CS >= red_bytes;
    static constexpr size_t off_coef = slice_bytes + slice2_bytes;
    static constexpr size_t off_vt = off_coef + coef_bytes;
    static constexpr size_t off_red = off_vt + vt_bytes;
    static constexpr size_t fixed = off_red + (red_in_halo ? 0 : red_bytes);
    static int cx_stride(int nxm) { return nxm | 1; }  // odd: conflict-free per-cell reads
    // line: x-lines of LINE nodes keep their c_x in registers (no c_x tables)
    static size_t total(int nxm, bool line)
    {
        return fixed + align16(sizeof(Real) * 2 * nxm) + (line ? 0 : 2 * align16(sizeof(Real) * SLICE * cx_stride(nxm)));
    }
};

// Coefficient prefetch: each thread moves 8 of the slice's SLICE*NCOEF values.
constexpr int CPF = SLICE * NCOEF / NT;
static_assert(CPF == 8, "coefficient prefetch assumes 8 values per thread");

// Partial of one (group, cell) as stored in global memory: FP64, or the FP32
// Kahan pair (sum, compensation) with value sum - compensation.
template <typename Real>
struct PartOut;
template <>
struct PartOut<double> {
    using T = double;
};
template <>
struct PartOut<float> {
    using T = float2;
};

// (s0 - c0) + (s1 - c1) as a Kahan pair (s, c), value s - c, with an exact
// two-sum of the leading parts.
__device__ __forceinline__ float2 pair_add(float s0, float c0, float s1, float c1)
{
    const float S = s0 + s1;
    const float bv = S - s0;
    const float E = ((s0 - (S - bv)) + (s1 - bv)) - (c0 + c1);
    const float hi = S + E;
    const float lo = E - (hi - S);
    return make_float2(hi, -lo);
}

// Face-plane load: in the persistent kernel the value may have been written
// by another CTA during the same launch, so it bypasses L1 (the acquire of the
// upwind block's completion flag orders it after that CTA's stores).
template <bool COHERENT, typename Real>
__device__ __forceinline__ Real ld_face(const Real *p)
{
    if constexpr (COHERENT)
        return __ldcg(p);
    else
        return *p;
}

// One work item: block w = (octant, reflected block coordinates) and
// velocity group vgy of that octant.  Called by every thread of the CTA.
//
// The item's moment partials go, per (group, cell), to a.part (staged sweep,
// COHERENT false) or, in the persistent sweep, to this CTA's scratch block
// [bz * SLICE][NPART] indexed by the cell's place in the block, from where
// chain_add moves them into the ordered accumulators.
//
// ORDER 2 (second-order upwind, single contexts on solid-free uniform grids):
// slice2 keeps slice k-2 at the block's cells, the halo is two cells wide,
// and FX2/FY2/FZ2 carry the block outflow one cell further upwind.
template <typename Real, int TV, int LINE, bool COHERENT, bool UNIF, int ORDER = 1, bool DEV = false>
__device__ __forceinline__ void sweep_item(const SweepArgs &a, const int4 w, const int vgy, unsigned char *smem,
                                           void *scratch)
{
    // the deviation-form FP32 source (uniform grids: it uses the width slots)
    constexpr bool DEVF = sizeof(Real) == 4 && (ORDER == 2 || DEV);
    static_assert(!DEVF || UNIF, "the deviation-form source needs a uniform grid");
    using L = SmemLayout<Real, TV, ORDER>;
    constexpr int VG = L::VG;
    constexpr int CS = L::CS;
    constexpr int H = L::H, PX = L::PX;
    const int nxm = a.nxo_max;
    Real *slice = reinterpret_cast<Real *>(smem);
    Real *slice2 = reinterpret_cast<Real *>(smem + L::slice_bytes);  // order 2 only
    Real *cs = reinterpret_cast<Real *>(smem + L::off_coef);
    Real *vt = reinterpret_cast<Real *>(smem + L::off_vt);
    double *mred = L::red_in_halo ? reinterpret_cast<double *>(smem) : reinterpret_cast<double *>(smem + L::off_red);
    const int cxs = nxm | 1;
    Real *xn = reinterpret_cast<Real *>(smem + L::fixed);  // [nxm][2]
    Real *cxh = reinterpret_cast<Real *>(smem + L::fixed + align16(sizeof(Real) * 2 * nxm));  // [SLICE][cxs]
    Real *cxl = cxh + align16(sizeof(Real) * SLICE * cxs) / sizeof(Real);                    // [SLICE][cxs]

    const int t = threadIdx.x;
    const int o = w.x;
    const int vcount = a.oct_vcount[o];
    const int v0 = vgy * VG;
    if (v0 >= vcount) return;
    const int nvg = min(VG, vcount - v0);
    const int gvbase = a.oct_vstart[o] + v0;
    const int vgid = a.oct_vgbase[o] + vgy;
    const int nxo = a.oct_nx[o];

    // Octant bit d set: xi_d >= 0, sweep towards +d.
    const bool px = (o & 1) != 0, py = (o & 2) != 0, pz = (o & 4) != 0;
    const int bxi = px ? w.y : a.nbx - 1 - w.y;
    const int byi = py ? w.z : a.nby - 1 - w.z;
    const int bzi = pz ? w.w : a.nbz - 1 - w.w;
    const int x0 = bxi * BX, ex = min(BX, a.nx - x0);
    const int y0 = byi * BY, ey = min(BY, a.ny - y0);
    const int z0 = bzi * a.bz, ez = min(a.bz, a.nz - z0);
    const bool xfirst = w.y == 0, yfirst = w.z == 0, zfirst = w.w == 0;
    const bool xlast = w.y == a.nbx - 1, ylast = w.z == a.nby - 1, zlast = w.w == a.nbz - 1;
    const int sidex = px ? 0 : 1, sidey = py ? 2 : 3, sidez = pz ? 4 : 5;  // upwind sides
    const int headx = px ? 1 : 0, heady = py ? 3 : 2, headz = pz ? 5 : 4;  // downwind sides
    const int nx = a.nx, ny = a.ny;
    const size_t ncell = a.ncell;
    const size_t Nv = (size_t)a.Nv;
    // solid cells or solid neighbours in this block (a.blk_plain marks the
    // physical blocks that have neither; without it every block of a problem
    // with solid cells counts as having them)
    const bool any_solid =
        a.any_solid != 0 && !(a.blk_plain != nullptr && a.blk_plain[((size_t)bzi * a.nby + byi) * a.nbx + bxi] != 0);

    auto GX = [&](int li) { return px ? x0 + li : x0 + ex - 1 - li; };
    auto GY = [&](int lj) { return py ? y0 + lj : y0 + ey - 1 - lj; };
    auto GZ = [&](int lk) { return pz ? z0 + lk : z0 + ez - 1 - lk; };
    auto SL = [&](int li, int lj) { return ((lj + H) * PX + (li + H)) * CS; };  // li, lj may be -1 (-2: order 2)
    auto CELL = [&](int x, int y, int z) { return (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z); };

    const Real *vel = static_cast<const Real *>(a.vel);
    const Real *velm = static_cast<const Real *>(a.velm);
    const Real *mt = static_cast<const Real *>(a.mtab);
    const Real *coef = static_cast<const Real *>(a.coef);
    Real *FXp = static_cast<Real *>(a.FX);
    Real *FYp = static_cast<Real *>(a.FY);
    Real *FZp = static_cast<Real *>(a.FZ);
    Real *FX2p = static_cast<Real *>(a.FX2);
    Real *FY2p = static_cast<Real *>(a.FY2);
    Real *FZ2p = static_cast<Real *>(a.FZ2);
    // order 2: index of the block's first cell along each sweep direction
    // (cells with index >= 2 have both upwind neighbours in the domain)
    const int sx0 = px ? x0 : nx - x0 - ex, sy0 = py ? y0 : ny - y0 - ey, sz0 = pz ? z0 : a.nz - z0 - ez;

    // ---- per-thread velocities (vl = t + m*NT) and the moment-phase tables ----
    // The FP32 sweep carries g = f - M_ref (mref: the reference Maxwellian of
    // the velocity); every ghost value enters as ghost - M_ref and the source
    // as f^S/tau - M_ref/tau.  The FP64 sweep carries f (mref unused).
    Real xi[TV][3], axi[TV][3], mgx[TV], mgy[TV], mgz[TV], msol[TV], mref[TV];
    Real dmref[TV];  // deviation-form source: the rounding error of M_ref
    size_t gv[TV];
    bool ok[TV];
    const int rowx = a.side_inflow[sidex] ? MT_INFLOW : sidex;
    const int rowy = a.side_inflow[sidey] ? MT_INFLOW : sidey;
    const int rowz = a.side_inflow[sidez] ? MT_INFLOW : sidez;
#pragma unroll
    for (int m = 0; m < TV; m++) {
        const int vl = t + m * NT;
        ok[m] = vl < nvg;
        gv[m] = (size_t)gvbase + (ok[m] ? vl : 0);
        xi[m][0] = vel[gv[m] * 4 + 0];
        xi[m][1] = vel[gv[m] * 4 + 1];
        xi[m][2] = vel[gv[m] * 4 + 2];
        axi[m][0] = fabs(xi[m][0]);
        axi[m][1] = fabs(xi[m][1]);
        axi[m][2] = fabs(xi[m][2]);
        // x-line factor w_x; line data for the fold: xi_y, xi_z (hi, lo), w_y w_z
        Real *e = vt + vl * VT;
        e[0] = ok[m] ? velm[gv[m] * 8 + 0] : Real(0);
        e[1] = xi[m][1];
        e[2] = xi[m][2];
        e[3] = ok[m] ? velm[gv[m] * 8 + 1] : Real(0);
        e[4] = velm[gv[m] * 8 + 3];
        e[5] = velm[gv[m] * 8 + 4];
        e[6] = Real(0);
        e[7] = Real(0);
        mgx[m] = mt[(size_t)rowx * Nv + gv[m]];
        mgy[m] = mt[(size_t)rowy * Nv + gv[m]];
        mgz[m] = mt[(size_t)rowz * Nv + gv[m]];
        msol[m] = mt[(size_t)MT_SOLID * Nv + gv[m]];
        mref[m] = sizeof(Real) == 4 ? velm[gv[m] * 8 + 5] : Real(0);
        if constexpr (DEVF) dmref[m] = velm[gv[m] * 8 + 6];
    }
    // ghost value rho_w * (unit wall or free-stream Maxwellian), as carried
    auto ghost = [&](Real rw, Real mg, int m) -> Real {
        if constexpr (sizeof(Real) == 4)
            return fma(rw, mg, -mref[m]);
        else
            return rw * mg;
    };
    // |xi|^2 of each velocity, rounded once from its FP64 value
    Real xsq[TV];
#pragma unroll
    for (int m = 0; m < TV; m++) {
        const double x0 = xi[m][0], x1 = xi[m][1], x2 = xi[m][2];
        xsq[m] = Real(x0 * x0 + x1 * x1 + x2 * x2);
    }
    // uniform grid: the upwind coefficients a_d = abs(xi_d) / dx_d and their
    // sum depend on the velocity only
    Real adx[TV][3], asum[TV];
#pragma unroll
    for (int m = 0; m < TV; m++) {
        if constexpr (UNIF) {
            adx[m][0] = axi[m][0] * Real(a.rd0[0]);
            adx[m][1] = axi[m][1] * Real(a.rd0[1]);
            adx[m][2] = axi[m][2] * Real(a.rd0[2]);
            asum[m] = adx[m][0] + adx[m][1] + adx[m][2];
        } else {
            adx[m][0] = adx[m][1] = adx[m][2] = asum[m] = Real(0);
        }
    }
    // x nodes of the octant in line order (the first nxo velocities of the octant)
    for (int ix = t; ix < nxo; ix += NT) {
        const size_t g = (size_t)a.oct_vstart[o] + ix;
        xn[ix * 2 + 0] = vel[g * 4 + 0];
        xn[ix * 2 + 1] = velm[g * 8 + 2];
    }

    // Ghost value entering through domain side `side` at cell `cell`:
    // free stream, or rho_w times the unit wall Maxwellian (Eq. (8)).
    auto wall_rho = [&](int side, size_t cell) -> Real {
        return a.side_inflow[side] ? Real(1) : Real(a.rho_w[side * ncell + cell]);
    };

    // ---- prefetch registers: coefficients and halos of one slice ----
    Real pc[CPF];
    Real phx[BY][TV], phy[BX][TV];
    Real phx2[ORDER == 2 ? BY : 1][TV], phy2[ORDER == 2 ? BX : 1][TV];  // order 2: second halo column / row
    auto prefetch = [&](int lk) {
        const int z = GZ(lk);
        const int cl = (t * CPF) / NCOEF, q0 = (t * CPF) % NCOEF;
        const int li = cl % BX, lj = cl / BX;
        if (li < ex && lj < ey) {
            const Real *src = coef + CELL(GX(li), GY(lj), z) * NCOEF + q0;
#pragma unroll
            for (int q = 0; q < CPF; q++) pc[q] = src[q];
        } else {
#pragma unroll
            for (int q = 0; q < CPF; q++) pc[q] = (q0 + q == C_FLAGS) ? flag_value<Real>(F_SOLID) : Real(0);
        }
        if (xfirst) {
#pragma unroll
            for (int lj2 = 0; lj2 < BY; lj2++) {
                if (lj2 >= ey) break;
                const Real rw = wall_rho(sidex, CELL(GX(0), GY(lj2), z));
#pragma unroll
                for (int m = 0; m < TV; m++) phx[lj2][m] = ghost(rw, mgx[m], m);
            }
        } else {
            const Real *fi = FXp + ((size_t)z * ny + GY(0)) * Nv;
            const long long step = py ? (long long)Nv : -(long long)Nv;
#pragma unroll
            for (int lj2 = 0; lj2 < BY; lj2++) {
                if (lj2 >= ey) break;
#pragma unroll
                for (int m = 0; m < TV; m++)
                    phx[lj2][m] = ok[m] ? ld_face<COHERENT>(fi + lj2 * step + (long long)gv[m]) : Real(0);
            }
            if constexpr (ORDER == 2) {
                const Real *fi2 = FX2p + ((size_t)z * ny + GY(0)) * Nv;
#pragma unroll
                for (int lj2 = 0; lj2 < BY; lj2++) {
                    if (lj2 >= ey) break;
#pragma unroll
                    for (int m = 0; m < TV; m++)
                        phx2[lj2][m] = ok[m] ? ld_face<COHERENT>(fi2 + lj2 * step + (long long)gv[m]) : Real(0);
                }
            }
        }
        if (yfirst) {
#pragma unroll
            for (int li2 = 0; li2 < BX; li2++) {
                if (li2 >= ex) break;
                const Real rw = wall_rho(sidey, CELL(GX(li2), GY(0), z));
#pragma unroll
                for (int m = 0; m < TV; m++) phy[li2][m] = ghost(rw, mgy[m], m);
            }
        } else {
            const Real *fi = FYp + ((size_t)z * nx + GX(0)) * Nv;
            const long long step = px ? (long long)Nv : -(long long)Nv;
#pragma unroll
            for (int li2 = 0; li2 < BX; li2++) {
                if (li2 >= ex) break;
#pragma unroll
                for (int m = 0; m < TV; m++)
                    phy[li2][m] = ok[m] ? ld_face<COHERENT>(fi + li2 * step + (long long)gv[m]) : Real(0);
            }
            if constexpr (ORDER == 2) {
                const Real *fi2 = FY2p + ((size_t)z * nx + GX(0)) * Nv;
#pragma unroll
                for (int li2 = 0; li2 < BX; li2++) {
                    if (li2 >= ex) break;
#pragma unroll
                    for (int m = 0; m < TV; m++)
                        phy2[li2][m] = ok[m] ? ld_face<COHERENT>(fi2 + li2 * step + (long long)gv[m]) : Real(0);
                }
            }
        }
    };
    prefetch(0);

    // z inflow of the block: the slice interior starts as slice k0-1.  A row
    // of cells is loaded before it is stored, so a row's loads are in flight
    // together.
    if (zfirst) {
        for (int lj = 0; lj < ey; lj++)
            for (int li = 0; li < ex; li++) {
                const Real rw = wall_rho(sidez, CELL(GX(li), GY(lj), GZ(0)));
#pragma unroll
                for (int m = 0; m < TV; m++)
                    if (ok[m]) slice[SL(li, lj) + t + m * NT] = ghost(rw, mgz[m], m);
            }
    } else {
        const long long sx = px ? (long long)Nv : -(long long)Nv;
        for (int lj = 0; lj < ey; lj++) {
            const Real *fi = FZp + ((size_t)GY(lj) * nx + GX(0)) * Nv;
            Real v[BX][TV];
#pragma unroll
            for (int li = 0; li < BX; li++) {
                if (li >= ex) break;
#pragma unroll
                for (int m = 0; m < TV; m++)
                    v[li][m] = ok[m] ? ld_face<COHERENT>(fi + li * sx + (long long)gv[m]) : Real(0);
            }
#pragma unroll
            for (int li = 0; li < BX; li++) {
                if (li >= ex) break;
#pragma unroll
                for (int m = 0; m < TV; m++)
                    if (ok[m]) slice[SL(li, lj) + t + m * NT] = v[li][m];
            }
            if constexpr (ORDER == 2) {
                // slice k0-2 (the upwind block's second-last slice)
                const Real *fi2 = FZ2p + ((size_t)GY(lj) * nx + GX(0)) * Nv;
#pragma unroll
                for (int li = 0; li < BX; li++) {
                    if (li >= ex) break;
#pragma unroll
                    for (int m = 0; m < TV; m++)
                        v[li][m] = ok[m] ? ld_face<COHERENT>(fi2 + li * sx + (long long)gv[m]) : Real(0);
                }
#pragma unroll
                for (int li = 0; li < BX; li++) {
                    if (li >= ex) break;
#pragma unroll
                    for (int m = 0; m < TV; m++)
                        if (ok[m]) slice2[(lj * BX + li) * CS + t + m * NT] = v[li][m];
                }
            }
        }
    }


    for (int lk = 0; lk < ez; lk++) {
        const int z = GZ(lk);
        // stage the prefetched slice data in shared memory
#pragma unroll
        for (int q = 0; q < CPF; q++) cs[t * CPF + q] = pc[q];
#pragma unroll
        for (int lj = 0; lj < BY; lj++) {
            if (lj >= ey) break;
#pragma unroll
            for (int m = 0; m < TV; m++)
                if (ok[m]) slice[SL(-1, lj) + t + m * NT] = phx[lj][m];
        }
#pragma unroll
        for (int li = 0; li < BX; li++) {
            if (li >= ex) break;
#pragma unroll
            for (int m = 0; m < TV; m++)
                if (ok[m]) slice[SL(li, -1) + t + m * NT] = phy[li][m];
        }
        if constexpr (ORDER == 2) {
            // the second halo column / row (read only by cells with both
            // upwind neighbours in the domain, so not in a first block)
            if (!xfirst) {
#pragma unroll
                for (int lj = 0; lj < BY; lj++) {
                    if (lj >= ey) break;
#pragma unroll
                    for (int m = 0; m < TV; m++)
                        if (ok[m]) slice[SL(-2, lj) + t + m * NT] = phx2[lj][m];
                }
            }
            if (!yfirst) {
#pragma unroll
                for (int li = 0; li < BX; li++) {
                    if (li >= ex) break;
#pragma unroll
                    for (int m = 0; m < TV; m++)
                        if (ok[m]) slice[SL(li, -2) + t + m * NT] = phy2[li][m];
                }
            }
        }
        __syncthreads();
        // c_x = xi_x - U_x of each cell of the slice as a float pair, per x node
        // (lines of LINE nodes keep theirs in registers instead)
        if constexpr (LINE == 0) {
            const int cl = t % SLICE, vp = t / SLICE;
            const Real ux = Real(-0.5) * cs[cl * NCOEF + C_M2UX];
            for (int ix = vp; ix < nxo; ix += NT / SLICE) {
                Real s, e;
                two_diff(xn[ix * 2], ux, s, e);
                cxh[cl * cxs + ix] = s;
                cxl[cl * cxs + ix] = e + xn[ix * 2 + 1];
            }
        }
        if (lk + 1 < ez) prefetch(lk + 1);

        // ---- sweep of the slice: Eq. (2) fused into Eq. (7), by anti-diagonals ----
        // FP32 deviation-form source (DEVF: order 2, or the dev_source
        // option): rtau (f^S - M_ref) evaluated as rtau M_ref (2^D shak - 1)
        // with D = log2(f^S_M / M_ref) built from per-cell terms that are small
        // near the reference state (coefficient slots C_RDX, C_RDY of uniform
        // grids), so that its rounding scales with the deviation g rather than
        // with f; the reference M_ref is the rest state and its own FP32
        // rounding error dmref is added back.
        auto dev_source = [&](const Quad<Real> &c0, const Quad<Real> &c1, const Quad<Real> &c2v,
                              const Quad<Real> &c3, int m, Real cq) -> Real {
            const Real dn = c2v.w, K = c3.x;
            const Real sd = fma(xi[m][0], c0.x, fma(xi[m][1], c0.y, xi[m][2] * c0.z));  // -2 U.xi
            const Real D = fma(xsq[m], dn, fma(sd, c1.x, K));
            const Real shm1 = cq * fma(xsq[m] + sd, c1.y, c3.z);  // Shakhov factor - 1
            const Real em = exp2m1(D);
            const Real X = fma(em, shm1, em + shm1);  // 2^D shak - 1
            return c1.z * fma(mref[m], X, dmref[m]);
        };
        // Eq. (2) fused into Eq. (7) for one cell of the slice (coefficients
        // c0..c3) and thread velocity m, from its three upwind values.
        auto cell_update = [&](const Quad<Real> &c0, const Quad<Real> &c1, const Quad<Real> &c2v,
                               const Quad<Real> &c3, int m, Real fx, Real fy, Real fz) -> Real {
          if constexpr (DEVF) {
            // uniform grids only (a_d per velocity); the update about the
            // upwind x value as below, with the deviation-form source
            const Real cq = fma(xi[m][0], c2v.x, fma(xi[m][1], c2v.y, fma(xi[m][2], c2v.z, c3.w)));
            const Real dsrc = dev_source(c0, c1, c2v, c3, m, cq);
            Real t = fma(-c1.z, fx, dsrc);
            t = fma(adx[m][1], fy - fx, t);
            t = fma(adx[m][2], fz - fx, t);
            return fma(t, rcp_approx(c1.z + asum[m]), fx);
          } else {
            const Real m2ux = c0.x, m2uy = c0.y, m2uz = c0.z, kappa = c0.w;
            const Real nexp = c1.x, rt1 = c1.y, rtau = c1.z;
            const Real qx = c2v.x, qy = c2v.y, qz = c2v.z, rdx = c2v.w;
            const Real rdy = c3.x, rdz = c3.y, shk0 = c3.z, muq = c3.w;
            // |c|^2 - |U|^2 = |xi|^2 - 2 U.xi and c.q' = xi.q' - U.q'
            const Real s = fma(xi[m][0], m2ux, fma(xi[m][1], m2uy, fma(xi[m][2], m2uz, xsq[m])));
            const Real cq = fma(xi[m][0], qx, fma(xi[m][1], qy, fma(xi[m][2], qz, muq)));
            const Real shak = fma(cq, fma(s, rt1, shk0), Real(1));
            Real src;
            if constexpr (sizeof(Real) == 4)  // kappa enters as log2(kappa) in the exponent
                src = eq_exp(fma(s, nexp, kappa)) * shak;
            else
                src = kappa * eq_exp(s * nexp) * shak;
            Real ax, ay, az, den;
            if constexpr (UNIF) {
                ax = adx[m][0];
                ay = adx[m][1];
                az = adx[m][2];
                den = rtau + asum[m];
            } else {
                ax = axi[m][0] * rdx;
                ay = axi[m][1] * rdy;
                az = axi[m][2] * rdz;
                den = rtau + ax + ay + az;
            }
            if constexpr (sizeof(Real) == 4) {
                // The same solution of Eq. (7) written about the upwind x value:
                //   f = f_x + (src - f_x/tau + a_y (f_y - f_x) + a_z (f_z - f_x)) / den.
                // On a smooth field the increment is small, so the one rounding
                // that matters is the final addition, which is unbiased.  The
                // plain form num * (1/den) scales f by the same rounding error of
                // 1/den in every cell of a velocity's characteristic, and that
                // error adds up along the sweep.
                (void)ax;
                Real t = fma(-rtau, fx + mref[m], src);
                t = fma(ay, fy - fx, t);
                t = fma(az, fz - fx, t);
                return fma(t, rcp_approx(den), fx);
            } else {
                return implicit_div(src + ax * fx + ay * fy + az * fz, den);
            }
          }
        };
        // Order 2: the three-point backward difference along an axis is
        //   a (3 f - 4 f_1 + f_2) / 2 = (3a/2) (f - h),  h = f_1 + (f_1 - f_2)/3,
        // so the update is that of Eq. (7) with the coefficient 3a/2 and the
        // extrapolated upwind value h on the axes where it applies (o2d).
        auto cell_update2 = [&](const Quad<Real> &c0, const Quad<Real> &c1, const Quad<Real> &c2v,
                                const Quad<Real> &c3, int m, Real hx, Real hy, Real hz, bool o2x, bool o2y,
                                bool o2z) -> Real {
            const Real m2ux = c0.x, m2uy = c0.y, m2uz = c0.z, kappa = c0.w;
            const Real nexp = c1.x, rt1 = c1.y, rtau = c1.z;
            const Real qx = c2v.x, qy = c2v.y, qz = c2v.z;
            const Real shk0 = c3.z, muq = c3.w;
            const Real cq = fma(xi[m][0], qx, fma(xi[m][1], qy, fma(xi[m][2], qz, muq)));
            // FP32: the deviation-form source; FP64: rtau f^S as in Eq. (7)
            Real dsrc;
            if constexpr (sizeof(Real) == 4) {
                dsrc = dev_source(c0, c1, c2v, c3, m, cq);
                (void)kappa;
            } else {
                const Real s = fma(xi[m][0], m2ux, fma(xi[m][1], m2uy, fma(xi[m][2], m2uz, xsq[m])));
                const Real shak = fma(cq, fma(s, rt1, shk0), Real(1));
                dsrc = kappa * eq_exp(s * nexp) * shak;
            }
            // uniform grids only: a_d per velocity
            const Real ax = o2x ? Real(1.5) * adx[m][0] : adx[m][0];
            const Real ay = o2y ? Real(1.5) * adx[m][1] : adx[m][1];
            const Real az = o2z ? Real(1.5) * adx[m][2] : adx[m][2];
            const Real den = rtau + ax + ay + az;
            if constexpr (sizeof(Real) == 4) {
                // about the upwind x value, as the first-order FP32 update
                Real t = fma(-rtau, hx, dsrc);
                t = fma(ay, hy - hx, t);
                t = fma(az, hz - hx, t);
                return fma(t, rcp_approx(den), hx);
            } else {
                return implicit_div(dsrc + ax * hx + ay * hy + az * hz, den);
            }
        };
        if constexpr (ORDER == 2) {
            // Generic diagonal loop with the second-order stencil.  The z
            // values of (i, j) are slice k-1 (in place) and k-2 (slice2);
            // once the cell is updated, its k-1 value moves to slice2.
            const int szk = sz0 + lk;
            const bool o2z = szk >= 2;
            const Real third = Real(1) / Real(3);
            for (int d = 0; d < ex + ey - 1; d++) {
                const int jhi = min(ey - 1, d), jlo = max(0, d - (ex - 1));
#pragma unroll
                for (int k = 0; k < BY; k++) {
                    const int lj = jhi - k;
                    if (lj >= jlo) {
                        const int li = d - lj;
                        const Real *c = cs + (lj * BX + li) * NCOEF;
                        const Quad<Real> c0 = load_quad(c), c1 = load_quad(c + 4), c2v = load_quad(c + 8),
                                         c3 = load_quad(c + 12);
                        const bool o2x = sx0 + li >= 2, o2y = sy0 + lj >= 2;
                        const int sidx = SL(li, lj), bidx = (lj * BX + li) * CS;
#pragma unroll
                        for (int m = 0; m < TV; m++) {
                            const int vl = t + m * NT;
                            const Real fz = slice[sidx + vl];
                            const Real fy = slice[sidx - PX * CS + vl];
                            const Real fx = slice[sidx - CS + vl];
                            const Real hx = o2x ? fma(fx - slice[sidx - 2 * CS + vl], third, fx) : fx;
                            const Real hy = o2y ? fma(fy - slice[sidx - 2 * PX * CS + vl], third, fy) : fy;
                            const Real hz = o2z ? fma(fz - slice2[bidx + vl], third, fz) : fz;
                            const Real f = cell_update2(c0, c1, c2v, c3, m, hx, hy, hz, o2x, o2y, o2z);
                            if (ok[m]) {
                                slice2[bidx + vl] = fz;
                                slice[sidx + vl] = f;
                            }
                        }
                    }
                }
            }
        } else if (ex == BX && ey == BY && !any_solid) {
            // Full block without solid cells: the 15 diagonals unrolled.  The
            // upwind x and y values of a cell were computed on the previous
            // diagonal by this thread and stay in registers (prev[row]); only
            // the z value (the cell itself in slice k-1) and the halo row and
            // column come from shared memory.  Every index is a compile-time
            // constant, so the cells of a diagonal form straight-line code whose
            // update chains the compiler can interleave, and a diagonal waits
            // only for register results of the one before.
            Real prev[BY][TV];
#pragma unroll
            for (int d = 0; d < BX + BY - 1; d++) {
#pragma unroll
                for (int k = 0; k < BY; k++) {
                    const int lj = (d < BY - 1 ? d : BY - 1) - k;
                    const int li = d - lj;
                    if (lj >= 0 && li < BX) {
                        const Real *c = cs + (lj * BX + li) * NCOEF;
                        const Quad<Real> c0 = load_quad(c), c1 = load_quad(c + 4), c2v = load_quad(c + 8),
                                         c3 = load_quad(c + 12);
                        const int sidx = SL(li, lj);
#pragma unroll
                        for (int m = 0; m < TV; m++) {
                            const int vl = t + m * NT;
                            const Real fz = slice[sidx + vl];
                            const Real fx = li == 0 ? slice[sidx - CS + vl] : prev[lj][m];
                            const Real fy = lj == 0 ? slice[sidx - PX * CS + vl] : prev[lj > 0 ? lj - 1 : 0][m];
                            const Real f = cell_update(c0, c1, c2v, c3, m, fx, fy, fz);
                            prev[lj][m] = f;
                            if (ok[m]) slice[sidx + vl] = f;
                        }
                    }
                }
            }
        } else {
        // The upwind values of cell (i, j) are read from the in-place slice:
        // (i-1, j) and (i, j-1) were updated on the previous diagonal, (i, j)
        // itself still holds slice k-1.  The cells of one diagonal are
        // independent, which gives up to BY update chains in flight.
        for (int d = 0; d < ex + ey - 1; d++) {
            const int jhi = min(ey - 1, d), jlo = max(0, d - (ex - 1));
#pragma unroll
            for (int k = 0; k < BY; k++) {
                const int lj = jhi - k;
                if (lj >= jlo) {
                    const int li = d - lj;
                    const Real *c = cs + (lj * BX + li) * NCOEF;
                    const Quad<Real> c0 = load_quad(c), c1 = load_quad(c + 4), c2v = load_quad(c + 8),
                                     c3 = load_quad(c + 12);
                    const int flags = flag_bits(c1.w);
                    if (!(flags & F_SOLID)) {
                        bool sol_x = false, sol_y = false, sol_z = false;
                        Real rwx = 0, rwy = 0, rwz = 0;
                        if (any_solid) {
                            const size_t cell = CELL(GX(li), GY(lj), z);
                            sol_x = flags & (F_SOLID_SIDE << sidex);
                            sol_y = flags & (F_SOLID_SIDE << sidey);
                            sol_z = flags & (F_SOLID_SIDE << sidez);
                            if (sol_x) rwx = Real(a.rho_w[sidex * ncell + cell]);
                            if (sol_y) rwy = Real(a.rho_w[sidey * ncell + cell]);
                            if (sol_z) rwz = Real(a.rho_w[sidez * ncell + cell]);
                        }
                        const int sidx = SL(li, lj);
#pragma unroll
                        for (int m = 0; m < TV; m++) {
                            const int vl = t + m * NT;
                            Real fz = slice[sidx + vl];
                            Real fy = slice[sidx - PX * CS + vl];
                            Real fx = slice[sidx - CS + vl];
                            if (any_solid) {
                                if (sol_x) fx = ghost(rwx, msol[m], m);
                                if (sol_y) fy = ghost(rwy, msol[m], m);
                                if (sol_z) fz = ghost(rwz, msol[m], m);
                            }
                            const Real f = cell_update(c0, c1, c2v, c3, m, fx, fy, fz);
                            if (ok[m]) slice[sidx + vl] = f;
                        }
                    }
                }
            }
        }
        }
        // outflow of the slice through the block's downwind x and y faces, for
        // the neighbouring blocks (own velocities, read back from the slice)
        if (!xlast) {
            Real *fo = FXp + ((size_t)z * ny + GY(0)) * Nv;
            const long long step = py ? (long long)Nv : -(long long)Nv;
#pragma unroll
            for (int lj = 0; lj < BY; lj++) {
                if (lj >= ey) break;
                const Real *src = slice + SL(ex - 1, lj) + t;
#pragma unroll
                for (int m = 0; m < TV; m++)
                    if (ok[m]) fo[lj * step + (long long)gv[m]] = src[m * NT];
            }
            if constexpr (ORDER == 2) {
                // the column before the last: the halo column when ex == 1
                Real *fo2 = FX2p + ((size_t)z * ny + GY(0)) * Nv;
#pragma unroll
                for (int lj = 0; lj < BY; lj++) {
                    if (lj >= ey) break;
                    const Real *src = slice + SL(ex - 2, lj) + t;
#pragma unroll
                    for (int m = 0; m < TV; m++)
                        if (ok[m]) fo2[lj * step + (long long)gv[m]] = src[m * NT];
                }
            }
        }
        if (!ylast) {
            Real *fo = FYp + ((size_t)z * nx + GX(0)) * Nv;
            const long long step = px ? (long long)Nv : -(long long)Nv;
#pragma unroll
            for (int li = 0; li < BX; li++) {
                if (li >= ex) break;
                const Real *src = slice + SL(li, ey - 1) + t;
#pragma unroll
                for (int m = 0; m < TV; m++)
                    if (ok[m]) fo[li * step + (long long)gv[m]] = src[m * NT];
            }
            if constexpr (ORDER == 2) {
                Real *fo2 = FY2p + ((size_t)z * nx + GX(0)) * Nv;
#pragma unroll
                for (int li = 0; li < BX; li++) {
                    if (li >= ex) break;
                    const Real *src = slice + SL(li, ey - 2) + t;
#pragma unroll
                    for (int m = 0; m < TV; m++)
                        if (ok[m]) fo2[li * step + (long long)gv[m]] = src[m * NT];
                }
            }
        }
        __syncthreads();

        // ---- moments of the slice over the group's velocities ----
        {
            const int cl = t % SLICE, vp = t / SLICE;  // NT = 2 * SLICE: two velocity halves
            const int li = cl % BX, lj = cl / BX;
            const bool valid = li < ex && lj < ey;
            const Real *c = cs + cl * NCOEF;
            const int flags = flag_bits(c[C_FLAGS + 0]);
            RunSum<Real> S[NPART];
            if (valid && !(flags & F_SOLID)) {
                const Real ux = Real(-0.5) * c[C_M2UX], uy = Real(-0.5) * c[C_M2UY], uz = Real(-0.5) * c[C_M2UZ];
                const bool wx = flags & (F_WALL_SIDE << headx);
                const bool wy = flags & (F_WALL_SIDE << heady);
                const bool wz = flags & (F_WALL_SIDE << headz);
                const Real sgnx = px ? Real(1) : Real(-1);
                const Real *sp = slice + SL(li, lj);
                const int vbeg = vp * (VG / 2);
                const int vend = min(vbeg + VG / 2, nvg);
                // fold the line sums P_a (x-line of the tensor-product grid ending at
                // velocity ve-1) with the line's c_y, c_z and w_y w_z
                if constexpr (sizeof(Real) == 4) {
                    // fold the line sums P_a (x-line of the tensor-product grid ending at
                    // velocity ve-1) with the line's c_y, c_z and w_y w_z
                    auto fold = [&](Real P0, Real P1, Real P2, Real P3, int ve) {
                        const Real *e = vt + (ve - 1) * VT;
                        Real cy, cyl, cz, czl;
                        two_diff(e[1], uy, cy, cyl);
                        two_diff(e[2], uz, cz, czl);
                        cyl += e[4];
                        czl += e[5];
                        const Real W = e[3];
                        const Real q0 = W * P0, q1 = W * P1, q2 = W * P2;
                        const Real r2 = fma(cy, cy, cz * cz);
                        const Real r2l = Real(2) * fma(cy, cyl, cz * czl);
                        S[P_S0].add(q0);
                        S[P_S1X].add(q1);
                        S[P_S1Y].add(fma(cy, q0, cyl * q0));
                        S[P_S1Z].add(fma(cz, q0, czl * q0));
                        S[P_S2XX].add(q2);
                        S[P_S2YY].add(fma(cy, cy, Real(2) * cy * cyl) * q0);
                        S[P_S2ZZ].add(fma(cz, cz, Real(2) * cz * czl) * q0);
                        S[P_S2XY].add(fma(cy, q1, cyl * q1));
                        S[P_S2XZ].add(fma(cz, q1, czl * q1));
                        S[P_S2YZ].add(fma(cy, cz, fma(cyl, cz, cy * czl)) * q0);
                        S[P_S3X].add(fma(W, P3, fma(r2, q1, r2l * q1)));
                        const Real e2 = fma(r2, q0, fma(r2l, q0, q2));
                        S[P_S3Y].add(fma(cy, e2, cyl * e2));
                        S[P_S3Z].add(fma(cz, e2, czl * e2));
                        // incoming flux w |xi_d| f towards the wall ahead
                        if (wx) S[P_FX].add(sgnx * fma(ux, q0, q1));
                        if (wy) S[P_FY].add(fabs(e[1]) * q0);
                        if (wz) S[P_FZ].add(fabs(e[2]) * q0);
                    };
                    if constexpr (LINE > 0) {
                        // Every x-line has LINE nodes and the thread's range holds whole
                        // lines: the c_x pairs and w_x of the LINE nodes stay in registers.
                        Real cxr[LINE], cxlr[LINE], wxr[LINE];
    #pragma unroll
                        for (int ix = 0; ix < LINE; ix++) {
                            Real hi, lo;
                            two_diff(xn[ix * 2], ux, hi, lo);
                            cxr[ix] = hi;
                            cxlr[ix] = lo + xn[ix * 2 + 1];
                            wxr[ix] = vt[(vbeg + ix) * VT];
                        }
                        for (int v = vbeg; v < vend; v += LINE) {
                            Real P0 = 0, P1 = 0, P2 = 0, P3 = 0, C1 = 0, C2 = 0, C3 = 0;
    #pragma unroll
                            for (int ix = 0; ix < LINE; ix++) {
                                const Real f = sp[v + ix];
                                const Real cx = cxr[ix];
                                const Real t0 = wxr[ix] * f;
                                const Real t1 = t0 * cx;
                                const Real t2 = t1 * cx;
                                P0 += t0;
                                P1 += t1;
                                P2 += t2;
                                P3 = fma(t2, cx, P3);
                                C1 = fma(t0, cxlr[ix], C1);
                                C2 = fma(t1, cxlr[ix], C2);
                                C3 = fma(t2, cxlr[ix], C3);
                            }
                            // first-order corrections for the low part of c_x
                            fold(P0, P1 + C1, fma(Real(2), C2, P2), fma(Real(3), C3, P3), v + LINE);
                        }
                    } else {
                        const Real *cxhc = cxh + cl * cxs, *cxlc = cxl + cl * cxs;
                        int v = vbeg;
                        while (v < vend) {
                            // one x-line segment [v, ve): velocities with the same (xi_y, xi_z)
                            const int ix0 = (v0 + v) % nxo;
                            const int ve = min(vend, v + (nxo - ix0));
                            Real P0 = 0, P1 = 0, P2 = 0, P3 = 0, C1 = 0, C2 = 0, C3 = 0;
    #pragma unroll 4
                            for (int vv = v; vv < ve; vv++) {
                                const int ix = ix0 + (vv - v);
                                const Real f = sp[vv];
                                const Real cx = cxhc[ix], cxlo = cxlc[ix];
                                const Real t0 = vt[vv * VT] * f;
                                const Real t1 = t0 * cx;
                                const Real t2 = t1 * cx;
                                P0 += t0;
                                P1 += t1;
                                P2 += t2;
                                P3 = fma(t2, cx, P3);
                                C1 = fma(t0, cxlo, C1);
                                C2 = fma(t1, cxlo, C2);
                                C3 = fma(t2, cxlo, C3);
                            }
                            fold(P0, P1 + C1, fma(Real(2), C2, P2), fma(Real(3), C3, P3), ve);
                            v = ve;
                        }
                    }
                } else {
                    // FP64: the rounding of c = xi - U^n is far below the path's
                    // tolerance, so the float-pair corrections of the FP32 path are
                    // left out (fewer operations and registers).
                    auto fold = [&](Real P0, Real P1, Real P2, Real P3, int ve) {
                        const Real *e = vt + (ve - 1) * VT;
                        const Real cy = e[1] - uy, cz = e[2] - uz;
                        const Real W = e[3];
                        const Real q0 = W * P0, q1 = W * P1, q2 = W * P2;
                        const Real r2 = fma(cy, cy, cz * cz);
                        S[P_S0].add(q0);
                        S[P_S1X].add(q1);
                        S[P_S1Y].add(cy * q0);
                        S[P_S1Z].add(cz * q0);
                        S[P_S2XX].add(q2);
                        S[P_S2YY].add(cy * cy * q0);
                        S[P_S2ZZ].add(cz * cz * q0);
                        S[P_S2XY].add(cy * q1);
                        S[P_S2XZ].add(cz * q1);
                        S[P_S2YZ].add(cy * cz * q0);
                        S[P_S3X].add(fma(W, P3, r2 * q1));
                        const Real e2 = fma(r2, q0, q2);
                        S[P_S3Y].add(cy * e2);
                        S[P_S3Z].add(cz * e2);
                        if (wx) S[P_FX].add(sgnx * fma(ux, q0, q1));
                        if (wy) S[P_FY].add(fabs(e[1]) * q0);
                        if (wz) S[P_FZ].add(fabs(e[2]) * q0);
                    };
                    if constexpr (LINE > 0) {
                        Real cxr[LINE], wxr[LINE];
    #pragma unroll
                        for (int ix = 0; ix < LINE; ix++) {
                            cxr[ix] = xn[ix * 2] - ux;
                            wxr[ix] = vt[(vbeg + ix) * VT];
                        }
                        for (int v = vbeg; v < vend; v += LINE) {
                            Real P0 = 0, P1 = 0, P2 = 0, P3 = 0;
    #pragma unroll
                            for (int ix = 0; ix < LINE; ix++) {
                                const Real f = sp[v + ix];
                                const Real cx = cxr[ix];
                                const Real t0 = wxr[ix] * f;
                                const Real t1 = t0 * cx;
                                const Real t2 = t1 * cx;
                                P0 += t0;
                                P1 += t1;
                                P2 += t2;
                                P3 = fma(t2, cx, P3);
                            }
                            fold(P0, P1, P2, P3, v + LINE);
                        }
                    } else {
                        const Real *cxhc = cxh + cl * cxs;
                        int v = vbeg;
                        while (v < vend) {
                            const int ix0 = (v0 + v) % nxo;
                            const int ve = min(vend, v + (nxo - ix0));
                            Real P0 = 0, P1 = 0, P2 = 0, P3 = 0;
    #pragma unroll 4
                            for (int vv = v; vv < ve; vv++) {
                                const int ix = ix0 + (vv - v);
                                const Real f = sp[vv];
                                const Real cx = cxhc[ix];
                                const Real t0 = vt[vv * VT] * f;
                                const Real t1 = t0 * cx;
                                const Real t2 = t1 * cx;
                                P0 += t0;
                                P1 += t1;
                                P2 += t2;
                                P3 = fma(t2, cx, P3);
                            }
                            fold(P0, P1, P2, P3, ve);
                            v = ve;
                        }
                    }
                }
            }
            // combine the two halves and write the (group, cell) partial
            using Out = typename PartOut<Real>::T;
            Out *red = reinterpret_cast<Out *>(mred);
            if (vp == 1) {
#pragma unroll
                for (int q = 0; q < NPART; q++) {
                    if constexpr (sizeof(Real) == 8)
                        red[q * SLICE + cl] = S[q].value();
                    else
                        red[q * SLICE + cl] = make_float2(S[q].s, S[q].c);
                }
            }
            __syncthreads();
            if (vp == 0 && valid) {
                // the cell's NPART partials are contiguous (128 bytes)
                Out *pp = COHERENT ? static_cast<Out *>(scratch) + ((size_t)lk * SLICE + cl) * NPART
                                   : static_cast<Out *>(a.part) + ((size_t)vgid * ncell + CELL(GX(li), GY(lj), z)) * NPART;
#pragma unroll
                for (int q = 0; q < NPART; q += 2) {
                    if constexpr (sizeof(Real) == 8) {
                        *reinterpret_cast<double2 *>(pp + q) = make_double2(S[q].value() + red[q * SLICE + cl],
                                                                            S[q + 1].value() + red[(q + 1) * SLICE + cl]);
                    } else {
                        const float2 o0 = red[q * SLICE + cl], o1 = red[(q + 1) * SLICE + cl];
                        const float2 r0 = pair_add(S[q].s, S[q].c, o0.x, o0.y);
                        const float2 r1 = pair_add(S[q + 1].s, S[q + 1].c, o1.x, o1.y);
                        *reinterpret_cast<float4 *>(pp + q) = make_float4(r0.x, r0.y, r1.x, r1.y);
                    }
                }
            }
        }
        // the next slice's halo row overwrites the reduction buffer
        if constexpr (L::red_in_halo) __syncthreads();
    }

    // z outflow of the block for the next stage (own velocities only)
    if (!zlast) {
        for (int cl = 0; cl < SLICE; cl++) {
            const int li = cl % BX, lj = cl / BX;
            if (li >= ex || lj >= ey) continue;
            const int x = GX(li), y = GY(lj);
#pragma unroll
            for (int m = 0; m < TV; m++) {
                if (!ok[m]) continue;
                FZp[((size_t)y * nx + x) * Nv + gv[m]] = slice[SL(li, lj) + t + m * NT];
                if constexpr (ORDER == 2)  // slice ez-2 (the inflow slice k0-1 when ez == 1)
                    FZ2p[((size_t)y * nx + x) * Nv + gv[m]] = slice2[(lj * BX + li) * CS + t + m * NT];
            }
        }
    }
}

// One wavefront stage: CTA (x, y) = (work item x of the stage, velocity group y).
template <typename Real, int TV, int LINE, bool UNIF>
__global__ void __launch_bounds__(NT, 2) sweep_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    sweep_item<Real, TV, LINE, false, UNIF>(a, a.work[blockIdx.x], blockIdx.y, smem, nullptr);
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait for a completion flag: true once it is set, false after
// `limit` polls (the caller then records an error and returns).
__device__ bool wait_flag(const int *p, long long limit)
{
    for (long long i = 0; i < limit; i++) {
        if (ld_acquire(p) != 0) return true;
        __nanosleep(100);
    }
    return false;
}

// Bounded wait for a chain token to reach `v` (tokens only grow).
__device__ bool wait_token(const int *p, int v, long long limit)
{
    for (long long i = 0; i < limit; i++) {
        if (ld_acquire(p) >= v) return true;
        __nanosleep(100);
    }
    return false;
}

// Ordered accumulation of one item's moment partials.  Velocity group g of
// an octant adds into accumulator k = g % nacc; the items of one (k, block)
// form a chain in the order they were claimed, and the item at place `pos`
// adds after the one at pos - 1 (the first one stores).  The order is fixed
// by the work list, so the sums are bit-reproducible, and no item waits for
// one claimed after it.  FP32 partials are Kahan pairs (s, c) with value
// s - c; the accumulator holds a float-float pair (hi, lo) with value hi + lo,
// hi updated by a two-sum.
template <typename Real>
struct Acc16;
template <>
struct Acc16<double> {
    using V = double2;  // two slots
    __device__ static V init(V s) { return s; }
    __device__ static V add(V a, V s) { return make_double2(a.x + s.x, a.y + s.y); }
};
template <>
struct Acc16<float> {
    using V = float4;  // two slots: (s0, c0, s1, c1) / (hi0, lo0, hi1, lo1)
    __device__ static V init(V s) { return make_float4(s.x, -s.y, s.z, -s.w); }
    __device__ static float2 ff(float hi, float lo, float s, float c)
    {
        const float t = hi + s;
        const float bp = t - hi;
        const float err = (hi - (t - bp)) + (s - bp);
        return make_float2(t, lo + (err - c));
    }
    __device__ static V add(V a, V s)
    {
        const float2 p = ff(a.x, a.y, s.x, s.y), q = ff(a.z, a.w, s.z, s.w);
        return make_float4(p.x, p.y, q.x, q.y);
    }
};

// Block geometry of an item for the chain: physical extents and origin.
struct BlockSpan {
    bool px, py, pz;
    int x0, ex, y0, ey, z0, ez;
    __device__ BlockSpan(const SweepArgs &a, int o, int bxr, int byr, int bzr)
    {
        px = (o & 1) != 0, py = (o & 2) != 0, pz = (o & 4) != 0;
        const int bxi = px ? bxr : a.nbx - 1 - bxr;
        const int byi = py ? byr : a.nby - 1 - byr;
        const int bzi = pz ? bzr : a.nbz - 1 - bzr;
        x0 = bxi * BX, ex = min(BX, a.nx - x0);
        y0 = byi * BY, ey = min(BY, a.ny - y0);
        z0 = bzi * a.bz, ez = min(a.bz, a.nz - z0);
    }
    // global cell of the block's local (march-order) cell cl of slice lk
    __device__ size_t cell(const SweepArgs &a, int cl, int lk) const
    {
        const int li = cl % BX, lj = cl / BX;
        const int x = px ? x0 + li : x0 + ex - 1 - li;
        const int y = py ? y0 + lj : y0 + ey - 1 - lj;
        const int z = pz ? z0 + lk : z0 + ez - 1 - lk;
        return (size_t)x + (size_t)a.nx * ((size_t)y + (size_t)a.ny * z);
    }
    __device__ bool valid(int cl) const { return cl % BX < ex && cl / BX < ey; }
};

// Before the chain wait: pull the block's accumulator records into L2.
template <typename Real>
__device__ void chain_prefetch(const SweepArgs &a, const BlockSpan &b, int vg)
{
    const unsigned char *acc = static_cast<const unsigned char *>(a.acc) +
                               (size_t)(vg % a.nacc) * a.ncell * a.acc_slots * 8;
    const int rec = a.acc_slots * 8;
    for (int r = threadIdx.x; r < b.ez * BY; r += NT) {  // one row of ex cells
        const int lj = r % BY, lk = r / BY;
        if (lj >= b.ey) continue;
        const unsigned char *p = acc + b.cell(a, lj * BX, lk) * rec;
        const unsigned char *q = acc + b.cell(a, lj * BX + b.ex - 1, lk) * rec;
        const unsigned char *lo = p < q ? p : q;
        for (int off = 0; off < b.ex * rec; off += 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(lo + off));
    }
}

template <typename Real>
__device__ void chain_add(const SweepArgs &a, int o, int bxr, int byr, int bzr, int vg, int pos,
                          const void *scratch)
{
    using Out = typename PartOut<Real>::T;
    const BlockSpan b(a, o, bxr, byr, bzr);
    const size_t ncell = a.ncell;
    if (a.acc_slots == ACC_COMPACT) {
        // the item's record and the accumulator record share one layout: add
        // them element-wise, 16 bytes (two slots) at a time, with CH vectors
        // of every thread in flight
        using A = Acc16<Real>;
        using V = typename A::V;
        constexpr int VPC = NPART * 8 / 16;  // vectors per cell record
        constexpr int CH = 4;
        const V *sc = static_cast<const V *>(scratch);
        V *acc = reinterpret_cast<V *>(static_cast<Out *>(a.acc) + (size_t)(vg % a.nacc) * ncell * ACC_COMPACT);
        const int n = b.ez * SLICE * VPC;
        for (int base = threadIdx.x; base < n; base += NT * CH) {
            V sv[CH], av[CH];
            size_t at[CH];
            bool live[CH];
#pragma unroll
            for (int u = 0; u < CH; u++) {
                const int e = base + u * NT;
                const int lc = e / VPC, cl = lc % SLICE;
                live[u] = e < n && b.valid(cl);
                at[u] = live[u] ? b.cell(a, cl, lc / SLICE) * VPC + e % VPC : 0;
                if (live[u]) sv[u] = sc[e];  // written by this CTA: the same L1 path
            }
            if (pos > 0) {
#pragma unroll
                for (int u = 0; u < CH; u++)
                    if (live[u]) av[u] = __ldcg(acc + at[u]);
            }
#pragma unroll
            for (int u = 0; u < CH; u++)
                if (live[u]) acc[at[u]] = pos == 0 ? A::init(sv[u]) : A::add(av[u], sv[u]);
        }
        return;
    }
    // ACC_SPLIT: the item's flux slots go to the slots of the sides ahead of
    // its octant; the first item of the chain stores zero on the other sides
    const Out *sc = static_cast<const Out *>(scratch);
    Out *acc = static_cast<Out *>(a.acc) + (size_t)(vg % a.nacc) * ncell * ACC_SPLIT;
    const int n = b.ez * SLICE * NPART;
#pragma unroll 4
    for (int e = threadIdx.x; e < n; e += NT) {
        const int q = e % NPART, cl = (e / NPART) % SLICE, lk = e / (NPART * SLICE);
        if (!b.valid(cl)) continue;
        const size_t cell = b.cell(a, cl, lk);
        const int slot = q < P_FX ? q : SUM_F0 + 2 * (q - P_FX) + ((o >> (q - P_FX)) & 1);
        const Out v = sc[e];  // written by this CTA: the same L1 path
        Out *dst = acc + cell * ACC_SPLIT + slot;
        if (pos == 0 && q >= P_FX) {
            Out *other = acc + cell * ACC_SPLIT + (SUM_F0 + 2 * (q - P_FX) + 1 - ((o >> (q - P_FX)) & 1));
            if constexpr (sizeof(Real) == 8)
                *other = 0.0;
            else
                *other = make_float2(0.f, 0.f);
        }
        if constexpr (sizeof(Real) == 8) {
            *dst = pos == 0 ? v : __ldcg(dst) + v;
        } else {
            if (pos == 0) {
                *dst = make_float2(v.x, -v.y);
            } else {
                const float2 cur = __ldcg(dst);
                const float t = cur.x + v.x;
                const float bp = t - cur.x;
                const float err = (cur.x - (t - bp)) + (v.x - bp);
                *dst = make_float2(t, cur.y + (err - v.y));
            }
        }
    }
}

// Persistent sweep over the items of many problem instances.  Items are
// claimed in list order (stage-major), so every item's upwind dependencies
// and its accumulator-chain predecessor were claimed earlier by CTAs that are
// running: the waits always end unless an error stopped a producer, and then
// they end at the poll limit.
template <typename Real, int TV, int LINE, bool UNIF, int ORDER, bool DEV>
__global__ void __launch_bounds__(NT, 2) sweep_persistent_kernel(const BatchSweepArgs b)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SweepArgs sa;
    __shared__ int s_item, s_go;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(b.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= b.n_items) break;
        const int4 item = b.items[it];
        const int inst = item.x, o = item.y >> 24, vg = item.y & 0xffffff;
        const int bxr = item.z & 1023, byr = (item.z >> 10) & 1023, bzr = (item.z >> 20) & 1023;
        // copy the instance's arguments to shared memory (words of the struct)
        {
            const int *src = reinterpret_cast<const int *>(b.inst + inst);
            int *dst = reinterpret_cast<int *>(&sa);
            for (int q = threadIdx.x; q < (int)(sizeof(SweepArgs) / sizeof(int)); q += NT) dst[q] = src[q];
        }
        int *fl = b.flags + b.flag_off[inst];
        if (threadIdx.x == 0) {
            const SweepArgs &a = b.inst[inst];
            const int vgg = item.w;  // global velocity-group index within the instance
            auto fidx = [&](int x, int y, int z) { return ((vgg * a.nbz + z) * a.nby + y) * a.nbx + x; };
            bool ok = *b.error == 0;
            if (ok && bxr > 0) ok = wait_flag(fl + fidx(bxr - 1, byr, bzr), b.spin_limit);
            if (ok && byr > 0) ok = wait_flag(fl + fidx(bxr, byr - 1, bzr), b.spin_limit);
            if (ok && bzr > 0) ok = wait_flag(fl + fidx(bxr, byr, bzr - 1), b.spin_limit);
            if (!ok) atomicExch(b.error, 1);
            s_go = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_go) break;
        void *scratch = static_cast<unsigned char *>(b.scratch) + (size_t)blockIdx.x * b.scratch_stride;
        sweep_item<Real, TV, LINE, true, UNIF, ORDER, DEV>(sa, make_int4(o, bxr, byr, bzr), vg, smem, scratch);
        __syncthreads();
        // the downwind blocks may start: the face planes are written
        if (threadIdx.x == 0 && it != b.skip_publish) {
            __threadfence();
            const int vgg = item.w;
            st_release(fl + ((vgg * sa.nbz + bzr) * sa.nby + byr) * sa.nbx + bxr, 1);
        }
        // then the item's turn in its accumulator chain
        const int pos = b.pos[it];
        const int bxi = (o & 1) ? bxr : sa.nbx - 1 - bxr;
        const int byi = (o & 2) ? byr : sa.nby - 1 - byr;
        const int bzi = (o & 4) ? bzr : sa.nbz - 1 - bzr;
        int *tk = sa.tok + (((size_t)(vg % sa.nacc) * sa.nbz + bzi) * sa.nby + byi) * sa.nbx + bxi;
        if (pos > 0) chain_prefetch<Real>(sa, BlockSpan(sa, o, bxr, byr, bzr), vg);
        if (threadIdx.x == 0) {
            bool ok = pos == 0 || wait_token(tk, pos, b.spin_limit);
            if (!ok) atomicExch(b.error, 1);
            s_go = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_go) break;
        chain_add<Real>(sa, o, bxr, byr, bzr, vg, pos, scratch);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(tk, pos + 1);
        }
    }
}

// The dynamic shared-memory limit is an attribute of a kernel on one device:
// it is raised (never lowered) on the current device before a launch that
// needs more than that device has been given, under a lock so that host
// threads launching the same kernel do not undo each other's setting.
std::mutex g_smem_mutex;
std::map<std::pair<int, const void *>, size_t> g_smem_set;

cudaError_t ensure_smem(const void *fn, size_t bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_smem_mutex);
    size_t &have = g_smem_set[std::make_pair(dev, fn)];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

template <typename Real, int TV, int LINE, bool UNIF>
cudaError_t launch_t(const SweepArgs &a, int n_items, int max_vg, cudaStream_t s)
{
    using L = SmemLayout<Real, TV>;
    const size_t bytes = L::total(a.nxo_max, LINE > 0);
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(sweep_kernel<Real, TV, LINE, UNIF>), bytes);
    if (e != cudaSuccess) return e;
    dim3 grid(n_items, max_vg);
    sweep_kernel<Real, TV, LINE, UNIF><<<grid, NT, bytes, s>>>(a);
    return cudaGetLastError();
}

template <typename Real, int TV>
cudaError_t launch_line(const SweepArgs &a, int n_items, int max_vg, cudaStream_t s)
{
    if (a.line16)
        return a.uniform ? launch_t<Real, TV, 16, true>(a, n_items, max_vg, s)
                         : launch_t<Real, TV, 16, false>(a, n_items, max_vg, s);
    return a.uniform ? launch_t<Real, TV, 0, true>(a, n_items, max_vg, s)
                     : launch_t<Real, TV, 0, false>(a, n_items, max_vg, s);
}

template <typename Real, int TV, int LINE, bool UNIF, int ORDER, bool DEV>
cudaError_t launch_persistent_t(const BatchSweepArgs &b, int nxo_max, int grid, cudaStream_t s)
{
    using L = SmemLayout<Real, TV, ORDER>;
    const size_t bytes = L::total(nxo_max, LINE > 0);
    const void *fn = reinterpret_cast<const void *>(sweep_persistent_kernel<Real, TV, LINE, UNIF, ORDER, DEV>);
    cudaError_t e = ensure_smem(fn, bytes);
    if (e != cudaSuccess) return e;
    sweep_persistent_kernel<Real, TV, LINE, UNIF, ORDER, DEV><<<grid, NT, bytes, s>>>(b);
    return cudaGetLastError();
}

template <typename Real, int TV, int LINE, bool UNIF, int ORDER, bool DEV>
int occupancy_t(size_t smem)
{
    int n = 0;
    const void *fn = reinterpret_cast<const void *>(sweep_persistent_kernel<Real, TV, LINE, UNIF, ORDER, DEV>);
    if (ensure_smem(fn, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_persistent_kernel<Real, TV, LINE, UNIF, ORDER, DEV>,
                                                      NT, smem) != cudaSuccess)
        return 0;
    return n;
}

// Instantiation for (precision, velocities per thread, line specialisation,
// uniform grid) chosen at run time, first-order sweep.
template <template <typename, int, int, bool, int, bool> class F, typename... Args>
auto dispatch(int precision, int tv, int line16, int uniform, Args &&...args)
{
#define KGS_CASES(R, T)                                                                                   \
    if (line16)                                                                                           \
        return uniform ? F<R, T, 16, true, 1, false>::run(args...) : F<R, T, 16, false, 1, false>::run(args...); \
    return uniform ? F<R, T, 0, true, 1, false>::run(args...) : F<R, T, 0, false, 1, false>::run(args...);
    if (precision == 0) {
        KGS_CASES(double, 1)
    }
    if (tv == 2) {
        KGS_CASES(float, 2)
    }
    KGS_CASES(float, 1)
#undef KGS_CASES
}

// The second-order sweep: one velocity per thread, uniform grids.
template <template <typename, int, int, bool, int, bool> class F, typename... Args>
auto dispatch_order2(int precision, int line16, Args &&...args)
{
    if (precision == 0)
        return line16 ? F<double, 1, 16, true, 2, false>::run(args...) : F<double, 1, 0, true, 2, false>::run(args...);
    return line16 ? F<float, 1, 16, true, 2, true>::run(args...) : F<float, 1, 0, true, 2, true>::run(args...);
}

// The first-order FP32 sweep with the deviation-form source, uniform grids.
template <template <typename, int, int, bool, int, bool> class F, typename... Args>
auto dispatch_dev(int tv, int line16, Args &&...args)
{
    if (tv == 2)
        return line16 ? F<float, 2, 16, true, 1, true>::run(args...) : F<float, 2, 0, true, 1, true>::run(args...);
    return line16 ? F<float, 1, 16, true, 1, true>::run(args...) : F<float, 1, 0, true, 1, true>::run(args...);
}

template <typename Real, int TV, int LINE, bool UNIF, int ORDER, bool DEV>
struct PersistentLaunch {
    static cudaError_t run(const BatchSweepArgs &b, int nxo_max, int grid, cudaStream_t s)
    {
        return launch_persistent_t<Real, TV, LINE, UNIF, ORDER, DEV>(b, nxo_max, grid, s);
    }
};

template <typename Real, int TV, int LINE, bool UNIF, int ORDER, bool DEV>
struct Occupancy {
    static int run(size_t smem) { return occupancy_t<Real, TV, LINE, UNIF, ORDER, DEV>(smem); }
};

}  // namespace

int sweep_persistent_occupancy(int precision, int tv, int line16, int uniform, size_t smem, int order, int dev)
{
    if (order == 2) return (tv == 1 && uniform) ? dispatch_order2<Occupancy>(precision, line16, smem) : 0;
    if (dev) return (precision != 0 && uniform) ? dispatch_dev<Occupancy>(tv, line16, smem) : 0;
    return dispatch<Occupancy>(precision, tv, line16, uniform, smem);
}

cudaError_t launch_sweep_persistent(int precision, int tv, int line16, int uniform, const BatchSweepArgs &b,
                                    int nxo_max, int grid, cudaStream_t s, int order, int dev)
{
    if (b.n_items == 0) return cudaSuccess;
    if (order == 2) {
        if (tv != 1 || !uniform) return cudaErrorInvalidValue;
        return dispatch_order2<PersistentLaunch>(precision, line16, b, nxo_max, grid, s);
    }
    if (dev) {
        if (precision == 0 || !uniform) return cudaErrorInvalidValue;
        return dispatch_dev<PersistentLaunch>(tv, line16, b, nxo_max, grid, s);
    }
    return dispatch<PersistentLaunch>(precision, tv, line16, uniform, b, nxo_max, grid, s);
}

size_t sweep_smem_bytes(int precision, int tv, int line16, int nxo_max, int order)
{
    const bool line = line16 != 0;
    if (order == 2)
        return precision == 0 ? SmemLayout<double, 1, 2>::total(nxo_max, line)
                              : SmemLayout<float, 1, 2>::total(nxo_max, line);
    if (precision == 0) return SmemLayout<double, 1>::total(nxo_max, line);
    return tv == 2 ? SmemLayout<float, 2>::total(nxo_max, line) : SmemLayout<float, 1>::total(nxo_max, line);
}

cudaError_t launch_sweep(int precision, int tv, const SweepArgs &a, int n_items, int max_vg, cudaStream_t s)
{
    if (n_items == 0 || max_vg == 0) return cudaSuccess;
    if (precision == 0) return launch_line<double, 1>(a, n_items, max_vg, s);
    if (tv == 2) return launch_line<float, 2>(a, n_items, max_vg, s);
    return launch_line<float, 1>(a, n_items, max_vg, s);
}

}  // namespace kgs
