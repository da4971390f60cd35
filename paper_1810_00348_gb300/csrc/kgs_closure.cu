// kgs_closure.cu -- per-iteration kernels around the sweep (arXiv 1810.00348):
//   coef_kernel      lagged cell coefficients of Eq. (2) and tau = mu/p (Eq. (10))
//   part_sums        fixed-order sum of the staged sweep's per-group partials
//   acc_sums         fixed-order sum of the persistent sweep's accumulators
//   closure          the macroscopic update of Eq. (5) and the wall densities
//                    of Eq. (9) from the per-cell sums
//   finalize_mass    global mass and the Section 3.4 rescale factor
//   scale_residual   rescale, divergence check and the Section 4.1 residual
//   finalize_residual
//   wall_flux_init   wall densities from the flux of the initial equilibrium
// All arithmetic in FP64.  Every reduction is a fixed-shape tree per block
// followed by an in-order sum over blocks, so results do not depend on
// scheduling.
#include "kgs_internal.h"

namespace kgs {
namespace {

constexpr double R_GAS = 0.5;
constexpr double LOG2E = 1.4426950408889634074;
constexpr int RED_THREADS = 256;

template <typename Real>
__global__ void coef_kernel(const double *__restrict__ mac, const uint8_t *__restrict__ solid,
                            const uint8_t *__restrict__ side_flags, const double *__restrict__ rdx,
                            const double *__restrict__ rdy, const double *__restrict__ rdz, int nx, int ny, int nz,
                            double mu_ref, double omega, double Pr, int dev_src, Real *__restrict__ coef)
{
    const size_t ncell = (size_t)nx * ny * nz;
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((size_t)nx * ny));
    Real out[NCOEF];
    for (int q = 0; q < NCOEF; q++) out[q] = Real(0);
    const int sf = side_flags[c];  // bits 0..5 solid neighbour, 6..11 wall face (packed in 2 bytes)
    const int wf = side_flags[ncell + c];
    int flags = ((sf & 63) * F_SOLID_SIDE) | ((wf & 63) << 7);
    if (solid && solid[c]) {
        flags |= F_SOLID;
    } else {
        const double rho = mac[c], T = mac[4 * ncell + c];
        const double RT = R_GAS * T;
        const double p = rho * RT;
        // tau = mu / p, mu = mu_ref T^omega (Sections 2.1 and 4)
        const double rtau = p / (mu_ref * pow(T, omega));
        const double tpr = 2.0 * M_PI * RT;
        const double A = rho / (tpr * sqrt(tpr));  // rho (2 pi R T)^(-3/2)
        const double sh = (1.0 - Pr) / (5.0 * p * RT);
        // centre U^n in the sweep precision, stored doubled and negated (exact)
        const double U[3] = {(double)(Real)mac[1 * ncell + c], (double)(Real)mac[2 * ncell + c],
                             (double)(Real)mac[3 * ncell + c]};
        const double q[3] = {(double)(Real)(sh * mac[5 * ncell + c]), (double)(Real)(sh * mac[6 * ncell + c]),
                             (double)(Real)(sh * mac[7 * ncell + c])};
        const double U2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
        out[C_M2UX] = (Real)(-2.0 * U[0]);
        out[C_M2UY] = (Real)(-2.0 * U[1]);
        out[C_M2UZ] = (Real)(-2.0 * U[2]);
        // exp(-|c|^2/(2RT)) = exp(-|U|^2/(2RT)) exp(-(|xi|^2 + s)/(2RT)); the FP32
        // sweep takes kappa as a base-2 logarithm inside its exponent
        out[C_KAPPA] = sizeof(Real) == 8 ? (Real)(rtau * A * exp(-U2 / (2.0 * RT)))
                                         : (Real)(log2(rtau * A) - LOG2E * U2 / (2.0 * RT));
        out[C_NEXP] = sizeof(Real) == 8 ? (Real)(-1.0 / (2.0 * RT)) : (Real)(-LOG2E / (2.0 * RT));
        out[C_RT1] = (Real)(1.0 / RT);
        out[C_QX] = (Real)q[0];
        out[C_QY] = (Real)q[1];
        out[C_QZ] = (Real)q[2];
        out[C_SHK0] = (Real)(U2 / RT - 5.0);
        out[C_MUQ] = (Real)(-(U[0] * q[0] + U[1] * q[1] + U[2] * q[2]));
        out[C_RTAU] = (Real)rtau;
        out[C_RDX] = (Real)rdx[i];
        out[C_RDY] = (Real)rdy[j];
        out[C_RDZ] = (Real)rdz[k];
        if (dev_src) {
            // FP32 second-order sweep (uniform grid: the widths are not read
            // per cell): the base-2 exponent of f^S_M / M_ref, against the
            // reference at rest (rho = 1, T = 1), is
            //   D = |xi|^2 (nexp - nexp_ref) + nexp (-2 U.xi) + K,
            //   nexp - nexp_ref = log2(e) (T - 1) / T,
            //   K = log2(rho) - 1.5 log2(T) - log2(e) |U|^2 / T,
            // both small where the gas is near the reference state
            out[C_RDX] = (Real)(LOG2E * (T - 1.0) / T);
            out[C_RDY] = (Real)(log2(rho) - 1.5 * log2(T) - LOG2E * U2 / (2.0 * RT));
        }
    }
    out[C_FLAGS] = flag_value<Real>(flags);
    for (int q = 0; q < NCOEF; q++) coef[c * NCOEF + q] = out[q];
}

// Block tree sum of NV doubles per thread into blk[blockIdx.x * NV + v].
template <int NV>
__device__ void block_sum(double (&v)[NV], double *blk)
{
    __shared__ double sh[NV][RED_THREADS];
    for (int q = 0; q < NV; q++) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int q = 0; q < NV; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < NV; q++) blk[(size_t)blockIdx.x * NV + q] = sh[q][0];
}

// Float-float accumulator: the running sum is hi + lo with |lo| <= ulp(hi)/2
// up to the rounding of lo itself; add(x, y) adds x - y.  hi is updated by
// Knuth's two-sum, whose rounding error is exact and goes to lo.
struct FFSum {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x, float y)
    {
        const float t = hi + x;
        const float bp = t - hi;
        const float err = (hi - (t - bp)) + (x - bp);
        hi = t;
        lo += err - y;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Sum w M_ref (xi_x - Ux)^A (xi_y - Uy)^B (xi_z - Uz)^C of the reference
// Maxwellian over the swept velocities: the binomial expansion of its raw
// moments about the cell's lagged velocity U (compile-time orders, so the
// loops unroll and the raw moments are read at constant offsets).
__host__ __device__ constexpr double binom3(int n, int k) { return (k == 0 || k == n) ? 1.0 : (n == 2 ? 2.0 : 3.0); }

template <int A, int B, int C>
__device__ __forceinline__ double ref_central(const RefMoments &r, const double U[3])
{
    double s = 0.0;
#pragma unroll
    for (int i = 0; i <= A; i++)
#pragma unroll
        for (int j = 0; j <= B; j++)
#pragma unroll
            for (int k = 0; k <= C; k++) {
                double f = binom3(A, i) * binom3(B, j) * binom3(C, k);
#pragma unroll
                for (int e = i; e < A; e++) f *= -U[0];
#pragma unroll
                for (int e = j; e < B; e++) f *= -U[1];
#pragma unroll
                for (int e = k; e < C; e++) f *= -U[2];
                s += f * r.raw[ref_index(i, j, k)];
            }
    return s;
}

// The reference Maxwellian's part of sum slot q (< SUM_F0) about U.
template <int Q>
__device__ __forceinline__ double ref_slot_of(const RefMoments &r, const double U[3])
{
    switch (Q) {
    case P_S0: return ref_central<0, 0, 0>(r, U);
    case P_S1X: return ref_central<1, 0, 0>(r, U);
    case P_S1Y: return ref_central<0, 1, 0>(r, U);
    case P_S1Z: return ref_central<0, 0, 1>(r, U);
    case P_S2XX: return ref_central<2, 0, 0>(r, U);
    case P_S2YY: return ref_central<0, 2, 0>(r, U);
    case P_S2ZZ: return ref_central<0, 0, 2>(r, U);
    case P_S2XY: return ref_central<1, 1, 0>(r, U);
    case P_S2XZ: return ref_central<1, 0, 1>(r, U);
    case P_S2YZ: return ref_central<0, 1, 1>(r, U);
    case P_S3X: return ref_central<3, 0, 0>(r, U) + ref_central<1, 2, 0>(r, U) + ref_central<1, 0, 2>(r, U);
    case P_S3Y: return ref_central<2, 1, 0>(r, U) + ref_central<0, 3, 0>(r, U) + ref_central<0, 1, 2>(r, U);
    default: return ref_central<2, 0, 1>(r, U) + ref_central<0, 2, 1>(r, U) + ref_central<0, 0, 3>(r, U);
    }
}

// All 13 reference parts of one cell.
__device__ __forceinline__ void ref_slots(const RefMoments &r, const double U[3], double (&out)[SUM_F0])
{
    out[P_S0] = ref_slot_of<P_S0>(r, U);
    out[P_S1X] = ref_slot_of<P_S1X>(r, U);
    out[P_S1Y] = ref_slot_of<P_S1Y>(r, U);
    out[P_S1Z] = ref_slot_of<P_S1Z>(r, U);
    out[P_S2XX] = ref_slot_of<P_S2XX>(r, U);
    out[P_S2YY] = ref_slot_of<P_S2YY>(r, U);
    out[P_S2ZZ] = ref_slot_of<P_S2ZZ>(r, U);
    out[P_S2XY] = ref_slot_of<P_S2XY>(r, U);
    out[P_S2XZ] = ref_slot_of<P_S2XZ>(r, U);
    out[P_S2YZ] = ref_slot_of<P_S2YZ>(r, U);
    out[P_S3X] = ref_slot_of<P_S3X>(r, U);
    out[P_S3Y] = ref_slot_of<P_S3Y>(r, U);
    out[P_S3Z] = ref_slot_of<P_S3Z>(r, U);
}

// Runtime slot index (the staged path's (cell, slot) threads).
__device__ double ref_slot(const RefMoments &r, int q, const double U[3])
{
    switch (q) {
    case P_S0: return ref_slot_of<P_S0>(r, U);
    case P_S1X: return ref_slot_of<P_S1X>(r, U);
    case P_S1Y: return ref_slot_of<P_S1Y>(r, U);
    case P_S1Z: return ref_slot_of<P_S1Z>(r, U);
    case P_S2XX: return ref_slot_of<P_S2XX>(r, U);
    case P_S2YY: return ref_slot_of<P_S2YY>(r, U);
    case P_S2ZZ: return ref_slot_of<P_S2ZZ>(r, U);
    case P_S2XY: return ref_slot_of<P_S2XY>(r, U);
    case P_S2XZ: return ref_slot_of<P_S2XZ>(r, U);
    case P_S2YZ: return ref_slot_of<P_S2YZ>(r, U);
    case P_S3X: return ref_slot_of<P_S3X>(r, U);
    case P_S3Y: return ref_slot_of<P_S3Y>(r, U);
    default: return ref_slot_of<P_S3Z>(r, U);
    }
}

// Lagged velocity centre of cell c as the FP32 sweep used it.
__device__ __forceinline__ void centre32(const void *coef, size_t c, double U[3])
{
    const float *cf = static_cast<const float *>(coef) + c * NCOEF;
    U[0] = -0.5 * (double)cf[C_M2UX];
    U[1] = -0.5 * (double)cf[C_M2UY];
    U[2] = -0.5 * (double)cf[C_M2UZ];
}

// Per-cell sums of the staged sweep's partials for CLOSE_CELLS cells per block:
// the first 13 warps hold (cell, moment slot) pairs, each thread summing one
// slot of one cell over all velocity groups in group order (a cell's slots
// are contiguous, so a warp's loads cover a few 128-byte rows); the last 3
// warps hold (cell, axis) pairs for the incoming wall fluxes, which split by
// the side of the group's octant.  The two kinds never share a warp, so
// neither takes the other's branch.
static_assert(CLOSE_CELLS * 13 % 32 == 0 && CLOSE_CELLS * 3 % 32 == 0, "slot warps must not mix");
template <typename Real>
__global__ void __launch_bounds__(CLOSE_CELLS * NPART) part_sums_kernel(const PartSumArgs a)
{
    const size_t ncell = a.ncell;
    const int t = threadIdx.x;
    const bool flux = t >= CLOSE_CELLS * P_FX;  // uniform per warp
    const int cl = flux ? (t - CLOSE_CELLS * P_FX) / 3 : t / P_FX;
    const int axis = flux ? (t - CLOSE_CELLS * P_FX) % 3 : 0;  // flux slots: incoming flux along x, y, z
    const int q = flux ? P_FX + axis : t % P_FX;
    const size_t c = (size_t)blockIdx.x * CLOSE_CELLS + cl;
    if (c >= ncell) return;
    double sum = 0.0, f_minus = 0.0, f_plus = 0.0;
    if (!(a.solid && a.solid[c])) {
        if (sizeof(Real) == 8) {
            const double *pp = static_cast<const double *>(a.part) + c * NPART + q;
            if (!flux) {
#pragma unroll 4
                for (int g = 0; g < a.n_vg; g++) sum += pp[(size_t)g * ncell * NPART];
            } else {
#pragma unroll 4
                for (int g = 0; g < a.n_vg; g++) {
                    const double v = pp[(size_t)g * ncell * NPART];
                    const bool ahead = (a.vg_oct[g] >> axis) & 1;  // the wall ahead of the group's octant
                    f_plus += ahead ? v : 0.0;                       // adding an exact zero changes nothing
                    f_minus += ahead ? 0.0 : v;
                }
            }
        } else {
            // FP32 partials are compensated pairs (value = x - y); they are
            // summed as float-float numbers (hi + lo, hi updated by an error-
            // free two-sum) on the FP32 pipe and widened once at the end.
            // The loads go in batches of CB groups into registers, the next
            // batch issued before the current one is summed, so that up to
            // 2 CB loads per thread are in flight.
            constexpr int CB = 16;
            FFSum acc0, acc1;  // flux slots: walls behind / ahead of the group's octant
            const float2 *pp = static_cast<const float2 *>(a.part) + c * NPART + q;
            const size_t gs = ncell * NPART;
            const int n_vg = a.n_vg;
            float2 cur[CB], nxt[CB];
            auto load = [&](float2 (&e)[CB], int g0) {
#pragma unroll
                for (int k = 0; k < CB; k++) e[k] = g0 + k < n_vg ? pp[(size_t)(g0 + k) * gs] : make_float2(0.f, 0.f);
            };
            load(cur, 0);
            for (int g0 = 0; g0 < n_vg; g0 += CB) {
                if (g0 + CB < n_vg) load(nxt, g0 + CB);
                if (!flux) {
#pragma unroll
                    for (int k = 0; k < CB; k++)
                        if (g0 + k < n_vg) acc0.add(cur[k].x, cur[k].y);
                } else {
                    // both sides take every group, one of them an exact zero
                    // pair, which leaves a float-float sum unchanged
#pragma unroll
                    for (int k = 0; k < CB; k++) {
                        const int g = g0 + k;
                        if (g < n_vg) {
                            const bool ahead = (a.vg_oct[g] >> axis) & 1;
                            acc1.add(ahead ? cur[k].x : 0.f, ahead ? cur[k].y : 0.f);
                            acc0.add(ahead ? 0.f : cur[k].x, ahead ? 0.f : cur[k].y);
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < CB; k++) cur[k] = nxt[k];
            }
            sum = f_minus = acc0.value();
            f_plus = acc1.value();
            // the FP32 sweep summed g = f - M_ref: add the reference's part
            if (!flux) {
                double U[3];
                centre32(a.coef, c, U);
                sum += ref_slot(a.ref, q, U);
            } else {
                if (a.wall_kind[(size_t)(2 * axis) * ncell + c] >= 0) f_minus += a.ref.flux[2 * axis];
                if (a.wall_kind[(size_t)(2 * axis + 1) * ncell + c] >= 0) f_plus += a.ref.flux[2 * axis + 1];
            }
        }
    }
    if (!flux) {
        a.sums[(size_t)q * ncell + c] = sum;
    } else {
        a.sums[(size_t)(SUM_F0 + 2 * axis) * ncell + c] = f_minus;
        a.sums[(size_t)(SUM_F0 + 2 * axis + 1) * ncell + c] = f_plus;
    }
}

// Per-cell sums of the persistent sweep's ordered accumulators, ACC_CELLS
// cells per block.  First the block's (cell, slot) pairs in address order
// (coalesced): each adds its slot's nacc accumulators in accumulator order
// (float-float for the FP32 path) into shared memory.  Then one thread per
// cell maps the accumulator slots to the NSUM sum slots, adds the reference
// Maxwellian's part (FP32 path) and writes the FP64 sums.
constexpr int ACC_CELLS = 128;
template <typename Real>
__global__ void __launch_bounds__(ACC_CELLS) acc_sums_kernel(const AccSumArgs a)
{
    __shared__ double tot[ACC_CELLS * ACC_SPLIT];
    const size_t ncell = a.ncell;
    const size_t c0 = (size_t)blockIdx.x * ACC_CELLS;
    const int nc = (int)min((size_t)ACC_CELLS, ncell - c0);
    const int ns = a.acc_slots, nacc = a.nacc;
    const size_t ks = ncell * ns;
    for (int j = threadIdx.x; j < nc * ns; j += ACC_CELLS) {
        const size_t at = c0 * ns + j;
        if (sizeof(Real) == 8) {
            const double *p = static_cast<const double *>(a.acc) + at;
            double e[NACC_MAX];
#pragma unroll
            for (int k = 0; k < NACC_MAX; k++) e[k] = k < nacc ? p[(size_t)k * ks] : 0.0;
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < NACC_MAX; k++)
                if (k < nacc) v += e[k];
            tot[j] = v;
        } else {
            const float2 *p = static_cast<const float2 *>(a.acc) + at;
            float2 e[NACC_MAX];
#pragma unroll
            for (int k = 0; k < NACC_MAX; k++) e[k] = k < nacc ? p[(size_t)k * ks] : make_float2(0.f, 0.f);
            FFSum t;
#pragma unroll
            for (int k = 0; k < NACC_MAX; k++)
                if (k < nacc) {
                    t.add(e[k].x, 0.f);
                    t.add(e[k].y, 0.f);
                }
            tot[j] = t.value();
        }
    }
    __syncthreads();
    const int cl = threadIdx.x;
    if (cl >= nc) return;
    const size_t c = c0 + cl;
    const double *tc = tot + (size_t)cl * ns;
    if (a.solid && a.solid[c]) {
        for (int q = 0; q < NSUM; q++) a.sums[(size_t)q * ncell + c] = 0.0;
        return;
    }
    if constexpr (sizeof(Real) == 4) {
        // the FP32 sweep summed g = f - M_ref: add the reference's part
        double U[3], ref[SUM_F0];
        centre32(a.coef, c, U);
        ref_slots(a.ref, U, ref);
#pragma unroll
        for (int q = 0; q < SUM_F0; q++) a.sums[(size_t)q * ncell + c] = tc[q] + ref[q];
    } else {
        for (int q = 0; q < SUM_F0; q++) a.sums[(size_t)q * ncell + c] = tc[q];
    }
#pragma unroll
    for (int side = 0; side < 6; side++) {
        // compact layout: the flux of an axis belongs to the side that has a
        // wall, zero on the other side
        const bool wall = a.wall_kind[(size_t)side * ncell + c] >= 0;
        double v;
        if (ns == ACC_COMPACT)
            v = wall ? tc[SUM_F0 + side / 2] : 0.0;
        else
            v = tc[SUM_F0 + side];
        if constexpr (sizeof(Real) == 4)
            if (wall) v += a.ref.flux[side];
        a.sums[(size_t)(SUM_F0 + side) * ncell + c] = v;
    }
}

// Closure of one outer iteration, one thread per cell (CLOSE_CELLS cells per
// block): the sums about U^n become the macroscopic fields of step n+1 and
// the wall densities (Eq. (5), Eq. (9)); the block's cell masses are summed
// in a fixed order for the Section 3.4 rescale.
__global__ void __launch_bounds__(CLOSE_CELLS) closure_kernel(const ClosureArgs a)
{
    const size_t ncell = a.ncell;
    const size_t c = (size_t)blockIdx.x * CLOSE_CELLS + threadIdx.x;
    const bool live = c < ncell && !(a.solid && a.solid[c]);
    double mass = 0.0;
    if (live) {
        double S[NSUM];
        for (int q = 0; q < NSUM; q++) S[q] = a.sums[(size_t)q * ncell + c];
        // The sums were taken about the lagged velocity U^n as stored in the
        // sweep precision; shift exactly to U^{n+1} = U^n + delta.
        double m2u[3];
        if (a.precision == 0) {
            const double *cf = static_cast<const double *>(a.coef) + c * NCOEF;
            m2u[0] = cf[C_M2UX], m2u[1] = cf[C_M2UY], m2u[2] = cf[C_M2UZ];
        } else {
            const float *cf = static_cast<const float *>(a.coef) + c * NCOEF;
            m2u[0] = cf[C_M2UX], m2u[1] = cf[C_M2UY], m2u[2] = cf[C_M2UZ];
        }
        const double Uc[3] = {-0.5 * m2u[0], -0.5 * m2u[1], -0.5 * m2u[2]};
        const double rho = S[P_S0];
        const double d[3] = {S[P_S1X] / rho, S[P_S1Y] / rho, S[P_S1Z] / rho};
        const double S2[3][3] = {{S[P_S2XX], S[P_S2XY], S[P_S2XZ]},
                                 {S[P_S2XY], S[P_S2YY], S[P_S2YZ]},
                                 {S[P_S2XZ], S[P_S2YZ], S[P_S2ZZ]}};
        const double S1[3] = {S[P_S1X], S[P_S1Y], S[P_S1Z]};
        const double S3[3] = {S[P_S3X], S[P_S3Y], S[P_S3Z]};
        const double trS2 = S2[0][0] + S2[1][1] + S2[2][2];
        const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double dS1 = d[0] * S1[0] + d[1] * S1[1] + d[2] * S1[2];
        // rho E - rho |U|^2 / 2 = tr(P)/2 with P = S2 - S0 delta delta^T, and
        // rho E = rho |U|^2/2 + (3/2) rho R T (Section 2.1)
        const double trP = trS2 - rho * d2;
        const double T = trP / (3.0 * rho * R_GAS);
        double qf[3];
        for (int i = 0; i < 3; i++) {
            if (a.q_lagged) {
                // the heat flux about the lagged velocity U^n (Algorithm 3's
                // eight moments, exact only at the fixed point)
                qf[i] = 0.5 * S3[i];
            } else {
                // q_i = 1/2 sum w f (c'-delta)_i |c'-delta|^2 expanded in the sums about U^n
                const double S2d = S2[i][0] * d[0] + S2[i][1] * d[1] + S2[i][2] * d[2];
                qf[i] = 0.5 * (S3[i] - 2.0 * S2d - d[i] * trS2 + 2.0 * d[i] * dS1 + d2 * S1[i] - rho * d2 * d[i]);
            }
        }
        double *mn = a.mac_new;
        mn[c] = rho;
        mn[1 * ncell + c] = Uc[0] + d[0];
        mn[2 * ncell + c] = Uc[1] + d[1];
        mn[3 * ncell + c] = Uc[2] + d[2];
        mn[4 * ncell + c] = T;
        mn[5 * ncell + c] = qf[0];
        mn[6 * ncell + c] = qf[1];
        mn[7 * ncell + c] = qf[2];
        for (int s = 0; s < 6; s++) {
            const int kind = a.wall_kind[s * ncell + c];
            a.rho_w_new[s * ncell + c] = kind >= 0 ? S[SUM_F0 + s] * a.wall_norm[kind * 6 + s] : 0.0;
        }
        const int i = (int)(c % a.nx), j = (int)((c / a.nx) % a.ny), k = (int)(c / ((size_t)a.nx * a.ny));
        mass = rho * a.dx[i] * a.dy[j] * a.dz[k];
    } else if (c < ncell) {
        for (int v = 0; v < 8; v++) a.mac_new[v * ncell + c] = 0.0;
        for (int s = 0; s < 6; s++) a.rho_w_new[s * ncell + c] = 0.0;
    }
    // fixed-order sum of the block's cell masses (lanes 0 .. CLOSE_CELLS-1)
    static_assert(CLOSE_CELLS == 32, "one warp per block's cells");
    for (int off = 16; off > 0; off >>= 1) mass += __shfl_down_sync(0xffffffffu, mass, off);
    if (threadIdx.x == 0) a.blk_mass[blockIdx.x] = mass;
}

// Total mass (fixed order: strided per-thread sums, then a tree) and the
// Section 3.4 rescale factor.
__global__ void __launch_bounds__(RED_THREADS)
    finalize_mass_kernel(const double *blk_mass, int n_blocks, double M0, int rescale, double *scale)
{
    __shared__ double sh[RED_THREADS];
    double M = 0.0;
    for (int b = threadIdx.x; b < n_blocks; b += RED_THREADS) M += blk_mass[b];
    sh[threadIdx.x] = M;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scale[0] = rescale ? M0 / sh[0] : 1.0;
        scale[1] = sh[0];
    }
}

__global__ void __launch_bounds__(RED_THREADS)
    scale_residual_kernel(double *mac_new, double *rho_w_new, const double *mac, const uint8_t *solid, size_t ncell,
                          const double *scale, double *blk_res, int *blk_bad)
{
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double s = scale[0];
    double v[10];
    for (int q = 0; q < 10; q++) v[q] = 0.0;
    int bad = 0;
    if (c < ncell && !(solid && solid[c])) {
        mac_new[c] *= s;
        for (int d = 0; d < 3; d++) mac_new[(5 + d) * ncell + c] *= s;
        for (int f = 0; f < 6; f++) rho_w_new[f * ncell + c] *= s;
        double pn[5], po[5];
        for (int t = 0; t < 2; t++) {
            const double *m = t ? mac : mac_new;
            double *phi = t ? po : pn;
            const double r = m[c], ux = m[ncell + c], uy = m[2 * ncell + c], uz = m[3 * ncell + c],
                         T = m[4 * ncell + c];
            phi[0] = r;
            phi[1] = r * ux;
            phi[2] = r * uy;
            phi[3] = r * uz;
            phi[4] = 0.5 * r * (ux * ux + uy * uy + uz * uz) + 1.5 * r * R_GAS * T;
        }
        for (int t = 0; t < 5; t++) {
            const double dd = pn[t] - po[t];
            v[t] = dd * dd;
            v[5 + t] = pn[t] * pn[t];
        }
        const double r = mac_new[c], T = mac_new[4 * ncell + c];
        bool finite = isfinite(r) && isfinite(T);
        for (int q = 1; q < 8; q++) finite = finite && isfinite(mac_new[q * ncell + c]);
        if (!(r > 0.0) || !(T > 0.0) || !finite) bad = 1;
    }
    block_sum<10>(v, blk_res);
    __shared__ int any_bad;
    if (threadIdx.x == 0) any_bad = 0;
    __syncthreads();
    if (bad) any_bad = 1;
    __syncthreads();
    if (threadIdx.x == 0) blk_bad[blockIdx.x] = any_bad;
}

__global__ void __launch_bounds__(RED_THREADS)
    finalize_residual_kernel(const double *blk_res, const int *blk_bad, int n_blocks, double *out)
{
    // fixed order: strided per-thread sums over the blocks, then a tree
    double v[10];
    for (int t = 0; t < 10; t++) v[t] = 0.0;
    int bad = 0;
    for (int b = threadIdx.x; b < n_blocks; b += RED_THREADS) {
        for (int t = 0; t < 10; t++) v[t] += blk_res[(size_t)b * 10 + t];
        bad |= blk_bad[b];
    }
    __shared__ double sh[10][RED_THREADS];
    __shared__ int any_bad;
    if (threadIdx.x == 0) any_bad = 0;
    for (int t = 0; t < 10; t++) sh[t][threadIdx.x] = v[t];
    __syncthreads();
    if (bad) any_bad = 1;
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int t = 0; t < 10; t++) sh[t][threadIdx.x] += sh[t][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double dn[5], nn[5];
    for (int t = 0; t < 5; t++) {
        dn[t] = sh[t][0];
        nn[t] = sh[5 + t][0];
    }
    bad = any_bad;
    // Section 4.1 reading: largest relative L2 change over rho, rho U, rho E;
    // denominators floored at 1e-8 ||rho||_2.
    double res = 0.0;
    const double fl = 1e-8 * sqrt(nn[0]);
    for (int t = 0; t < 5; t++) {
        double den = sqrt(nn[t]);
        if (den < fl) den = fl;
        const double r = sqrt(dn[t]) / den;
        if (r > res) res = r;
    }
    out[0] = res;
    out[1] = bad ? 1.0 : 0.0;
}

// rho_w^0 from the flux of f^{S,0} through each wall face (Eq. (9) with the
// initial state).  On the tensor-product grid the Maxwellian factorises by
// axis and the Shakhov factor is a cubic polynomial in c, so the flux is a sum
// of products of 1D sums S_e^a = sum_i w_i c_i^a exp(-c_i^2 / (2RT)), a = 0..3,
// along the two tangential axes and of the half-range sums with the extra
// factor |xi_n| (only velocities pointing into the wall) along the normal
// axis.  One warp per (side, cell) face; the lanes split the nodes of each
// axis and the warp sums them in a fixed order.
__global__ void __launch_bounds__(128) wall_flux_init_kernel(const double *mac, const int8_t *wall_kind,
                                                             const double *wall_norm, const double *axis64, int nvx,
                                                             int nvy, int nvz, size_t ncell, double R, double Pr,
                                                             double *rho_w)
{
    const size_t idx = (size_t)blockIdx.x * 4 + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (idx >= 6 * ncell) return;
    const int s = (int)(idx / ncell);
    const size_t c = idx % ncell;
    const int kind = wall_kind[idx];
    if (kind < 0) {
        if (lane == 0) rho_w[idx] = 0.0;
        return;
    }
    const double rho = mac[c], T = mac[4 * ncell + c];
    const double U[3] = {mac[ncell + c], mac[2 * ncell + c], mac[3 * ncell + c]};
    const double q[3] = {mac[5 * ncell + c], mac[6 * ncell + c], mac[7 * ncell + c]};
    const double RT = R * T, p = rho * RT;
    const double A = rho / pow(2.0 * M_PI * RT, 1.5);
    const int d = s / 2;
    const double nrm = (s % 2) ? -1.0 : 1.0;  // normal from the wall into the gas
    const int nv[3] = {nvx, nvy, nvz};
    const int off[3] = {0, nvx, nvx + nvy};
    const double *w = axis64 + nvx + nvy + nvz;
    double S[3][4];
    for (int e = 0; e < 3; e++) {
        double m[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = lane; i < nv[e]; i += 32) {
            const double x = axis64[off[e] + i], ce = x - U[e];
            double g = w[off[e] + i] * exp(-ce * ce / (2.0 * RT));
            if (e == d) g = (x * nrm < 0.0) ? g * (-x * nrm) : 0.0;
            m[0] += g;
            m[1] += g * ce;
            m[2] += g * ce * ce;
            m[3] += g * ce * ce * ce;
        }
        for (int a = 0; a < 4; a++) {
            for (int o = 16; o > 0; o >>= 1) m[a] += __shfl_xor_sync(0xffffffffu, m[a], o);
            S[e][a] = m[a];
        }
    }
    auto P = [&](int px, int py, int pz) { return S[0][px] * S[1][py] * S[2][pz]; };
    // sum over incoming velocities of w |xi_n| e (c.q) |c|^2 and of w |xi_n| e (c.q)
    const double cq3 = q[0] * (P(3, 0, 0) + P(1, 2, 0) + P(1, 0, 2)) + q[1] * (P(2, 1, 0) + P(0, 3, 0) + P(0, 1, 2)) +
                       q[2] * (P(2, 0, 1) + P(0, 2, 1) + P(0, 0, 3));
    const double cq1 = q[0] * P(1, 0, 0) + q[1] * P(0, 1, 0) + q[2] * P(0, 0, 1);
    const double k = (1.0 - Pr) / (5.0 * p * RT);
    const double F = A * (P(0, 0, 0) + k * (cq3 / RT - 5.0 * cq1));
    if (lane == 0) rho_w[idx] = F * wall_norm[kind * 6 + s];
}

__global__ void fill_kernel(double *p, size_t n, double v)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_coef(int precision, const double *mac, const uint8_t *solid, const uint8_t *side_flags,
                        const double *rdx, const double *rdy, const double *rdz, int nx, int ny, int nz,
                        double mu_ref, double omega, double Pr, void *coef, cudaStream_t s, int dev_src)
{
    const size_t n = (size_t)nx * ny * nz;
    if (precision == 0)
        coef_kernel<double><<<nblk(n, 256), 256, 0, s>>>(mac, solid, side_flags, rdx, rdy, rdz, nx, ny, nz, mu_ref,
                                                          omega, Pr, 0, static_cast<double *>(coef));
    else
        coef_kernel<float><<<nblk(n, 256), 256, 0, s>>>(mac, solid, side_flags, rdx, rdy, rdz, nx, ny, nz, mu_ref,
                                                         omega, Pr, dev_src, static_cast<float *>(coef));
    return cudaGetLastError();
}

cudaError_t launch_part_sums(const PartSumArgs &a, cudaStream_t s)
{
    const unsigned nb = (unsigned)close_blocks(a.ncell);
    if (a.precision == 0)
        part_sums_kernel<double><<<nb, CLOSE_CELLS * NPART, 0, s>>>(a);
    else
        part_sums_kernel<float><<<nb, CLOSE_CELLS * NPART, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_acc_sums(const AccSumArgs &a, cudaStream_t s)
{
    const unsigned nb = nblk((size_t)a.ncell, ACC_CELLS);
    if (a.precision == 0)
        acc_sums_kernel<double><<<nb, ACC_CELLS, 0, s>>>(a);
    else
        acc_sums_kernel<float><<<nb, ACC_CELLS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_closure(const ClosureArgs &a, cudaStream_t s)
{
    closure_kernel<<<(unsigned)close_blocks(a.ncell), CLOSE_CELLS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_finalize_mass(const double *blk_mass, int n_blocks, double M0, int rescale, double *scale,
                                 cudaStream_t s)
{
    finalize_mass_kernel<<<1, RED_THREADS, 0, s>>>(blk_mass, n_blocks, M0, rescale, scale);
    return cudaGetLastError();
}

cudaError_t launch_scale_residual(double *mac_new, double *rho_w_new, const double *mac, const uint8_t *solid,
                                  unsigned long long ncell, const double *scale, double *blk_res, int *blk_bad,
                                  int n_blocks, cudaStream_t s)
{
    scale_residual_kernel<<<n_blocks, RED_THREADS, 0, s>>>(mac_new, rho_w_new, mac, solid, ncell, scale, blk_res,
                                                           blk_bad);
    return cudaGetLastError();
}

cudaError_t launch_finalize_residual(const double *blk_res, const int *blk_bad, int n_blocks, double *out2,
                                     cudaStream_t s)
{
    finalize_residual_kernel<<<1, RED_THREADS, 0, s>>>(blk_res, blk_bad, n_blocks, out2);
    return cudaGetLastError();
}

cudaError_t launch_wall_flux_init(const double *mac, const int8_t *wall_kind, const double *wall_norm,
                                  const double *axis64, int nvx, int nvy, int nvz, unsigned long long ncell, double R,
                                  double Pr, double *rho_w, cudaStream_t s)
{
    wall_flux_init_kernel<<<nblk(6 * ncell, 4), 128, 0, s>>>(mac, wall_kind, wall_norm, axis64, nvx, nvy, nvz, ncell, R,
                                                              Pr, rho_w);
    return cudaGetLastError();
}

cudaError_t launch_fill(double *p, unsigned long long n, double v, cudaStream_t s)
{
    fill_kernel<<<nblk(n, 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

}  // namespace kgs
