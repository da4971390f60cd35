// kgs_sweep.cu -- the fused equilibrium + upwind implicit sweep + moment
// kernel of one outer iteration (arXiv 1810.00348, Eqs. (2), (5), (7), (9)).
//
// Work decomposition.  The physical grid is cut into blocks of BX x BY x bz
// cells.  For the velocities of octant o (signs of xi_x, xi_y, xi_z) a block
// depends only on its three upwind neighbour blocks, so the blocks are swept
// in diagonal stages (block coordinates reflected so that the sweep runs
// towards +x, +y, +z): stage s holds every block whose reflected coordinates
// sum to s, for all eight octants at once.  One launch per stage; one CTA per
// (octant, block, group of vg_size velocities of that octant).  Velocities
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
// Each update is the pointwise solution of Eq. (7):
//     f = (f^S/tau + sum_d a_d f_up,d) / (1/tau + sum_d a_d),  a_d = |xi_d|/dx_d,
// with the Shakhov equilibrium f^S of Eq. (2) computed on the fly from the
// lagged coefficients of the cell.  After each slice the threads switch to a
// cell-per-thread layout and sum the slice's moments over the group's
// velocities (the 13 sums about the lagged velocity U^n and the incoming
// wall fluxes of Eq. (9)); the per-(group, cell) partials go to global
// memory in FP64 and a fixed-order reduction closes the iteration (no
// atomics).  Block faces between stages go through three face planes in
// global memory indexed by the cell position on the face: a block reads the
// plane entries written by its upwind neighbour in the previous stage before
// overwriting them with its own outflow.
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

// exp of the scaled exponent: FP64 uses exp(), FP32 the hardware 2^x with the
// log2(e) factor already folded into the coefficient C_NEXP.
__device__ __forceinline__ double eq_exp(double x) { return exp(x); }
__device__ __forceinline__ float eq_exp(float x) { return ex2_approx(x); }
__device__ __forceinline__ double implicit_div(double num, double den) { return num / den; }
__device__ __forceinline__ float implicit_div(float num, float den) { return num * rcp_approx(den); }

__host__ __device__ constexpr size_t align16(size_t n) { return (n + 15) & ~size_t(15); }

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

template <typename Real, int TV>
struct SmemLayout {
    static constexpr int VG = NT * TV;
    static constexpr int CS = VG + 1;  // odd cell stride: conflict-free per-cell reads
    static constexpr size_t slice_bytes = align16(sizeof(Real) * (BY + 1) * (BX + 1) * CS);
    static constexpr size_t coef_bytes = align16(sizeof(Real) * SLICE * NCOEF);
    static constexpr size_t vel_bytes = align16(sizeof(Real) * VG * 8);
    static constexpr size_t red_bytes = sizeof(double) * NPART * SLICE;
    static constexpr size_t total = slice_bytes + coef_bytes + vel_bytes + red_bytes;
};

template <typename Real, int TV>
__global__ void __launch_bounds__(NT) sweep_kernel(const SweepArgs a)
{
    using L = SmemLayout<Real, TV>;
    constexpr int VG = L::VG;
    constexpr int CS = L::CS;
    extern __shared__ __align__(16) unsigned char smem[];
    Real *slice = reinterpret_cast<Real *>(smem);
    Real *cs = reinterpret_cast<Real *>(smem + L::slice_bytes);
    Real *vs = reinterpret_cast<Real *>(smem + L::slice_bytes + L::coef_bytes);
    double *mred = reinterpret_cast<double *>(smem + L::slice_bytes + L::coef_bytes + L::vel_bytes);

    const int t = threadIdx.x;
    const int4 w = a.work[blockIdx.x];
    const int o = w.x;
    const int vcount = a.oct_vcount[o];
    const int v0 = blockIdx.y * VG;
    if (v0 >= vcount) return;
    const int nvg = min(VG, vcount - v0);
    const int gvbase = a.oct_vstart[o] + v0;
    const int vgid = a.oct_vgbase[o] + blockIdx.y;

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
    const int sidex = px ? 0 : 1, sidey = py ? 2 : 3, sidez = pz ? 4 : 5;      // upwind sides
    const int headx = px ? 1 : 0, heady = py ? 3 : 2, headz = pz ? 5 : 4;      // downwind sides
    const int nx = a.nx, ny = a.ny;
    const size_t ncell = a.ncell;
    const size_t Nv = (size_t)a.Nv;

    auto GX = [&](int li) { return px ? x0 + li : x0 + ex - 1 - li; };
    auto GY = [&](int lj) { return py ? y0 + lj : y0 + ey - 1 - lj; };
    auto GZ = [&](int lk) { return pz ? z0 + lk : z0 + ez - 1 - lk; };
    auto SL = [&](int li, int lj) { return ((lj + 1) * (BX + 1) + (li + 1)) * CS; };  // li, lj may be -1

    const Real *vel = static_cast<const Real *>(a.vel);
    const Real *mt = static_cast<const Real *>(a.mtab);
    const Real *coef = static_cast<const Real *>(a.coef);
    Real *FXp = static_cast<Real *>(a.FX);
    Real *FYp = static_cast<Real *>(a.FY);
    Real *FZp = static_cast<Real *>(a.FZ);

    // Per-thread velocities: vl = t + m*NT.
    const Real *velw = static_cast<const Real *>(a.velw);
    const int nxo = a.oct_nx[o];
    Real xi[TV][3], mgx[TV], mgy[TV], mgz[TV], msol[TV];
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
        Real w4[4];
#pragma unroll
        for (int q = 0; q < 4; q++) w4[q] = vel[gv[m] * 4 + q];
        xi[m][0] = w4[0];
        xi[m][1] = w4[1];
        xi[m][2] = w4[2];
        // moment-phase table: xi_x, w_x, x-line end flag, -, xi_y, xi_z, w_y w_z, -
        Real *vt = vs + vl * 8;
        vt[0] = w4[0];
        vt[1] = ok[m] ? velw[gv[m] * 2 + 0] : Real(0);
        vt[2] = ((v0 + vl) % nxo == nxo - 1) ? Real(1) : Real(0);
        vt[3] = Real(0);
        vt[4] = w4[1];
        vt[5] = w4[2];
        vt[6] = ok[m] ? velw[gv[m] * 2 + 1] : Real(0);
        vt[7] = Real(0);
        mgx[m] = mt[(size_t)rowx * Nv + gv[m]];
        mgy[m] = mt[(size_t)rowy * Nv + gv[m]];
        mgz[m] = mt[(size_t)rowz * Nv + gv[m]];
        msol[m] = mt[(size_t)MT_SOLID * Nv + gv[m]];
    }

    // Ghost value entering through domain side `side` at cell `cell`:
    // free stream, or rho_w times the unit wall Maxwellian (Eq. (8)).
    auto wall_rho = [&](int side, size_t cell) -> Real {
        return a.side_inflow[side] ? Real(1) : Real(a.rho_w[side * ncell + cell]);
    };

    // z inflow of the block: the slice interior starts as slice k0-1.
    for (int cl = 0; cl < SLICE; cl++) {
        const int li = cl % BX, lj = cl / BX;
        if (li >= ex || lj >= ey) continue;
        const int x = GX(li), y = GY(lj), z = GZ(0);
        const size_t cell = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z);
        const Real rw = zfirst ? wall_rho(sidez, cell) : Real(0);
#pragma unroll
        for (int m = 0; m < TV; m++) {
            if (!ok[m]) continue;
            Real v = zfirst ? rw * mgz[m] : FZp[((size_t)y * nx + x) * Nv + gv[m]];
            slice[SL(li, lj) + t + m * NT] = v;
        }
    }

    for (int lk = 0; lk < ez; lk++) {
        const int z = GZ(lk);
        __syncthreads();  // the previous slice's moment phase is done with smem
        // coefficients of the slice's cells (invalid cells flagged solid)
        for (int idx = t; idx < SLICE * NCOEF; idx += NT) {
            const int cl = idx / NCOEF, q = idx % NCOEF;
            const int li = cl % BX, lj = cl / BX;
            Real v;
            if (li < ex && lj < ey) {
                const size_t cell = (size_t)GX(li) + (size_t)nx * ((size_t)GY(lj) + (size_t)ny * z);
                v = coef[cell * NCOEF + q];
            } else {
                v = (q == C_FLAGS) ? Real(F_SOLID) : Real(0);
            }
            cs[idx] = v;
        }
        // halo column (x inflow) and halo row (y inflow) of this slice
        for (int lj = 0; lj < ey; lj++) {
            const int y = GY(lj), x = GX(0);
            const size_t cell = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z);
            const Real rw = xfirst ? wall_rho(sidex, cell) : Real(0);
#pragma unroll
            for (int m = 0; m < TV; m++) {
                if (!ok[m]) continue;
                Real v = xfirst ? rw * mgx[m] : FXp[((size_t)z * ny + y) * Nv + gv[m]];
                slice[SL(-1, lj) + t + m * NT] = v;
            }
        }
        for (int li = 0; li < ex; li++) {
            const int x = GX(li), y = GY(0);
            const size_t cell = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z);
            const Real rw = yfirst ? wall_rho(sidey, cell) : Real(0);
#pragma unroll
            for (int m = 0; m < TV; m++) {
                if (!ok[m]) continue;
                Real v = yfirst ? rw * mgy[m] : FYp[((size_t)z * nx + x) * Nv + gv[m]];
                slice[SL(li, -1) + t + m * NT] = v;
            }
        }
        __syncthreads();

        // ---- sweep of the slice: Eq. (2) fused into Eq. (7) ----
        for (int lj = 0; lj < ey; lj++) {
            const int y = GY(lj);
            Real fprev[TV];
#pragma unroll
            for (int m = 0; m < TV; m++) fprev[m] = slice[SL(-1, lj) + t + m * NT];
            for (int li = 0; li < ex; li++) {
                const Real *c = cs + (lj * BX + li) * NCOEF;
                const int flags = (int)c[C_FLAGS];
                if (flags & F_SOLID) continue;
                const Real ux = c[C_UX], uy = c[C_UY], uz = c[C_UZ];
                const Real kappa = c[C_KAPPA], nexp = c[C_NEXP], rt1 = c[C_RT1];
                const Real qx = c[C_QX], qy = c[C_QY], qz = c[C_QZ];
                const Real rtau = c[C_RTAU], rdx = c[C_RDX], rdy = c[C_RDY], rdz = c[C_RDZ];
                const int x = GX(li);
                const size_t cell = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z);
                const bool sol_x = flags & (F_SOLID_SIDE << sidex);
                const bool sol_y = flags & (F_SOLID_SIDE << sidey);
                const bool sol_z = flags & (F_SOLID_SIDE << sidez);
                Real rwx = 0, rwy = 0, rwz = 0;
                if (sol_x) rwx = Real(a.rho_w[sidex * ncell + cell]);
                if (sol_y) rwy = Real(a.rho_w[sidey * ncell + cell]);
                if (sol_z) rwz = Real(a.rho_w[sidez * ncell + cell]);
                const int sidx = SL(li, lj);
#pragma unroll
                for (int m = 0; m < TV; m++) {
                    const int vl = t + m * NT;
                    Real fz = slice[sidx + vl];
                    Real fy = slice[sidx - (BX + 1) * CS + vl];
                    Real fx = fprev[m];
                    if (sol_x) fx = rwx * msol[m];
                    if (sol_y) fy = rwy * msol[m];
                    if (sol_z) fz = rwz * msol[m];
                    const Real cx = xi[m][0] - ux, cy = xi[m][1] - uy, cz = xi[m][2] - uz;
                    const Real c2 = cx * cx + cy * cy + cz * cz;
                    const Real cq = cx * qx + cy * qy + cz * qz;
                    const Real E = eq_exp(c2 * nexp);
                    const Real src = kappa * E * (Real(1) + cq * (c2 * rt1 - Real(5)));
                    const Real ax = fabs(xi[m][0]) * rdx, ay = fabs(xi[m][1]) * rdy, az = fabs(xi[m][2]) * rdz;
                    const Real num = src + ax * fx + ay * fy + az * fz;
                    const Real den = rtau + ax + ay + az;
                    const Real f = implicit_div(num, den);
                    fprev[m] = f;
                    if (ok[m]) {
                        slice[sidx + vl] = f;
                        if (li == ex - 1 && !xlast) FXp[((size_t)z * ny + y) * Nv + gv[m]] = f;
                        if (lj == ey - 1 && !ylast) FYp[((size_t)z * nx + x) * Nv + gv[m]] = f;
                    }
                }
            }
        }
        __syncthreads();

        // ---- moments of the slice over the group's velocities ----
        // Thread (cell, half) sums its half of the group's velocities.  The
        // velocities come in x-lines of the tensor-product grid (ix fastest):
        // along a line only c_x changes, so the thread keeps the four line
        // sums P_a = sum w_x c_x^a f (a = 0..3) and, at the end of each line,
        // folds them with the line's c_y, c_z, w_y w_z into the 13 sums about
        // U^n and the three incoming wall fluxes (Eq. (5), Eq. (9)).
        {
            const int cl = t % SLICE, vp = t / SLICE;  // NT = 2 * SLICE: two velocity halves
            const int li = cl % BX, lj = cl / BX;
            const bool valid = li < ex && lj < ey;
            double acc[NPART];
#pragma unroll
            for (int q = 0; q < NPART; q++) acc[q] = 0.0;
            if (valid) {
                const Real *c = cs + cl * NCOEF;
                const int flags = (int)c[C_FLAGS];
                if (!(flags & F_SOLID)) {
                    const Real ux = c[C_UX], uy = c[C_UY], uz = c[C_UZ];
                    const bool wx = flags & (F_WALL_SIDE << headx);
                    const bool wy = flags & (F_WALL_SIDE << heady);
                    const bool wz = flags & (F_WALL_SIDE << headz);
                    const Real sgnx = px ? Real(1) : Real(-1);
                    RunSum<Real> S[NPART];
                    Real P0 = 0, P1 = 0, P2 = 0, P3 = 0;
                    const Real *sp = slice + SL(li, lj);
                    const int vbeg = vp * (VG / 2);
                    const int vend = min(vbeg + VG / 2, nvg);
                    for (int v = vbeg; v < vend; v++) {
                        const Real f = sp[v];
                        const Real *vt = vs + v * 8;
                        const Real cx = vt[0] - ux;
                        const Real t0 = vt[1] * f;
                        const Real t1 = t0 * cx;
                        const Real t2 = t1 * cx;
                        P0 += t0;
                        P1 += t1;
                        P2 += t2;
                        P3 += t2 * cx;
                        if (vt[2] != Real(0) || v == vend - 1) {  // end of an x-line (warp-uniform)
                            const Real cy = vt[4] - uy, cz = vt[5] - uz, W = vt[6];
                            const Real q0 = W * P0, q1 = W * P1, q2 = W * P2;
                            const Real r2 = cy * cy + cz * cz;
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
                            S[P_S3X].add(W * P3 + r2 * q1);
                            const Real e2 = q2 + r2 * q0;
                            S[P_S3Y].add(cy * e2);
                            S[P_S3Z].add(cz * e2);
                            // incoming flux w |xi_d| f towards the wall ahead
                            if (wx) S[P_FX].add(sgnx * (q1 + ux * q0));
                            if (wy) S[P_FY].add(fabs(vt[4]) * q0);
                            if (wz) S[P_FZ].add(fabs(vt[5]) * q0);
                            P0 = P1 = P2 = P3 = Real(0);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < NPART; q++) acc[q] = S[q].value();
                }
            }
            if (vp == 1) {
#pragma unroll
                for (int q = 0; q < NPART; q++) mred[q * SLICE + cl] = acc[q];
            }
            __syncthreads();
            if (vp == 0 && valid) {
                const size_t cell = (size_t)GX(li) + (size_t)nx * ((size_t)GY(lj) + (size_t)ny * z);
                double *pp = a.part + (size_t)vgid * NPART * ncell + cell;
#pragma unroll
                for (int q = 0; q < NPART; q++) pp[(size_t)q * ncell] = acc[q] + mred[q * SLICE + cl];
            }
        }
    }

    // z outflow of the block for the next stage
    if (!zlast) {
        __syncthreads();
        const int z = GZ(ez - 1);
        (void)z;
        for (int cl = 0; cl < SLICE; cl++) {
            const int li = cl % BX, lj = cl / BX;
            if (li >= ex || lj >= ey) continue;
            const int x = GX(li), y = GY(lj);
#pragma unroll
            for (int m = 0; m < TV; m++) {
                if (!ok[m]) continue;
                FZp[((size_t)y * nx + x) * Nv + gv[m]] = slice[SL(li, lj) + t + m * NT];
            }
        }
    }
}

template <typename Real, int TV>
cudaError_t launch_t(const SweepArgs &a, int n_items, int max_vg, cudaStream_t s)
{
    using L = SmemLayout<Real, TV>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<Real, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L::total);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid(n_items, max_vg);
    sweep_kernel<Real, TV><<<grid, NT, L::total, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t sweep_smem_bytes(int precision, int tv)
{
    if (precision == 0) return SmemLayout<double, 1>::total;
    return tv == 2 ? SmemLayout<float, 2>::total : SmemLayout<float, 1>::total;
}

cudaError_t launch_sweep(int precision, int tv, const SweepArgs &a, int n_items, int max_vg, cudaStream_t s)
{
    if (n_items == 0 || max_vg == 0) return cudaSuccess;
    if (precision == 0) return launch_t<double, 1>(a, n_items, max_vg, s);
    if (tv == 2) return launch_t<float, 2>(a, n_items, max_vg, s);
    return launch_t<float, 1>(a, n_items, max_vg, s);
}

}  // namespace kgs
