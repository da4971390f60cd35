"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
moments of Maxwellians (Eqs. (2), (5)), the textbook hard-sphere viscosity
(Eq. (10) at omega = 1/2), a dense LU solve of the upwind system (Eq. (7))
and of its second-order variant, the convergence order of both on a
relaxation problem with a closed-form solution,
the rest state, mass conservation (Section 3.4), the cavity's mirror
symmetries (Section 4.1), and the free-molecular fixed point obtained by a
separate power iteration.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_1810_00348_gb300 import inputs
from tests import brute


def _fine_problem(**kw):
    # 52 nodes on [-8, 8] (h = 0.31): the trapezoid rule integrates Gaussians
    # of variance 0.3..0.8 to ~1e-15 and the cut tails are below 1e-15, so
    # these moments are exact up to rounding
    return inputs.cavity(2, 52, L_v=8.0, **kw)


# ---------------------------------------------------------------------------
# Eq. (2) and Eq. (5)

def test_units_of_the_maxwellian():
    """Velocity unit sqrt(2 R T0): f^M(1, 0, 1) = pi^{-3/2} exp(-|xi|^2)."""
    p = inputs.cavity(2, 5, L_v=2.0, Pr=1.0)
    o = Oracle(p)
    f = o.equilibrium([1.0, 0, 0, 0, 1.0, 0, 0, 0])
    xi, _ = brute.velocities(p)
    expect = math.pi ** -1.5 * np.exp(-np.sum(xi ** 2, axis=1))
    np.testing.assert_allclose(f, expect, rtol=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bgk_limit_is_the_maxwellian(seed):
    """Pr = 1 removes the Shakhov factor: f^S equals the textbook Maxwellian."""
    rng = np.random.default_rng(seed)
    p = inputs.cavity(2, 9, L_v=4.0, Pr=1.0)
    o = Oracle(p)
    rho, T = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
    U = rng.uniform(-0.5, 0.5, 3)
    q = rng.uniform(-0.2, 0.2, 3)
    f = o.equilibrium([rho, *U, T, *q])
    xi, _ = brute.velocities(p)
    np.testing.assert_allclose(f, brute.maxwellian(rho, U, T, xi), rtol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_quadrature_reproduces_maxwellian_moments(seed):
    """Eq. (5) on f^M recovers (rho, U, T) and q = 0 (closed form)."""
    rng = np.random.default_rng(seed)
    p = _fine_problem(Pr=1.0)
    o = Oracle(p)
    rho, T = rng.uniform(0.5, 2.0), rng.uniform(0.6, 1.6)
    U = rng.uniform(-0.4, 0.4, 3)
    m = o.moments(o.equilibrium([rho, *U, T, 0, 0, 0]))
    np.testing.assert_allclose(m[0], rho, rtol=1e-12)
    np.testing.assert_allclose(m[1:4], U, atol=1e-12)
    np.testing.assert_allclose(m[4], T, rtol=1e-11)
    np.testing.assert_allclose(m[5:8], 0.0, atol=2e-11)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_shakhov_moments(seed):
    """The Shakhov correction leaves rho, U, T unchanged and gives
    q(f^S) = (1 - Pr) q (the design property of Eq. (2))."""
    rng = np.random.default_rng(seed)
    Pr = 2.0 / 3.0
    p = _fine_problem(Pr=Pr)
    o = Oracle(p)
    rho, T = rng.uniform(0.5, 2.0), rng.uniform(0.7, 1.4)
    U = rng.uniform(-0.3, 0.3, 3)
    q = rng.uniform(-0.05, 0.05, 3)
    m = o.moments(o.equilibrium([rho, *U, T, *q]))
    np.testing.assert_allclose(m[0], rho, rtol=1e-12)
    np.testing.assert_allclose(m[1:4], U, atol=1e-12)
    np.testing.assert_allclose(m[4], T, rtol=1e-11)
    np.testing.assert_allclose(m[5:8], (1.0 - Pr) * q, atol=2e-11)


def test_coarse_grid_quadrature_error_scale():
    """12 nodes on [-4, 4] (the small cavity's grid): the density of the
    discrete unit Maxwellian differs from 1 by the trapezoid error, which is
    below 1e-6 but not zero."""
    p = inputs.cavity(2, 12, L_v=4.0, Pr=1.0)
    o = Oracle(p)
    m = o.moments(o.equilibrium([1.0, 0, 0, 0, 1.0, 0, 0, 0]))
    assert 1e-9 < abs(m[0] - 1.0) < 1e-6


# ---------------------------------------------------------------------------
# Eq. (10)

def test_mu_ref_reduces_to_hard_sphere_relation():
    """At omega = 1/2, Eq. (10) is the hard-sphere mean free path relation
    lambda = (16/5) mu / (rho sqrt(2 pi R T)), i.e. mu = (5/16) rho lambda
    sqrt(2 pi R T) with rho = T = 1, R = 1/2, lambda = Kn."""
    for Kn in (0.1, 1.0, 3.0):
        p = inputs.cavity(2, 4, Kn=Kn, omega=0.5)
        o = Oracle(p)
        np.testing.assert_allclose(o.mu_ref(), 5.0 / 16.0 * Kn * math.sqrt(2 * math.pi * 0.5), rtol=1e-14)


def test_mu_ref_argon():
    """omega = 0.81 (argon, Section 4): mu_ref = 15 sqrt(pi) (1/2) Kn / ((5-2w)(7-2w))."""
    p = inputs.cavity(2, 4, Kn=1.0, omega=0.81)
    np.testing.assert_allclose(Oracle(p).mu_ref(), 0.7310329, rtol=1e-6)


def _sheared_column(rho0, T0, Kn, shear):
    """A column of 32 cells across a unit gap in y whose cells are 1e6 wide in
    x and z (the side walls then reach the middle cells only through upwind
    weights of order 1e-7), with the lagged state rho0, T0, q = 0 and the
    weak shear U_x = shear (y - 1/2).  The walls at y = 0 and y = 1 move with
    the gas next to them, at T0."""
    ny = 32
    p = inputs.cavity([1, ny, 1], 28, L_v=6.5, Kn=Kn, T_w=T0)
    p.dx = np.array([1e6])
    p.dz = np.array([1e6])
    p.U_w[2] = [-0.5 * shear, 0.0, 0.0]
    p.U_w[3] = [0.5 * shear, 0.0, 0.0]
    y = (np.arange(ny) + 0.5) / ny
    mac = np.zeros((8, 1, ny, 1))
    mac[0] = rho0
    mac[4] = T0
    mac[1, 0, :, 0] = shear * (y - 0.5)
    return p, mac


@pytest.mark.parametrize("rho0,T0", [(1.0, 1.0), (2.0, 1.0), (1.0, 2.0), (0.5, 1.5)])
def test_relaxation_time_gives_the_viscosity(rho0, T0):
    """tau = mu / p with mu = mu_ref T^omega and p = rho R T (Section 2.1,
    Eq. (10)), checked through a consequence: the shear stress of a weakly
    sheared gas.  Away from the walls the first-order upwind solution of an
    equilibrium that is affine in y is exactly f = f^S - tau xi_y df^S/dy (the
    Chapman-Enskog solution: the upwind difference of an affine profile is
    its exact derivative), whose shear stress is P_xy = -p tau dU_x/dy.  So
    the swept field of the middle cells must carry the viscosity
    mu(T) = mu_ref T^omega: independent of the density (the classic kinetic
    theory result), growing as T^omega with the temperature.  mu_ref is pinned
    by the hard-sphere relation above."""
    shear, Kn = 0.02, 0.004
    p, mac = _sheared_column(rho0, T0, Kn, shear)
    o = Oracle(p, mac)
    xi, w = brute.velocities(p)
    ny = p.ny
    f = np.array([o.sweep(a).reshape(-1) for a in range(p.nvel)])  # [nvel][ny]
    for j in (ny // 2 - 1, ny // 2):
        U = mac[1:4, 0, j, 0]
        c = xi - U[None, :]
        Pxy = np.sum(w * c[:, 0] * c[:, 1] * f[:, j])
        mu = o.mu_ref() * T0 ** p.omega
        assert abs(-Pxy / (mu * shear) - 1.0) < 1e-5, (rho0, T0, -Pxy / shear, mu)


# ---------------------------------------------------------------------------
# Section 3.4 boundary values

def test_wall_and_inflow_ghosts():
    """Eq. (8) with the wall velocity: ghost = rho_w f^M(1, U_w, T_w);
    free-stream face: ghost = f^M(rho_inf, U_inf, T_inf)."""
    p = inputs.cavity(3, 5, L_v=3.0, lid=0.3)
    p.T_w = [1.0, 1.2, 0.9, 1.1, 1.0, 0.8]
    p.face_type[4] = inputs.FACE_INFLOW
    p.rho_in, p.U_in, p.T_in = 0.7, [0.2, -0.1, 0.3], 1.3
    o = Oracle(p)
    rw = inputs.random_rho_w(p, 3)
    o.set_rho_w(rw)
    rw = rw.reshape(6, -1)
    xi, _ = brute.velocities(p)
    c = brute.cell_index(p, 1, 2, 0)  # on the +y lid and the -z inflow side
    for a in (0, 17, 60, 124):
        np.testing.assert_allclose(o.ghost(c, 3, a), rw[3, c] * brute.maxwellian(1.0, [0.3, 0, 0], 1.1, xi[a]),
                                   rtol=1e-14)
        np.testing.assert_allclose(o.ghost(c, 4, a), brute.maxwellian(0.7, [0.2, -0.1, 0.3], 1.3, xi[a]),
                                   rtol=1e-14)
        assert o.ghost(c, 0, a) == 0.0  # interior face


def test_discrete_wall_density_at_rest_is_one():
    """A gas at rest at the wall temperature: the discrete normalisation of
    Eq. (9) gives rho_w = 1 exactly (symmetric velocity grid)."""
    p = inputs.cavity(3, 8, L_v=4.0, lid=0.0)
    rw = Oracle(p).rho_w()
    wall = rw != 0.0
    np.testing.assert_allclose(rw[wall], 1.0, rtol=1e-14)
    assert wall.sum() == 6 * 9


def test_analytic_wall_density_converges_second_order():
    """Printed Eq. (9) (analytic normalisation) at rest: rho_w -> 1 as the
    velocity grid is refined, with the O(h^2) error of the trapezoid rule on
    the half-range flux (the kink of |xi_n| at 0)."""
    errs = []
    for n in (16, 32, 64):
        p = inputs.cavity(1, [n, 40, 40], L_v=6.0, lid=0.0, wall_mode=inputs.WALL_ANALYTIC)
        rw = Oracle(p).rho_w()
        errs.append(abs(rw[0, 0, 0, 0] - 1.0))
    assert errs[0] > errs[1] > errs[2]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5


# ---------------------------------------------------------------------------
# Eq. (7): the sweep against a dense solve

def _rtau(o, p, mac):
    """1/tau = p/mu with mu = mu_ref T^omega (Sections 2.1 and 4); mu_ref is
    pinned by test_mu_ref_reduces_to_hard_sphere_relation."""
    rho, T = mac[0].reshape(-1), mac[4].reshape(-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = rho * 0.5 * T / (o.mu_ref() * T ** p.omega)
    return np.nan_to_num(r)


@pytest.mark.parametrize("case", ["cube3", "ragged_nonuniform", "solid"])
def test_sweep_matches_dense_solve(case):
    if case == "cube3":
        p = inputs.cavity(3, 5, L_v=3.0, lid=0.2, Kn=0.3)
    elif case == "ragged_nonuniform":
        p = inputs.cavity([4, 2, 3], [4, 5, 6], L_v=3.0, lid=0.2, Kn=0.7)
        p.dx = np.array([0.1, 0.3, 0.2, 0.4])
        p.dy = np.array([0.6, 0.4])
        p.dz = np.array([0.25, 0.5, 0.25])
    else:
        p = inputs.cavity([4, 3, 3], 5, L_v=3.0, lid=0.2, Kn=0.5)
        p.solid = np.zeros((3, 3, 4), np.uint8)
        p.solid[1, 1, 1] = 1
        p.solid[2, 0, 3] = 1
    mac = inputs.random_macros(p, 11)
    o = Oracle(p, mac)
    o.set_rho_w(inputs.random_rho_w(p, 12))
    xi, _ = brute.velocities(p)
    rtau = _rtau(o, p, mac)
    m = mac.reshape(8, -1)
    nc = p.ncell
    for a in range(p.nvel):
        fS = np.array([o.equilibrium(m[:, c])[a] if rtau[c] > 0 else 0.0 for c in range(nc)])
        f_ref = brute.dense_upwind_solve(p, xi[a], rtau, fS, lambda c, face: o.ghost(c, face, a))
        f = o.sweep(a).reshape(-1)
        np.testing.assert_allclose(f, f_ref, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("case", ["cube4", "ragged", "solid"])
def test_second_order_sweep_matches_dense_solve(case):
    """The order-2 sweep (three-point upwind differences, Section 6's next
    step) equals an LU solve of the same system assembled row by row."""
    if case == "cube4":
        p = inputs.cavity(4, 5, L_v=3.0, lid=0.2, Kn=0.3)
    elif case == "ragged":
        p = inputs.cavity([5, 2, 4], [4, 5, 6], L_v=3.0, lid=0.2, Kn=0.7)
        p.dx = np.full(5, 0.3)
        p.dy = np.full(2, 0.45)
        p.dz = np.full(4, 0.2)
    else:
        p = inputs.cavity([5, 4, 3], 5, L_v=3.0, lid=0.2, Kn=0.5)
        p.solid = np.zeros((3, 4, 5), np.uint8)
        p.solid[1, 1, 2] = 1
        p.solid[2, 0, 4] = 1
    p.order = 2
    mac = inputs.random_macros(p, 21)
    o = Oracle(p, mac)
    o.set_rho_w(inputs.random_rho_w(p, 22))
    xi, _ = brute.velocities(p)
    rtau = _rtau(o, p, mac)
    m = mac.reshape(8, -1)
    nc = p.ncell
    for a in range(p.nvel):
        fS = np.array([o.equilibrium(m[:, c])[a] if rtau[c] > 0 else 0.0 for c in range(nc)])
        f_ref = brute.dense_upwind2_solve(p, xi[a], rtau, fS, lambda c, face: o.ghost(c, face, a))
        f = o.sweep(a).reshape(-1)
        np.testing.assert_allclose(f, f_ref, rtol=1e-12, atol=1e-15)


def _relaxation_column(n, order):
    """One velocity (1.5, 0, 0) crossing n cells of width 1/n from a free
    stream (rho 2, T 1.2) into gas in uniform equilibrium (rho 1, T 1)."""
    p = inputs.cavity([n, 1, 1], 5, L_v=3.0, lid=0.0, Kn=0.5)
    p.face_type = [inputs.FACE_INFLOW] * 6
    p.rho_in, p.T_in, p.U_in = 2.0, 1.2, [0.0, 0.0, 0.0]
    p.order = order
    mac = np.zeros((8, 1, 1, n))
    mac[0], mac[4] = 1.0, 1.0
    return p, Oracle(p, mac)


@pytest.mark.parametrize("order,lo,hi", [(1, 1.8, 2.2), (2, 3.4, 4.6)])
def test_sweep_converges_at_its_order(order, lo, hi):
    """xi f' = (S - f)/tau with S and tau uniform has the solution
    f = S + (g - S) exp(-(x - x_g)/(xi tau)); the ghost g enters as the value
    one cell upwind of the first cell (x_g = -dx/2).  Halving dx halves the
    first-order error and quarters the second-order one."""
    xi = np.array([1.5, 0.0, 0.0])
    errs = []
    for n in (32, 64, 128):
        p, o = _relaxation_column(n, order)
        v, _ = brute.velocities(p)
        a = int(np.flatnonzero((v == xi).all(axis=1))[0])
        S = brute.maxwellian(1.0, [0, 0, 0], 1.0, xi)
        g = brute.maxwellian(2.0, [0, 0, 0], 1.2, xi)
        tau = o.mu_ref() / 0.5  # mu / (rho R T) at rho = T = 1
        x = (np.arange(n) + 0.5) / n
        exact = S + (g - S) * np.exp(-(x + 0.5 / n) / (xi[0] * tau))
        errs.append(np.abs(o.sweep(a).reshape(-1) - exact).max() / abs(g - S))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert lo < r1 < hi and lo < r2 < hi, (errs, r1, r2)


def test_sweep_is_a_convex_combination():
    """Maximum principle of the implicit upwind update: each f lies between
    the smallest and largest of the ghosts and f^S values it mixes."""
    p = inputs.cavity(5, 6, L_v=3.0, lid=0.2, Kn=0.2)
    mac = inputs.random_macros(p, 5)
    o = Oracle(p, mac)
    m = mac.reshape(8, -1)
    for a in (0, 100, 215):
        fS = np.array([o.equilibrium(m[:, c])[a] for c in range(p.ncell)])
        g = [o.ghost(c, face, a) for c in range(p.ncell) for face in range(6) if brute.neighbour(p, c, face) < 0]
        lo, hi = min(fS.min(), min(g)), max(fS.max(), max(g))
        f = o.sweep(a)
        assert f.min() >= lo * (1 - 1e-14) and f.max() <= hi * (1 + 1e-14)


# ---------------------------------------------------------------------------
# whole iterations: invariants

@pytest.mark.parametrize("order", [1, 2])
def test_rest_state_stays_at_rest(order):
    """Gas at rest between walls at its own temperature stays at rest to
    1e-12 (24 nodes on [-6, 6], discrete walls), for either upwind order."""
    p = inputs.cavity(4, 24, L_v=6.0, lid=0.0, Kn=0.5)
    p.order = order
    o = Oracle(p)
    o.iterate(6)
    m = o.macros()
    assert np.abs(m[0] - 1).max() < 1e-12
    assert np.abs(m[4] - 1).max() < 1e-12
    assert np.abs(m[1:4]).max() < 1e-12
    assert np.abs(m[5:8]).max() < 1e-12


def test_rest_state_drift_is_quadrature_error_on_coarse_grid():
    p = inputs.cavity(4, 12, L_v=4.0, lid=0.0, Kn=1.0)
    o = Oracle(p)
    o.iterate(4)
    m = o.macros()
    assert np.abs(m[4] - 1).max() < 5e-6
    # the quadrature error varies near walls and drives flows of its own size
    assert np.abs(m[1:4]).max() < 1e-6


def test_mass_rescale_keeps_total_mass():
    p = inputs.cavity(4, 8, L_v=4.0, lid=0.3, Kn=0.5, wall_mode=inputs.WALL_ANALYTIC)
    o = Oracle(p)
    M0 = o.total_mass()
    for _ in range(3):
        o.iterate()
        np.testing.assert_allclose(o.total_mass(), M0, rtol=1e-14)


def test_mass_without_rescale_conserved_at_convergence():
    """Discrete walls, no rescaling: the upwind scheme is conservative and the
    discrete wall flux is balanced, so the mass change per iteration falls
    to the quadrature error of the equilibrium's density (~1e-14 with 26
    nodes on [-6, 6]) as the iteration converges."""
    p = inputs.cavity(3, 26, L_v=6.0, lid=0.2, Kn=2.0, mass_rescale=0)
    o = Oracle(p)
    drift = []
    res = 1.0
    for _ in range(60):
        M = o.total_mass()
        res = o.iterate()
        drift.append(abs(o.total_mass() - M))
        if res < 1e-11:
            break
    assert res < 1e-11
    assert drift[-1] < 1e-13
    assert drift[-1] < 1e-9 * max(drift[:3])


def test_cavity_mirror_symmetry():
    """Lid on the +y face moving along +x: the z -> 1-z mirror maps the field
    to itself (rho, T, Ux, Uy, qx, qy even; Uz, qz odd), every iteration."""
    p = inputs.cavity([4, 4, 5], 6, L_v=4.0, lid=0.3, Kn=0.5)
    o = Oracle(p)
    o.iterate(3)
    m = o.macros()
    mz = m[:, ::-1]
    for q, sign in zip(range(8), [1, 1, 1, -1, 1, 1, 1, -1]):
        np.testing.assert_allclose(mz[q], sign * m[q], atol=1e-13)


def test_lid_reversal_is_the_x_mirror():
    p1 = inputs.cavity([4, 3, 3], 6, L_v=4.0, lid=0.3, Kn=0.5)
    p2 = inputs.cavity([4, 3, 3], 6, L_v=4.0, lid=-0.3, Kn=0.5)
    o1, o2 = Oracle(p1), Oracle(p2)
    o1.iterate(2)
    o2.iterate(2)
    m1, m2 = o1.macros(), o2.macros()[:, :, :, ::-1]
    for q, sign in zip(range(8), [1, -1, 1, 1, 1, -1, 1, 1]):
        np.testing.assert_allclose(m2[q], sign * m1[q], atol=1e-13)


# ---------------------------------------------------------------------------
# free-molecular limit: a separately solved linear fixed point

def _free_molecular_fixed_point(p):
    """Kn = inf: every f is a fixed mix of wall ghosts, so the wall densities
    obey a linear map rho_w -> F_in(rho_w)/D with D the discrete outgoing flux
    of each unit wall Maxwellian (Eq. (9), discrete normalisation).  Build the
    map column by column with dense solves, then run the power iteration
    with the mass normalisation of Section 3.4."""
    xi, w = brute.velocities(p)
    nc = p.ncell
    faces = [(c, f) for c in range(nc) for f in range(6) if brute.neighbour(p, c, f) == -1]
    idx = {cf: n for n, cf in enumerate(faces)}
    wallU = [np.array(u) for u in p.U_w]
    nf = len(faces)
    # ghost_unit[a, n]: unit-density emission of wall face n for velocity a
    A = np.zeros((nf, nf))   # F_in[m] = sum_n A[m, n] rho_w[n]
    fields = np.zeros((nf, len(w), nc))  # f per unit rho_w of face n
    for n, (c0, f0) in enumerate(faces):
        for a in range(len(w)):
            def ghost(c, face):
                return brute.maxwellian(1.0, wallU[face], p.T_w[face], xi[a]) if (c, face) == (c0, f0) else 0.0
            fields[n, a] = brute.dense_upwind_solve(p, xi[a], np.zeros(nc), np.zeros(nc), ghost)
    for m_, (c, f) in enumerate(faces):
        d = f // 2
        nrm = 1.0 if f % 2 == 0 else -1.0
        xn = xi[:, d] * nrm
        inc = xn < 0
        A[m_] = np.einsum("a,na->n", (w * -xn)[inc], fields[:, inc, c])
    D = np.zeros(nf)
    for m_, (c, f) in enumerate(faces):
        d = f // 2
        nrm = 1.0 if f % 2 == 0 else -1.0
        xn = xi[:, d] * nrm
        out = xn > 0
        D[m_] = np.sum(w[out] * xn[out] * brute.maxwellian(1.0, wallU[f], p.T_w[f], xi[out]))
    vol = np.multiply.outer(np.multiply.outer(p.dz, p.dy), p.dx).reshape(-1)
    rw = np.ones(nf)  # the rest equilibrium emits with rho_w = 1 at step 0
    for _ in range(5000):
        # density of the field swept with the current rho_w, and the rescale
        # factor that brings its mass back to M0 = 1 (uniform rho = 1 start)
        rho_cur = np.einsum("n,a,nac->c", rw, w, fields)
        s = np.sum(vol) / np.sum(rho_cur * vol)
        new = s * (A @ rw) / D
        done = np.abs(new - rw).max() < 1e-15
        rw = new
        if done:
            break
    rho = np.einsum("n,a,nac->c", rw, w, fields)
    return faces, rw, rho


@pytest.mark.parametrize("n", [1, 2])
def test_free_molecular_limit(n):
    p = inputs.cavity(n, 6, L_v=3.0, lid=0.4, Kn=math.inf)
    p.T_w = [1.0, 1.3, 1.0, 0.9, 1.1, 1.0]
    faces, rw_ref, rho_ref = _free_molecular_fixed_point(p)
    o = Oracle(p)
    for _ in range(400):
        res = o.iterate()
        if res < 1e-14:
            break
    rw = o.rho_w().reshape(6, -1)
    got = np.array([rw[f, c] for c, f in faces])
    np.testing.assert_allclose(got, rw_ref, rtol=1e-12)
    np.testing.assert_allclose(o.macros()[0].reshape(-1), rho_ref, rtol=1e-12)


# ---------------------------------------------------------------------------
# the outer iteration assembles Eq. (5) from the sweeps of Eq. (7)

def test_iteration_moments_are_eq5_of_the_swept_field():
    """One outer iteration (Eq. (6)) gives, at every cell, the Eq. (5)
    moments of the distribution obtained by sweeping each velocity with the
    step-n state; the moments function is pinned by the closed-form tests."""
    p = inputs.cavity([3, 4, 3], 7, L_v=3.5, lid=0.25, Kn=0.4, mass_rescale=0)
    mac = inputs.random_macros(p, 21)
    o = Oracle(p, mac)
    o.set_rho_w(inputs.random_rho_w(p, 22))
    F = np.stack([o.sweep(a).reshape(-1) for a in range(p.nvel)])  # [nvel, ncell]
    o.iterate()
    new = o.macros().reshape(8, -1)
    for c in range(p.ncell):
        np.testing.assert_allclose(new[:, c], o.moments(F[:, c]), rtol=1e-12, atol=1e-14)


def test_mass_rescale_scales_rho_q_and_wall_density_only():
    """Section 3.4 rescaling, read as scaling f: after one iteration from the
    same state, rescaling multiplies rho, q and rho_w by M0/M and leaves U, T."""
    mac = None
    out = {}
    for flag in (0, 1):
        p = inputs.cavity([3, 3, 4], 6, L_v=3.5, lid=0.3, Kn=0.3, mass_rescale=flag,
                          wall_mode=inputs.WALL_ANALYTIC)
        if mac is None:
            mac = inputs.random_macros(p, 31)
        o = Oracle(p, mac)
        M0 = o.total_mass()
        o.iterate()
        out[flag] = (o.macros(), o.rho_w(), M0)
    (m0, rw0, M0), (m1, rw1, _) = out[0], out[1]
    vol = (1.0 / 3) * (1.0 / 3) * (1.0 / 4)
    s = M0 / (m0[0].sum() * vol)
    assert abs(s - 1.0) > 1e-4  # the case does exercise the rescale
    np.testing.assert_allclose(m1[0], s * m0[0], rtol=1e-13)
    np.testing.assert_allclose(m1[5:8], s * m0[5:8], rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(m1[1:5], m0[1:5], rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(rw1, s * rw0, rtol=1e-13)


def test_concurrent_velocity_ranges_match_the_serial_loop():
    # the optional concurrent ranges change only the order in which the
    # per-velocity contributions are added
    from tests.parity import field_errors
    p = inputs.cavity([9, 7, 10], 12, Kn=0.5, lid=0.2)
    mac = inputs.random_macros(p, 5)
    serial, ranged = Oracle(p, mac), Oracle(p, mac, threads=4)
    serial.iterate(2)
    ranged.iterate(2)
    err = field_errors(ranged.macros(), serial.macros())
    assert max(err.values()) < 1e-12, err
    assert np.max(np.abs(ranged.rho_w() - serial.rho_w())) < 1e-12


# ---------------------------------------------------------------------------
# Algorithm 3's heat flux about the lagged velocity (option)

def test_lagged_heat_flux_is_the_moment_about_the_old_velocity():
    """With q_lagged the heat flux of step n+1 is 1/2 sum w (xi - U^n)
    |xi - U^n|^2 f^{n+1}, the lagged U^n of the input state (Algorithm 3
    accumulates its moments in one pass, before the new U is known); rho, U
    and T are those of the exact form.  The reference sums the oracle's swept
    distribution with numpy."""
    p = inputs.cavity([4, 3, 5], [6, 5, 7], L_v=3.5, lid=0.2, Kn=0.4, mass_rescale=0)
    mac = inputs.random_macros(p, 71)
    exact = Oracle(p, mac)
    p.q_lagged = 1
    lag = Oracle(p, mac)
    xi, w = brute.velocities(p)
    f = np.array([lag.sweep(a).reshape(-1) for a in range(p.nvel)])  # [nvel][ncell]
    exact.iterate()
    lag.iterate()
    m_e, m_l = exact.macros().reshape(8, -1), lag.macros().reshape(8, -1)
    np.testing.assert_allclose(m_l[:5], m_e[:5], rtol=1e-13, atol=1e-15)
    U = mac.reshape(8, -1)[1:4]
    c = xi[:, :, None] - U[None, :, :]  # [nvel][3][ncell]
    c2 = np.sum(c * c, axis=1)
    q_ref = 0.5 * np.einsum("a,adc,ac,ac->dc", w, c, c2, f)
    np.testing.assert_allclose(m_l[5:8], q_ref, rtol=1e-12, atol=1e-14)
    assert np.max(np.abs(m_l[5:8] - m_e[5:8])) > 1e-6  # the two forms differ away from the fixed point


def test_lagged_heat_flux_has_the_same_fixed_point():
    """At the fixed point U^{n+1} = U^n, so both heat-flux forms converge to
    the same fields."""
    out = []
    for lagged in (0, 1):
        p = inputs.cavity(4, 8, L_v=4.0, lid=0.2, Kn=0.5)
        p.q_lagged = lagged
        o = Oracle(p)
        for _ in range(400):
            if o.iterate() < 1e-13:
                break
        out.append(o.macros())
    np.testing.assert_allclose(out[1], out[0], rtol=0, atol=1e-11)
