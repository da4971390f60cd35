"""Brute-force references used to pin the oracle (test code only).

They are deliberately built a different way from the oracle: the upwind
scheme of Eq. (7) is assembled as one sparse-as-dense linear system over all
fluid cells and solved with LU, instead of being swept cell by cell; the
Maxwellian is evaluated with numpy from its textbook form.
"""
import numpy as np

R = 0.5  # velocity unit sqrt(2 R T0)


def maxwellian(rho, U, T, xi):
    """Textbook Maxwellian rho (2 pi R T)^(-3/2) exp(-|xi-U|^2/(2 R T)); xi [..., 3]."""
    c2 = np.sum((np.asarray(xi) - np.asarray(U)) ** 2, axis=-1)
    return rho * (2 * np.pi * R * T) ** -1.5 * np.exp(-c2 / (2 * R * T))


def velocities(prob):
    """All discrete velocities [nvel, 3] and weights [nvel], index ix fastest."""
    X, Y, Z = np.meshgrid(prob.xi_x, prob.xi_y, prob.xi_z, indexing="ij")
    WX, WY, WZ = np.meshgrid(prob.w_x, prob.w_y, prob.w_z, indexing="ij")
    xi = np.stack([X, Y, Z], axis=-1).transpose(2, 1, 0, 3).reshape(-1, 3)
    w = (WX * WY * WZ).transpose(2, 1, 0).reshape(-1)
    return xi, w


def cell_index(prob, i, j, k):
    return i + prob.nx * (j + prob.ny * k)


def neighbour(prob, c, face):
    i = c % prob.nx
    j = (c // prob.nx) % prob.ny
    k = c // (prob.nx * prob.ny)
    ijk = [i, j, k]
    d, step = face // 2, (1 if face % 2 else -1)
    ijk[d] += step
    n = [prob.nx, prob.ny, prob.nz]
    if ijk[d] < 0 or ijk[d] >= n[d]:
        return -1
    nb = cell_index(prob, *ijk)
    if prob.solid is not None and prob.solid.reshape(-1)[nb]:
        return -2
    return nb


def dense_upwind_solve(prob, xi, rtau, fS, ghost):
    """Solve Eq. (7) for one velocity xi as a linear system over fluid cells.

    rtau[c]: 1/tau; fS[c]: equilibrium; ghost(c, face): boundary value.
    Row c:  (1/tau_c + sum_d a_d) f_c - sum_{d interior} a_d f_up(c,d)
            = fS_c/tau_c + sum_{d boundary} a_d ghost(c, d)
    with a_d = |xi_d| / width_d(c) and the upwind side fixed by sign(xi_d).
    """
    nc = prob.nx * prob.ny * prob.nz
    widths = [prob.dx, prob.dy, prob.dz]
    solid = np.zeros(nc, bool) if prob.solid is None else prob.solid.reshape(-1).astype(bool)
    A = np.zeros((nc, nc))
    b = np.zeros(nc)
    for c in range(nc):
        if solid[c]:
            A[c, c] = 1.0
            continue
        ijk = [c % prob.nx, (c // prob.nx) % prob.ny, c // (prob.nx * prob.ny)]
        A[c, c] += rtau[c]
        b[c] += rtau[c] * fS[c]
        for d in range(3):
            if xi[d] == 0.0:
                continue
            a = abs(xi[d]) / widths[d][ijk[d]]
            face = 2 * d + (0 if xi[d] > 0 else 1)
            A[c, c] += a
            nb = neighbour(prob, c, face)
            if nb >= 0:
                A[c, nb] -= a
            else:
                b[c] += a * ghost(c, face)
    f = np.linalg.solve(A, b)
    f[solid] = 0.0
    return f


def dense_upwind2_solve(prob, xi, rtau, fS, ghost):
    """The second-order upwind system for one velocity xi, assembled over all
    fluid cells and solved with LU.  Along an axis with both upwind
    neighbours fluid, the derivative is the three-point backward difference
    (3 f_c - 4 f_n1 + f_n2) / (2 dx), which puts 3a/2 on the diagonal, -2a on
    n1 and +a/2 on n2 (a = |xi_d| / dx_d); elsewhere the row is the
    first-order one of dense_upwind_solve."""
    nc = prob.nx * prob.ny * prob.nz
    widths = [prob.dx, prob.dy, prob.dz]
    solid = np.zeros(nc, bool) if prob.solid is None else prob.solid.reshape(-1).astype(bool)
    A = np.zeros((nc, nc))
    b = np.zeros(nc)
    for c in range(nc):
        if solid[c]:
            A[c, c] = 1.0
            continue
        ijk = [c % prob.nx, (c // prob.nx) % prob.ny, c // (prob.nx * prob.ny)]
        A[c, c] += rtau[c]
        b[c] += rtau[c] * fS[c]
        for d in range(3):
            if xi[d] == 0.0:
                continue
            a = abs(xi[d]) / widths[d][ijk[d]]
            face = 2 * d + (0 if xi[d] > 0 else 1)
            n1 = neighbour(prob, c, face)
            n2 = neighbour(prob, n1, face) if n1 >= 0 else -1
            if n2 >= 0:
                A[c, c] += 1.5 * a
                A[c, n1] -= 2.0 * a
                A[c, n2] += 0.5 * a
            elif n1 >= 0:
                A[c, c] += a
                A[c, n1] -= a
            else:
                A[c, c] += a
                b[c] += a * ghost(c, face)
    f = np.linalg.solve(A, b)
    f[solid] = 0.0
    return f
