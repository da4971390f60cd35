"""The seeded synthetic workloads are what the design states: the
splitmix64 generator against its published outputs, the batch draw ranges,
the cube's geometry and free stream, and the velocity quadratures."""
import math

import numpy as np

from paper_1810_00348_gb300 import inputs


def test_splitmix64_published_outputs():
    # splitmix64 from state 0 (Steele, Lea & Flood 2014; the usual seeding
    # generator of the xoshiro family): its first three outputs
    g = inputs.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_batch_draws_ranges_and_determinism():
    a = inputs.batch_cavities(64, seed=0)
    b = inputs.batch_cavities(64, seed=0)
    c = inputs.batch_cavities(64, seed=1)
    key = lambda ps: [(p.nx, len(p.xi_x), p.Kn, p.U_w[3][0]) for p in ps]
    assert key(a) == key(b) and key(a) != key(c)
    for p in a:
        assert 0.05 <= p.Kn <= 10.0
        assert 16 <= p.nx <= 48 and p.nx == p.ny == p.nz
        assert 16 <= len(p.xi_x) <= 32
        assert 0.05 <= p.U_w[3][0] <= 0.3   # lid: the +y face moving along x
    # log-uniform Kn: both decades ends are visited over 64 draws
    assert min(p.Kn for p in a) < 0.2 and max(p.Kn for p in a) > 2.0


def test_cube_geometry_and_free_stream():
    p = inputs.cube()
    assert (p.nx, p.ny, p.nz) == (96, 64, 64)
    solid = p.solid.astype(bool)
    assert solid.sum() == 16 ** 3
    zs, ys, xs = np.nonzero(solid)
    for idx in (xs, ys, zs):  # [1.5, 2.5] in cells of 1/16
        assert idx.min() == 24 and idx.max() == 39
    assert math.isclose(p.U_in[0], 2.0 * math.sqrt(5.0 / 6.0)) and p.U_in[1] == p.U_in[2] == 0.0
    assert all(f == inputs.FACE_INFLOW for f in p.face_type) and p.mass_rescale == 0


def test_velocity_axes():
    # uniform trapezoid on [-4, 4]: end nodes with half weights, total 8
    x, w = inputs.uniform_axis(32, 4.0)
    assert x[0] == -4.0 and x[-1] == 4.0 and np.allclose(np.diff(x), 8.0 / 31)
    assert math.isclose(w[0], w[1] / 2) and math.isclose(w.sum(), 8.0)
    # stretched: symmetric, ends at +-L, finer at the origin, weights integrate 1 exactly
    x, w = inputs.stretched_axis(48, 8.0, 3.0)
    assert np.allclose(x, -x[::-1]) and math.isclose(x[-1], 8.0)
    d = np.diff(x)
    assert d[len(d) // 2] < d[0] / 5 and np.all(w > 0) and math.isclose(w.sum(), 16.0)


def test_cube_on_the_papers_stretched_mesh():
    """Section 4.2's mesh: 181 x 181 x 191 cells whose widths grow cell by
    cell by 1.02 in front of and beside the unit cube and by 1.03 behind it
    (flow along x), the cube spanned by equal cells, 48^3 uniform velocities
    on [-4, 4]^3, Kn 1, Ma 2."""
    p = inputs.cube_paper_mesh()
    assert (p.nx, p.ny, p.nz) == (191, 181, 181)
    assert len(p.xi_x) == 48 and p.xi_x[0] == -4.0 and p.xi_x[-1] == 4.0
    assert p.Kn == 1.0 and abs(p.U_in[0] - 2.0 * np.sqrt(5.0 / 6.0)) < 1e-15
    zs, ys, xs = np.nonzero(p.solid)
    n = 31
    assert p.solid.sum() == n ** 3
    for w, lo in ((p.dx, xs.min()), (p.dy, ys.min()), (p.dz, zs.min())):
        assert np.allclose(w[lo:lo + n], 1.0 / n)          # equal cells across the cube
        assert abs(np.sum(w[lo:lo + n]) - 1.0) < 1e-12      # unit side
    ratio = lambda w: w[1:] / w[:-1]
    x0 = xs.min()
    assert np.allclose(ratio(p.dx[:x0 + 1]), 1.0 / 1.02)     # front: growing away from the cube
    assert np.allclose(ratio(p.dx[x0 + n - 1:]), 1.03)       # rear
    y0 = ys.min()
    assert np.allclose(ratio(p.dy[:y0 + 1]), 1.0 / 1.02) and np.allclose(ratio(p.dy[y0 + n - 1:]), 1.02)
