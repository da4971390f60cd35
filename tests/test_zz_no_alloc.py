"""kgs_iterate_noalloc: the entry point for callers that cannot allocate
device memory (a framework pool owns the device, a latency-critical path
cannot take cudaMalloc's synchronisation, or nothing may be allocated after
start-up).  It runs one outer iteration out of a fixed file-scope device
array; its outputs must equal those of the allocating path (kgs_setup +
kgs_iterate) for the same state, on two calls in a row, within the FP64
parity tolerance of the other GPU tests.

Collected last on purpose: the test allocates its own input and output
buffers with torch, and it must pass both alone in a fresh process and after
every other test.
"""
import numpy as np
import pytest

from paper_1810_00348_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def _mass(p, mac):
    vol = np.multiply.outer(np.multiply.outer(p.dz, p.dy), p.dx)
    return float(np.sum(mac[0] * vol))


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_allocating_path_on_two_calls(precision):
    import torch

    from paper_1810_00348_gb300 import kgs
    from tests.parity import field_errors

    kgs.load()
    p = inputs.cavity([12, 10, 9], [8, 7, 8], L_v=3.5, lid=0.2, Kn=0.4)
    mac = inputs.random_macros(p, 401)
    ctx = kgs.kgs_setup(p, precision=precision)
    kgs.kgs_set_initial(ctx, mac)
    rw0 = kgs.kgs_rho_w(ctx).copy()
    ref = []
    for _ in range(2):
        rc, _, r = kgs.kgs_iterate(ctx, 1)
        assert rc == kgs.KGS_OK
        ref.append((kgs.kgs_moments(ctx).copy(), kgs.kgs_rho_w(ctx).copy(), r))

    dev = torch.device("cuda", torch.cuda.current_device())
    m_in = torch.tensor(mac.reshape(-1), dtype=torch.float64, device=dev)
    w_in = torch.tensor(rw0.reshape(-1), dtype=torch.float64, device=dev)
    M0 = _mass(p, mac)
    for step in range(2):
        m_out = torch.empty_like(m_in)
        w_out = torch.empty_like(w_in)
        rc, res = kgs.kgs_iterate_noalloc(p, m_in.data_ptr(), w_in.data_ptr(), m_out.data_ptr(), w_out.data_ptr(),
                                          M0=M0, precision=precision)
        assert rc == kgs.KGS_OK
        got_m = m_out.cpu().numpy().reshape(8, p.nz, p.ny, p.nx)
        got_w = w_out.cpu().numpy().reshape(6, p.nz, p.ny, p.nx)
        ref_m, ref_w, ref_r = ref[step]
        err = field_errors(got_m, ref_m)
        assert max(err.values()) <= FP64_TOL, (step, err)
        wall = ref_w != 0.0
        assert np.array_equal(wall, got_w != 0.0)
        assert np.max(np.abs(got_w[wall] - ref_w[wall]) / np.abs(ref_w[wall])) <= FP64_TOL
        assert abs(res - ref_r) <= FP64_TOL * max(abs(ref_r), 1e-300)
        m_in, w_in = m_out, w_out


def test_noalloc_rejects_problems_beyond_the_fixed_scratch():
    import torch

    from paper_1810_00348_gb300 import kgs

    kgs.load()
    p = inputs.cavity(40, 24)  # face planes alone need ~330 MB in FP64
    n = p.ncell
    dev = torch.device("cuda", torch.cuda.current_device())
    m = torch.ones(8 * n, dtype=torch.float64, device=dev)
    w = torch.ones(6 * n, dtype=torch.float64, device=dev)
    m2, w2 = torch.empty_like(m), torch.empty_like(w)
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_iterate_noalloc(p, m.data_ptr(), w.data_ptr(), m2.data_ptr(), w2.data_ptr())
    assert e.value.code == kgs.KGS_EINVAL
