"""The velocity-space partition of an outer iteration, the one exchange the
method has (the paper's MPI_Allreduce of the moment and wall-flux sums), on
two gloo processes on the CPU.  Velocities are independent within an
iteration (Eq. (6) lags f^S, tau and rho_w), so each rank sweeps its half of
the velocities with the oracle, the first-pass sums (rho, rho U, rho E,
incoming wall fluxes) are all-reduced, U^{n+1} follows, and the heat-flux
sums of the second pass are all-reduced in turn.  The reduced sums must
equal, bit for bit, the same two partial sums added in one process, and the
serial loop over all velocities to rounding.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle  # noqa: E402
from paper_1810_00348_gb300 import inputs  # noqa: E402


def _problem():
    p = inputs.cavity([7, 6, 5], 8, L_v=3.5, lid=0.2, Kn=0.5)
    return p, inputs.random_macros(p, 11)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _halves(nv, world):
    return [(r * nv // world, (r + 1) * nv // world) for r in range(world)]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, mac = _problem()
    o = Oracle(p, mac)
    a0, a1 = _halves(o.nvel, world)[rank]
    s1 = torch.from_numpy(o.pass1_range(a0, a1))
    dist.all_reduce(s1)
    U = (s1[1:4] / s1[0]).numpy()
    s2 = torch.from_numpy(o.pass2_range(a0, a1, U))
    dist.all_reduce(s2)
    out[rank] = (s1.numpy().tobytes(), s2.numpy().tobytes())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_the_velocity_partition():
    import torch.multiprocessing as mp

    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        res = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), res), nprocs=world, join=True)
        res = dict(res)
    assert res[0] == res[1]  # every rank holds the same reduced sums
    s1 = np.frombuffer(res[0][0]).reshape(11, -1)
    s2 = np.frombuffer(res[0][1]).reshape(3, -1)

    p, mac = _problem()
    o = Oracle(p, mac)
    parts = [o.pass1_range(a0, a1) for a0, a1 in _halves(o.nvel, world)]
    ref1 = parts[0] + parts[1]
    assert np.array_equal(s1, ref1)
    U = ref1[1:4] / ref1[0]
    qparts = [o.pass2_range(a0, a1, U) for a0, a1 in _halves(o.nvel, world)]
    assert np.array_equal(s2, qparts[0] + qparts[1])

    # the partition changes only the order of the additions
    full1 = o.pass1_range(0, o.nvel)
    assert np.max(np.abs(s1 - full1)) <= 1e-13 * np.max(np.abs(full1))
    full2 = o.pass2_range(0, o.nvel, U)
    assert np.max(np.abs(s2 - full2)) <= 1e-13 * np.max(np.abs(full2))
