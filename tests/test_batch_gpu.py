"""Batched instances in one persistent sweep launch per outer iteration
(kgs_batch_*): results must equal, bit for bit, those of single contexts with
the same sweep shape (same arithmetic in the same order), match the FP64
oracle, retire converged instances, report an expired bounded wait as
KGS_ETIMEOUT without faulting, and stay usable afterwards.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1810_00348_gb300 import inputs
from tests.parity import assert_fields_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


def small_batch(n=5, seed=3):
    # uneven instances drawn with splitmix64, at sizes the oracle handles
    return inputs.batch_cavities(n=n, seed=seed, cells=(5, 12), vels=(8, 12))


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single_contexts(kgs, precision):
    probs = small_batch()
    b = kgs.kgs_batch_setup(probs, precision=precision, v_per_cta=128, block_z=8)
    rc, done, res = kgs.kgs_batch_iterate(b, 3)
    assert rc == kgs.KGS_OK and done == [3] * len(probs)
    for i, p in enumerate(probs):
        c = kgs.kgs_setup(p, precision=precision, v_per_cta=128, block_z=8)
        rc1, _, r1 = kgs.kgs_iterate(c, 3)
        assert rc1 == kgs.KGS_OK
        assert np.array_equal(kgs.kgs_batch_moments(b, i), kgs.kgs_moments(c)), i
        assert res[i] == r1


def test_batch_fp64_matches_oracle(kgs):
    probs = small_batch(n=3, seed=5)
    b = kgs.kgs_batch_setup(probs, precision=0, v_per_cta=128, block_z=4)
    kgs.kgs_batch_iterate(b, 2)
    for i, p in enumerate(probs):
        o = Oracle(p)
        o.iterate(2)
        assert_fields_close(kgs.kgs_batch_moments(b, i), o.macros(), 1e-10, what="batch instance %d" % i)


def test_batch_convergence_retires_instances(kgs):
    probs = small_batch(n=4, seed=7)
    b = kgs.kgs_batch_setup(probs, precision=0, v_per_cta=128, block_z=8, tol=1e-6, max_iters=300)
    rc, done, res = kgs.kgs_batch_iterate(b, 0)
    assert rc == kgs.KGS_OK
    assert all(r < 1e-6 for r in res)
    for i, p in enumerate(probs):
        c = kgs.kgs_setup(p, precision=0, v_per_cta=128, block_z=8, tol=1e-6, max_iters=300)
        rc1, n1, r1 = kgs.kgs_iterate(c, 0)
        assert done[i] == n1  # retired exactly when the single run converges
        assert np.array_equal(kgs.kgs_batch_moments(b, i), kgs.kgs_moments(c))


def test_batch_wait_timeout_is_reported_and_recoverable(kgs):
    probs = small_batch(n=3, seed=11)
    b = kgs.kgs_batch_setup(probs, precision=1, v_per_cta=128, block_z=4)
    # item 0 (stage 0) never announces completion: its dependents give up
    kgs.kgs_batch_fault(b, spin_limit=20000, unpublished_item=0)
    rc, _, _ = kgs.kgs_batch_iterate(b, 1)
    assert rc == kgs.KGS_ETIMEOUT
    kgs.kgs_batch_fault(b)  # normal operation again
    for i in range(len(probs)):
        kgs.kgs_batch_set_initial(b, i)
    rc, done, _ = kgs.kgs_batch_iterate(b, 2)
    assert rc == kgs.KGS_OK and done == [2] * len(probs)
    for i, p in enumerate(probs):
        c = kgs.kgs_setup(p, precision=1, v_per_cta=128, block_z=4)
        kgs.kgs_iterate(c, 2)
        assert np.array_equal(kgs.kgs_batch_moments(b, i), kgs.kgs_moments(c))


def test_autotune_picks_a_valid_cached_shape(kgs):
    import time

    p = inputs.cavity(12, 8, Kn=0.5)
    t0 = time.perf_counter()
    vpc, bz = kgs.kgs_autotune(p, precision=1)
    t1 = time.perf_counter()
    assert vpc in (128, 256) and bz in (8, 16, 32)
    assert kgs.kgs_autotune(p, precision=1) == (vpc, bz)
    assert time.perf_counter() - t1 < 0.1 * max(t1 - t0, 1e-3) + 0.05  # second call is a cache hit
    vpc64, _ = kgs.kgs_autotune(p, precision=0)
    assert vpc64 == 128
    # a batch with v_per_cta = block_z = 0 uses the tuned shape of its largest instance
    b = kgs.kgs_batch_setup([p, inputs.cavity(6, 6)], precision=1)
    info = kgs.kgs_batch_info(b, 0)
    assert (info["v_per_cta"], info["block_z"]) == (vpc, bz)


def test_batch_solve_equals_kgs_solve_per_instance(kgs):
    """kgs_batch_solve applies kgs_solve's switch rule to every instance of a
    batch: with the same sweep shapes (256 velocities per thread block in the
    mixed phase, 128 in FP64, blocks 32 cells deep) each instance follows the
    same mixed iterations, switches at the same iteration and ends on the same
    FP64 state, bit for bit."""
    probs = inputs.batch_cavities(n=4, seed=11, cells=(6, 12), vels=(8, 12))
    rc, b, nm, nd, res = kgs.kgs_batch_solve(probs, tol=1e-6, max_iters=2000, v_per_cta=256, block_z=32)
    assert rc == kgs.KGS_OK
    assert all(r < 1e-6 for r in res)
    for i, p in enumerate(probs):
        rc1, m1, nm1, nd1, r1 = kgs.kgs_solve(p, tol=1e-6, max_iters=2000)
        assert rc1 == kgs.KGS_OK
        assert (nm[i], nd[i]) == (nm1, nd1), i
        assert res[i] == r1
        assert np.array_equal(kgs.kgs_batch_moments(b, i), m1), i
