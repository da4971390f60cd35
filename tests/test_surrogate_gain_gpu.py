"""The learned initial guess end to end on small cavities: training data from
the solver, a short training run of the full-size network, then held-out
solves from the uniform state, from the upsampled coarse solution alone (the
network's input) and from the guess; and the fallback that rejects a guess
which is not a physical state.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CELLS, VELS, TOL = 12, 12, 1e-6


@pytest.fixture(scope="module")
def sur():
    from paper_1810_00348_gb300 import kgs, surrogate
    kgs.load()
    return surrogate


@pytest.fixture(scope="module")
def trained(sur):
    from paper_1810_00348_gb300 import kgs
    probs = sur.draw_cavities(64, seed=100, cells=CELLS, vels=VELS)
    samples = sur.make_samples(probs, precision=kgs.KGS_FP64, tol=TOL, max_iters=3000)
    assert all(s.iters_fine < 3000 and s.iters_coarse < 3000 for s in samples)
    s = sur.Surrogate(seed=0)
    assert 0.9e6 < s.num_params() < 1.1e6
    losses = s.train(samples, steps=600, batch=16, lr=1e-3, seed=0)
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10])
    return s


def test_guess_saves_iterations_on_held_out_cavities(sur, trained):
    from paper_1810_00348_gb300 import kgs
    held = sur.draw_cavities(3, seed=999, cells=CELLS, vels=VELS)
    coarse, _, _, rc = sur.solve([sur.coarse_problem(p) for p in held], kgs.KGS_FP64, TOL, 3000)
    assert rc == kgs.KGS_OK
    gains = []
    for p, c in zip(held, coarse):
        n_uniform, _, r_u, rc_u = sur.iterations_to(p, None, kgs.KGS_FP64, TOL, 3000)
        _, up = sur.upsample(p, c)
        n_up, _, r_up, rc_up = sur.iterations_to(p, up.cpu().numpy(), kgs.KGS_FP64, TOL, 3000)
        guess, n_bad = trained.guess(p, c)
        assert n_bad == 0 and guess is not None
        n_guess, _, r_g, rc_g = sur.iterations_to(p, guess, kgs.KGS_FP64, TOL, 3000)
        assert rc_u == kgs.KGS_OK and rc_g == kgs.KGS_OK and rc_up == kgs.KGS_OK
        assert r_u < TOL and r_g < TOL and r_up < TOL
        assert n_guess < n_uniform, (p.name, n_guess, n_uniform)
        # the network must add to its own input: fewer iterations than from
        # the upsampled coarse solution it corrects
        assert n_guess <= n_up, (p.name, n_guess, n_up)
        gains.append(n_up - n_guess)
        # both starts converge to the same fixed point
        ctx_u = kgs.kgs_setup(p, precision=kgs.KGS_FP64, tol=TOL, max_iters=3000)
        kgs.kgs_iterate(ctx_u, 0)
        ctx_g = kgs.kgs_setup(p, precision=kgs.KGS_FP64, tol=TOL, max_iters=3000)
        kgs.kgs_set_initial(ctx_g, guess)
        kgs.kgs_iterate(ctx_g, 0)
        mu, mg = kgs.kgs_moments(ctx_u), kgs.kgs_moments(ctx_g)
        assert np.abs(mu[0] - mg[0]).max() < 1e-3
    assert sum(gains) > 0, gains


def test_unphysical_guess_is_rejected(sur):
    from paper_1810_00348_gb300 import kgs
    s = sur.Surrogate(channels=(11, 16, 8), seed=1)
    n, _ = kgs.kgs_net_num_params(s.net)
    params = np.zeros(n, np.float32)
    params[-8] = -1e4   # bias of the density correction: rho = up - 1e3
    kgs.kgs_net_set_params(s.net, params)
    p = sur.draw_cavities(1, seed=5, cells=8, vels=8)[0]
    coarse = np.zeros((8, 4, 4, 4))
    coarse[0] = coarse[4] = 1.0
    guess, n_bad = s.guess(p, coarse)
    assert guess is None and n_bad == p.ncell
